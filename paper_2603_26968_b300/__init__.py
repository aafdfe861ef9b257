"""LOPC hot path on B300: error-bounded quantization, local-order repair, lossless
coding of bins and subbins, and the matching decompressor, as hand-written CUDA for
sm_103a behind a C ABI (``include/lopc.h``)."""
