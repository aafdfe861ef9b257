"""The full-size workloads whose streams and reconstructions are pinned by hash.

Each case is (name, group, spec): the seeded field ``synth.make_field(spec)``
compressed with the NOA bound ``spec.eb``.  Group "single" is one field per call
(the 2D image, the 512^3 float32 field at three bounds, the 256x384x384 float64
field with ties); group "batch" is the 64-field mixed batch, compressed in one
batched call.  ``tests/golden/make_full_hashes.py`` writes the oracle's SHA-256
of every field, stream and reconstruction to ``tests/golden/full_hashes.json``;
``tests/test_gpu_full_hashes.py`` compares the CUDA path's against them.
"""
from paper_2603_26968_b300 import synth as S


def cases():
    out = [("c1_f32_256x256_noa1e-3", "single", S.spec_2d_small())]
    for eb in (1e-2, 1e-3, 1e-4):
        out.append((f"c2_f32_512_noa{eb:.0e}", "single", S.spec_3d_f32(n=512, eb=eb)))
    out.append(("c3_f64_256x384x384_noa5e-4", "single", S.spec_3d_f64_ties()))
    for j, sp in enumerate(S.spec_batch()):
        out.append((f"c4_field{j:02d}", "batch", sp))
    return out


def field_key(spec):
    """Specs that differ only in their bound make the same field."""
    return (spec.name, spec.shape, spec.dtype, spec.recipe, spec.n_bumps, spec.sigma, spec.seed, spec.noise,
            tuple(sorted((k, tuple(v) if isinstance(v, (list, tuple)) else v) for k, v in spec.extra.items())))
