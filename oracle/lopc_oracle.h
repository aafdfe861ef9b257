/* lopc_oracle.h -- plain, slow CPU oracle of the LOPC hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link or call
 * this; only the tests, the smoke check and the benchmark's CPU-baseline leg do.
 * It shares no code, header, table or constant generator with the CUDA library.
 *
 * What it computes (the paper is "Fast Topology-Aware Lossy Data Compression with
 * Full Preservation of Critical Points and Local Order", LOPC):
 *   - error bound resolution, ABS or NOA (Sec. III-A);
 *   - the half-width quantizer b = round(x / eps) (Sec. III-A);
 *   - flags and the subbin repair of Algorithms 1 and 2, as the least fixpoint
 *     (Sec. III-B, III-E) and, as a cross-check, as the paper's own iteration;
 *   - lossless coding: a Lorenzo or 1D-difference residual (format 2; DIFFNB only in
 *     format 1), NB mapping, BIT, RZE_1 for bins, BIT.RZE_w.RZE_1 for subbins over
 *     16 KiB chunks (Sec. III-C);
 *   - the decoder: subbin k of bin b decodes to the k-th representable value above
 *     the lowest value of the bin (Sec. III-E);
 *   - checkers: neighbour-order preservation and critical-point types (Sec. II).
 *
 * Status codes match the library's numeric values but are defined here on their own.
 */
#ifndef LOPC_ORACLE_H
#define LOPC_ORACLE_H
#include <stddef.h>
#include <stdint.h>

#define ORC_OK 0
#define ORC_INVALID_ARG (-1)
#define ORC_NONFINITE (-2)
#define ORC_RANGE (-3)
#define ORC_CAPACITY (-4)
#define ORC_CORRUPT (-5)

typedef struct {
  int32_t dtype;   /* 0 = float32, 1 = float64 */
  int32_t ndim;    /* 2 or 3 */
  int64_t dims[3]; /* slowest first; a 2D field uses dims[0..1] */
  int32_t mode;    /* 0 = ABS, 1 = NOA */
  int32_t pad_;
  double eb;
} orc_desc;

/* Error bound: eps, the shrunk quantizer width eps_q and inv = 1/eps_q; *constant = 1
 * when NOA meets a zero value range. */
int orc_resolve_eps(const orc_desc* d, const void* x, double* eps, double* eps_q, double* inv,
                    int* constant, double* const_value);
/* b[i] = round-half-even of the exact product x[i]*inv. */
int orc_quantize(int dtype, const void* x, int64_t n, double inv, int64_t* b);
/* Same for a single value (used by the decoder and by tests). */
int64_t orc_q1(int dtype, double v, double inv);
/* Smallest value v of the dtype with q(v) == b; returns 0 on success. */
int orc_lowest_in_bin(int dtype, int64_t b, double inv, double* v);
/* k-th successor in the total order of the dtype's values (+0 canonical). */
double orc_succ_k(int dtype, double v, uint64_t k);

/* Per point, bit k = neighbour k exists, is in the same bin and precedes p. */
void orc_constraint_masks(const orc_desc* d, const void* x, const int64_t* b, uint16_t* cmask);
/* Least fixpoint of the subbin constraints, by one pass in ascending (value, index). */
int orc_repair_lfp(const orc_desc* d, const void* x, const int64_t* b, uint64_t* s);
/* The paper's worklist iteration (Algorithms 1-2), run serially; returns #iterations. */
int64_t orc_repair_alg2(const orc_desc* d, const void* x, const int64_t* b, uint64_t* s);
/* xhat[i] = succ^s[i](lowest value in bin b[i]). */
int orc_reconstruct(int dtype, int64_t n, const int64_t* b, const uint64_t* s, double inv, void* xhat);

/* Codec stages on byte buffers (w = word bytes, 4 or 8). */
size_t orc_diffnb(int w, const int64_t* v, int64_t n, uint8_t* out);
void orc_undiffnb(int w, const uint8_t* in, int64_t n, int64_t* v);
size_t orc_bit(int w, const uint8_t* words, int64_t n, uint8_t* out);
void orc_unbit(int w, const uint8_t* in, int64_t n32, uint8_t* words);
size_t orc_rze(int g, const uint8_t* in, size_t L, uint8_t* out);
int orc_unrze(int g, const uint8_t* in, size_t in_len, size_t L, uint8_t* out);

/* One chunk's records (Sec. III-C): bins and subbins of its points in chunk order,
 * the chunk being dims[0] x dims[1] x dims[2] points (2D: dims[0] = 1); each record
 * buffer needs n*w bytes; sizes carry the raw flag (bit 31) and, for bins, the flag
 * of the 1D-difference predictor (bit 30; otherwise the Lorenzo residual). */
void orc_encode_chunk(int dtype, const int64_t* b, const uint64_t* s, const int64_t dims[3], uint8_t* bin_rec,
                      uint32_t* bin_size, uint8_t* sub_rec, uint32_t* sub_size);

/* Whole stream. */
size_t orc_compress_bound(const orc_desc* d);
int orc_compress(const orc_desc* d, const void* x, uint8_t* out, size_t cap, size_t* out_size);
int orc_peek(const uint8_t* in, size_t n, orc_desc* d);
int orc_decompress(const uint8_t* in, size_t n, void* xhat, size_t cap_bytes);

/* Checkers: number of neighbour pairs whose order differs between x and y (same
 * dtype); critical-point types as (#lower-link components, #upper-link components). */
int64_t orc_order_violations(const orc_desc* d, const void* x, const void* y);
void orc_critical_types(const orc_desc* d, const void* x, uint8_t* lower_cc, uint8_t* upper_cc);

#endif
