/* lopc_oracle.c -- plain, slow, single-threaded CPU oracle of the LOPC hot path.
 *
 * TEST INFRASTRUCTURE ONLY (see lopc_oracle.h).  Every function follows a passage of
 * the paper or one of the stated readings of it; nothing here is blocked, fused or
 * reordered for speed.  Build:  gcc -O2 -ffp-contract=off -shared -fPIC ... -lquadmath
 * A second build adds -fopenmp: the loops whose iterations are independent (points
 * of the quantizer, chunks of the coder and decoder) are then split over threads,
 * each iteration computing exactly what it computes alone, so both builds give the
 * same bytes.  The repair stays one sequential pass in (value, index) order.
 *
 * Readings of the paper that this file fixes (the paper is silent or garbled there):
 *   neighbourhood   Freudenthal triangulation of the grid (Sec. II, "as in prior
 *                   work"): neighbours of v are v +- d, d in {0,1}^ndim \ {0};
 *   tie-break       Simulation of Simplicity by linear index (Sec. II, Alg. 1):
 *                   n precedes p iff x_n < x_p, or x_n == x_p and idx_n < idx_p,
 *                   compared numerically (-0 == +0);
 *   quantizer       b = round-half-even(x * inv) of the EXACT real product, with
 *                   eps_q = eps*(1 - 2^-16) and inv = 1/eps_q in IEEE binary64
 *                   (Sec. III-A says "multiply by 1/eps and round to nearest");
 *                   |b| must stay below 2^30 (float32) or 2^52 (float64);
 *   constant field  NOA with a zero range stores the value itself;
 *   repair          the least non-negative s with s(p) >= s(n) + [idx_n > idx_p] for
 *                   every same-bin neighbour n preceding p (Sec. III-B, III-E:
 *                   "as low as possible");
 *   decode          subbin k of bin b is the k-th value above the lowest value v of
 *                   the dtype with q(v) == b (Sec. III-E);
 *   format          16 KiB chunks (Sec. II-C on PFPL) taken as fixed tiles; stage
 *                   layouts of DIFFNB, BIT, RZE as written below.
 */
#include "lopc_oracle.h"

#include <math.h>
#include <quadmath.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ values, keys */

static double val_at(int dtype, const void* x, int64_t i) {
  return dtype == 0 ? (double)((const float*)x)[i] : ((const double*)x)[i];
}

static int64_t max_key(int dtype) {
  return dtype == 0 ? (int64_t)0x7f7fffff : (int64_t)0x7fefffffffffffffLL;
}

/* Position of a finite value in the total order of the dtype's values, with -0 and
 * +0 sharing position 0. */
static int64_t key_of(int dtype, double v) {
  if (dtype == 0) {
    float f = (float)v;
    uint32_t u;
    memcpy(&u, &f, 4);
    int64_t m = (int64_t)(u & 0x7fffffffu);
    return (u >> 31) ? -m : m;
  } else {
    uint64_t u;
    memcpy(&u, &v, 8);
    int64_t m = (int64_t)(u & 0x7fffffffffffffffULL);
    return (u >> 63) ? -m : m;
  }
}

static double val_of_key(int dtype, int64_t k) {
  if (dtype == 0) {
    uint32_t u = k >= 0 ? (uint32_t)k : (0x80000000u | (uint32_t)(-k));
    float f;
    memcpy(&f, &u, 4);
    return (double)f;
  } else {
    uint64_t u = k >= 0 ? (uint64_t)k : (0x8000000000000000ULL | (uint64_t)(-k));
    double d;
    memcpy(&d, &u, 8);
    return d;
  }
}

double orc_succ_k(int dtype, double v, uint64_t k) {
  int64_t key = key_of(dtype, v);
  if (k > (uint64_t)(max_key(dtype) - key)) return INFINITY;
  return val_of_key(dtype, key + (int64_t)k);
}

/* ------------------------------------------------------------------- quantizer */

static int64_t bin_limit(int dtype) { return dtype == 0 ? ((int64_t)1 << 30) : ((int64_t)1 << 52); }

/* Sec. III-A: bin = round(x * (1/eps)).  The product of two binary64 significands
 * has at most 106 bits, so binary128 (113-bit significand) holds it exactly and
 * rintq rounds it half-to-even.  Returns INT64_MIN when |x*inv| >= 2^62. */
int64_t orc_q1(int dtype, double v, double inv) {
  (void)dtype;
  __float128 t = (__float128)v * (__float128)inv;
  if (fabsq(t) >= 4611686018427387904.0Q) return INT64_MIN;
  return (int64_t)rintq(t);
}

int orc_quantize(int dtype, const void* x, int64_t n, double inv, int64_t* b) {
  int64_t lim = bin_limit(dtype);
  int bad = 0; /* every point is independent: the OpenMP build splits the loop */
#pragma omp parallel for schedule(static) reduction(| : bad)
  for (int64_t i = 0; i < n; i++) {
    int64_t q = orc_q1(dtype, val_at(dtype, x, i), inv);
    if (q == INT64_MIN || q >= lim || q <= -lim)
      bad = 1;
    else
      b[i] = q;
  }
  return bad ? ORC_RANGE : ORC_OK;
}

/* Sec. III-E: subbin 0 is the lowest representable value of the bin.  The
 * quantizer is monotone in the value, hence in the key, so bisection over the keys
 * finds the smallest key whose value quantizes to >= b. */
int orc_lowest_in_bin(int dtype, int64_t b, double inv, double* v) {
  int64_t lo = -max_key(dtype), hi = max_key(dtype);
  int64_t qh = orc_q1(dtype, val_of_key(dtype, hi), inv);
  if (qh != INT64_MIN && qh < b) return ORC_CORRUPT;
  while (lo < hi) {
    int64_t mid = (int64_t)(((__int128)lo + (__int128)hi) >> 1); /* floor, so mid < hi */
    int64_t q = orc_q1(dtype, val_of_key(dtype, mid), inv);
    if (q == INT64_MIN) q = val_of_key(dtype, mid) < 0 ? INT64_MIN : INT64_MAX;
    if (q >= b) hi = mid; else lo = mid + 1;
  }
  double r = val_of_key(dtype, lo);
  if (orc_q1(dtype, r, inv) != b) return ORC_CORRUPT;
  *v = r;
  return ORC_OK;
}

/* -------------------------------------------------------------- error bound */

static int desc_ok(const orc_desc* d) {
  if (!d) return 0;
  if (d->dtype != 0 && d->dtype != 1) return 0;
  if (d->ndim != 2 && d->ndim != 3) return 0;
  for (int k = 0; k < d->ndim; k++)
    if (d->dims[k] <= 0) return 0;
  if (d->mode != 0 && d->mode != 1) return 0;
  if (!(d->eb > 0.0) || !isfinite(d->eb)) return 0;
  return 1;
}

static int64_t npoints(const orc_desc* d) {
  int64_t n = 1;
  for (int k = 0; k < d->ndim; k++) n *= d->dims[k];
  return n;
}

/* Sec. III-A: ABS eps = eb; NOA eps = eb * (x_max - x_min). */
int orc_resolve_eps(const orc_desc* d, const void* x, double* eps, double* eps_q, double* inv,
                    int* constant, double* const_value) {
  if (!desc_ok(d)) return ORC_INVALID_ARG;
  int64_t n = npoints(d);
  for (int64_t i = 0; i < n; i++)
    if (!isfinite(val_at(d->dtype, x, i))) return ORC_NONFINITE;
  *constant = 0;
  *const_value = 0.0;
  double e;
  if (d->mode == 0) {
    e = d->eb;
  } else {
    double mn = val_at(d->dtype, x, 0), mx = mn;
    for (int64_t i = 1; i < n; i++) {
      double v = val_at(d->dtype, x, i);
      if (v < mn) mn = v;
      if (v > mx) mx = v;
    }
    double r = mx - mn;
    if (!isfinite(r)) return ORC_RANGE;
    if (r == 0.0) {
      *constant = 1;
      *const_value = mn + 0.0; /* +0 is canonical */
      *eps = 0.0;
      *eps_q = 0.0;
      *inv = 0.0;
      return ORC_OK;
    }
    e = d->eb * r;
  }
  if (!(e > 0.0) || !isfinite(e)) return ORC_RANGE;
  double eq = e * (1.0 - 0x1p-16);
  double iv = 1.0 / eq;
  if (!(eq > 0.0) || !isfinite(iv)) return ORC_RANGE;
  *eps = e;
  *eps_q = eq;
  *inv = iv;
  return ORC_OK;
}

/* --------------------------------------------------------------- neighbourhood */

/* Freudenthal triangulation: the 7 non-zero 0/1 offsets (dz, dy, dx); direction
 * k < 7 is -P[k], direction k >= 7 is +P[k-7].  A 2D field is a 3D field with one
 * slab, so offsets with dz != 0 leave the domain. */
static const int P7[7][3] = {{0, 0, 1}, {0, 1, 0}, {0, 1, 1}, {1, 0, 0}, {1, 0, 1}, {1, 1, 0}, {1, 1, 1}};

typedef struct {
  int64_t nz, ny, nx;
} grid3;

static grid3 grid_of(const orc_desc* d) {
  grid3 g;
  if (d->ndim == 2) {
    g.nz = 1;
    g.ny = d->dims[0];
    g.nx = d->dims[1];
  } else {
    g.nz = d->dims[0];
    g.ny = d->dims[1];
    g.nx = d->dims[2];
  }
  return g;
}

static void dir_offset(int k, int* dz, int* dy, int* dx) {
  int s = k < 7 ? -1 : 1;
  const int* p = P7[k % 7];
  *dz = s * p[0];
  *dy = s * p[1];
  *dx = s * p[2];
}

/* Index of neighbour k of point i, or -1 outside the domain. */
static int64_t neighbour(grid3 g, int64_t i, int k) {
  int64_t x = i % g.nx, y = (i / g.nx) % g.ny, z = i / (g.nx * g.ny);
  int dz, dy, dx;
  dir_offset(k, &dz, &dy, &dx);
  x += dx;
  y += dy;
  z += dz;
  if (x < 0 || y < 0 || z < 0 || x >= g.nx || y >= g.ny || z >= g.nz) return -1;
  return (z * g.ny + y) * g.nx + x;
}

/* Simulation of Simplicity: never equal, ties broken by the lower index. */
static int precedes(int dtype, const void* x, int64_t n, int64_t p) {
  double vn = val_at(dtype, x, n), vp = val_at(dtype, x, p);
  return vn < vp || (vn == vp && n < p);
}

/* Alg. 1, second loop: per neighbour, same bin and "n < p". */
void orc_constraint_masks(const orc_desc* d, const void* x, const int64_t* b, uint16_t* cmask) {
  grid3 g = grid_of(d);
  int64_t n = g.nx * g.ny * g.nz;
  for (int64_t p = 0; p < n; p++) {
    uint16_t m = 0;
    for (int k = 0; k < 14; k++) {
      int64_t q = neighbour(g, p, k);
      if (q >= 0 && b[q] == b[p] && precedes(d->dtype, x, q, p)) m |= (uint16_t)(1u << k);
    }
    cmask[p] = m;
  }
}

/* ------------------------------------------------------------------- repair */

typedef struct {
  double v;
  int64_t i;
} vi_t;

static int cmp_vi(const void* a, const void* b) {
  const vi_t* x = (const vi_t*)a;
  const vi_t* y = (const vi_t*)b;
  if (x->v < y->v) return -1;
  if (x->v > y->v) return 1;
  return (x->i > y->i) - (x->i < y->i);
}

/* Sec. III-B and III-E: the subbins are the least values that satisfy every
 * same-bin "n < p" relation, s(p) >= s(n) + [idx_n > idx_p].  The relations are
 * acyclic and follow the ascending (value, index) order, so one pass in that order
 * computes the least solution directly (a longest path in the DAG). */
int orc_repair_lfp(const orc_desc* d, const void* x, const int64_t* b, uint64_t* s) {
  grid3 g = grid_of(d);
  int64_t n = g.nx * g.ny * g.nz;
  vi_t* ord = (vi_t*)malloc(sizeof(vi_t) * (size_t)n);
  if (!ord) return ORC_CAPACITY;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; i++) {
    ord[i].v = val_at(d->dtype, x, i);
    ord[i].i = i;
  }
  qsort(ord, (size_t)n, sizeof(vi_t), cmp_vi);
  for (int64_t r = 0; r < n; r++) {
    int64_t p = ord[r].i;
    uint64_t m = 0;
    for (int k = 0; k < 14; k++) {
      int64_t q = neighbour(g, p, k);
      if (q < 0 || b[q] != b[p] || !precedes(d->dtype, x, q, p)) continue;
      uint64_t c = s[q] + (uint64_t)(q > p);
      if (c > m) m = c;
    }
    s[p] = m;
  }
  free(ord);
  return ORC_OK;
}

/* Algorithms 1 and 2 as printed, run serially: worklist 1 holds all points; each
 * iteration raises s(p) to the largest s(n) + tie over its same-bin lower
 * neighbours and, if it was raised, queues p's greater same-bin neighbours once
 * (a per-point stamp of the last iteration it was queued in).  Returns the number
 * of iterations. */
int64_t orc_repair_alg2(const orc_desc* d, const void* x, const int64_t* b, uint64_t* s) {
  grid3 g = grid_of(d);
  int64_t n = g.nx * g.ny * g.nz;
  int64_t* wl1 = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  int64_t* wl2 = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  int64_t* stamp = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  if (!wl1 || !wl2 || !stamp) {
    free(wl1);
    free(wl2);
    free(stamp);
    return -1;
  }
  int64_t n1 = n, iter = 0;
  for (int64_t i = 0; i < n; i++) {
    s[i] = 0;
    wl1[i] = i;
    stamp[i] = -1;
  }
  while (n1 > 0) {
    int64_t n2 = 0;
    for (int64_t w = 0; w < n1; w++) {
      int64_t p = wl1[w];
      uint64_t nmax = 0;
      for (int k = 0; k < 14; k++) {
        int64_t q = neighbour(g, p, k);
        if (q < 0 || b[q] != b[p] || !precedes(d->dtype, x, q, p)) continue;
        uint64_t c = s[q] + (uint64_t)(q > p);
        if (c > nmax) nmax = c;
      }
      if (s[p] < nmax) {
        s[p] = nmax;
        for (int k = 0; k < 14; k++) {
          int64_t q = neighbour(g, p, k);
          if (q < 0 || b[q] != b[p] || !precedes(d->dtype, x, p, q)) continue;
          if (stamp[q] != iter) {
            stamp[q] = iter;
            wl2[n2++] = q;
          }
        }
      }
    }
    int64_t* t = wl1;
    wl1 = wl2;
    wl2 = t;
    n1 = n2;
    iter++;
  }
  free(wl1);
  free(wl2);
  free(stamp);
  return iter;
}

int orc_reconstruct(int dtype, int64_t n, const int64_t* b, const uint64_t* s, double inv, void* xhat) {
  for (int64_t i = 0; i < n; i++) {
    double lo;
    if (orc_lowest_in_bin(dtype, b[i], inv, &lo) != ORC_OK) return ORC_CORRUPT;
    double v = orc_succ_k(dtype, lo, s[i]);
    if (!isfinite(v)) return ORC_CORRUPT;
    if (dtype == 0)
      ((float*)xhat)[i] = (float)v;
    else
      ((double*)xhat)[i] = v;
  }
  return ORC_OK;
}

/* -------------------------------------------------------------------- codec */

static uint64_t wmask(int w) { return w == 4 ? 0xffffffffULL : 0xffffffffffffffffULL; }

static void put_word(uint8_t* p, int w, uint64_t v) {
  for (int k = 0; k < w; k++) p[k] = (uint8_t)(v >> (8 * k));
}

static uint64_t get_word(const uint8_t* p, int w) {
  uint64_t v = 0;
  for (int k = 0; k < w; k++) v |= (uint64_t)p[k] << (8 * k);
  return v;
}

/* DIFFNB_w (PFPL's delta + negabinary): d_i = v_i - v_{i-1} modulo 2^(8w) with
 * v_{-1} = 0, then u_i = (d_i + M) XOR M with M = 0xAA..A. */
size_t orc_diffnb(int w, const int64_t* v, int64_t n, uint8_t* out) {
  uint64_t msk = wmask(w), M = 0xAAAAAAAAAAAAAAAAULL & msk;
  uint64_t prev = 0;
  for (int64_t i = 0; i < n; i++) {
    uint64_t cur = (uint64_t)v[i];
    uint64_t dd = (cur - prev) & msk;
    uint64_t u = ((dd + M) & msk) ^ M;
    put_word(out + i * w, w, u);
    prev = cur;
  }
  return (size_t)n * (size_t)w;
}

void orc_undiffnb(int w, const uint8_t* in, int64_t n, int64_t* v) {
  uint64_t msk = wmask(w), M = 0xAAAAAAAAAAAAAAAAULL & msk;
  uint64_t prev = 0;
  for (int64_t i = 0; i < n; i++) {
    uint64_t u = get_word(in + i * w, w);
    uint64_t dd = ((u ^ M) - M) & msk;
    uint64_t cur = (prev + dd) & msk;
    v[i] = w == 4 ? (int64_t)(int32_t)(uint32_t)cur : (int64_t)cur;
    prev = cur;
  }
}

/* BIT_w: pad to a multiple of 32 words with zeros; plane k (k = 0 is the least
 * significant bit) is n32/32 little-endian u32 words whose bit j of word g is bit k
 * of input word 32g + j.  Output length w * n32 bytes. */
size_t orc_bit(int w, const uint8_t* words, int64_t n, uint8_t* out) {
  int64_t n32 = (n + 31) / 32 * 32, G = n32 / 32;
  for (int k = 0; k < 8 * w; k++) {
    for (int64_t g = 0; g < G; g++) {
      uint32_t acc = 0;
      for (int j = 0; j < 32; j++) {
        int64_t i = 32 * g + j;
        if (i >= n) break;
        uint32_t bit = (words[i * w + k / 8] >> (k % 8)) & 1u;
        acc |= bit << j;
      }
      put_word(out + (k * G + g) * 4, 4, acc);
    }
  }
  return (size_t)w * (size_t)n32;
}

void orc_unbit(int w, const uint8_t* in, int64_t n32, uint8_t* words) {
  int64_t G = n32 / 32;
  memset(words, 0, (size_t)n32 * (size_t)w);
  for (int k = 0; k < 8 * w; k++)
    for (int64_t g = 0; g < G; g++) {
      uint32_t acc = (uint32_t)get_word(in + (k * G + g) * 4, 4);
      for (int j = 0; j < 32; j++)
        if ((acc >> j) & 1u) words[(32 * g + j) * w + k / 8] |= (uint8_t)(1u << (k % 8));
    }
}

/* Repeat elimination of a byte string (how RZE compresses its bitmap): bit j of the
 * new bitmap is set when byte j differs from byte j-1 (byte -1 being 0); only those
 * bytes are kept. */
static size_t repeat_elim(const uint8_t* a, size_t len, uint8_t* bm, uint8_t* kept) {
  size_t nk = 0;
  memset(bm, 0, (len + 7) / 8);
  for (size_t j = 0; j < len; j++) {
    uint8_t prev = j ? a[j - 1] : 0;
    if (a[j] != prev) {
      bm[j / 8] |= (uint8_t)(1u << (j % 8));
      kept[nk++] = a[j];
    }
  }
  return nk;
}

/* RZE_g: a bitmap with one bit per g-byte unit (1 = non-zero, least significant
 * bit first) and the non-zero units; the bitmap is repeat-eliminated twice.
 * Output: [level-2 bitmap][level-1 kept][level-0 kept][non-zero units]. */
size_t orc_rze(int g, const uint8_t* in, size_t L, uint8_t* out) {
  size_t U = L / (size_t)g;
  size_t l0 = (U + 7) / 8, l1 = (l0 + 7) / 8, l2 = (l1 + 7) / 8;
  uint8_t* m0 = (uint8_t*)calloc(l0 + 1, 1);
  uint8_t* m1 = (uint8_t*)calloc(l1 + 1, 1);
  uint8_t* m2 = (uint8_t*)calloc(l2 + 1, 1);
  uint8_t* k0 = (uint8_t*)malloc(l0 + 1);
  uint8_t* k1 = (uint8_t*)malloc(l1 + 1);
  uint8_t* pay = (uint8_t*)malloc(L + 1);
  size_t np = 0;
  for (size_t j = 0; j < U; j++) {
    int nz = 0;
    for (int t = 0; t < g; t++) nz |= in[j * g + t] != 0;
    if (nz) {
      m0[j / 8] |= (uint8_t)(1u << (j % 8));
      memcpy(pay + np * g, in + j * g, (size_t)g);
      np++;
    }
  }
  size_t nk0 = repeat_elim(m0, l0, m1, k0);
  size_t nk1 = repeat_elim(m1, l1, m2, k1);
  size_t o = 0;
  memcpy(out + o, m2, l2);
  o += l2;
  memcpy(out + o, k1, nk1);
  o += nk1;
  memcpy(out + o, k0, nk0);
  o += nk0;
  memcpy(out + o, pay, np * (size_t)g);
  o += np * (size_t)g;
  free(m0);
  free(m1);
  free(m2);
  free(k0);
  free(k1);
  free(pay);
  return o;
}

static int tail_bits_zero(const uint8_t* bm, size_t nbits) {
  size_t nbytes = (nbits + 7) / 8;
  for (size_t j = nbits; j < nbytes * 8; j++)
    if ((bm[j / 8] >> (j % 8)) & 1u) return 0;
  return 1;
}

static size_t popcount_bits(const uint8_t* bm, size_t nbits) {
  size_t c = 0;
  for (size_t j = 0; j < nbits; j++) c += (bm[j / 8] >> (j % 8)) & 1u;
  return c;
}

/* Inverse of repeat elimination: byte j is the next kept byte where the bitmap bit
 * is set, else byte j-1. */
static int repeat_restore(const uint8_t* bm, size_t len, const uint8_t* kept, size_t nk, uint8_t* a) {
  size_t c = 0;
  uint8_t prev = 0;
  for (size_t j = 0; j < len; j++) {
    if ((bm[j / 8] >> (j % 8)) & 1u) {
      if (c >= nk) return ORC_CORRUPT;
      prev = kept[c++];
    }
    a[j] = prev;
  }
  return c == nk ? ORC_OK : ORC_CORRUPT;
}

int orc_unrze(int g, const uint8_t* in, size_t in_len, size_t L, uint8_t* out) {
  size_t U = L / (size_t)g;
  size_t l0 = (U + 7) / 8, l1 = (l0 + 7) / 8, l2 = (l1 + 7) / 8;
  int rc = ORC_CORRUPT;
  uint8_t* m0 = (uint8_t*)calloc(l0 + 1, 1);
  uint8_t* m1 = (uint8_t*)calloc(l1 + 1, 1);
  size_t o = 0;
  if (in_len < l2) goto done;
  const uint8_t* m2 = in;
  o = l2;
  if (!tail_bits_zero(m2, l1)) goto done;
  size_t nk1 = popcount_bits(m2, l1);
  if (o + nk1 > in_len) goto done;
  if (repeat_restore(m2, l1, in + o, nk1, m1) != ORC_OK) goto done;
  o += nk1;
  if (!tail_bits_zero(m1, l0)) goto done;
  size_t nk0 = popcount_bits(m1, l0);
  if (o + nk0 > in_len) goto done;
  if (repeat_restore(m1, l0, in + o, nk0, m0) != ORC_OK) goto done;
  o += nk0;
  if (!tail_bits_zero(m0, U)) goto done;
  size_t np = popcount_bits(m0, U);
  if (o + np * (size_t)g != in_len) goto done;
  {
    size_t c = 0;
    for (size_t j = 0; j < U; j++) {
      if ((m0[j / 8] >> (j % 8)) & 1u) {
        memcpy(out + j * g, in + o + c * g, (size_t)g);
        c++;
      } else {
        memset(out + j * g, 0, (size_t)g);
      }
    }
  }
  rc = ORC_OK;
done:
  free(m0);
  free(m1);
  return rc;
}

/* ---------------------------------------------------------------- chunks */

#define RAW_FLAG 0x80000000u
#define DIFF_FLAG 0x40000000u /* format 2: this bin record uses the 1D difference */
#define SIZE_MASK 0x3FFFFFFFu
#define NB_MASK 0xAAAAAAAAAAAAAAAAull

static int popcount64(uint64_t v) {
  int c = 0;
  for (; v; v &= v - 1) c++;
  return c;
}

/* The 3D Lorenzo residual of a chunk's bins (cz x cy x cx points, row-major; a 2D
 * chunk has cz = 1): r[z][y][x] = sum over (a, b, c) in {0,1}^3 of
 * (-1)^(a+b+c) bins[z-a][y-b][x-c], bins outside the chunk taken as 0, in w-byte
 * wrapping arithmetic.  Written as NB-mapped words, (r + M) xor M. */
static void lorenzo_nb(int w, const int64_t* b, const int64_t d[3], uint8_t* out) {
  for (int64_t z = 0; z < d[0]; z++)
    for (int64_t y = 0; y < d[1]; y++)
      for (int64_t x = 0; x < d[2]; x++) {
        uint64_t acc = 0;
        for (int a = 0; a < 2; a++)
          for (int bb = 0; bb < 2; bb++)
            for (int c = 0; c < 2; c++) {
              int64_t zz = z - a, yy = y - bb, xx = x - c;
              if (zz < 0 || yy < 0 || xx < 0) continue;
              uint64_t v = (uint64_t)b[(zz * d[1] + yy) * d[2] + xx];
              acc = ((a + bb + c) & 1) ? acc - v : acc + v;
            }
        uint64_t u = ((acc + NB_MASK) ^ NB_MASK) & wmask(w);
        put_word(out + ((z * d[1] + y) * d[2] + x) * w, w, u);
      }
}

/* Inverse of lorenzo_nb: unmap, then inclusive prefix sums along x, y and z. */
static void unlorenzo_nb(int w, const uint8_t* in, const int64_t d[3], int64_t* b) {
  int64_t n = d[0] * d[1] * d[2];
  uint64_t* r = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(n ? n : 1));
  for (int64_t i = 0; i < n; i++) r[i] = ((get_word(in + i * w, w) ^ NB_MASK) - NB_MASK) & wmask(w);
  for (int64_t z = 0; z < d[0]; z++)
    for (int64_t y = 0; y < d[1]; y++)
      for (int64_t x = 1; x < d[2]; x++) {
        int64_t i = (z * d[1] + y) * d[2] + x;
        r[i] = (r[i] + r[i - 1]) & wmask(w);
      }
  for (int64_t z = 0; z < d[0]; z++)
    for (int64_t y = 1; y < d[1]; y++)
      for (int64_t x = 0; x < d[2]; x++) {
        int64_t i = (z * d[1] + y) * d[2] + x;
        r[i] = (r[i] + r[i - d[2]]) & wmask(w);
      }
  for (int64_t z = 1; z < d[0]; z++)
    for (int64_t y = 0; y < d[1]; y++)
      for (int64_t x = 0; x < d[2]; x++) {
        int64_t i = (z * d[1] + y) * d[2] + x;
        r[i] = (r[i] + r[i - d[1] * d[2]]) & wmask(w);
      }
  for (int64_t i = 0; i < n; i++) b[i] = w == 4 ? (int64_t)(int32_t)(uint32_t)r[i] : (int64_t)r[i];
  free(r);
}

/* Bins (Sec. III-C; format 2): a predictor's residual, NB-mapped, then BIT_w and
 * RZE_1.  The predictor is the chunk's Lorenzo residual, or the 1D difference along
 * the chunk's point order (DIFFNB_w, the only one of format 1) when its mapped words
 * hold strictly fewer one bits.  Stored raw when the encoding is not smaller. */
static uint32_t enc_bins(int w, const int64_t* b, const int64_t d[3], uint8_t* rec) {
  int64_t n = d[0] * d[1] * d[2];
  int64_t n32 = (n + 31) / 32 * 32;
  uint8_t* tl = (uint8_t*)calloc((size_t)n32 * w, 1);
  uint8_t* td = (uint8_t*)calloc((size_t)n32 * w, 1);
  uint8_t* t2 = (uint8_t*)malloc((size_t)n32 * w);
  uint8_t* t3 = (uint8_t*)malloc((size_t)n32 * w * 2 + 64);
  lorenzo_nb(w, b, d, tl);
  orc_diffnb(w, b, n, td);
  int64_t cost_l = 0, cost_d = 0;
  for (int64_t i = 0; i < n; i++) {
    cost_l += popcount64(get_word(tl + i * w, w));
    cost_d += popcount64(get_word(td + i * w, w));
  }
  int use_diff = cost_d < cost_l;
  size_t L = orc_bit(w, use_diff ? td : tl, n, t2);
  size_t R = orc_rze(1, t2, L, t3);
  uint32_t sz;
  if (R >= (size_t)n * w) {
    for (int64_t i = 0; i < n; i++) put_word(rec + i * w, w, (uint64_t)b[i] & wmask(w));
    sz = (uint32_t)(n * w) | RAW_FLAG;
  } else {
    memcpy(rec, t3, R);
    sz = (uint32_t)R | (use_diff ? DIFF_FLAG : 0u);
  }
  free(tl);
  free(td);
  free(t2);
  free(t3);
  return sz;
}

/* Subbins (Sec. III-C, LC-generated): BIT_w, RZE_w, RZE_1; the record starts with
 * the u32 length of the RZE_w output. */
static uint32_t enc_subbins(int w, const uint64_t* s, int64_t n, uint8_t* rec) {
  int64_t n32 = (n + 31) / 32 * 32;
  uint8_t* t0 = (uint8_t*)calloc((size_t)n32 * w, 1);
  uint8_t* t1 = (uint8_t*)malloc((size_t)n32 * w);
  uint8_t* t2 = (uint8_t*)malloc((size_t)n32 * w * 2 + 64);
  uint8_t* t3 = (uint8_t*)malloc((size_t)n32 * w * 3 + 64);
  for (int64_t i = 0; i < n; i++) put_word(t0 + i * w, w, s[i] & wmask(w));
  size_t L = orc_bit(w, t0, n, t1);
  size_t L2 = orc_rze(w, t1, L, t2);
  size_t R = orc_rze(1, t2, L2, t3);
  uint32_t sz;
  if (4 + R >= (size_t)n * w) {
    memcpy(rec, t0, (size_t)n * w);
    sz = (uint32_t)(n * w) | RAW_FLAG;
  } else {
    put_word(rec, 4, (uint64_t)L2);
    memcpy(rec + 4, t3, R);
    sz = (uint32_t)(4 + R);
  }
  free(t0);
  free(t1);
  free(t2);
  free(t3);
  return sz;
}

static int dec_bins(int w, int version, const uint8_t* rec, uint32_t sz, const int64_t d[3], int64_t* b) {
  int64_t n = d[0] * d[1] * d[2];
  int64_t n32 = (n + 31) / 32 * 32;
  uint32_t len = sz & SIZE_MASK;
  if ((sz & DIFF_FLAG) && (version == 1 || (sz & RAW_FLAG))) return ORC_CORRUPT;
  int use_diff = version == 1 || (sz & DIFF_FLAG);
  if (sz & RAW_FLAG) {
    if (len != (uint32_t)(n * w)) return ORC_CORRUPT;
    for (int64_t i = 0; i < n; i++) {
      uint64_t u = get_word(rec + i * w, w);
      b[i] = w == 4 ? (int64_t)(int32_t)(uint32_t)u : (int64_t)u;
    }
    return ORC_OK;
  }
  size_t L = (size_t)n32 * w;
  uint8_t* t2 = (uint8_t*)malloc(L);
  uint8_t* t1 = (uint8_t*)malloc(L);
  int rc = orc_unrze(1, rec, len, L, t2);
  if (rc == ORC_OK) {
    orc_unbit(w, t2, n32, t1);
    for (int64_t i = n * w; i < n32 * w; i++)
      if (t1[i]) rc = ORC_CORRUPT;
    if (rc == ORC_OK) {
      if (use_diff)
        orc_undiffnb(w, t1, n, b);
      else
        unlorenzo_nb(w, t1, d, b);
    }
  }
  free(t1);
  free(t2);
  return rc;
}

static int dec_subbins(int w, const uint8_t* rec, uint32_t sz, int64_t n, uint64_t* s) {
  int64_t n32 = (n + 31) / 32 * 32;
  if (sz & DIFF_FLAG) return ORC_CORRUPT;
  uint32_t len = sz & SIZE_MASK;
  if (sz & RAW_FLAG) {
    if (len != (uint32_t)(n * w)) return ORC_CORRUPT;
    for (int64_t i = 0; i < n; i++) s[i] = get_word(rec + i * w, w);
    return ORC_OK;
  }
  if (len < 4) return ORC_CORRUPT;
  size_t L = (size_t)n32 * w;
  size_t L2 = (size_t)get_word(rec, 4);
  if (L2 > 2 * L + 64) return ORC_CORRUPT;
  uint8_t* t2 = (uint8_t*)malloc(L2 + 1);
  uint8_t* t1 = (uint8_t*)malloc(L);
  uint8_t* t0 = (uint8_t*)malloc(L);
  int rc = orc_unrze(1, rec + 4, len - 4, L2, t2);
  if (rc == ORC_OK) rc = orc_unrze(w, t2, L2, L, t1);
  if (rc == ORC_OK) {
    orc_unbit(w, t1, n32, t0);
    for (int64_t i = n * w; i < n32 * w; i++)
      if (t0[i]) rc = ORC_CORRUPT;
    if (rc == ORC_OK)
      for (int64_t i = 0; i < n; i++) s[i] = get_word(t0 + i * w, w);
  }
  free(t0);
  free(t1);
  free(t2);
  return rc;
}

void orc_encode_chunk(int dtype, const int64_t* b, const uint64_t* s, const int64_t dims[3], uint8_t* bin_rec,
                      uint32_t* bin_size, uint8_t* sub_rec, uint32_t* sub_size) {
  int w = dtype == 0 ? 4 : 8;
  *bin_size = enc_bins(w, b, dims, bin_rec);
  *sub_size = enc_subbins(w, s, dims[0] * dims[1] * dims[2], sub_rec);
}

/* ---------------------------------------------------------------- stream */

#define HDR 128
#define MAGIC 0x43504F4Cu /* "LOPC" */
#define VERSION 2 /* format 1 (bin records DIFFNB only) is still read */

static size_t pad16(size_t v) { return (v + 15) & ~(size_t)15; }

/* Chunk geometry: 16 KiB of words per chunk (4096 float32 or 2048 float64 points),
 * as a fixed tile: 2D 64x64 / 32x64, 3D 16x16x16 / 8x16x16. */
static void tile_of(int dtype, int ndim, int64_t t[3]) {
  if (ndim == 2) {
    t[0] = 1;
    t[1] = dtype == 0 ? 64 : 32;
    t[2] = 64;
  } else {
    t[0] = dtype == 0 ? 16 : 8;
    t[1] = 16;
    t[2] = 16;
  }
}

typedef struct {
  grid3 g;
  int64_t t[3];
  int64_t nt[3];
  int64_t ntiles;
} tiling;

static tiling tiling_of(const orc_desc* d) {
  tiling T;
  T.g = grid_of(d);
  tile_of(d->dtype, d->ndim, T.t);
  int64_t n[3] = {T.g.nz, T.g.ny, T.g.nx};
  T.ntiles = 1;
  for (int k = 0; k < 3; k++) {
    T.nt[k] = (n[k] + T.t[k] - 1) / T.t[k];
    T.ntiles *= T.nt[k];
  }
  return T;
}

/* Linear indices of the points of tile `tid`, row-major inside the (clipped) tile. */
/* Flat indices of chunk tid's points in chunk order; dims receives its clipped shape. */
static int64_t tile_points(const tiling* T, int64_t tid, int64_t* idx, int64_t dims[3]) {
  int64_t tx = tid % T->nt[2], ty = (tid / T->nt[2]) % T->nt[1], tz = tid / (T->nt[2] * T->nt[1]);
  int64_t z0 = tz * T->t[0], y0 = ty * T->t[1], x0 = tx * T->t[2];
  int64_t z1 = z0 + T->t[0] < T->g.nz ? z0 + T->t[0] : T->g.nz;
  int64_t y1 = y0 + T->t[1] < T->g.ny ? y0 + T->t[1] : T->g.ny;
  int64_t x1 = x0 + T->t[2] < T->g.nx ? x0 + T->t[2] : T->g.nx;
  int64_t c = 0;
  for (int64_t z = z0; z < z1; z++)
    for (int64_t y = y0; y < y1; y++)
      for (int64_t x = x0; x < x1; x++) idx[c++] = (z * T->g.ny + y) * T->g.nx + x;
  dims[0] = z1 - z0;
  dims[1] = y1 - y0;
  dims[2] = x1 - x0;
  return c;
}

size_t orc_compress_bound(const orc_desc* d) {
  if (!desc_ok(d)) return 0;
  tiling T = tiling_of(d);
  int w = d->dtype == 0 ? 4 : 8;
  return HDR + pad16((size_t)T.ntiles * 8) + 2 * ((size_t)npoints(d) * w + 16 * (size_t)T.ntiles);
}

static void put_u16(uint8_t* p, uint16_t v) { put_word(p, 2, v); }
static void put_u32(uint8_t* p, uint32_t v) { put_word(p, 4, v); }
static void put_u64(uint8_t* p, uint64_t v) { put_word(p, 8, v); }
static void put_f64(uint8_t* p, double v) {
  uint64_t u;
  memcpy(&u, &v, 8);
  put_u64(p, u);
}
static double get_f64(const uint8_t* p) {
  uint64_t u = get_word(p, 8);
  double v;
  memcpy(&v, &u, 8);
  return v;
}

static void write_header(uint8_t* h, const orc_desc* d, const tiling* T, int constant, double eps, double inv,
                         double cval, uint64_t total) {
  memset(h, 0, HDR);
  put_u32(h + 0, MAGIC);
  put_u16(h + 4, VERSION);
  h[6] = (uint8_t)d->dtype;
  h[7] = (uint8_t)d->ndim;
  for (int k = 0; k < 3; k++) put_u64(h + 8 + 8 * k, (uint64_t)(k < d->ndim ? d->dims[k] : 0));
  h[32] = (uint8_t)d->mode;
  h[33] = (uint8_t)constant;
  for (int k = 0; k < 3; k++) put_u32(h + 36 + 4 * k, (uint32_t)T->t[k]);
  put_f64(h + 48, d->eb);
  put_f64(h + 56, eps);
  put_f64(h + 64, inv);
  if (d->dtype == 0) {
    float f = (float)cval;
    uint32_t u;
    memcpy(&u, &f, 4);
    put_u64(h + 72, u);
  } else {
    put_f64(h + 72, cval);
  }
  put_u64(h + 80, constant ? 0 : (uint64_t)T->ntiles);
  put_u64(h + 88, total);
}

int orc_compress(const orc_desc* d, const void* x, uint8_t* out, size_t cap, size_t* out_size) {
  if (!desc_ok(d)) return ORC_INVALID_ARG;
  double eps, eps_q, inv, cval;
  int constant;
  int rc = orc_resolve_eps(d, x, &eps, &eps_q, &inv, &constant, &cval);
  if (rc != ORC_OK) return rc;
  tiling T = tiling_of(d);
  int w = d->dtype == 0 ? 4 : 8;
  int64_t n = npoints(d);
  if (constant) {
    if (cap < HDR) return ORC_CAPACITY;
    write_header(out, d, &T, 1, 0.0, 0.0, cval, HDR);
    *out_size = HDR;
    return ORC_OK;
  }
  int64_t* b = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  uint64_t* s = (uint64_t*)calloc((size_t)n, sizeof(uint64_t));
  rc = orc_quantize(d->dtype, x, n, inv, b);
  if (rc == ORC_OK) rc = orc_repair_lfp(d, x, b, s);
  if (rc != ORC_OK) {
    free(b);
    free(s);
    return rc;
  }
  int64_t cmax = T.t[0] * T.t[1] * T.t[2];
  uint32_t* sizes = (uint32_t*)malloc(sizeof(uint32_t) * 2 * (size_t)T.ntiles);
  uint8_t** recs = (uint8_t**)malloc(sizeof(uint8_t*) * 2 * (size_t)T.ntiles);
  /* chunks are coded independently (Sec. II-C): the OpenMP build splits this loop */
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t c = 0; c < T.ntiles; c++) {
    int64_t* idx = (int64_t*)malloc(sizeof(int64_t) * (size_t)cmax);
    int64_t* tb = (int64_t*)malloc(sizeof(int64_t) * (size_t)cmax);
    uint64_t* ts = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)cmax);
    int64_t dims[3];
    int64_t m = tile_points(&T, c, idx, dims);
    for (int64_t i = 0; i < m; i++) {
      tb[i] = b[idx[i]];
      ts[i] = s[idx[i]];
    }
    recs[c] = (uint8_t*)malloc((size_t)m * w + 64);
    recs[T.ntiles + c] = (uint8_t*)malloc((size_t)m * w + 64);
    sizes[c] = enc_bins(w, tb, dims, recs[c]);
    sizes[T.ntiles + c] = enc_subbins(w, ts, m, recs[T.ntiles + c]);
    free(idx);
    free(tb);
    free(ts);
  }
  size_t table = pad16((size_t)T.ntiles * 8);
  size_t total = HDR + table;
  for (int64_t c = 0; c < 2 * T.ntiles; c++) total += pad16(sizes[c] & SIZE_MASK);
  if (total > cap) {
    rc = ORC_CAPACITY;
  } else {
    memset(out, 0, total);
    write_header(out, d, &T, 0, eps, inv, 0.0, total);
    for (int64_t c = 0; c < 2 * T.ntiles; c++) put_u32(out + HDR + 4 * c, sizes[c]);
    size_t o = HDR + table;
    for (int64_t c = 0; c < 2 * T.ntiles; c++) {
      uint32_t len = sizes[c] & SIZE_MASK;
      memcpy(out + o, recs[c], len);
      o += pad16(len);
    }
    *out_size = total;
  }
  for (int64_t c = 0; c < 2 * T.ntiles; c++) free(recs[c]);
  free(recs);
  free(sizes);
  free(b);
  free(s);
  return rc;
}

typedef struct {
  orc_desc d;
  int version;
  int constant;
  double eps, inv, cval;
  uint64_t nchunks, total;
} hdr_t;

static int parse_header(const uint8_t* in, size_t n, hdr_t* H) {
  if (!in || n < HDR) return ORC_CORRUPT;
  uint64_t version = get_word(in + 4, 2);
  if (get_word(in, 4) != MAGIC || version < 1 || version > VERSION) return ORC_CORRUPT;
  memset(H, 0, sizeof(*H));
  H->version = (int)version;
  H->d.dtype = in[6];
  H->d.ndim = in[7];
  if (H->d.dtype > 1 || (H->d.ndim != 2 && H->d.ndim != 3)) return ORC_CORRUPT;
  for (int k = 0; k < 3; k++) {
    int64_t v = (int64_t)get_word(in + 8 + 8 * k, 8);
    if (k < H->d.ndim ? (v <= 0 || v > ((int64_t)1 << 40)) : v != 0) return ORC_CORRUPT;
    H->d.dims[k] = v;
  }
  H->d.mode = in[32];
  H->constant = in[33];
  if (H->d.mode > 1 || H->constant > 1) return ORC_CORRUPT;
  int64_t t[3];
  tile_of(H->d.dtype, H->d.ndim, t);
  for (int k = 0; k < 3; k++)
    if ((int64_t)get_word(in + 36 + 4 * k, 4) != t[k]) return ORC_CORRUPT;
  H->d.eb = get_f64(in + 48);
  H->eps = get_f64(in + 56);
  H->inv = get_f64(in + 64);
  if (H->d.dtype == 0) {
    uint32_t u = (uint32_t)get_word(in + 72, 8);
    float f;
    memcpy(&f, &u, 4);
    H->cval = f;
  } else {
    H->cval = get_f64(in + 72);
  }
  H->nchunks = get_word(in + 80, 8);
  H->total = get_word(in + 88, 8);
  if (H->total > n || H->total < HDR) return ORC_CORRUPT;
  tiling T = tiling_of(&H->d);
  if (H->constant ? H->nchunks != 0 : H->nchunks != (uint64_t)T.ntiles) return ORC_CORRUPT;
  if (!H->constant && (!(H->inv > 0.0) || !isfinite(H->inv))) return ORC_CORRUPT;
  return ORC_OK;
}

int orc_peek(const uint8_t* in, size_t n, orc_desc* d) {
  hdr_t H;
  int rc = parse_header(in, n, &H);
  if (rc == ORC_OK) *d = H.d;
  return rc;
}

int orc_decompress(const uint8_t* in, size_t n, void* xhat, size_t cap_bytes) {
  hdr_t H;
  int rc = parse_header(in, n, &H);
  if (rc != ORC_OK) return rc;
  int w = H.d.dtype == 0 ? 4 : 8;
  int64_t np = npoints(&H.d);
  if (cap_bytes < (size_t)np * w) return ORC_CAPACITY;
  if (H.constant) {
    if (H.total != HDR) return ORC_CORRUPT;
    for (int64_t i = 0; i < np; i++) {
      if (H.d.dtype == 0)
        ((float*)xhat)[i] = (float)H.cval;
      else
        ((double*)xhat)[i] = H.cval;
    }
    return ORC_OK;
  }
  tiling T = tiling_of(&H.d);
  size_t table = pad16((size_t)T.ntiles * 8);
  if (HDR + table > H.total) return ORC_CORRUPT;
  const uint8_t* tab = in + HDR;
  size_t* off = (size_t*)malloc(sizeof(size_t) * 2 * (size_t)T.ntiles);
  size_t o = HDR + table;
  for (int64_t c = 0; c < 2 * T.ntiles; c++) {
    off[c] = o;
    o += pad16((uint32_t)get_word(tab + 4 * c, 4) & SIZE_MASK);
  }
  if (o != H.total) {
    free(off);
    return ORC_CORRUPT;
  }
  int64_t cmax = T.t[0] * T.t[1] * T.t[2];
  int bad = 0; /* every decoder error is a corrupt stream */
  /* chunks decode independently (Sec. III-E): the OpenMP build splits this loop */
#pragma omp parallel for schedule(dynamic, 16) reduction(| : bad)
  for (int64_t c = 0; c < T.ntiles; c++) {
    int64_t* idx = (int64_t*)malloc(sizeof(int64_t) * (size_t)cmax);
    int64_t* tb = (int64_t*)malloc(sizeof(int64_t) * (size_t)cmax);
    uint64_t* ts = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)cmax);
    int64_t dims[3];
    int64_t m = tile_points(&T, c, idx, dims);
    uint32_t sb = (uint32_t)get_word(tab + 4 * c, 4), ss = (uint32_t)get_word(tab + 4 * (T.ntiles + c), 4);
    int crc = dec_bins(w, H.version, in + off[c], sb, dims, tb);
    if (crc == ORC_OK) crc = dec_subbins(w, in + off[T.ntiles + c], ss, m, ts);
    for (int64_t i = 0; i < m && crc == ORC_OK; i++) {
      double lo;
      if (orc_lowest_in_bin(H.d.dtype, tb[i], H.inv, &lo) != ORC_OK) {
        crc = ORC_CORRUPT;
        break;
      }
      double v = orc_succ_k(H.d.dtype, lo, ts[i]);
      if (!isfinite(v)) {
        crc = ORC_CORRUPT;
        break;
      }
      if (H.d.dtype == 0)
        ((float*)xhat)[idx[i]] = (float)v;
      else
        ((double*)xhat)[idx[i]] = v;
    }
    if (crc != ORC_OK) bad = 1;
    free(idx);
    free(tb);
    free(ts);
  }
  free(off);
  return bad ? ORC_CORRUPT : ORC_OK;
}

/* ---------------------------------------------------------------- checkers */

int64_t orc_order_violations(const orc_desc* d, const void* x, const void* y) {
  grid3 g = grid_of(d);
  int64_t n = g.nx * g.ny * g.nz, bad = 0;
  for (int64_t p = 0; p < n; p++)
    for (int k = 7; k < 14; k++) {
      int64_t q = neighbour(g, p, k);
      if (q < 0) continue;
      if (precedes(d->dtype, x, q, p) != precedes(d->dtype, y, q, p)) bad++;
    }
  return bad;
}

/* Two link vertices are adjacent when their offsets differ by a neighbour offset
 * (the triangulation is a flag complex). */
static int offsets_adjacent(int ka, int kb) {
  int a[3], b[3];
  dir_offset(ka, &a[0], &a[1], &a[2]);
  dir_offset(kb, &b[0], &b[1], &b[2]);
  int dz = b[0] - a[0], dy = b[1] - a[1], dx = b[2] - a[2];
  if (dz == 0 && dy == 0 && dx == 0) return 0;
  int allpos = (dz == 0 || dz == 1) && (dy == 0 || dy == 1) && (dx == 0 || dx == 1);
  int allneg = (dz == 0 || dz == -1) && (dy == 0 || dy == -1) && (dx == 0 || dx == -1);
  return allpos || allneg;
}

static int uf_find(int* par, int i) {
  while (par[i] != i) i = par[i];
  return i;
}

static uint8_t count_components(const int* ks, int m) {
  int par[14];
  for (int i = 0; i < m; i++) par[i] = i;
  for (int i = 0; i < m; i++)
    for (int j = i + 1; j < m; j++)
      if (offsets_adjacent(ks[i], ks[j])) {
        int a = uf_find(par, i), b = uf_find(par, j);
        if (a != b) par[a] = b;
      }
  int c = 0;
  for (int i = 0; i < m; i++) c += uf_find(par, i) == i;
  return (uint8_t)c;
}

/* Sec. II: lower link = neighbours below v, upper link = neighbours above v (SoS
 * order); minimum if the lower link is empty, maximum if the upper link is empty,
 * regular if each is one connected piece, saddle otherwise. */
void orc_critical_types(const orc_desc* d, const void* x, uint8_t* lower_cc, uint8_t* upper_cc) {
  grid3 g = grid_of(d);
  int64_t n = g.nx * g.ny * g.nz;
  for (int64_t p = 0; p < n; p++) {
    int lo[14], up[14], nl = 0, nu = 0;
    for (int k = 0; k < 14; k++) {
      int64_t q = neighbour(g, p, k);
      if (q < 0) continue;
      if (precedes(d->dtype, x, q, p))
        lo[nl++] = k;
      else
        up[nu++] = k;
    }
    lower_cc[p] = count_components(lo, nl);
    upper_cc[p] = count_components(up, nu);
  }
}
