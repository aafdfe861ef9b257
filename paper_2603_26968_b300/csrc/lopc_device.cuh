// lopc_device.cuh -- device building blocks of the LOPC hot path on sm_103a:
// value keys, the exact quantizer, tile geometry, block scans and the lossless
// stages (DIFFNB, BIT, RZE) as block-cooperative routines on shared memory.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "lopc.h"

namespace lopc {

// ------------------------------------------------------------------ constants

constexpr int kHeaderBytes = 128;
constexpr uint32_t kMagic = 0x43504F4Cu;  // "LOPC"
constexpr uint32_t kRawFlag = 0x80000000u;   // size-table entry: the record is stored raw
constexpr uint32_t kDiffFlag = 0x40000000u;  // bin record of format 2 coded with the 1D difference
constexpr uint32_t kSizeMask = 0x3FFFFFFFu;  // the record length

// Status bits collected on the device and mapped to a return code on the host.
enum : uint32_t {
  kErrNonfinite = 1u,
  kErrRange = 2u,
  kErrCorrupt = 4u,
  kErrNotConverged = 8u,
  kErrInternal = 16u,
};

// Per-call state that lives at the start of the workspace.
struct Params {
  unsigned long long kmin, kmax;  // biased order keys (key + 2^63) of the extremes
  double eb;
  double eps, eps_q, inv;         // eps_q = eps (1 - 2^-16), inv = 1 / eps_q
  unsigned long long inv_m;       // inv = inv_m * 2^inv_e, inv_m < 2^53
  int inv_e;
  int mode;
  int constant;                   // NOA with a zero range
  unsigned int status;            // kErr* bits
  unsigned long long const_bits;  // the constant's bits (float32: low 32 bits)
  int fast_ok;                    // inv_f is a normal float: the fast quantizer path may run
  float inv_f;                    // inv rounded to float
  unsigned int pass_ordered;       // the tile pass takes the tiles in ascending tile key (k_order decides)
  unsigned long long total;       // stream bytes
  unsigned long long rounds;
  unsigned long long fix_iters;   // sum over tile runs of fixpoint sweeps
  unsigned long long fix_iters_max;
  unsigned long long phase[9];    // SM cycles spent per kernel phase (block-summed, for measurement)
  unsigned long long work[6];     // fixpoint evaluations and raises: tile pass, reruns; rerun tiles run, of them idle
};

// Adds a and b, summed over the block, to dst[0] and dst[1] (all threads call it).
__device__ __forceinline__ void block_add2(unsigned long long a, unsigned long long b, unsigned long long* dst) {
  __shared__ unsigned long long acc[2];
  if (threadIdx.x == 0) acc[0] = acc[1] = 0;
  __syncthreads();
  a = __reduce_add_sync(0xffffffffu, (unsigned)a);
  b = __reduce_add_sync(0xffffffffu, (unsigned)b);
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&acc[0], a);
    atomicAdd(&acc[1], b);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    atomicAdd(&dst[0], acc[0]);
    atomicAdd(&dst[1], acc[1]);
  }
}

// Adds the cycles since `t0` to phase counter `k` (thread 0 of the block only).
__device__ __forceinline__ void phase_mark(Params* P, int k, long long& t0) {
  if (threadIdx.x == 0) {
    const long long t = clock64();
    atomicAdd(&P->phase[k], (unsigned long long)(t - t0));
    t0 = t;
  }
}

// ------------------------------------------------------------------- traits

template <typename T>
struct Traits;

template <>
struct Traits<float> {
  using Key = int32_t;
  using Bits = uint32_t;
  using Bin = int32_t;
  static constexpr int W = 4;
  static constexpr int64_t kBinLimit = int64_t(1) << 30;
  static constexpr Key kMaxKey = 0x7f7fffff;
  static constexpr Bin kAbsent = INT32_MIN;
  static constexpr float kMaxFinite = 3.40282347e+38f;
  __device__ static Bits bits(float v) { return __float_as_uint(v); }
  __device__ static float from_bits(Bits u) { return __uint_as_float(u); }
};

template <>
struct Traits<double> {
  using Key = int64_t;
  using Bits = uint64_t;
  using Bin = int64_t;
  static constexpr int W = 8;
  static constexpr int64_t kBinLimit = int64_t(1) << 52;
  static constexpr Key kMaxKey = 0x7fefffffffffffffLL;
  static constexpr Bin kAbsent = INT64_MIN;
  static constexpr double kMaxFinite = 1.7976931348623157e+308;
  __device__ static Bits bits(double v) { return (Bits)__double_as_longlong(v); }
  __device__ static double from_bits(Bits u) { return __longlong_as_double((long long)u); }
};

// Position of a value in the dtype's total order; -0 and +0 share position 0, so
// comparing keys compares values numerically (Sec. II, Simulation of Simplicity
// then breaks ties by index).
template <typename T>
__device__ __forceinline__ typename Traits<T>::Key order_key(T v) {
  using K = typename Traits<T>::Key;
  using B = typename Traits<T>::Bits;
  const B u = Traits<T>::bits(v);
  constexpr int sh = 8 * sizeof(B) - 1;
  const K m = (K)(u & ~(B(1) << sh));
  return (u >> sh) ? -m : m;
}

template <typename T>
__device__ __forceinline__ T value_of_key(typename Traits<T>::Key k) {
  using B = typename Traits<T>::Bits;
  constexpr int sh = 8 * sizeof(B) - 1;
  const B u = k >= 0 ? (B)k : ((B(1) << sh) | (B)(-k));
  return Traits<T>::from_bits(u);
}

template <typename T>
__device__ __forceinline__ bool is_finite_bits(T v) {
  using B = typename Traits<T>::Bits;
  const B u = Traits<T>::bits(v);
  if (sizeof(T) == 4) return ((uint32_t)u & 0x7f800000u) != 0x7f800000u;
  return ((uint64_t)u & 0x7ff0000000000000ULL) != 0x7ff0000000000000ULL;
}

// ------------------------------------------------------------------ quantizer

// Bin of a value (Sec. III-A: multiply by 1/eps and round to nearest): the exact
// product of the value's significand and inv's 53-bit significand (at most 106
// bits) rounded half to even, all in integer arithmetic.  Returns false when
// |x * inv| >= 2^62.
template <typename T>
__device__ __forceinline__ bool quantize_exact(T x, unsigned long long inv_m, int inv_e, long long& bin) {
  uint64_t m;
  int e;
  bool neg;
  if (sizeof(T) == 4) {
    const uint32_t u = __float_as_uint((float)x);
    neg = u >> 31;
    const int ex = (u >> 23) & 0xff;
    m = u & 0x7fffffu;
    if (ex) {
      m |= 0x800000u;
      e = ex - 150;
    } else {
      e = -149;
    }
  } else {
    const uint64_t u = (uint64_t)__double_as_longlong((double)x);
    neg = u >> 63;
    const int ex = (int)((u >> 52) & 0x7ff);
    m = u & 0xfffffffffffffULL;
    if (ex) {
      m |= 0x10000000000000ULL;
      e = ex - 1075;
    } else {
      e = -1074;
    }
  }
  if (m == 0) {
    bin = 0;
    return true;
  }
  const unsigned __int128 P = (unsigned __int128)m * (unsigned __int128)inv_m;
  const int sh = -(e + inv_e);  // x * inv = P * 2^-sh
  uint64_t q;
  if (sh <= 0) {
    const uint64_t hi = (uint64_t)(P >> 64), lo = (uint64_t)P;
    const int nbits = hi ? 128 - __clzll((long long)hi) : 64 - __clzll((long long)lo);
    if (nbits - sh > 62) return false;
    q = (uint64_t)(P << (-sh));
  } else if (sh >= 128) {
    q = 0;
  } else {
    unsigned __int128 qq = P >> sh;
    const unsigned __int128 r = P - (qq << sh);
    const unsigned __int128 half = (unsigned __int128)1 << (sh - 1);
    if (r > half || (r == half && ((uint64_t)qq & 1))) qq += 1;
    if ((uint64_t)(qq >> 62) != 0) return false;
    q = (uint64_t)qq;
  }
  bin = neg ? -(long long)q : (long long)q;
  return true;
}

// Bin of a value, fast path first: t = x * inv in binary32 carries a relative error
// below 2^-22.4 (x rounded to float when it is float64, inv rounded to float, one
// product rounding).  When t lies farther than |t| * 2^-20 from every half-integer
// the rounding of the exact product is the rounding of t; otherwise, and outside
// the ranges where that bound holds, the exact integer path decides.
template <typename T>
__device__ __forceinline__ bool quantize_fast(T x, float inv_f, int fast_ok, unsigned long long inv_m, int inv_e,
                                              long long& bin) {
  if (fast_ok) {
    float xf;
    bool in_range;
    if (sizeof(T) == 4) {
      xf = (float)x;
      in_range = true;
    } else {
      const double ax = fabs((double)x);
      in_range = ax == 0.0 || (ax >= 1.1754943508222875e-38 && ax < 1.7014118346046923e38);
      xf = __double2float_rn((double)x);
    }
    if (in_range) {
      const float t = __fmul_rn(xf, inv_f);
      const float at = fabsf(t);
      if (at < 2097152.0f) {  // 2^21: rint(t) and t - rint(t) are exact
        const float r = rintf(t);
        const float room = __fsub_rn(0.5f, fabsf(__fsub_rn(t, r)));
        if (room > __fmul_rn(at, 9.5367431640625e-07f)) {  // 2^-20
          bin = (long long)__float2int_rn(r);  // |r| < 2^21 and integral: exact in 32 bits
          return true;
        }
      }
    }
  }
  return quantize_exact<T>(x, inv_m, inv_e, bin);
}

// Significand and exponent of a finite value: |v| = m * 2^e.
template <typename T>
__device__ __forceinline__ void split_value(T v, uint64_t& m, int& e, bool& neg) {
  if (sizeof(T) == 4) {
    const uint32_t u = __float_as_uint((float)v);
    neg = u >> 31;
    const int ex = (u >> 23) & 0xff;
    m = u & 0x7fffffu;
    if (ex) {
      m |= 0x800000u;
      e = ex - 150;
    } else {
      e = -149;
    }
  } else {
    const uint64_t u = (uint64_t)__double_as_longlong((double)v);
    neg = u >> 63;
    const int ex = (int)((u >> 52) & 0x7ff);
    m = u & 0xfffffffffffffULL;
    if (ex) {
      m |= 0x10000000000000ULL;
      e = ex - 1075;
    } else {
      e = -1074;
    }
  }
}

// Sign of (P * 2^sh - C) for a 128-bit P = (ph, pl), any shift, and 0 < C < 2^63.
__device__ __forceinline__ int cmp_scaled(uint64_t ph, uint64_t pl, int sh, uint64_t C) {
  const int pbits = ph ? 128 - __clzll((long long)ph) : (pl ? 64 - __clzll((long long)pl) : 0);
  if (pbits == 0) return -1;
  if (sh >= 0) {
    if (pbits + sh > 63) return 1;
    const uint64_t a = pl << sh;
    return a > C ? 1 : (a < C ? -1 : 0);
  }
  const int r = -sh;
  const int cbits = 64 - __clzll((long long)C);
  if (cbits + r > 127) return -1;  // C * 2^r >= 2^127 > P
  const unsigned __int128 c = (unsigned __int128)C << r;
  const unsigned __int128 p = ((unsigned __int128)ph << 64) | pl;
  return p > c ? 1 : (p < c ? -1 : 0);
}

// q(v) >= b, exactly: with t = v * inv, q(v) = round-half-even(t) is >= b iff
// 2t > 2b - 1, or 2t == 2b - 1 and b is even.
template <typename T>
__device__ __forceinline__ bool bin_at_least(T v, long long b, unsigned long long inv_m, int inv_e) {
  uint64_t m;
  int e;
  bool neg;
  split_value<T>(v, m, e, neg);
  const long long c = 2 * b - 1;
  if (m == 0) return 0 >= b;
  const uint64_t pl = m * (uint64_t)inv_m, ph = __umul64hi(m, (uint64_t)inv_m);
  const int sh = e + inv_e + 1;  // |2t| = (m * inv_m) * 2^sh
  if (!neg) {
    if (c < 0) return true;
    const int r = cmp_scaled(ph, pl, sh, (uint64_t)c);
    return r > 0 || (r == 0 && (b & 1) == 0);
  }
  if (c > 0) return false;
  const int r = cmp_scaled(ph, pl, sh, (uint64_t)(-c));
  return r < 0 || (r == 0 && (b & 1) == 0);
}

// Lowest value of the dtype whose bin is b (Sec. III-E: subbin 0 decodes to the
// lowest representable value within the bin), as an order key.  For float64 the bin's
// lower boundary is the real t = (b - 1/2) / inv, and the division rounded up gives the
// smallest float64 at or above t, which is in bin b unless it equals t and b is odd (a
// tie goes to the even bin b - 1); then the next value is.  Otherwise (float32, where
// the float64 division costs more than the steps it saves, or an infinite boundary) a
// guess from (b - 1/2) eps_q, a few exact steps, and bisection over all keys if that
// fails.  Returns false if bin b holds no value.
template <typename T>
__device__ bool lowest_key_in_bin(long long b, double eps_q, unsigned long long inv_m, int inv_e,
                                  typename Traits<T>::Key& out) {
  using K = typename Traits<T>::Key;
  const K kmax = Traits<T>::kMaxKey;
  K k;
  if (sizeof(T) == 8) {
    const double t = __ddiv_ru((double)b - 0.5, scalbn((double)inv_m, inv_e));  // |b| < 2^52: b - 1/2 is exact
    const bool fin = is_finite_bits<double>(t);
    k = fin ? (K)order_key<double>(t) : kmax;
    if (fin) {
      bool here = bin_at_least<T>(value_of_key<T>(k), b, inv_m, inv_e);
      if (!here && k < kmax) here = bin_at_least<T>(value_of_key<T>(++k), b, inv_m, inv_e);
      if (here) {
        if (bin_at_least<T>(value_of_key<T>(k), b + 1, inv_m, inv_e)) return false;  // bin b is empty
        out = k;
        return true;
      }
    }
  }
  if (sizeof(T) == 4) {
    const float g = __fmul_rn(__fsub_rn((float)b, 0.5f), (float)eps_q);
    k = is_finite_bits<float>(g) ? (K)order_key<float>(g) : (g > 0.f ? kmax : -kmax);
  } else {
    const double g = __dmul_rn(__dsub_rn((double)b, 0.5), eps_q);
    k = is_finite_bits<double>(g) ? (K)order_key<double>(g) : (g > 0.0 ? kmax : -kmax);
  }
  bool ok = false;
  for (int step = 0; step < 8; ++step) {
    const bool here = bin_at_least<T>(value_of_key<T>(k), b, inv_m, inv_e);
    if (!here) {
      if (k >= kmax) break;
      ++k;
      continue;
    }
    if (k <= -kmax) {
      ok = true;
      break;
    }
    const bool below = bin_at_least<T>(value_of_key<T>(k - 1), b, inv_m, inv_e);
    if (!below) {
      ok = true;
      break;
    }
    --k;
  }
  if (!ok) {  // bisection: smallest key with q >= b
    K lo = -kmax, hi = kmax;
    if (!bin_at_least<T>(value_of_key<T>(hi), b, inv_m, inv_e)) return false;
    while (lo < hi) {
      const K mid = (K)((lo >> 1) + (hi >> 1) + (lo & hi & 1));  // floor((lo+hi)/2)
      if (bin_at_least<T>(value_of_key<T>(mid), b, inv_m, inv_e))
        hi = mid;
      else
        lo = mid + 1;
    }
    k = lo;
  }
  if (bin_at_least<T>(value_of_key<T>(k), b + 1, inv_m, inv_e)) return false;  // bin b is empty
  out = k;
  return true;
}

// ----------------------------------------------------------------- geometry

struct Geometry {
  int64_t nz, ny, nx;      // a 2D field has nz = 1
  int64_t ntz, nty, ntx;   // tiles per dimension
  int64_t ntiles;
  int tz, ty, tx;          // tile (chunk) shape
  int ndim, dtype;
};

__host__ __device__ inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

struct HeaderInfo {
  int32_t dtype, ndim, mode;
  int64_t dims[3];
  int32_t tile[3];
  double eb;
};

// One field of a launch.  Every kernel serves a table of fields whose tiles share
// one global index space (a single field is a batch of one); a field's tiles are
// [tile_base, tile_base + g.ntiles).
struct FieldInfo {
  Geometry g;
  HeaderInfo hdr;
  const void* x;          // input values
  uint8_t* out;           // stream
  uint64_t out_cap;
  Params* P;              // per-field state (in the workspace)
  uint32_t* s;            // subbins, one per point
  uint32_t* cm;           // per point: lower same-bin neighbours (bits 0-13), in-tile upper ones (16-29)
  uint8_t* slots;         // 2 x ntiles record slots of 16 KiB
  uint32_t* sizes;        // 2 x ntiles record sizes
  uint64_t* offs;         // 2 x ntiles record offsets
  int64_t* bins_out;      // optional export of the bins (may be null)
  uint64_t* size_out;     // device: this field's stream length (may be null)
  int* status_out;        // device: this field's LOPC status (may be null)
  uint32_t* dirty;        // tiles to rerun next round: one byte flag per rank (below), ceil(ntiles / 4) words
  uint32_t* tkey;         // per tile: the top 32 bits of the smallest order key of its sample points
  uint32_t* order;        // the tiles in ascending tkey (the order the pass and the reruns visit them in): rank -> tile
  uint32_t* rank;         // the inverse: tile -> rank
  int64_t tile_base;      // first tile in the table's tile index space
  int64_t word_base;      // first dirty word in the table's flat word space
  int64_t round_cap;
};

__host__ __device__ inline int64_t dirty_words(int64_t ntiles) { return (ntiles + 3) / 4; }

// Field class of a table entry: 0 = f32 2D, 1 = f32 3D, 2 = f64 2D, 3 = f64 3D.
__host__ __device__ inline int class_of_geometry(const Geometry& g) {
  return (g.dtype == LOPC_F64 ? 2 : 0) + (g.ndim == 3 ? 1 : 0);
}

// State shared by all fields of a launch.
struct BatchState {
  unsigned int count[4];      // tiles to rerun per class this round
  unsigned int off[4];        // their first position in the list
  unsigned int next[4];       // per class: the next listed item a rerun block takes
  unsigned int next_all[4];   // per class: the next tile of the all-tile round
  unsigned int app[4];        // per class: tiles reruns appended to the round in progress
  unsigned long long rounds;  // repair rounds done
  unsigned long long runs;    // tile runs launched (first round included)
  unsigned int cap_hit;
  unsigned int pad;
};

// Field of flat dirty word w among fields F[0 .. nf), sorted by word_base.
__device__ __forceinline__ int field_of_word(const FieldInfo* F, int nf, int64_t w) {
  int lo = 0, hi = nf - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (F[mid].word_base <= w)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// Field of global tile gt among fields F[f0 .. f0+nf), sorted by tile_base.
__device__ __forceinline__ int field_of_tile(const FieldInfo* F, int f0, int nf, int64_t gt) {
  int lo = f0, hi = f0 + nf - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (F[mid].tile_base <= gt)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// The chunk of a tile: its origin and clipped extent.
struct TileBox {
  int64_t z0, y0, x0;
  int cz, cy, cx;
  int n;
};

// (A field has fewer than 2^32 points, so tile indices and counts fit 32 bits and
// the divisions are 32-bit ones.)
__device__ __forceinline__ TileBox tile_box(const Geometry& g, int64_t tid) {
  TileBox t;
  const uint32_t i = (uint32_t)tid, ntx = (uint32_t)g.ntx, nty = (uint32_t)g.nty;
  const uint32_t row = i / ntx;
  const int64_t tx = i - row * ntx, tz = row / nty, ty = row - (uint32_t)tz * nty;
  t.z0 = tz * g.tz;
  t.y0 = ty * g.ty;
  t.x0 = tx * g.tx;
  t.cz = (int)min((int64_t)g.tz, g.nz - t.z0);
  t.cy = (int)min((int64_t)g.ty, g.ny - t.y0);
  t.cx = (int)min((int64_t)g.tx, g.nx - t.x0);
  t.n = t.cz * t.cy * t.cx;
  return t;
}

// ------------------------------------------------------------------ block scan

// Exclusive prefix sum over the block, in thread order; *total receives the sum.
// `tmp` holds one slot per warp plus one.
template <int NT, typename V>
__device__ __forceinline__ V block_exclusive_scan(V v, V* tmp, V* total) {
  constexpr int NW = NT / 32;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  V x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const V y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) tmp[wid] = x;
  __syncthreads();
  if (wid == 0) {
    V w = lane < NW ? tmp[lane] : V(0);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const V y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < NW) tmp[lane] = w;  // inclusive warp totals
    if (lane == NW - 1) tmp[NW] = w;
  }
  __syncthreads();
  const V base = wid ? tmp[wid - 1] : V(0);
  const V res = base + x - v;
  if (total) *total = tmp[NW];
  __syncthreads();
  return res;
}

// Stream offsets of m records placed back to back from `base`, each taking its size
// (kSizeMask bits of sizes[i]) padded to 16 bytes: offs[i] = base + the padded sizes
// before i.  The block walks the table in chunks of 8 NT sizes, eight consecutive ones
// per thread (coalesced), with one block scan per chunk and a running carry; the next
// chunk's sizes are loaded before this chunk's scan, so their latency overlaps it.
// Sums are 64-bit: a corrupt table's sizes cannot wrap around.  Returns base + the
// padded total (in every thread).
__host__ __device__ constexpr uint64_t pad16_u(uint64_t v) { return (v + 15) & ~(uint64_t)15; }

template <int NT>
__device__ __forceinline__ uint64_t record_offsets(const uint32_t* __restrict__ sizes, int64_t m, uint64_t base,
                                                   uint64_t* __restrict__ offs, uint64_t* tmp) {
  constexpr int PT = 8;
  uint64_t carry = base;
  uint32_t nx[PT];
  auto load = [&](int64_t c0) {
    const int64_t i0 = c0 + PT * (int64_t)threadIdx.x;
#pragma unroll
    for (int u = 0; u < PT; ++u) nx[u] = i0 + u < m ? (uint32_t)pad16_u(sizes[i0 + u] & kSizeMask) : 0u;
  };
  if (m > 0) load(0);
  for (int64_t c0 = 0; c0 < m; c0 += PT * NT) {
    uint64_t p[PT], sum = 0;
#pragma unroll
    for (int u = 0; u < PT; ++u) {
      p[u] = sum;
      sum += nx[u];
    }
    if (c0 + PT * NT < m) load(c0 + PT * NT);  // in flight during the scan
    uint64_t tot;
    const uint64_t ex = carry + block_exclusive_scan<NT, uint64_t>(sum, tmp, &tot);
    const int64_t i0 = c0 + PT * (int64_t)threadIdx.x;
#pragma unroll
    for (int u = 0; u < PT; ++u)
      if (i0 + u < m) offs[i0 + u] = ex + p[u];
    carry += tot;
  }
  return carry;
}

}  // namespace lopc
