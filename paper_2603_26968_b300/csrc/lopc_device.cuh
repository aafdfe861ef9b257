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
constexpr uint32_t kRawFlag = 0x80000000u;
constexpr int kSegment = 16;  // points a thread owns along x in a tile

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
  unsigned int dirty_count;
  unsigned int pad0;
  unsigned long long total;       // stream bytes
  unsigned long long rounds;
};

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

// q(v) >= b, comparing through the exact quantizer (overflow counts as +-inf).
template <typename T>
__device__ __forceinline__ bool bin_at_least(T v, long long b, unsigned long long inv_m, int inv_e) {
  long long q;
  if (!quantize_exact<T>(v, inv_m, inv_e, q)) return !(v < (T)0);
  return q >= b;
}

// Lowest value of the dtype whose bin is b (Sec. III-E: subbin 0 decodes to the
// lowest representable value within the bin), as an order key.  A guess from
// (b - 1/2) eps_q, a few exact steps, and bisection over all keys if that fails.
// Returns false if bin b holds no value.
template <typename T>
__device__ bool lowest_key_in_bin(long long b, double eps_q, unsigned long long inv_m, int inv_e,
                                  typename Traits<T>::Key& out) {
  using K = typename Traits<T>::Key;
  const K kmax = Traits<T>::kMaxKey;
  const double g = __dmul_rn(__dsub_rn((double)b, 0.5), eps_q);
  K k;
  if (!(g == g) || g > 1e300 || g < -1e300) {
    k = 0;
  } else {
    const T gv = (T)g;
    k = is_finite_bits<T>(gv) ? order_key<T>(gv) : (gv > (T)0 ? kmax : -kmax);
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
  long long q;
  if (!quantize_exact<T>(value_of_key<T>(k), inv_m, inv_e, q) || q != b) return false;
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

// The chunk of a tile: its origin and clipped extent.
struct TileBox {
  int64_t z0, y0, x0;
  int cz, cy, cx;
  int n;
};

__device__ __forceinline__ TileBox tile_box(const Geometry& g, int64_t tid) {
  TileBox t;
  const int64_t tx = tid % g.ntx, ty = (tid / g.ntx) % g.nty, tz = tid / (g.ntx * g.nty);
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

// ------------------------------------------------------------- BIT_w stage

// Bit-plane transpose of n32 words (a multiple of 32): plane k (k = 0 least
// significant) is n32/32 u32 words, bit j of word g being bit k of word 32g+j.
// `word(i)` supplies input word i (zero for padding).  One warp per group of 32.
template <int NT, int W, typename WordFn>
__device__ __forceinline__ void bit_transpose(int n32, WordFn word, uint32_t* planes) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int G = n32 >> 5;
  for (int g = wid; g < G; g += NT / 32) {
    const uint64_t v = word(32 * g + lane);
    uint32_t lo_plane = 0, hi_plane = 0;
#pragma unroll
    for (int k = 0; k < 32; ++k) {
      const uint32_t r = __ballot_sync(0xffffffffu, (uint32_t)(v >> k) & 1u);
      if (lane == k) lo_plane = r;
    }
    planes[lane * G + g] = lo_plane;
    if (W == 8) {
#pragma unroll
      for (int k = 0; k < 32; ++k) {
        const uint32_t r = __ballot_sync(0xffffffffu, (uint32_t)(v >> (32 + k)) & 1u);
        if (lane == k) hi_plane = r;
      }
      planes[(32 + lane) * G + g] = hi_plane;
    }
  }
}

// Inverse of bit_transpose: `emit(i, word)` receives word i of the n32.
template <int NT, int W, typename EmitFn>
__device__ __forceinline__ void bit_untranspose(int n32, const uint32_t* planes, EmitFn emit) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int G = n32 >> 5;
  for (int g = wid; g < G; g += NT / 32) {
    const uint32_t lo_plane = planes[lane * G + g];
    const uint32_t hi_plane = W == 8 ? planes[(32 + lane) * G + g] : 0u;
    uint32_t lo = 0, hi = 0;
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const uint32_t r = __ballot_sync(0xffffffffu, (lo_plane >> j) & 1u);
      if (lane == j) lo = r;
    }
    if (W == 8) {
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const uint32_t r = __ballot_sync(0xffffffffu, (hi_plane >> j) & 1u);
        if (lane == j) hi = r;
      }
    }
    emit(32 * g + lane, (uint64_t)lo | ((uint64_t)hi << 32));
  }
}

// ------------------------------------------------------------- RZE_g stage

struct RzeScratch {
  uint8_t* m0;   // level-0 bitmap (>= ceil(U/8) bytes)
  uint8_t* m1;   // level-1 bitmap
  uint8_t* m2;   // level-2 bitmap
  uint32_t* pre; // per-word prefix counts (>= ceil(l0/4) + 1 words)
  uint32_t* tmp; // scan scratch (NT/32 + 1)
};

__device__ __forceinline__ uint32_t bytes_ceil8(uint32_t n) { return (n + 7u) >> 3; }

// Encodes `in` (L bytes, shared memory) with RZE_g: [level-2 bitmap][level-1 kept]
// [level-0 kept][non-zero units].  If the encoding would not be shorter than
// `limit` bytes nothing is written.  Returns the encoded length.
template <int NT>
__device__ uint32_t rze_encode(const uint8_t* in, uint32_t L, int g, uint8_t* out, uint32_t limit,
                               const RzeScratch& sc) {
  const uint32_t U = L / (uint32_t)g;
  const uint32_t l0 = bytes_ceil8(U), l1 = bytes_ceil8(l0), l2 = bytes_ceil8(l1);
  const int t = threadIdx.x;
  // level 0: contiguous ranges of bitmap bytes per thread
  const uint32_t per0 = (l0 + NT - 1) / NT;
  const uint32_t a0 = min(l0, t * per0), b0 = min(l0, a0 + per0);
  uint32_t cnt = 0;
  for (uint32_t j = a0; j < b0; ++j) {
    uint32_t byte = 0;
    for (int bit = 0; bit < 8; ++bit) {
      const uint32_t u = 8 * j + bit;
      if (u >= U) break;
      uint32_t nz = 0;
      for (int k = 0; k < g; ++k) nz |= in[u * g + k];
      if (nz) {
        byte |= 1u << bit;
        ++cnt;
      }
    }
    sc.m0[j] = (uint8_t)byte;
  }
  uint32_t np;
  const uint32_t pay_off = block_exclusive_scan<NT, uint32_t>(cnt, sc.tmp, &np);
  // level 1: repeat elimination of m0
  const uint32_t per1 = (l1 + NT - 1) / NT;
  const uint32_t a1 = min(l1, t * per1), b1 = min(l1, a1 + per1);
  uint32_t c1 = 0;
  for (uint32_t jj = a1; jj < b1; ++jj) {
    uint32_t byte = 0;
    for (int bit = 0; bit < 8; ++bit) {
      const uint32_t j = 8 * jj + bit;
      if (j >= l0) break;
      const uint8_t prev = j ? sc.m0[j - 1] : 0;
      if (sc.m0[j] != prev) {
        byte |= 1u << bit;
        ++c1;
      }
    }
    sc.m1[jj] = (uint8_t)byte;
  }
  uint32_t nk0;
  const uint32_t k0_off = block_exclusive_scan<NT, uint32_t>(c1, sc.tmp, &nk0);
  // level 2: repeat elimination of m1
  const uint32_t per2 = (l2 + NT - 1) / NT;
  const uint32_t a2 = min(l2, t * per2), b2 = min(l2, a2 + per2);
  uint32_t c2 = 0;
  for (uint32_t jj = a2; jj < b2; ++jj) {
    uint32_t byte = 0;
    for (int bit = 0; bit < 8; ++bit) {
      const uint32_t j = 8 * jj + bit;
      if (j >= l1) break;
      const uint8_t prev = j ? sc.m1[j - 1] : 0;
      if (sc.m1[j] != prev) {
        byte |= 1u << bit;
        ++c2;
      }
    }
    sc.m2[jj] = (uint8_t)byte;
  }
  uint32_t nk1;
  const uint32_t k1_off = block_exclusive_scan<NT, uint32_t>(c2, sc.tmp, &nk1);
  const uint32_t total = l2 + nk1 + nk0 + np * (uint32_t)g;
  if (total >= limit) return total;
  // write
  for (uint32_t j = t; j < l2; j += NT) out[j] = sc.m2[j];
  {
    uint32_t r = 0;
    for (uint32_t jj = a2; jj < b2; ++jj)
      for (int bit = 0; bit < 8; ++bit) {
        const uint32_t j = 8 * jj + bit;
        if (j >= l1) break;
        if ((sc.m2[jj] >> bit) & 1u) out[l2 + k1_off + r++] = sc.m1[j];
      }
  }
  {
    uint32_t r = 0;
    for (uint32_t jj = a1; jj < b1; ++jj)
      for (int bit = 0; bit < 8; ++bit) {
        const uint32_t j = 8 * jj + bit;
        if (j >= l0) break;
        if ((sc.m1[jj] >> bit) & 1u) out[l2 + nk1 + k0_off + r++] = sc.m0[j];
      }
  }
  {
    uint32_t r = 0;
    uint8_t* pay = out + l2 + nk1 + nk0;
    for (uint32_t j = a0; j < b0; ++j)
      for (int bit = 0; bit < 8; ++bit) {
        const uint32_t u = 8 * j + bit;
        if (u >= U) break;
        if ((sc.m0[j] >> bit) & 1u) {
          for (int k = 0; k < g; ++k) pay[(pay_off + r) * g + k] = in[u * g + k];
          ++r;
        }
      }
  }
  return total;
}

// Counts set bits of `bm` (nbits valid) into prefix words: pre[w] = set bits in
// words [0, w), pre[nw] = total.  Bitmap bytes are read little-endian into words.
template <int NT>
__device__ uint32_t bitmap_prefix(const uint8_t* bm, uint32_t nbytes, uint32_t* pre, uint32_t* tmp) {
  const uint32_t nw = (nbytes + 3) >> 2;
  const uint32_t per = (nw + NT - 1) / NT;
  const uint32_t a = min(nw, threadIdx.x * per), b = min(nw, a + per);
  uint32_t c = 0;
  for (uint32_t w = a; w < b; ++w) {
    uint32_t v = 0;
    for (int k = 0; k < 4; ++k) {
      const uint32_t i = 4 * w + k;
      if (i < nbytes) v |= (uint32_t)bm[i] << (8 * k);
    }
    c += __popc(v);
  }
  uint32_t total;
  uint32_t run = block_exclusive_scan<NT, uint32_t>(c, tmp, &total);
  for (uint32_t w = a; w < b; ++w) {
    pre[w] = run;
    uint32_t v = 0;
    for (int k = 0; k < 4; ++k) {
      const uint32_t i = 4 * w + k;
      if (i < nbytes) v |= (uint32_t)bm[i] << (8 * k);
    }
    run += __popc(v);
  }
  if (threadIdx.x == 0) pre[nw] = total;
  __syncthreads();
  return total;
}

// Set bits of bm strictly before position j, from the prefix words.
__device__ __forceinline__ uint32_t rank_before(const uint8_t* bm, uint32_t nbytes, const uint32_t* pre,
                                                uint32_t j) {
  const uint32_t w = j >> 5, off = j & 31;
  uint32_t v = 0;
  for (int k = 0; k < 4; ++k) {
    const uint32_t i = 4 * w + k;
    if (i < nbytes) v |= (uint32_t)bm[i] << (8 * k);
  }
  const uint32_t below = off ? (v & ((1u << off) - 1u)) : 0u;
  return pre[w] + __popc(below);
}

__device__ __forceinline__ bool bit_of(const uint8_t* bm, uint32_t j) { return (bm[j >> 3] >> (j & 7)) & 1u; }

// Tail bits [nbits, 8*ceil(nbits/8)) of a bitmap are zero.
__device__ __forceinline__ bool tail_zero(const uint8_t* bm, uint32_t nbits) {
  const uint32_t r = nbits & 7;
  if (!r) return true;
  return (bm[nbits >> 3] >> r) == 0;
}

// Inverse of rze_encode: `in` holds exactly in_len bytes (global or shared), `out`
// receives L bytes (shared).  Returns false when the record is inconsistent.
template <int NT>
__device__ bool rze_decode(const uint8_t* in, uint32_t in_len, uint32_t L, int g, uint8_t* out,
                           const RzeScratch& sc) {
  const uint32_t U = L / (uint32_t)g;
  const uint32_t l0 = bytes_ceil8(U), l1 = bytes_ceil8(l0), l2 = bytes_ceil8(l1);
  __shared__ int bad;
  if (threadIdx.x == 0) bad = in_len < l2;
  __syncthreads();
  if (bad) return false;
  for (uint32_t j = threadIdx.x; j < l2; j += NT) sc.m2[j] = in[j];
  __syncthreads();
  if (threadIdx.x == 0 && !tail_zero(sc.m2, l1)) bad = 1;
  const uint32_t nk1 = bitmap_prefix<NT>(sc.m2, l2, sc.pre, sc.tmp);
  if (bad || l2 + nk1 > in_len) return false;
  // level 1 bitmap: byte j = last kept byte at or before j
  for (uint32_t j = threadIdx.x; j < l1; j += NT) {
    const uint32_t r = rank_before(sc.m2, l2, sc.pre, j) + (bit_of(sc.m2, j) ? 1u : 0u);
    sc.m1[j] = r ? in[l2 + r - 1] : 0;
  }
  __syncthreads();
  if (threadIdx.x == 0 && !tail_zero(sc.m1, l0)) bad = 1;
  const uint32_t nk0 = bitmap_prefix<NT>(sc.m1, l1, sc.pre, sc.tmp);
  if (bad || l2 + nk1 + nk0 > in_len) return false;
  const uint8_t* k0 = in + l2 + nk1;
  for (uint32_t j = threadIdx.x; j < l0; j += NT) {
    const uint32_t r = rank_before(sc.m1, l1, sc.pre, j) + (bit_of(sc.m1, j) ? 1u : 0u);
    sc.m0[j] = r ? k0[r - 1] : 0;
  }
  __syncthreads();
  if (threadIdx.x == 0 && !tail_zero(sc.m0, U)) bad = 1;
  const uint32_t np = bitmap_prefix<NT>(sc.m0, l0, sc.pre, sc.tmp);
  if (bad || (uint64_t)l2 + nk1 + nk0 + (uint64_t)np * g != in_len) return false;
  const uint8_t* pay = in + l2 + nk1 + nk0;
  for (uint32_t u = threadIdx.x; u < U; u += NT) {
    if (bit_of(sc.m0, u)) {
      const uint32_t r = rank_before(sc.m0, l0, sc.pre, u);
      for (int k = 0; k < g; ++k) out[u * g + k] = pay[r * g + k];
    } else {
      for (int k = 0; k < g; ++k) out[u * g + k] = 0;
    }
  }
  __syncthreads();
  return true;
}

}  // namespace lopc
