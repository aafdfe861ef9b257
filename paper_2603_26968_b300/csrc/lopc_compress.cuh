// lopc_compress.cuh -- compression kernels: value range (NOA), error-bound
// resolution, the tile pass (quantize, flags, tile-local least fixpoint), reruns of
// tiles whose halo changed, the chunk encoder, the size scan and the stream pack.
#pragma once
#include "lopc_codec.cuh"

namespace lopc {

// Compile-time tile configuration (Sec. II-C chunk of 16 KiB of words, as a tile).
template <typename T, int ND>
struct TileCfg;
// TZ x TY x TX: the chunk tile; HZ: z halo (0 for 2D); NT threads and SEG y-points per
// thread in the tile pass and reruns (NT = TZ * (TY / SEG) * TX); MINB, MINB_RERUN:
// blocks per SM those kernels are built for; NTC: threads of the chunk codecs.
template <>
struct TileCfg<float, 3> {
  static constexpr int TZ = 16, TY = 16, TX = 16, HZ = 1, NT = 256, SEG = 16, MINB = 3, MINB_RERUN = 4, NTC = 256;
};
template <>
struct TileCfg<double, 3> {
  static constexpr int TZ = 8, TY = 16, TX = 16, HZ = 1, NT = 128, SEG = 16, MINB = 3, MINB_RERUN = 6, NTC = 128;
};
template <>
struct TileCfg<float, 2> {
  static constexpr int TZ = 1, TY = 64, TX = 64, HZ = 0, NT = 256, SEG = 16, MINB = 3, MINB_RERUN = 4, NTC = 256;
};
template <>
struct TileCfg<double, 2> {
  static constexpr int TZ = 1, TY = 32, TX = 64, HZ = 0, NT = 128, SEG = 16, MINB = 5, MINB_RERUN = 6, NTC = 128;
};

// ------------------------------------------------------------------ range

// Per-field state reset and cleared dirty flags; blockIdx.y is the field.
__global__ void k_init_params(const FieldInfo* F, int nf) {
  const int f = blockIdx.y;
  if (f >= nf) return;
  const int64_t nw = dirty_words(F[f].g.ntiles);
  for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nw; w += (int64_t)gridDim.x * blockDim.x)
    F[f].dirty[w] = 0u;
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  Params* P = F[f].P;
  P->kmin = ~0ULL;
  P->kmax = 0ULL;
  P->eb = F[f].hdr.eb;
  P->mode = F[f].hdr.mode;
  P->status = 0;
  P->constant = 0;
  P->pass_ordered = 0;
  P->total = 0;
  P->rounds = 0;
  P->fix_iters = 0;
  P->fix_iters_max = 0;
  for (int k = 0; k < 9; ++k) P->phase[k] = 0;
  for (int k = 0; k < 6; ++k) P->work[k] = 0;
  P->fast_ok = 0;
  P->inv_f = 0.f;
}

template <typename T>
__device__ __forceinline__ unsigned long long biased(typename Traits<T>::Key k) {
  return (unsigned long long)((long long)k) ^ 0x8000000000000000ULL;
}

// Sec. III-A (NOA): x_min and x_max over each field, as order keys; blockIdx.y is
// the field within the class.
template <typename T>
__global__ void k_range(const FieldInfo* F, int f0) {
  using K = typename Traits<T>::Key;
  const FieldInfo& fi = F[f0 + blockIdx.y];
  if (fi.hdr.mode != LOPC_NOA) return;
  const T* __restrict__ x = reinterpret_cast<const T*>(fi.x);
  const int64_t n = fi.g.nz * fi.g.ny * fi.g.nx;
  Params* P = fi.P;
  K lo = Traits<T>::kMaxKey, hi = -Traits<T>::kMaxKey;
  bool bad = false;
  auto take = [&](T v) {
    if (!is_finite_bits<T>(v)) {
      bad = true;
      return;
    }
    const K k = order_key<T>(v);
    lo = min(lo, k);
    hi = max(hi, k);
  };
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  // 16-byte loads over the aligned body, single values over the head and tail
  constexpr int V = 16 / (int)sizeof(T);
  const int64_t head = (int64_t)(((16 - (reinterpret_cast<uintptr_t>(x) & 15)) & 15) / sizeof(T));
  const int64_t h = head < n ? head : n;
  const int64_t nv = (n - h) / V;
  const uint4* xv = reinterpret_cast<const uint4*>(x + h);
  for (int64_t i = t0; i < nv; i += stride) {
    const uint4 u = __ldg(&xv[i]);
    if constexpr (sizeof(T) == 4) {
      take(__uint_as_float(u.x));
      take(__uint_as_float(u.y));
      take(__uint_as_float(u.z));
      take(__uint_as_float(u.w));
    } else {
      take(Traits<T>::from_bits(((uint64_t)u.y << 32) | u.x));
      take(Traits<T>::from_bits(((uint64_t)u.w << 32) | u.z));
    }
  }
  for (int64_t i = t0; i < h; i += stride) take(x[i]);
  for (int64_t i = h + nv * V + t0; i < n; i += stride) take(x[i]);
  unsigned long long blo = biased<T>(lo), bhi = biased<T>(hi);
  for (int o = 16; o; o >>= 1) {
    blo = min(blo, __shfl_xor_sync(0xffffffffu, blo, o));
    bhi = max(bhi, __shfl_xor_sync(0xffffffffu, bhi, o));
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&P->status, kErrNonfinite);
  if ((threadIdx.x & 31) == 0) {
    atomicMin(&P->kmin, blo);
    atomicMax(&P->kmax, bhi);
  }
}

// Sec. III-A: eps = eb (ABS) or eb * (x_max - x_min) (NOA); eps_q = eps (1 - 2^-16);
// inv = 1 / eps_q.  IEEE binary64, correctly rounded, no contraction.  One thread
// per field of the class.
template <typename T>
__global__ void k_resolve_eps(const FieldInfo* F, int f0, int nf) {
  using K = typename Traits<T>::Key;
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= nf) return;
  Params* P = F[f0 + f].P;
  if (P->status & kErrNonfinite) return;
  double eps = P->eb;
  if (P->mode == LOPC_NOA) {
    const K kmin = (K)(long long)(P->kmin ^ 0x8000000000000000ULL);
    const K kmax = (K)(long long)(P->kmax ^ 0x8000000000000000ULL);
    const double xmin = (double)value_of_key<T>(kmin), xmax = (double)value_of_key<T>(kmax);
    const double r = __dsub_rn(xmax, xmin);
    if (!(r <= 1.79e308)) {
      P->status |= kErrRange;
      return;
    }
    if (r == 0.0) {
      P->constant = 1;
      const T c = (T)__dadd_rn(xmin, 0.0);
      P->const_bits = (unsigned long long)Traits<T>::bits(c);
      P->eps = P->eps_q = P->inv = 0.0;
      return;
    }
    eps = __dmul_rn(P->eb, r);
  }
  if (!(eps > 0.0) || !(eps <= 1.79e308)) {
    P->status |= kErrRange;
    return;
  }
  const double eq = __dmul_rn(eps, 1.0 - 0x1p-16);
  const double inv = __ddiv_rn(1.0, eq);
  if (!(eq > 0.0) || !(inv <= 1.79e308)) {
    P->status |= kErrRange;
    return;
  }
  P->eps = eps;
  P->eps_q = eq;
  P->inv = inv;
  const unsigned long long u = (unsigned long long)__double_as_longlong(inv);
  const int ex = (int)((u >> 52) & 0x7ff);
  P->inv_m = (u & 0xfffffffffffffULL) | (ex ? 0x10000000000000ULL : 0ULL);
  P->inv_e = ex ? ex - 1075 : -1074;
  const float inv_f = __double2float_rn(inv);
  P->inv_f = inv_f;
  P->fast_ok = inv_f >= 1.1754943508222875e-38f && inv_f <= 3.4028234663852886e38f;
}

// ---------------------------------------------------------------- tile pass

constexpr uint32_t kSlotBytes = 16384;  // a record never exceeds the raw chunk (16 KiB)

// Shared-memory geometry of a tile with its 1-point halo, and the thread mapping:
// thread t owns the SEG points (lz, SEG*sy + j, lx), j = 0..SEG-1, of one y-segment,
// with t = (lz * SEGY + sy) * TX + lx, so the lanes of a warp walk consecutive x.
// Z-planes have a pitch = 16 (mod 32) so that the two x-runs of 16 lanes a warp
// touches fall in distinct banks.  Rows have an odd pitch (A16 = false, the tightest
// layout), or a pitch that is a multiple of 4 words with the first interior point
// at entry 4 (A16 = true), so that interior rows start on 16-byte boundaries.
template <typename T, int ND, bool A16 = false>
struct TileGeom {
  using C = TileCfg<T, ND>;
  static constexpr int TZ = C::TZ, TY = C::TY, TX = C::TX, HZ = C::HZ, NT = C::NT, SEG = C::SEG;
  static constexpr int BZ = TZ + 2 * HZ, BY = TY + 2, BX = TX + 2;
  static constexpr int XO = A16 ? 4 : 1;  // entry of interior column 0 within a row
  static constexpr int BXP = A16 ? ((TX + 8 + 3) & ~3) : ((BX % 2) ? BX : BX + 1);
  static constexpr int PP = HZ ? ((BY * BXP + 15) / 32) * 32 + 16 : BY * BXP;
  static constexpr int E = BZ * PP;               // shared-memory entries
  static constexpr int NP = TZ * TY * TX;         // points of a full tile
  static constexpr int SEGY = TY / SEG;           // y-segments per column
  static_assert(TZ * SEGY * TX == NT, "one y-segment per thread");
  static_assert(TX >= 16, "a half warp spans one x-run");
  __device__ static constexpr int off(int dz, int dy, int dx) { return dz * PP + dy * BXP + dx; }
  __device__ static constexpr int entry(int lz, int ly, int lx) { return (lz + HZ) * PP + (ly + 1) * BXP + lx + XO; }
  // linear index of a tile point (masks are kept for the tile's own points only)
  __device__ static constexpr int lin(int lz, int ly, int lx) { return (lz * TY + ly) * TX + lx; }
  __device__ static constexpr int loff(int dz, int dy, int dx) { return (dz * TY + dy) * TX + dx; }
};

struct SegPos {
  int lz, ly0, lx;  // local coordinates of the thread's first point
  int e0;           // its shared-memory entry; point j is at e0 + j * BXP
  int o0;           // its linear index (and frontier bit); point j is o0 + j * TX
};

template <typename G>
__device__ __forceinline__ SegPos seg_pos() {
  SegPos s;
  const int t = threadIdx.x;
  s.lx = t % G::TX;
  const int r = t / G::TX;
  s.lz = r / G::SEGY;
  s.ly0 = (r % G::SEGY) * G::SEG;
  s.e0 = G::entry(s.lz, s.ly0, s.lx);
  s.o0 = G::lin(s.lz, s.ly0, s.lx);
  return s;
}

// Direction k (0..13) of the Freudenthal neighbourhood (Sec. II): k < 7 is -D[k]
// (lower linear index), k >= 7 is +D[k-7]; D[d] has bits (z, y, x) of d + 1.
__host__ __device__ constexpr int dz_of(int k) { return (k < 7 ? -1 : 1) * ((((k % 7) + 1) >> 2) & 1); }
__host__ __device__ constexpr int dy_of(int k) { return (k < 7 ? -1 : 1) * ((((k % 7) + 1) >> 1) & 1); }
__host__ __device__ constexpr int dx_of(int k) { return (k < 7 ? -1 : 1) * (((k % 7) + 1) & 1); }

// Asynchronous global -> shared copies (cp.async); a false predicate writes zeros and
// reads nothing (the source must still be a valid address).
__device__ __forceinline__ void cp_async4(void* dst, const void* src, bool pred) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(pred ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src, bool pred) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(src), "r"(pred ? 8 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// A word copy into shared memory for a box load: asynchronous through L1
// (cp.async.ca) for data no block changes during the kernel, or else a load from L2
// (ld.global.cg; L1 is not coherent across SMs, so a line it cached earlier in the
// same kernel could hold a value another block has raised since) and a store.
template <bool MUTABLE, typename Word>
__device__ __forceinline__ void box_word(Word* dst, const Word* src, bool in) {
  if (MUTABLE) {
    *dst = in ? __ldcg(src) : (Word)0;
  } else if (sizeof(Word) == 4) {
    cp_async4(dst, src, in);
  } else {
    cp_async8(dst, src, in);
  }
}

// Loads of words other blocks may change (ld.global.cg, from L2) into dst[], B per
// thread issued together before their shared-memory stores, so that a thread waits for
// one round trip per B loads rather than per load.  at(i, e, src) gives item i's entry
// of dst (-1: none) and source (null: outside the field, stored as 0); i runs over
// [0, n).
template <int NT, int B, typename Word, typename At>
__device__ __forceinline__ void gather_l2(Word* dst, int n, At at) {
  for (int i0 = threadIdx.x; i0 < n; i0 += B * NT) {
    Word v[B];
    int e[B];
#pragma unroll
    for (int u = 0; u < B; ++u) {
      const int i = i0 + u * NT;
      const Word* sp = nullptr;
      e[u] = -1;
      if (i < n) at(i, e[u], sp);
      v[u] = sp ? __ldcg(sp) : (Word)0;
    }
#pragma unroll
    for (int u = 0; u < B; ++u)
      if (e[u] >= 0) dst[e[u]] = v[u];
  }
}

// Copy of a tile's box (the tile and a one-point halo; 2D tiles have no z halo) of
// `src` (row-major field of nz x ny x nx elements of `Word`) into shared memory at
// `dst` (entry layout of G).  Rows are walked as (row, column) with one row base per
// row: the interior columns go to lanes (asynchronous 16-byte copies of four words,
// which bypass L1, when the layout and the field allow it), the two halo columns are
// a second loop.  Absent points read nothing and are zero.  MUTABLE: `src` may be
// changed by other blocks during the kernel (see box_word).  The caller waits for
// the asynchronous copies.
template <typename G, typename Word, bool MUTABLE = false>
__device__ __forceinline__ void load_box_async(Word* dst, const Word* __restrict__ src, const Geometry& g,
                                               const TileBox& tb) {
  static_assert(G::TX == 16 || G::TX == 64, "interior columns are whole lane groups");
  constexpr int NT = G::NT, ROWS = G::BZ * G::BY;
  const int64_t plane = g.ny * g.nx;
  constexpr int V = 16 / (int)sizeof(Word);  // words per 16-byte copy
  if (G::XO % V == 0 && G::BXP % V == 0 && G::PP % V == 0 && g.nx % V == 0) {
    // every interior row starts on a 16-byte boundary in shared and global memory,
    // and a copy of V words is either wholly inside the field or wholly outside
    constexpr int CW = G::TX / V;  // copies per row
    constexpr int RPP = NT / CW;
    const int c = threadIdx.x % CW;
    for (int r = threadIdx.x / CW; r < ROWS; r += RPP) {
      const int ly = r % G::BY, lz = r / G::BY;
      const int64_t gz = tb.z0 + lz - G::HZ, gy = tb.y0 + ly - 1;
      const int64_t gx = tb.x0 + (int64_t)c * V;
      const bool in = gz >= 0 && gz < g.nz && gy >= 0 && gy < g.ny && gx < g.nx;
      const unsigned d = (unsigned)__cvta_generic_to_shared(dst + lz * G::PP + ly * G::BXP + G::XO + c * V);
      const Word* sp = in ? src + gz * plane + gy * g.nx + gx : src;
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(sp), "r"(in ? 16 : 0) : "memory");
    }
  } else if (!MUTABLE) {
    constexpr int CW = G::TX < 32 ? G::TX : 32;  // lanes per row
    constexpr int RPP = NT / CW;                 // rows per pass
    const int c = threadIdx.x % CW;
    for (int r = threadIdx.x / CW; r < ROWS; r += RPP) {
      const int ly = r % G::BY, lz = r / G::BY;
      const int64_t gz = tb.z0 + lz - G::HZ, gy = tb.y0 + ly - 1;
      const bool row_in = gz >= 0 && gz < g.nz && gy >= 0 && gy < g.ny;
      const Word* row = src + (row_in ? gz * plane + gy * g.nx : 0);
      Word* drow = dst + lz * G::PP + ly * G::BXP + G::XO;
#pragma unroll
      for (int lx = c; lx < G::TX; lx += CW) {
        const int64_t gx = tb.x0 + lx;
        const bool in = row_in && gx < g.nx;
        box_word<MUTABLE>(&drow[lx], in ? row + gx : src, in);
      }
    }
  } else {
    // loads from L2, four per thread in flight before their stores
    gather_l2<NT, 4, Word>(dst, ROWS * G::TX, [&](int i, int& d, const Word*& sp) {
      const int r = i / G::TX, lx = i - r * G::TX;
      const int ly = r % G::BY, lz = r / G::BY;
      const int64_t gz = tb.z0 + lz - G::HZ, gy = tb.y0 + ly - 1, gx = tb.x0 + lx;
      d = lz * G::PP + ly * G::BXP + G::XO + lx;
      sp = gz >= 0 && gz < g.nz && gy >= 0 && gy < g.ny && gx < g.nx ? src + gz * plane + gy * g.nx + gx : nullptr;
    });
  }
  // the halo columns x0 - 1 and x0 + TX
  auto halo = [&](int i, int& d, const Word*& sp) {
    const int r = i >> 1, side = i & 1;
    const int ly = r % G::BY, lz = r / G::BY;
    const int64_t gz = tb.z0 + lz - G::HZ, gy = tb.y0 + ly - 1;
    const int64_t gx = side ? tb.x0 + G::TX : tb.x0 - 1;
    const bool in = gz >= 0 && gz < g.nz && gy >= 0 && gy < g.ny && gx >= 0 && gx < g.nx;
    d = lz * G::PP + ly * G::BXP + (side ? G::XO + G::TX : G::XO - 1);
    sp = in ? src + gz * plane + gy * g.nx + gx : nullptr;
  };
  if (MUTABLE) {
    gather_l2<NT, (2 * ROWS + NT - 1) / NT, Word>(dst, 2 * ROWS, halo);  // every load in flight at once
  } else {
    for (int i = threadIdx.x; i < 2 * ROWS; i += NT) {
      int d;
      const Word* sp;
      halo(i, d, sp);
      box_word<false>(dst + d, sp ? sp : src, sp != nullptr);
    }
  }
}

// Calls fn(e, in) for every entry e of a tile's box (in: the point is in the field),
// walking rows as load_box_async does.
template <typename G, typename Fn>
__device__ __forceinline__ void for_box(const Geometry& g, const TileBox& tb, Fn fn) {
  constexpr int NT = G::NT, ROWS = G::BZ * G::BY;
  constexpr int CW = G::TX < 32 ? G::TX : 32;
  constexpr int RPP = NT / CW;
  const int c = threadIdx.x % CW;
  for (int r = threadIdx.x / CW; r < ROWS; r += RPP) {
    const int ly = r % G::BY, lz = r / G::BY;
    const int64_t gz = tb.z0 + lz - G::HZ, gy = tb.y0 + ly - 1;
    const bool row_in = gz >= 0 && gz < g.nz && gy >= 0 && gy < g.ny;
    const int e0 = lz * G::PP + ly * G::BXP;
#pragma unroll
    for (int lx = c; lx < G::TX; lx += CW) fn(e0 + G::XO + lx, row_in && tb.x0 + lx < g.nx);
  }
  for (int i = threadIdx.x; i < 2 * ROWS; i += NT) {
    const int r = i >> 1, side = i & 1;
    const int ly = r % G::BY, lz = r / G::BY;
    const int64_t gz = tb.z0 + lz - G::HZ, gy = tb.y0 + ly - 1;
    const int64_t gx = side ? tb.x0 + G::TX : tb.x0 - 1;
    fn(lz * G::PP + ly * G::BXP + (side ? G::XO + G::TX : G::XO - 1),
       gz >= 0 && gz < g.nz && gy >= 0 && gy < g.ny && gx >= 0 && gx < g.nx);
  }
}

// Direction bits whose offset along an axis is -1 (lo) or +1 (hi).
__host__ __device__ constexpr uint32_t dir_mask(int axis, int sign) {
  uint32_t r = 0;
  for (int k = 0; k < 14; ++k) {
    const int d = axis == 0 ? dz_of(k) : axis == 1 ? dy_of(k) : dx_of(k);
    if (d == sign) r |= 1u << k;
  }
  return r;
}

// Bits of the directions that leave the tile box, for a point at local (lz, ly, lx):
// the directions stepping below a face the point lies on, or above one.
template <typename G>
__device__ __forceinline__ uint32_t out_of_box_bits(int lz, int ly, int lx) {
  constexpr uint32_t zl = dir_mask(0, -1), zh = dir_mask(0, 1), yl = dir_mask(1, -1), yh = dir_mask(1, 1);
  constexpr uint32_t xl = dir_mask(2, -1), xh = dir_mask(2, 1);
  uint32_t r = (ly == 0 ? yl : 0u) | (ly == G::TY - 1 ? yh : 0u) | (lx == 0 ? xl : 0u) | (lx == G::TX - 1 ? xh : 0u);
  if (G::HZ) r |= (lz == 0 ? zl : 0u) | (lz == G::TZ - 1 ? zh : 0u);
  return r;
}

// Bit (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1) of the neighbour tile (dz, dy, dx in
// {-1, 0, 1}) that holds the box entry at local (lz, ly, lx) of a tile.
template <typename G>
__device__ __forceinline__ uint32_t tile_dir_bit(int lz, int ly, int lx) {
  const int dz = lz < 0 ? -1 : lz >= G::TZ ? 1 : 0, dy = ly < 0 ? -1 : ly >= G::TY ? 1 : 0;
  const int dx = lx < 0 ? -1 : lx >= G::TX ? 1 : 0;
  return 1u << ((dz + 1) * 9 + (dy + 1) * 3 + (dx + 1));
}

// Tile index of the neighbour in direction d (a tile_dir_bit position) of tile tid,
// or -1 when it lies outside the field's tiles.
__device__ __forceinline__ int64_t neighbour_tile(const Geometry& g, int64_t tid, int d) {
  const int64_t tz = tid / (g.ntx * g.nty), ty = (tid / g.ntx) % g.nty, tx = tid % g.ntx;
  const int64_t nz = tz + d / 9 - 1, ny = ty + (d / 3) % 3 - 1, nx = tx + d % 3 - 1;
  if (nz < 0 || nz >= g.ntz || ny < 0 || ny >= g.nty || nx < 0 || nx >= g.ntx) return -1;
  return (nz * g.nty + ny) * g.ntx + nx;
}

// Neighbour-tile bits of the constraints that the thread's segment points violate
// after a rerun: a point p of the segment that rose in this run constrains each
// out-of-tile upper same-bin neighbour q to s(q) >= s(p) + [p after q]; q's value in
// the box is what this run loaded (a lower bound of its current value), so a tile
// whose constraint holds there is never marked, and one whose constraint fails may
// be marked when it need not be (its rerun then finds every constraint held).
// `cm(o)` gives point o's lower bits 0-13 and same-bin bits 16-29; `risen(j)`
// whether segment point j rose.
template <typename G, typename CmFn, typename RisenFn>
__device__ __forceinline__ uint32_t violated_tile_bits(const uint32_t* sv, const TileBox& tb, int lz, int ly0, int lx,
                                                       int e0, int o0, CmFn cm, RisenFn risen) {
  uint32_t bits = 0;
  if (lz >= tb.cz || lx >= tb.cx) return 0;
#pragma unroll 1
  for (int j = 0; j < G::SEG; ++j) {
    const int ly = ly0 + j;
    if (ly >= tb.cy) break;
    const uint32_t ob = out_of_box_bits<G>(lz, ly, lx);
    if (!ob || !risen(j)) continue;
    const uint32_t m = cm(o0 + j * G::TX);
    const uint32_t upo = (m >> 16) & ~m & ob & 0x3FFFu;
    if (!upo) continue;
    const int e = e0 + j * G::BXP;
    const uint32_t v = sv[e];
#pragma unroll
    for (int k = 0; k < 14; ++k) {
      if (!G::HZ && dz_of(k) != 0) continue;
      if (((upo >> k) & 1u) && sv[e + G::off(dz_of(k), dy_of(k), dx_of(k))] < v + (k < 7 ? 1u : 0u))
        bits |= tile_dir_bit<G>(lz + dz_of(k), ly + dy_of(k), lx + dx_of(k));
    }
  }
  return bits;
}

// Local coordinates of tile point o (linear order: x fastest).
template <typename G>
__device__ __forceinline__ void point_of_lin(int o, int& lz, int& ly, int& lx) {
  lx = o % G::TX;
  ly = (o / G::TX) % G::TY;
  lz = o / (G::TX * G::TY);
}

// Shared state of the list-driven fixpoint: two frontiers and the risen points (one
// bit per tile point, linear order), two list counters, the frontier list.
template <typename G>
struct FixSmem {
  static constexpr int NW = G::NP / 32;
  static constexpr size_t bits_bytes() { return (size_t)3 * NW * 4 + 16; }
  static constexpr size_t list_bytes() { return ((size_t)G::NP * 2 + 15) & ~(size_t)15; }
};

// Tile-local least fixpoint of Alg. 2's update, by sweeps over a frontier list:
//   s(p) = max(s(p), max over lower same-bin n of s(n) + [n after p]),
// recomputed only for points whose lower same-bin neighbours rose; a point that
// rises puts its greater same-bin neighbours of the tile on the next frontier.  Each
// sweep compacts the frontier bitmap into a list that all threads share evenly, so a
// sweep costs about one evaluation per thread.  Once a frontier is small (the thin
// tail of the chains), warp 0 runs the sweeps alone with warp barriers, and hands a
// frontier that has grown again back to the block.  Raised subbins are visible to
// the rest of the sweep at once; a neighbour read before it rose is queued again by
// that rise.  `over` is set, with the last frontier not evaluated, after `limit`
// sweeps or before the evaluations would exceed `eval_budget`.  Chaotic relaxation
// from lower bounds reaches the unique least fixpoint (Sec. III-E) whatever the
// schedule.  `cml[o]` holds, for tile point o (linear order), its lower same-bin
// neighbours in bits 0-13, and in bits 16-29 its same-bin upper neighbours inside the
// tile (SAME = false) or all its same-bin neighbours (SAME = true; the in-tile upper
// ones are derived).  `fa` holds the first frontier, `fb` and `rb` must be clear;
// `rb` receives the points that rose; cnt[0..3] are scratch.  Returns the number of
// sweeps.
template <typename G, bool SAME>
__device__ __forceinline__ int frontier_fixpoint(uint32_t* sv, const uint32_t* cml, uint32_t* fa, uint32_t* fb,
                                                 uint32_t* rb, unsigned* cnt, uint16_t* list, int limit, bool& over,
                                                 unsigned& evals, unsigned& raises,
                                                 unsigned eval_budget = 0xffffffffu) {
  constexpr int NW = G::NP / 32, NT = G::NT;
  constexpr unsigned kTail = 16, kBack = 32;  // warp 0 alone below kTail points, until above kBack
  static_assert(NW <= NT && NW % 32 == 0, "one frontier word per thread; whole words per lane");
  volatile uint32_t* vs = sv;
  const int lane = threadIdx.x & 31;
  // evaluates tile point o; a rise records o and queues o's in-tile upper neighbours in `next`
  auto eval_point = [&](int o, uint32_t* next) {
    int lz, ly, lx;
    point_of_lin<G>(o, lz, ly, lx);
    const int e = G::entry(lz, ly, lx);
    const uint32_t m = cml[o];
    const uint32_t before = vs[e];
    ++evals;
    uint32_t best = before;
#pragma unroll
    for (int k = 0; k < 14; ++k) {  // predicated loads at constant offsets, all in flight together
      if (!G::HZ && dz_of(k) != 0) continue;
      if (m & (1u << k)) {
        const uint32_t cand = vs[e + G::off(dz_of(k), dy_of(k), dx_of(k))] + (k >= 7 ? 1u : 0u);
        best = cand > best ? cand : best;
      }
    }
    if (best == before) return;
    vs[e] = best;
    ++raises;
    atomicOr(&rb[o >> 5], 1u << (o & 31));
    // in-tile upper neighbours: stored as such, or derived from the same-bin bits
    const uint32_t um = SAME ? ((m >> 16) & ~m & ~out_of_box_bits<G>(lz, ly, lx)) : (m >> 16);
#pragma unroll
    for (int k = 0; k < 14; ++k) {
      if (!G::HZ && dz_of(k) != 0) continue;
      if (um & (1u << k)) {
        const int qn = o + G::loff(dz_of(k), dy_of(k), dx_of(k));
        atomicOr(&next[qn >> 5], 1u << (qn & 31));
      }
    }
  };
  if (threadIdx.x == 0) cnt[0] = cnt[1] = 0;
  __syncthreads();
  int iter = 0;
  unsigned spent = 0;  // evaluations so far (the same value in every thread)
  while (true) {
    // compact the frontier into the list; clear it for reuse two sweeps later
    uint32_t word = 0;
    if (threadIdx.x < NW) {
      word = fa[threadIdx.x];
      if (word) fa[threadIdx.x] = 0u;
    }
    const int c = __popc(word);
    int incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const int wtot = __shfl_sync(0xffffffffu, incl, 31);
    unsigned base = 0;
    if (lane == 31 && wtot) base = atomicAdd(&cnt[iter & 1], (unsigned)wtot);
    base = __shfl_sync(0xffffffffu, base, 31);
    unsigned pos = base + (unsigned)(incl - c);
    for (uint32_t b = word; b; b &= b - 1) list[pos++] = (uint16_t)(threadIdx.x * 32 + __ffs(b) - 1);
    __syncthreads();
    const unsigned n = cnt[iter & 1];
    if (n == 0) break;
    if (++iter > limit || spent + n > eval_budget) {
      over = true;
      break;
    }
    spent += n;
    if (n <= kTail) {
      // the tail: warp 0 sweeps alone from this list (fa and fb are clear)
      if (threadIdx.x < 32) {
        unsigned wn = n, wspent = spent;
        int wit = iter;
        unsigned flags = 0;  // 1: over, 2: done
        while (true) {
          for (unsigned i = lane; i < wn; i += 32) eval_point(list[i], fb);
          __syncwarp();
          // compact fb into the list, lane by lane over contiguous words
          constexpr int WPL = NW / 32;
          uint32_t wv[WPL];
          unsigned cw = 0;
#pragma unroll
          for (int r = 0; r < WPL; ++r) {
            wv[r] = fb[lane * WPL + r];
            cw += __popc(wv[r]);
          }
          unsigned wi = cw;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
          }
          const unsigned total = __shfl_sync(0xffffffffu, wi, 31);
          unsigned wp = wi - cw;
#pragma unroll
          for (int r = 0; r < WPL; ++r) {
            if (wv[r]) fb[lane * WPL + r] = 0u;
            for (uint32_t b = wv[r]; b; b &= b - 1) list[wp++] = (uint16_t)((lane * WPL + r) * 32 + __ffs(b) - 1);
          }
          __syncwarp();
          wn = total;
          if (wn == 0) {
            flags = 2;
            break;
          }
          if (wn > kBack) {  // grown again: back to the block, as frontier bits (counted there)
            for (unsigned i = lane; i < wn; i += 32) {
              const int o = list[i];
              atomicOr(&fa[o >> 5], 1u << (o & 31));
            }
            break;
          }
          if (++wit > limit || wspent + wn > eval_budget) {
            flags = 1;
            break;
          }
          wspent += wn;
        }
        __syncwarp();
        if (lane == 0) {
          cnt[0] = cnt[1] = 0;
          cnt[2] = (unsigned)wit | (flags << 30);
          cnt[3] = wspent;
        }
      }
      __syncthreads();
      const unsigned st = cnt[2];
      iter = (int)(st & 0x3FFFFFFFu);
      spent = cnt[3];
      if (st >> 30) {
        over = (st >> 30) == 1u;
        break;
      }
      continue;
    }
    if (threadIdx.x == 0) cnt[iter & 1] = 0;  // the counter of the next sweep
    for (unsigned i = threadIdx.x; i < n; i += NT) eval_point(list[i], fb);
    __syncthreads();
    uint32_t* t = fa;
    fa = fb;
    fb = t;
  }
  return iter;
}


// Tile-local least fixpoint in topological order (Kahn's algorithm), for the tile pass
// where every point must be computed: a point is evaluated once, when all its
// lower same-bin neighbours inside the tile are final, as
//   s(p) = max over lower same-bin n of s(n) + [n after p]
// (halo neighbours hold constants).  Each wave takes the ready list; a point's
// evaluation releases its in-tile upper neighbours, and those whose last lower
// neighbour it was form the next list.  The constraint graph is acyclic, so this is
// the unique least fixpoint.  `cml[o]`: lower bits 0-13, in-tile upper bits 16-29;
// `indeg`: NP bytes of scratch (read as words); `la`, `lb`: two lists of NP entries;
// `cnt`: two counters.  Returns the number of waves.
template <typename G, bool SAME>
__device__ __forceinline__ int topo_fixpoint(uint32_t* sv, const uint32_t* cml, uint32_t* indeg, uint16_t* la,
                                             uint16_t* lb, unsigned* cnt, const TileBox& tb, uint32_t* rb,
                                             unsigned& evals, unsigned& raises) {
  constexpr int NT = G::NT;
  const int lane = threadIdx.x & 31;
  if (threadIdx.x == 0) cnt[0] = cnt[1] = 0;
  __syncthreads();
  // in-degrees (in-tile lower same-bin neighbours) and the first ready list
  static_assert(G::NP % NT == 0, "a whole number of points per thread");
  for (int o4 = threadIdx.x; o4 < G::NP / 4; o4 += NT) {
    uint32_t word = 0;
    unsigned readym = 0;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int o = 4 * o4 + u;
      int lz, ly, lx;
      point_of_lin<G>(o, lz, ly, lx);
      const bool real = lz < tb.cz && ly < tb.cy && lx < tb.cx;
      const uint32_t d = real ? (uint32_t)__popc(cml[o] & 0x3FFFu & ~out_of_box_bits<G>(lz, ly, lx)) : 0xFFu;
      word |= d << (8 * u);
      readym |= (real && d == 0 ? 1u : 0u) << u;
    }
    indeg[o4] = word;
    const unsigned r = __popc(readym);
    unsigned incl = r;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const unsigned y = __shfl_up_sync(0xffffffffu, incl, off);
      if (lane >= off) incl += y;
    }
    const unsigned wt = __shfl_sync(0xffffffffu, incl, 31);
    unsigned base = 0;
    if (lane == 31 && wt) base = atomicAdd(&cnt[0], wt);
    base = __shfl_sync(0xffffffffu, base, 31) + incl - r;
    for (unsigned m = readym; m; m &= m - 1) la[base++] = (uint16_t)(4 * o4 + __ffs(m) - 1);
  }
  __syncthreads();
  // one warp's share of a wave: item i of the ready list `lin_` (n items); the points
  // it makes ready go to `lout` (counter `cout`), appended by the warp as a whole
  auto step = [&](unsigned i, unsigned n, const uint16_t* lin_, uint16_t* lout, unsigned* cout) {
    unsigned readym = 0;
    int o = 0;
    uint32_t m = 0;
    if (i < n) {
      o = lin_[i];
      int lz, ly, lx;
      point_of_lin<G>(o, lz, ly, lx);
      const int e = G::entry(lz, ly, lx);
      m = cml[o];
      const uint32_t before = sv[e];
      uint32_t best = before;
#pragma unroll
      for (int k = 0; k < 14; ++k) {
        if (!G::HZ && dz_of(k) != 0) continue;
        if (m & (1u << k)) {
          const uint32_t cand = sv[e + G::off(dz_of(k), dy_of(k), dx_of(k))] + (k >= 7 ? 1u : 0u);
          best = cand > best ? cand : best;
        }
      }
      if (best != before) {
        ++raises;
        sv[e] = best;
        if (rb) atomicOr(&rb[o >> 5], 1u << (o & 31));
      }
      ++evals;
      // release the in-tile upper neighbours; record those this point made ready
      const uint32_t um = SAME ? ((m >> 16) & ~m & ~out_of_box_bits<G>(lz, ly, lx)) : (m >> 16);
#pragma unroll
      for (int k = 0; k < 14; ++k) {
        if (!G::HZ && dz_of(k) != 0) continue;
        if (um & (1u << k)) {
          const int q = o + G::loff(dz_of(k), dy_of(k), dx_of(k));
          const uint32_t sh = 8u * (uint32_t)(q & 3);
          const uint32_t old = atomicSub(&indeg[q >> 2], 1u << sh);
          if (((old >> sh) & 0xFFu) == 1u) readym |= 1u << k;
        }
      }
    }
    const unsigned r = __popc(readym);
    unsigned incl = r;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const unsigned y = __shfl_up_sync(0xffffffffu, incl, off);
      if (lane >= off) incl += y;
    }
    const unsigned wt = __shfl_sync(0xffffffffu, incl, 31);
    unsigned base = 0;
    if (lane == 31 && wt) base = atomicAdd(cout, wt);
    base = __shfl_sync(0xffffffffu, base, 31) + incl - r;
#pragma unroll
    for (int k = 0; k < 14; ++k) {
      if (!G::HZ && dz_of(k) != 0) continue;
      if (readym & (1u << k)) lout[base++] = (uint16_t)(o + G::loff(dz_of(k), dy_of(k), dx_of(k)));
    }
  };
  constexpr unsigned kTail = 16, kBack = 32;  // warp 0 alone below kTail ready points, until above kBack
  unsigned n = cnt[0];
  int cur = 0;
  int wave = 0;
  while (n) {
    if (n <= kTail) {
      // the thin waves: warp 0 alone, with warp barriers; the same list protocol
      // (input count in cnt[cur], output counter cnt[cur ^ 1] clear)
      if (threadIdx.x < 32) {
        unsigned wn = n;
        int wcur = cur, wwave = wave;
        while (wn && wn <= kBack) {
          ++wwave;
          const uint16_t* lin_ = wcur ? lb : la;
          uint16_t* lout = wcur ? la : lb;
          unsigned* cout = &cnt[wcur ^ 1];
          for (unsigned b0 = 0; b0 < wn; b0 += 32) step(b0 + lane, wn, lin_, lout, cout);
          __syncwarp();
          wn = *reinterpret_cast<volatile unsigned*>(cout);
          __syncwarp();
          if (lane == 0) cnt[wcur] = 0;
          wcur ^= 1;
          __syncwarp();
        }
        if (lane == 0) {
          cnt[2] = wn;
          cnt[3] = (unsigned)wcur | ((unsigned)wwave << 1);
        }
      }
      __syncthreads();
      n = cnt[2];
      cur = (int)(cnt[3] & 1u);
      wave = (int)(cnt[3] >> 1);
      __syncthreads();
      continue;
    }
    ++wave;
    const uint16_t* lin_ = cur ? lb : la;
    uint16_t* lout = cur ? la : lb;
    unsigned* cout = &cnt[cur ^ 1];
    for (unsigned b0 = 0; b0 < n; b0 += NT) step(b0 + threadIdx.x, n, lin_, lout, cout);  // uniform trip count
    __syncthreads();
    n = *cout;
    if (threadIdx.x == 0) cnt[cur] = 0;  // the counter of the wave after next
    cur ^= 1;
    __syncthreads();
  }
  return wave;
}

template <typename T, int ND>
struct PassSmem {
  using G = TileGeom<T, ND>;
  using K = typename Traits<T>::Key;
  using B = typename Traits<T>::Bin;
  static constexpr uint32_t L = (uint32_t)G::NP * Traits<T>::W;  // BIT output of a full tile
  static constexpr size_t up16(size_t v) { return (v + 15) & ~(size_t)15; }
  // RA: keys -> subbins -> bit planes + RZE work;  RB: bins -> staged bin record
  static constexpr size_t RAa = (size_t)G::E * (sizeof(K) > 4 ? sizeof(K) : 4);
  static constexpr size_t RAb = (size_t)L + RzeWork::bytes(L);
  static constexpr size_t RA = up16(RAa > RAb ? RAa : RAb);
  // after the bin record, the bins' region holds the in-degrees and two ready lists
  static constexpr size_t TOPO = (size_t)G::NP + 2 * FixSmem<G>::list_bytes();
  static constexpr size_t max3(size_t a, size_t b, size_t c) { return a > b ? (a > c ? a : c) : (b > c ? b : c); }
  static constexpr size_t RB = up16(max3((size_t)G::E * sizeof(B), (size_t)L, TOPO));
  static constexpr size_t RC = up16((size_t)G::NP * 4);                 // neighbour masks of the tile's points
  static constexpr size_t RD = up16(FixSmem<G>::bits_bytes());         // frontier bits, counters
  static constexpr size_t bytes() { return RA + RB + RC + RD; }
};

// Tile pass (one block per chunk-tile):
//   1. load x on the tile and its halo, quantize (Sec. III-A) and take order keys;
//   2. flags (Alg. 1): the lower same-bin neighbours of every point;
//   3. encode the tile's bin record (Sec. III-C; bins are final once quantized);
//   4. tile-local least fixpoint with halo subbins taken as 0 (a lower bound), unless
//      fix = 0 (the worklist schedule starts from subbins 0);
//   5. write subbins and lower masks (what reruns and the boundary check need).
template <typename T, int ND>
__global__ void __launch_bounds__(TileCfg<T, ND>::NT, TileCfg<T, ND>::MINB)
    k_pass(const FieldInfo* __restrict__ F, int f0, int nf, int64_t tile0, unsigned budget16, unsigned dense16,
           int fix) {
  using G = TileGeom<T, ND>;
  using PS = PassSmem<T, ND>;
  using K = typename Traits<T>::Key;
  using B = typename Traits<T>::Bin;
  using WordT = typename Traits<T>::Bits;
  constexpr int NT = G::NT, W = Traits<T>::W;
  const int64_t gt0 = tile0 + blockIdx.x;
  const FieldInfo& fi = F[field_of_tile(F, f0, nf, gt0)];
  Params* P = fi.P;
  // in an ordered pass the blocks take the field's tiles in ascending tile key, so that a
  // tile's lower-valued neighbours, whose subbins its halo reads, have usually been
  // passed already; otherwise in index order, with halo subbins 0
  const bool ordered = P->pass_ordered != 0;
  const int64_t gt = ordered ? fi.tile_base + (int64_t)fi.order[gt0 - fi.tile_base] : gt0;
  if (P->status & kErrNonfinite) return;
  if (P->constant) return;
  const Geometry g = fi.g;
  const T* __restrict__ x = reinterpret_cast<const T*>(fi.x);
  uint32_t* __restrict__ s_glob = fi.s;
  uint32_t* __restrict__ cm_glob = fi.cm;
  int64_t* __restrict__ bins_out = fi.bins_out;
  uint8_t* __restrict__ slots = fi.slots;
  uint32_t* __restrict__ sizes = fi.sizes;
  extern __shared__ __align__(16) unsigned char smem[];
  K* key = reinterpret_cast<K*>(smem);
  uint32_t* sv = reinterpret_cast<uint32_t*>(smem);
  B* bin = reinterpret_cast<B*>(smem + PS::RA);
  uint32_t* cml = reinterpret_cast<uint32_t*>(smem + PS::RA + PS::RB);
  uint32_t* fa = reinterpret_cast<uint32_t*>(smem + PS::RA + PS::RB + PS::RC);
  uint32_t* fb = fa + G::NP / 32;
  uint32_t* rb = fb + G::NP / 32;
  unsigned* cnt = rb + G::NP / 32;
  // the fixpoint's lists, in the bins' region once they are dead: the frontier list,
  // or (for a tile that needs the topological order) in-degrees and two ready lists
  uint16_t* flist = reinterpret_cast<uint16_t*>(smem + PS::RA);
  uint32_t* indeg = reinterpret_cast<uint32_t*>(smem + PS::RA);
  uint16_t* la = reinterpret_cast<uint16_t*>(smem + PS::RA + G::NP);
  uint16_t* lb = la + FixSmem<G>::list_bytes() / 2;

  const int64_t tid = gt - fi.tile_base;
  if (tid < 0 || tid >= g.ntiles) return;  // never for a consistent plan
  const TileBox tb = tile_box(g, tid);
  const unsigned long long inv_m = P->inv_m;
  const int inv_e = P->inv_e;
  const float inv_f = P->inv_f;
  const int fast_ok = P->fast_ok;
  const int64_t plane = g.ny * g.nx;
  long long t0 = clock64();

  // 1. load x on the box with asynchronous copies (absent points read nothing), then
  //    quantize and take order keys in place (absent points get a bin no value has)
  using Raw = typename Traits<T>::Bits;
  Raw* raw = reinterpret_cast<Raw*>(smem);  // the keys' region holds the raw values first
  constexpr int NBOX = G::BZ * G::BY * G::BX;  // entries of the box (the rare error path walks them)
  load_box_async<G, Raw>(raw, reinterpret_cast<const Raw*>(x), g, tb);
  for (int i = threadIdx.x; i < 3 * (G::NP / 32); i += NT) fa[i] = 0;  // both frontiers, risen bits
  // ORs of the two predictors' mapped words: the bit planes each can reach
  __shared__ unsigned long long s_orl, s_ord;
  if (threadIdx.x == 0) {
    cnt[0] = cnt[2] = cnt[3] = 0;  // same-bin pairs; the bin predictors' costs
    s_orl = s_ord = 0ull;
  }
  cp_async_wait_all();
  __syncthreads();
  bool bad = false;
  for_box<G>(g, tb, [&](int e, bool in) {
    B b = Traits<T>::kAbsent;
    K k = 0;
    if (in) {
      const T v = Traits<T>::from_bits(raw[e]);
      long long q;
      if (is_finite_bits<T>(v) && quantize_fast<T>(v, inv_f, fast_ok, inv_m, inv_e, q) &&
          q < Traits<T>::kBinLimit && q > -Traits<T>::kBinLimit) {
        b = (B)q;
        k = order_key<T>(v);
      } else {
        bad = true;
      }
    }
    key[e] = k;
    bin[e] = b;
  });
  if (__syncthreads_or(bad)) {  // tell non-finite from out-of-range, off the fast path (whole block)
    for (int i = threadIdx.x; i < NBOX; i += NT) {
      const int lx = i % G::BX, ly = (i / G::BX) % G::BY, lz = i / (G::BX * G::BY);
      const int64_t gz = tb.z0 + lz - G::HZ, gy = tb.y0 + ly - 1, gx = tb.x0 + lx - 1;
      if (gz >= 0 && gz < g.nz && gy >= 0 && gy < g.ny && gx >= 0 && gx < g.nx) {
        const T v = x[gz * plane + gy * g.nx + gx];
        long long q;
        if (!is_finite_bits<T>(v))
          atomicOr(&P->status, kErrNonfinite);
        else if (!quantize_exact<T>(v, inv_m, inv_e, q) || q >= Traits<T>::kBinLimit || q <= -Traits<T>::kBinLimit)
          atomicOr(&P->status, kErrRange);
      }
    }
  }
  __syncthreads();
  phase_mark(P, 0, t0);

  // 2. flags of the thread's y-segment: the lower same-bin neighbours, and the upper
  //    ones inside the tile (a same-bin neighbour that is not lower is upper), which a
  //    rise requeues or the topological order releases.
  const SegPos sp = seg_pos<G>();
  const bool col_in = sp.lz < tb.cz && sp.lx < tb.cx;
  const int64_t gz = tb.z0 + sp.lz, gx = tb.x0 + sp.lx;
  unsigned same_pairs = 0;  // same-bin neighbour pairs of the thread's points
  // the bin record's predictor costs: one bits of the NB-mapped Lorenzo residuals and
  // 1D differences of the thread's points (the Lorenzo stencil's seven lower-octant
  // points are the neighbours -D[0..6] the flags load anyway)
  unsigned cost_l = 0, cost_d = 0;
  uint64_t or_l = 0, or_d = 0;
  constexpr WordT NBM = (WordT)0xAAAAAAAAAAAAAAAAULL;
#pragma unroll 1
  for (int j = 0; j < G::SEG; ++j) {
    uint32_t same = 0, lo = 0;
    const int e = sp.e0 + j * G::BXP;
    const int ly = sp.ly0 + j;
    if (col_in && ly < tb.cy) {
      const B bp = bin[e];
      const K kp = key[e];
      B nbin[14];
#pragma unroll
      for (int k = 0; k < 14; ++k) {
        if (!G::HZ && dz_of(k) != 0) continue;
        const int e2 = e + G::off(dz_of(k), dy_of(k), dx_of(k));
        nbin[k] = bin[e2];
        if (nbin[k] == bp) {
          same |= 1u << k;
          const K kn = key[e2];
          if (kn < kp || (kn == kp && k < 7)) lo |= 1u << k;
        }
      }
      const bool hx = sp.lx > 0, hy = ly > 0, hz = G::HZ && sp.lz > 0;
      WordT r = (WordT)bp;
      r -= hx ? (WordT)nbin[0] : (WordT)0;
      r -= hy ? (WordT)nbin[1] : (WordT)0;
      r += (hx && hy) ? (WordT)nbin[2] : (WordT)0;
      if (G::HZ) {
        r -= hz ? (WordT)nbin[3] : (WordT)0;
        r += (hz && hx) ? (WordT)nbin[4] : (WordT)0;
        r += (hz && hy) ? (WordT)nbin[5] : (WordT)0;
        r -= (hz && hy && hx) ? (WordT)nbin[6] : (WordT)0;
      }
      WordT prev = 0;  // the point before this one in the chunk's point order
      if (hx)
        prev = (WordT)nbin[0];
      else if (hy)
        prev = (WordT)bin[G::entry(sp.lz, ly - 1, tb.cx - 1)];
      else if (hz)
        prev = (WordT)bin[G::entry(sp.lz - 1, tb.cy - 1, tb.cx - 1)];
      const uint64_t ml = (uint64_t)((WordT)(r + NBM) ^ NBM), md = (uint64_t)((WordT)((WordT)bp - prev + NBM) ^ NBM);
      cost_l += __popcll(ml);
      cost_d += __popcll(md);
      or_l |= ml;
      or_d |= md;
    }
    const uint32_t up = same & ~lo & ~out_of_box_bits<G>(sp.lz, ly, sp.lx);
    const int o = sp.o0 + j * G::TX;
    same_pairs += __popc(same);
    cml[o] = lo | (up << 16);
    // the global copy (for reruns) keeps the lower and all the same-bin bits
    if (col_in && ly < tb.cy) cm_glob[gz * plane + (tb.y0 + ly) * g.nx + gx] = lo | (same << 16);
    // first-frontier bits: the tile's own subbins start at 0, so a point can rise first
    // only through a +1 constraint or, in an ordered pass, a lower neighbour outside the
    // tile (whose subbin the halo holds); one ballot per warp: a row of lanes holds
    // consecutive points
    const uint32_t bal = __ballot_sync(
        0xffffffffu, (lo >> 7) != 0 || (ordered && (lo & out_of_box_bits<G>(sp.lz, ly, sp.lx)) != 0));
    if (G::TX >= 32) {
      if ((threadIdx.x & 31) == 0 && bal) atomicOr(&fa[o >> 5], bal);
    } else if ((threadIdx.x & 15) == 0) {
      const uint32_t half = (bal >> (threadIdx.x & 16)) & 0xFFFFu;
      if (half) atomicOr(&fa[o >> 5], half << (o & 31));
    }
  }
  if (bins_out && col_in) {
    for (int j = 0; j < G::SEG && sp.ly0 + j < tb.cy; ++j)
      bins_out[gz * plane + (tb.y0 + sp.ly0 + j) * g.nx + gx] = (int64_t)bin[sp.e0 + j * G::BXP];
  }
  {
    const unsigned wsum = __reduce_add_sync(0xffffffffu, same_pairs);
    const unsigned wl = __reduce_add_sync(0xffffffffu, cost_l), wd = __reduce_add_sync(0xffffffffu, cost_d);

    if ((threadIdx.x & 31) == 0) {
      atomicAdd(&cnt[0], wsum);
      atomicAdd(&cnt[2], wl);
      atomicAdd(&cnt[3], wd);
    }
    block_or_into(or_l, &s_orl);
    block_or_into(or_d, &s_ord);
  }
  __syncthreads();  // keys are dead from here on
  // same-bin pairs over the tile's points, against 16ths of the neighbour pairs a full
  // tile has (each pair is seen from both ends)
  const unsigned pairs_full = (unsigned)G::NP * (G::HZ ? 14u : 6u);
  const bool dense_tile = (unsigned long long)cnt[0] * 16ull > (unsigned long long)pairs_full * dense16;
  phase_mark(P, 1, t0);

  // 3. bin record (format 2): a predictor's residual, NB-mapped, BIT_w, RZE_1; raw if
  //    that is not shorter.  The predictor is the chunk's Lorenzo residual (bins
  //    outside the chunk count as 0), or the 1D difference along the chunk's point
  //    order when its mapped words hold strictly fewer one bits.
  {
    const int n = tb.n, n32 = (n + 31) & ~31;
    const uint32_t raw = (uint32_t)n * W;
    const bool full = n == G::NP;
    auto coords = [&](int i, int& lz2, int& ly2, int& lx2) {
      if (full) {
        lx2 = i % G::TX;
        ly2 = (i / G::TX) % G::TY;
        lz2 = i / (G::TX * G::TY);
      } else {
        lx2 = i % tb.cx;
        ly2 = (i / tb.cx) % tb.cy;
        lz2 = i / (tb.cx * tb.cy);
      }
    };
    auto bin_of = [&](int i) -> WordT {
      int lx2, ly2, lz2;
      coords(i, lz2, ly2, lx2);
      return (WordT)bin[G::entry(lz2, ly2, lx2)];
    };
    auto diff_of = [&](int i) -> WordT { return bin_of(i) - (i ? bin_of(i - 1) : (WordT)0); };
    // sum over (a, b, c) in {0,1}^3 of (-1)^(a+b+c) bins[z-a][y-b][x-c], in the chunk
    auto lorenzo_of = [&](int i) -> WordT {
      int lx2, ly2, lz2;
      coords(i, lz2, ly2, lx2);
      const int e = G::entry(lz2, ly2, lx2);
      const bool hx = lx2 > 0, hy = ly2 > 0;
      WordT r = (WordT)bin[e];
      r -= hx ? (WordT)bin[e - 1] : (WordT)0;
      r -= hy ? (WordT)bin[e - G::BXP] : (WordT)0;
      r += (hx && hy) ? (WordT)bin[e - G::BXP - 1] : (WordT)0;
      if (G::HZ && lz2 > 0) {
        const int ez = e - G::PP;
        r -= (WordT)bin[ez];
        r += hx ? (WordT)bin[ez - 1] : (WordT)0;
        r += hy ? (WordT)bin[ez - G::BXP] : (WordT)0;
        r -= (hx && hy) ? (WordT)bin[ez - G::BXP - 1] : (WordT)0;
      }
      return r;
    };
    constexpr WordT M = (WordT)0xAAAAAAAAAAAAAAAAULL;
    auto nb = [&](WordT d) -> uint64_t { return (uint64_t)((WordT)(d + M) ^ M); };
    const bool use_diff = cnt[3] < cnt[2];  // the costs summed during the flags
    uint32_t* planes = reinterpret_cast<uint32_t*>(smem);
    const RzeWork w = rze_work_at(smem + PS::L, PS::L);
    // planes above those the chosen predictor's mapped words reach (their OR, taken
    // during the flags) are zero: the transpose packs the planes below, and the coder
    // does not read the rest
    const int Pnz = planes_of(use_diff ? s_ord : s_orl);
    bit_transpose_planes<NT, W>(n32, Pnz, [&](int i) -> uint64_t {
      if (i >= n) return 0;
      return nb(use_diff ? diff_of(i) : lorenzo_of(i));
    }, planes);
    __syncthreads();
    uint8_t* slot = slots + (size_t)tid * kSlotBytes;
    uint8_t* stage = reinterpret_cast<uint8_t*>(bin);  // bins are dead once the record is written
    const uint32_t Lnz = plane_bytes_of(n32, Pnz, (uint32_t)W * n32);
    const uint32_t len = rze_encode<NT, 1>(reinterpret_cast<const uint8_t*>(planes), W * n32, stage, raw, w, Lnz);
    if (len >= raw) {  // nothing was staged: bins are intact
      for (int i = threadIdx.x; i < n; i += NT) reinterpret_cast<WordT*>(slot)[i] = bin_of(i);
      if (threadIdx.x == 0) sizes[tid] = raw | kRawFlag;
    } else {
      zero_tail16<NT>(stage, len);
      __syncthreads();
      copy16<NT>(slot, stage, len);
      if (threadIdx.x == 0) sizes[tid] = len | (use_diff ? kDiffFlag : 0u);
    }
  }
  __syncthreads();  // bins, planes and the staged record are dead from here on
  phase_mark(P, 4, t0);

  // 4. tile-local least fixpoint from subbins 0 on the tile and, on the halo of an
  //    ordered pass, the subbins neighbours have written so far (cleared before the
  //    pass; any value read is a lower bound, so the result is one too)
  for (int e = threadIdx.x; e < G::E; e += NT) sv[e] = 0;
  __syncthreads();
  if (fix && ordered) {
    // only neighbour tiles passed before this one (lower rank) have written subbins
    __shared__ uint32_t earlier;  // bit (dz+1)*9 + (dy+1)*3 + (dx+1) per neighbour tile
    if (threadIdx.x == 0) earlier = 0u;
    __syncthreads();
    const int64_t tz = tid / (g.ntx * g.nty), ty = (tid / g.ntx) % g.nty, tx = tid % g.ntx;
    const uint32_t my_rank = gt0 - fi.tile_base;
    if (threadIdx.x < 27) {
      const int dz = threadIdx.x / 9 - 1, dy = (threadIdx.x / 3) % 3 - 1, dx = threadIdx.x % 3 - 1;
      const int64_t nz_ = tz + dz, ny_ = ty + dy, nx_ = tx + dx;
      if ((dz | dy | dx) != 0 && (G::HZ || dz == 0) && nz_ >= 0 && nz_ < g.ntz && ny_ >= 0 && ny_ < g.nty &&
          nx_ >= 0 && nx_ < g.ntx && fi.rank[(nz_ * g.nty + ny_) * g.ntx + nx_] < my_rank)
        atomicOr(&earlier, 1u << threadIdx.x);
    }
    __syncthreads();
    const uint32_t ebits = earlier;
    if (ebits) {
      constexpr int NZF = G::HZ ? 2 * G::BY * G::BX : 0;  // z faces (whole planes)
      constexpr int NYF = 2 * G::TZ * G::BX;              // y faces of the tile's planes
      constexpr int NXF = 2 * G::TZ * G::TY;              // x faces of the tile's rows
      // from L2 (other blocks write them during the pass), several loads in flight
      gather_l2<NT, 4, uint32_t>(sv, NZF + NYF + NXF, [&](int i, int& d, const uint32_t*& sp) {
        int lz, ly, lx;
        if (i < NZF) {
          const int r = i % (G::BY * G::BX);
          lz = i < G::BY * G::BX ? -1 : G::TZ;
          ly = r / G::BX - 1;
          lx = r % G::BX - 1;
        } else if (i < NZF + NYF) {
          const int jj = i - NZF, r = jj % (G::TZ * G::BX);
          lz = r / G::BX;
          ly = jj < G::TZ * G::BX ? -1 : G::TY;
          lx = r % G::BX - 1;
        } else {
          const int jj = i - NZF - NYF, r = jj % (G::TZ * G::TY);
          lz = r / G::TY;
          ly = r % G::TY;
          lx = jj < G::TZ * G::TY ? -1 : G::TX;
        }
        // a later tile's subbins are still 0, as the entry is: neither is read
        const int64_t qz = tb.z0 + lz, qy = tb.y0 + ly, qx = tb.x0 + lx;
        if ((ebits & tile_dir_bit<G>(lz, ly, lx)) && qz >= 0 && qz < g.nz && qy >= 0 && qy < g.ny && qx >= 0 &&
            qx < g.nx) {
          d = G::entry(lz, ly, lx);
          sp = &s_glob[qz * plane + qy * g.nx + qx];
        }
      });
    }
    __syncthreads();
  }
  // frontier sweeps (cheaper while chains are short), and for a tile whose chains
  // outlast the evaluation budget (budget16 / 16 evaluations per point) the
  // topological order, which evaluates each point once, from the values reached so
  // far (lower bounds of the result)
  unsigned evals = 0, raises = 0;
  bool over = false;
  int iters = 0;
  // a tile whose neighbour pairs are mostly same-bin (thick bins, long chains) takes
  // the topological order at once
  if (fix && !dense_tile) {
    iters = frontier_fixpoint<G, false>(sv, cml, fa, fb, rb, cnt, flist, 4 * G::NP + 64, over, evals, raises,
                                        (unsigned)G::NP * budget16 / 16u);
  }
  if (fix && (over || dense_tile)) {
    __syncthreads();
    iters += topo_fixpoint<G, false>(sv, cml, indeg, la, lb, cnt, tb, nullptr, evals, raises);
  }
  if (threadIdx.x == 0) {
    atomicAdd(&P->fix_iters, (unsigned long long)iters);
    atomicMax(&P->fix_iters_max, (unsigned long long)iters);
  }
  block_add2(evals, raises, &P->work[0]);
  phase_mark(P, 2, t0);

  // 5. write the subbins reruns start from (cross-tile constraints are checked afterwards)
  if (col_in) {
#pragma unroll 4
    for (int j = 0; j < G::SEG; ++j) {
      if (sp.ly0 + j >= tb.cy) break;
      const int e = sp.e0 + j * G::BXP;
      const int64_t gi = gz * plane + (tb.y0 + sp.ly0 + j) * g.nx + gx;
      s_glob[gi] = sv[e];
    }
  }
  phase_mark(P, 3, t0);
}

template <typename T, int ND>
struct RerunSmem {
  using G = TileGeom<T, ND, true>;
  static constexpr size_t up16(size_t v) { return (v + 15) & ~(size_t)15; }
  static constexpr size_t CM = (size_t)G::E * 4;                      // subbins, then lower masks
  static constexpr size_t BITS = CM + up16((size_t)G::NP * 4);        // frontiers, risen bits, counters
  static constexpr size_t LIST = BITS + up16(FixSmem<G>::bits_bytes());
  static constexpr size_t bytes() { return LIST + FixSmem<G>::list_bytes(); }
};

// Rerun of a tile whose halo subbins may have risen: the stored lower-neighbour
// masks and the current subbins of the tile and its halo are all it needs.  After
// the pass every tile holds its tile-local least fixpoint with halo subbins 0, so
// the first round visits every tile (list == nullptr); later rounds visit the tiles
// marked by the round before.  The first frontier is the boundary points whose
// constraint from a lower same-bin neighbour in another tile is violated; a tile
// without one returns at once.  Writes the subbins that rose and marks the tiles
// whose constraints from risen boundary points are now violated.
template <typename T, int ND>
__global__ void __launch_bounds__(TileCfg<T, ND>::NT, TileCfg<T, ND>::MINB_RERUN)
    k_rerun(const FieldInfo* __restrict__ F, int f0, int nf, int64_t tile0, int64_t ntile_cls, int cls,
            BatchState* __restrict__ B, const uint32_t* __restrict__ list, uint32_t* __restrict__ app) {
  using G = TileGeom<T, ND, true>;  // interior rows on 16-byte boundaries
  using RS = RerunSmem<T, ND>;
  constexpr int NT = G::NT;
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t* sv = reinterpret_cast<uint32_t*>(smem);
  uint32_t* cm = reinterpret_cast<uint32_t*>(smem + RS::CM);
  uint32_t* fa0 = reinterpret_cast<uint32_t*>(smem + RS::BITS);
  uint32_t* rb = fa0 + 2 * (G::NP / 32);
  unsigned* cnt = rb + G::NP / 32;
  uint16_t* flist = reinterpret_cast<uint16_t*>(smem + RS::LIST);
  __shared__ uint32_t marks;
  __shared__ unsigned s_item, s_claimed, s_lim;
  __shared__ long long s_app_gt;
  // the first round (list == nullptr) visits every tile of the class; blocks take
  // items from a counter, so a slow tile holds up only its own block.  Items past the
  // list are tiles that reruns of this round marked (app, the class's segment of a
  // table-wide array): a block takes them while any are left and never waits, and a
  // tile marked after the last block has gone keeps its flag for the next round.
  const int64_t count = list ? (int64_t)B->count[cls] : ntile_cls;
  const uint32_t* lst = list ? list + B->off[cls] : nullptr;
  unsigned* next = list ? &B->next[cls] : &B->next_all[cls];
  uint32_t* app_seg = app ? app + tile0 : nullptr;
  volatile unsigned* napp = &B->app[cls];
  // thread 0 takes the following item while the block works on this one, so the
  // counter's latency is hidden
  unsigned ahead = 0;
  if (threadIdx.x == 0) ahead = atomicAdd(next, 1u);
#pragma unroll 1
  while (true) {
    if (threadIdx.x == 0) {
      const long long appended = app_seg ? (long long)min(*napp, (unsigned)ntile_cls) : 0ll;
      const long long lim = (long long)count + appended;
      long long agt = -1;
      if ((long long)ahead < lim) {
        // an appended tile, read once for the block (the entry may not be written yet:
        // then it is stale and checked below, and the tile itself keeps its flag)
        if ((long long)ahead >= count) agt = (long long)reinterpret_cast<volatile uint32_t*>(app_seg)[ahead - count];
      }
      s_item = ahead;
      s_lim = (unsigned)lim;  // count + appended <= 2 * the class's tiles < 2^32
      s_app_gt = agt;
      if ((long long)ahead < lim) ahead = atomicAdd(next, 1u);
    }
    __syncthreads();  // also: the last item's shared state is no longer read
    const int64_t item = (int64_t)s_item;
    const int64_t lim = (int64_t)s_lim;
    const int64_t agt = (int64_t)s_app_gt;
    __syncthreads();  // s_item is rewritten for the next item
    if (item >= lim) break;
    int64_t gt;
    if (item < count) {
      gt = lst ? (int64_t)lst[item] : tile0 + item;
    } else {
      gt = agt;
      if (gt < tile0 || gt >= tile0 + ntile_cls) continue;  // uniform per block
    }
    const FieldInfo& fi = F[field_of_tile(F, f0, nf, gt)];
    if (!lst && item < count) gt = fi.tile_base + (int64_t)fi.order[gt - fi.tile_base];  // in ascending tile key
    Params* P = fi.P;
    if ((P->status & kErrNonfinite) || P->constant) continue;  // uniform per block
    if (app_seg) {
      // claim the tile: clear its flag, so that a mark from now on queues it again; an
      // appended copy whose flag is already clear was taken by another block
      if (threadIdx.x == 0) {
        const uint32_t r = fi.rank[gt - fi.tile_base], sh = 8u * (r & 3u);
        const uint32_t old = atomicAnd(&fi.dirty[r >> 2], ~(0xFFu << sh));
        __threadfence();  // a marker's raised subbins, fenced before its flag, are read after this
        s_claimed = (old >> sh) & 0xFFu;
      }
      __syncthreads();
      const bool claimed = s_claimed != 0u;
      __syncthreads();
      if (item >= count && !claimed) continue;
    }
    const Geometry g = fi.g;
    uint32_t* __restrict__ s_glob = fi.s;
    const uint32_t* __restrict__ cm_glob = fi.cm;
    uint32_t* fa = fa0;
    uint32_t* fb = fa0 + G::NP / 32;
    const int64_t tid = gt - fi.tile_base;
    if (tid < 0 || tid >= g.ntiles) continue;  // never for a consistent plan (uniform per block)
    const TileBox tb = tile_box(g, tid);
    const int64_t plane = g.ny * g.nx;
    long long t0 = clock64();
    // subbins of the box and lower masks of the tile's own points, by asynchronous
    // copies (absent points read nothing and are zero)
    load_box_async<G, uint32_t, true>(sv, s_glob, g, tb);  // other blocks of this round raise subbins
    if ((g.nx & 3) == 0) {  // four masks per 16-byte copy (a copy is wholly inside or outside)
      for (int i = threadIdx.x; i < G::NP / 4; i += NT) {
        const int o = 4 * i;
        const int lx = o % G::TX, ly = (o / G::TX) % G::TY, lz = o / (G::TX * G::TY);
        const bool in = lz < tb.cz && ly < tb.cy && lx < tb.cx;
        const int64_t gi = (tb.z0 + lz) * plane + (tb.y0 + ly) * g.nx + tb.x0 + lx;
        const unsigned d = (unsigned)__cvta_generic_to_shared(&cm[o]);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(in ? &cm_glob[gi] : cm_glob),
                     "r"(in ? 16 : 0)
                     : "memory");
      }
    } else {
      for (int o = threadIdx.x; o < G::NP; o += NT) {
        const int lx = o % G::TX, ly = (o / G::TX) % G::TY, lz = o / (G::TX * G::TY);
        const bool in = lz < tb.cz && ly < tb.cy && lx < tb.cx;
        const int64_t gi = (tb.z0 + lz) * plane + (tb.y0 + ly) * g.nx + tb.x0 + lx;
        cp_async4(&cm[o], in ? &cm_glob[gi] : cm_glob, in);
      }
    }
    for (int i = threadIdx.x; i < 3 * (G::NP / 32); i += NT) fa0[i] = 0;  // frontiers, risen bits
    uint32_t nb_rank = ~0u;  // thread d < 27: rank of neighbour tile d (~0u: none), for marking
    if (threadIdx.x < 27) {
      const int64_t nt = threadIdx.x == 13 ? -1 : neighbour_tile(g, tid, threadIdx.x);
      if (nt >= 0) nb_rank = fi.rank[nt];
    }
    if (threadIdx.x == 0) marks = 0u;
    cp_async_wait_all();
    __syncthreads();
    const SegPos sp = seg_pos<G>();
    const bool col_in = sp.lz < tb.cz && sp.lx < tb.cx;
    // the first frontier: boundary points whose constraint from a lower same-bin
    // neighbour outside the tile is violated by the current subbins (points outside
    // a clipped tile are out of the domain: their masks were loaded as 0)
    bool first = false;
    if (col_in) {
#pragma unroll 1
      for (int j = 0; j < G::SEG; ++j) {
        const int e = sp.e0 + j * G::BXP;
        const int o = sp.o0 + j * G::TX;
        const uint32_t mo = cm[o] & out_of_box_bits<G>(sp.lz, sp.ly0 + j, sp.lx);
        if (!mo) continue;
        const uint32_t sp_ = sv[e];
        bool viol = false;
#pragma unroll
        for (int k = 0; k < 14; ++k) {
          if ((mo >> k) & 1u) {
            if (sv[e + G::off(dz_of(k), dy_of(k), dx_of(k))] + (k >= 7 ? 1u : 0u) > sp_) viol = true;
          }
        }
        if (viol) {
          atomicOr(&fa[o >> 5], 1u << (o & 31));
          first = true;
        }
      }
    }
    const bool idle = !__syncthreads_or(first);
    if (threadIdx.x == 0) {
      atomicAdd(&P->work[4], 1ull);
      if (idle) atomicAdd(&P->work[5], 1ull);
    }
    if (idle) {  // every constraint into this tile holds
      phase_mark(P, 7, t0);
      continue;
    }
    phase_mark(P, 5, t0);
    bool over = false;
    unsigned evals = 0, raises = 0;
    const int iters = frontier_fixpoint<G, true>(sv, cm, fa, fb, rb, cnt, flist, 4 * G::NP + 64, over, evals, raises);
    uint32_t risen = 0;  // the thread's segment points that rose
    for (int j = 0; j < G::SEG; ++j) {
      const int o = sp.o0 + j * G::TX;
      risen |= ((rb[o >> 5] >> (o & 31)) & 1u) << j;
    }
    if (threadIdx.x == 0) {
      if (over) atomicOr(&P->status, kErrNotConverged);
      atomicAdd(&P->fix_iters, (unsigned long long)iters);
      atomicMax(&P->fix_iters_max, (unsigned long long)iters);
    }
    block_add2(evals, raises, &P->work[2]);
    phase_mark(P, 6, t0);
    // write the subbins that rose.  With appended tiles two blocks can hold the same
    // tile at once, each from its own snapshot: the write takes the larger value, and
    // the elementwise max of two tile-local fixpoints is again one (each is a lower
    // bound of the least fixpoint)
    const int64_t gz = tb.z0 + sp.lz, gx = tb.x0 + sp.lx;
    if (col_in && risen) {
#pragma unroll 1
      for (int j = 0; j < G::SEG; ++j) {
        if (!((risen >> j) & 1u)) continue;
        const int ly = sp.ly0 + j;
        atomicMax(&s_glob[gz * plane + (tb.y0 + ly) * g.nx + gx], sv[sp.e0 + j * G::BXP]);
      }
    }
    // the neighbour tiles to mark: those holding an upper same-bin neighbour q of a
    // risen boundary point p whose constraint s(q) >= s(p) + [p after q] no longer
    // holds.  q's subbin is read from the halo loaded at the start: it can only have
    // risen since, so a tile is sometimes marked when it need not be (its rerun then
    // finds every constraint held) but never missed.
    const uint32_t mine = risen ? violated_tile_bits<G>(sv, tb, sp.lz, sp.ly0, sp.lx, sp.e0, sp.o0,
                                                        [&](int o) { return cm[o]; },
                                                        [&](int j) { return ((risen >> j) & 1u) != 0u; })
                                : 0u;
    if (mine) atomicOr(&marks, mine);
    __threadfence();  // the raised subbins are visible before any tile is marked
    __syncthreads();
    if (threadIdx.x < 27 && ((marks >> threadIdx.x) & 1u) && nb_rank != ~0u) {
      const uint32_t r = nb_rank;
      if (!app_seg) {
        reinterpret_cast<volatile uint8_t*>(fi.dirty)[r] = 1;  // every writer stores the same value
      } else {
        // newly dirty: also offer the tile to this round
        const uint32_t sh = 8u * (r & 3u);
        const uint32_t old = atomicOr(&fi.dirty[r >> 2], 1u << sh);
        if (!((old >> sh) & 0xFFu)) {
          const unsigned pos = atomicAdd(&B->app[cls], 1u);
          if ((int64_t)pos < ntile_cls) app_seg[pos] = (uint32_t)(fi.tile_base + fi.order[r]);
        }
      }
    }
    phase_mark(P, 8, t0);  // the next item's first barrier separates this item's reads from its writes
  }
}

// Dirty flags -> the next round's list (one block).  Flags are kept per rank (a
// tile's position in its field's rerun order, ascending tile key), so the list holds
// the fields in table order and each field's tiles in rerun order: within a round a
// tile is then usually visited after the lower-valued tiles its constraints come
// from.  Per class the count and first position, flags cleared.  The table is sorted
// by class, so the list is grouped by class.  Counts a round for every field of the
// table; a field past its round cap drops its dirty tiles and is reported as not
// converged.  field_counts (optional, one per table entry) receives how many tiles
// each field has in the list: 0 means its subbins are final.  Tells the graph's
// while-node whether to run another round.
template <int NT>
__global__ void __launch_bounds__(NT) k_compact(const FieldInfo* __restrict__ F, int nf, int64_t total_words,
                                                uint32_t* __restrict__ list, BatchState* B,
                                                unsigned int* __restrict__ field_counts,
                                                cudaGraphConditionalHandle handle, int use_handle) {
  __shared__ unsigned int tmp[NT / 32 + 1];
  __shared__ unsigned int cnt[4];
  __shared__ int capped;
  if (threadIdx.x < 4) cnt[threadIdx.x] = 0;
  if (threadIdx.x == 0) capped = 0;
  for (int f = threadIdx.x; f < nf; f += NT) {
    F[f].P->rounds += 1;
    if (field_counts) field_counts[f] = 0;
  }
  __syncthreads();
  // each thread owns a contiguous range of flag words: count, one scan, then list
  const int64_t per = (total_words + NT - 1) / NT;
  const int64_t a = min(total_words, (int64_t)threadIdx.x * per), b = min(total_words, a + per);
  auto bits_of = [](uint32_t v) {  // four byte flags -> four bits
    return (v & 0xffu ? 1u : 0u) | (v & 0xff00u ? 2u : 0u) | (v & 0xff0000u ? 4u : 0u) | (v & 0xff000000u ? 8u : 0u);
  };
  // the thread's words are read KW at a time, every load of a batch in flight before
  // any is used, with the field of each; a thread with at most KW words keeps them in
  // registers for the listing pass
  constexpr int KW = 8;
  uint32_t v[KW];
  int fk[KW];
  int k = a < b ? field_of_word(F, nf, a) : 0;
  auto batch = [&](int64_t w0) {
#pragma unroll
    for (int u = 0; u < KW; ++u) {
      const int64_t w = w0 + u;
      v[u] = 0u;
      fk[u] = k;
      if (w < b) {
        while (k + 1 < nf && F[k + 1].word_base <= w) ++k;
        fk[u] = k;
        v[u] = F[k].dirty[w - F[k].word_base];
      }
    }
  };
  int lf = -1;  // the field whose round-cap verdict `live` holds
  bool live = false;
  auto live_of = [&](int f) {
    if (f != lf) {
      lf = f;
      live = (long long)F[f].P->rounds <= F[f].round_cap;
    }
    return live;
  };
  unsigned int n = 0;
  for (int64_t w0 = a; w0 < b; w0 += KW) {
    batch(w0);
#pragma unroll
    for (int u = 0; u < KW; ++u)
      if (v[u] && live_of(fk[u])) n += __popc(bits_of(v[u]));
  }
  const bool kept = b - a <= KW;
  unsigned int tot;
  unsigned int pos = block_exclusive_scan<NT, unsigned int>(n, tmp, &tot);
  k = a < b ? field_of_word(F, nf, a) : 0;
  for (int64_t w0 = a; w0 < b; w0 += KW) {
    if (!kept) batch(w0);
#pragma unroll
    for (int u = 0; u < KW; ++u) {
      if (!v[u]) continue;
      const int f = fk[u];
      const int64_t wl = w0 + u - F[f].word_base;  // the word within its field
      F[f].dirty[wl] = 0u;
      if (!live_of(f)) {  // past the cap: drop the tiles, fail the field
        atomicOr(&F[f].P->status, kErrNotConverged);
        capped = 1;
        continue;
      }
      const uint32_t bits = bits_of(v[u]);
      const uint32_t* ord = F[f].order + 4 * wl;  // the word's first rank
      const int64_t base = F[f].tile_base;
      for (uint32_t bb = bits; bb; bb &= bb - 1) list[pos++] = (uint32_t)(base + ord[__ffs(bb) - 1]);
      const unsigned int c = __popc(bits);
      atomicAdd(&cnt[class_of_geometry(F[f].g)], c);
      if (field_counts) atomicAdd(&field_counts[f], c);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned int o = 0;
    for (int c = 0; c < 4; ++c) {
      B->count[c] = cnt[c];
      B->off[c] = o;
      B->next[c] = 0;
      B->app[c] = 0;
      o += cnt[c];
    }
    B->rounds += 1;
    B->runs += tot;
    B->cap_hit |= (unsigned int)capped;
    if (use_handle) cudaGraphSetConditional(handle, tot ? 1u : 0u);
  }
}

// Tile keys for the rerun order: the top 32 bits of the smallest order key among 64
// sample points of the tile (a 4 x 4 x 4 grid over the clipped tile, 8 x 8 in 2D); one
// block of 64 threads per tile.  Only an approximate value order is needed.  The block
// also measures how many bins the samples span, (max - min) * inv clamped to
// kSpanClamp bins, in sixteenths of a bin, and leaves it in rank[tile] for k_order.
constexpr unsigned kSpanClamp = 256;
template <typename T, int ND>
__global__ void __launch_bounds__(64) k_tile_keys(const FieldInfo* __restrict__ F, int f0, int nf, int64_t tile0) {
  using K = typename Traits<T>::Key;
  __shared__ uint32_t wmin[2], wmax[2];
  const int64_t gt = tile0 + blockIdx.x;
  const FieldInfo& fi = F[field_of_tile(F, f0, nf, gt)];
  const int64_t tid = gt - fi.tile_base;
  const Geometry g = fi.g;
  if (tid < 0 || tid >= g.ntiles) return;  // never for a consistent plan
  const TileBox tb = tile_box(g, tid);
  const int t = threadIdx.x;
  int lz, ly, lx;
  if (ND == 3) {
    lz = (t >> 4) * (tb.cz - 1) / 3;
    ly = ((t >> 2) & 3) * (tb.cy - 1) / 3;
    lx = (t & 3) * (tb.cx - 1) / 3;
  } else {
    lz = 0;
    ly = (t >> 3) * (tb.cy - 1) / 7;
    lx = (t & 7) * (tb.cx - 1) / 7;
  }
  constexpr uint64_t kBias = sizeof(K) == 4 ? 0x80000000ull : 0x8000000000000000ull;
  constexpr int kShift = 8 * (int)sizeof(K) - 32;
  const T v = reinterpret_cast<const T*>(fi.x)[((tb.z0 + lz) * g.ny + tb.y0 + ly) * g.nx + tb.x0 + lx];
  uint32_t kmin = 0xFFFFFFFFu, kmax = 0u;  // top 32 bits of the biased order keys
  if (is_finite_bits<T>(v)) kmin = kmax = (uint32_t)(((uint64_t)order_key<T>(v) ^ kBias) >> kShift);
  kmin = __reduce_min_sync(0xffffffffu, kmin);
  kmax = __reduce_max_sync(0xffffffffu, kmax);
  if ((t & 31) == 0) {
    wmin[t >> 5] = kmin;
    wmax[t >> 5] = kmax;
  }
  __syncthreads();
  if (t == 0) {
    kmin = wmin[0] < wmin[1] ? wmin[0] : wmin[1];
    kmax = wmax[0] > wmax[1] ? wmax[0] : wmax[1];
    fi.tkey[tid] = kmin;
    double c = 0.0;  // constant fields (inv undefined) and tiles without finite samples count as 0
    const Params* P = fi.P;
    if (kmin <= kmax && !P->constant) {
      // the keys' dropped low bits (f64) only round the span down a little
      const double lo = (double)value_of_key<T>((K)((((uint64_t)kmin) << kShift) ^ kBias));
      const double hi = (double)value_of_key<T>((K)((((uint64_t)kmax) << kShift) ^ kBias));
      const double span = (hi - lo) * P->inv;
      c = span >= 0.0 ? fmin(span, (double)kSpanClamp) : 0.0;
    }
    fi.rank[tid] = (uint32_t)(c * 16.0);
  }
}

// Mean sample span (k_tile_keys), in bins, below which the tile pass of a field takes
// its tiles in tile-key order: thick bins relative to a tile's values, so same-bin
// chains cross many tile faces and a halo read from lower-valued neighbours already
// passed saves rerun rounds.  With thin bins the chains end inside their tiles, and
// the index order keeps neighbouring boxes in L2.
constexpr unsigned kOrderedSpan = 48;

// pass_order: two bits per field class (0 f32 2D, 1 f32 3D, 2 f64 2D, 3 f64 3D): 0 the
// span decides, 1 index order, 2 tile-key order.
template <int NT>
__global__ void __launch_bounds__(NT) k_order(const FieldInfo* __restrict__ F, unsigned pass_order) {
  constexpr int NB = 4096, PER = NB / NT;
  static_assert(NB % NT == 0, "whole bucket runs per thread");
  __shared__ unsigned int hist[NB];
  __shared__ unsigned int tmp[NT / 32 + 1];
  __shared__ unsigned int red[2][NT / 32];
  const FieldInfo& fi = F[blockIdx.x];
  const int64_t n = fi.g.ntiles;
  uint32_t* __restrict__ order = fi.order;
  uint32_t* __restrict__ rank = fi.rank;
  const uint32_t* __restrict__ tkey = fi.tkey;
  if (fi.P->constant || (fi.P->status & kErrNonfinite)) {
    for (int64_t t = threadIdx.x; t < n; t += NT) order[t] = rank[t] = (uint32_t)t;
    if (threadIdx.x == 0) fi.P->pass_ordered = 0u;
    return;
  }
  // every pass over the tiles reads KB keys per thread at a time, all in flight together
  constexpr int KB = 8;
  uint32_t lo = 0xFFFFFFFFu, hi = 0u;
  unsigned long long span16 = 0;  // sum of the tiles' sample spans (sixteenths of a bin)
  for (int64_t t0 = threadIdx.x; t0 < n; t0 += (int64_t)KB * NT) {
    uint32_t k[KB], sp[KB];
#pragma unroll
    for (int u = 0; u < KB; ++u) {
      const int64_t t = t0 + (int64_t)u * NT;
      k[u] = t < n ? tkey[t] : lo;
      sp[u] = t < n ? rank[t] : 0u;
    }
#pragma unroll
    for (int u = 0; u < KB; ++u) {
      if (t0 + (int64_t)u * NT >= n) break;
      lo = k[u] < lo ? k[u] : lo;
      hi = k[u] > hi ? k[u] : hi;
      span16 += sp[u];
    }
  }
  {
    __shared__ unsigned long long tmp64[NT / 32 + 1];
    unsigned long long tot;
    block_exclusive_scan<NT, unsigned long long>(span16, tmp64, &tot);
    if (threadIdx.x == 0) {
      const int cls = 2 * (fi.g.dtype == 1) + (fi.g.ndim == 3);
      const unsigned mode = (pass_order >> (2 * cls)) & 3u;
      fi.P->pass_ordered = mode == 2u || (mode == 0u && tot < 16ull * kOrderedSpan * (unsigned long long)n);
    }
  }
  lo = __reduce_min_sync(0xffffffffu, lo);
  hi = __reduce_max_sync(0xffffffffu, hi);
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = lo;
    red[1][threadIdx.x >> 5] = hi;
  }
  for (int i = threadIdx.x; i < NB; i += NT) hist[i] = 0u;
  __syncthreads();
  lo = red[0][0];
  hi = red[1][0];
  for (int w = 1; w < NT / 32; ++w) {
    lo = red[0][w] < lo ? red[0][w] : lo;
    hi = red[1][w] > hi ? red[1][w] : hi;
  }
  const uint64_t span = (uint64_t)(hi - lo) + 1u;
  auto bucket = [&](uint32_t k) { return (unsigned int)(((uint64_t)(k - lo) * NB) / span); };
  for (int64_t t0 = threadIdx.x; t0 < n; t0 += (int64_t)KB * NT) {
    uint32_t k[KB];
#pragma unroll
    for (int u = 0; u < KB; ++u) {
      const int64_t t = t0 + (int64_t)u * NT;
      k[u] = t < n ? tkey[t] : 0u;
    }
#pragma unroll
    for (int u = 0; u < KB; ++u)
      if (t0 + (int64_t)u * NT < n) atomicAdd(&hist[bucket(k[u])], 1u);
  }
  __syncthreads();
  unsigned int v[PER], sum = 0;
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    v[u] = hist[PER * threadIdx.x + u];
    sum += v[u];
  }
  unsigned int total;
  unsigned int start = block_exclusive_scan<NT, unsigned int>(sum, tmp, &total);
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    hist[PER * threadIdx.x + u] = start;  // first position of the bucket
    start += v[u];
  }
  __syncthreads();
  for (int64_t t0 = threadIdx.x; t0 < n; t0 += (int64_t)KB * NT) {
    uint32_t k[KB];
#pragma unroll
    for (int u = 0; u < KB; ++u) {
      const int64_t t = t0 + (int64_t)u * NT;
      k[u] = t < n ? tkey[t] : 0u;
    }
#pragma unroll
    for (int u = 0; u < KB; ++u) {
      const int64_t t = t0 + (int64_t)u * NT;
      if (t >= n) break;
      const unsigned int r = atomicAdd(&hist[bucket(k[u])], 1u);
      order[r] = (uint32_t)t;
      rank[t] = r;
    }
  }
}

// Clears the subbins of every field whose tile pass is ordered (the pass reads its
// neighbours' subbins as they are written, so unwritten ones must read 0); other
// fields' passes write every subbin before anything reads it.  blockIdx.y is the field.
__global__ void __launch_bounds__(256) k_clear_subbins(const FieldInfo* __restrict__ F) {
  const FieldInfo& f = F[blockIdx.y];
  if (!f.P->pass_ordered) return;
  const int64_t n = f.g.nz * f.g.ny * f.g.nx;
  uint32_t* __restrict__ s = f.s;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n4 = ((uintptr_t)s & 15u) ? 0 : n / 4;  // 16-byte stores where aligned
  for (int64_t i = i0; i < n4; i += stride) reinterpret_cast<uint4*>(s)[i] = make_uint4(0u, 0u, 0u, 0u);
  for (int64_t i = n4 * 4 + i0; i < n; i += stride) s[i] = 0u;
}

// ----------------------------------------------------------------- subbin encoder

// A raw subbin record: the tile's subbins as words, in the chunk's point order (kept
// out of line: the encoder's registers are budgeted for five blocks per SM).
template <typename W_t>
__device__ __noinline__ void store_raw_subbins(W_t* slot, const uint32_t* s_glob, TileBox tb, int64_t nx,
                                               int64_t plane) {
  for (int i = threadIdx.x; i < tb.n; i += blockDim.x) {
    const int lx = i % tb.cx, ly = (i / tb.cx) % tb.cy, lz = i / (tb.cx * tb.cy);
    slot[i] = (W_t)s_glob[(tb.z0 + lz) * plane + (tb.y0 + ly) * nx + tb.x0 + lx];
  }
}

template <typename T, int ND>
struct EncSmem {
  using G = TileGeom<T, ND>;
  static constexpr int NP = G::NP;
  static constexpr int W = Traits<T>::W;
  static constexpr uint32_t L = (uint32_t)NP * W;                    // BIT output bytes of a full tile
  static constexpr uint32_t LR = (L + L / 8 + L / 64 + L / 512 + 16 + 15) & ~15u;  // RZE_w output bound
  // A: words -> RZE_w output; B: planes -> staged record; work (five blocks per SM for
  // float32 tiles)
  static constexpr size_t bytes() { return (size_t)LR + L + RzeWork::bytes(LR) + 16; }
};

// Subbin record of each chunk (Sec. III-C, LC-generated pipeline): BIT_w, RZE_w,
// RZE_1, prefixed by the u32 length of the RZE_w output; raw if not shorter.
template <typename T, int ND>
__global__ void __launch_bounds__(TileCfg<T, ND>::NTC, 5) k_encode_sub(const FieldInfo* __restrict__ F, int f0, int nf,
                                                                   int64_t tile0) {
  using G = TileGeom<T, ND>;
  using ES = EncSmem<T, ND>;
  using W_t = typename Traits<T>::Bits;
  constexpr int NT = TileCfg<T, ND>::NTC, W = Traits<T>::W;
  const int64_t gt = tile0 + blockIdx.x;
  const FieldInfo& fi = F[field_of_tile(F, f0, nf, gt)];
  const Params* P = fi.P;
  if (P->status & kErrNonfinite) return;
  if (P->constant) return;
  const Geometry g = fi.g;
  const uint32_t* __restrict__ s_glob = fi.s;
  uint8_t* __restrict__ slots = fi.slots;
  uint32_t* __restrict__ sizes = fi.sizes;
  extern __shared__ __align__(16) unsigned char smem[];
  W_t* ws = reinterpret_cast<W_t*>(smem);
  uint8_t* rzw = smem;  // the words are dead once transposed
  uint32_t* planes = reinterpret_cast<uint32_t*>(smem + ES::LR);
  uint8_t* stage = smem + ES::LR;  // the planes are dead once RZE_w has read them
  const RzeWork w = rze_work_at(smem + ES::LR + ES::L, ES::LR);

  const int64_t tid = gt - fi.tile_base;
  if (tid < 0 || tid >= g.ntiles) return;  // never for a consistent plan
  const TileBox tb = tile_box(g, tid);
  const int n = tb.n, n32 = (n + 31) & ~31;
  const int64_t plane = g.ny * g.nx;
  if (n == G::NP && W == 4 && (g.nx & 3) == 0 && ((uintptr_t)s_glob & 15u) == 0) {
    // subbins are already words, and every row of four starts on a 16-byte boundary
    // (x0 and TX are multiples of 16): 16-byte asynchronous copies
    static_assert(G::TX % 4 == 0, "rows of whole 16-byte copies");
    for (int i = 4 * threadIdx.x; i < n; i += 4 * NT) {
      const int lx = i % G::TX, ly = (i / G::TX) % G::TY, lz = i / (G::TX * G::TY);
      const unsigned d = (unsigned)__cvta_generic_to_shared(&ws[i]);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d),
                   "l"(&s_glob[(tb.z0 + lz) * plane + (tb.y0 + ly) * g.nx + tb.x0 + lx])
                   : "memory");
    }
    cp_async_wait_all();
  } else if (n == G::NP && W == 4) {  // subbins are already words: 4-byte asynchronous copies
    for (int i = threadIdx.x; i < n; i += NT) {
      const int lx = i % G::TX, ly = (i / G::TX) % G::TY, lz = i / (G::TX * G::TY);
      cp_async4(&ws[i], &s_glob[(tb.z0 + lz) * plane + (tb.y0 + ly) * g.nx + tb.x0 + lx], true);
    }
    cp_async_wait_all();
  } else if (n == G::NP) {
#pragma unroll 4
    for (int i = threadIdx.x; i < n; i += NT) {
      const int lx = i % G::TX, ly = (i / G::TX) % G::TY, lz = i / (G::TX * G::TY);
      ws[i] = (W_t)s_glob[(tb.z0 + lz) * plane + (tb.y0 + ly) * g.nx + tb.x0 + lx];
    }
  } else {
    for (int i = threadIdx.x; i < n; i += NT) {
      const int lx = i % tb.cx, ly = (i / tb.cx) % tb.cy, lz = i / (tb.cx * tb.cy);
      ws[i] = (W_t)s_glob[(tb.z0 + lz) * plane + (tb.y0 + ly) * g.nx + tb.x0 + lx];
    }
  }
  const uint32_t raw = (uint32_t)n * W;
  uint8_t* slot = slots + ((size_t)g.ntiles + tid) * kSlotBytes;
  __shared__ unsigned long long s_or;  // OR of the subbins: the planes they reach
  if (threadIdx.x == 0) s_or = 0ull;
  __syncthreads();
  {
    uint64_t o = 0;
    for (int i = threadIdx.x; i < n; i += NT) o |= (uint64_t)ws[i];
    block_or_into(o, &s_or);
  }
  __syncthreads();
  // planes above those the subbins reach are zero: the transpose packs the planes
  // below, and the coder does not read the rest
  const int Pnz = planes_of(s_or);
  bit_transpose_planes<NT, W>(n32, Pnz, [&](int i) -> uint64_t { return i < n ? (uint64_t)ws[i] : 0ULL; }, planes);
  __syncthreads();
  const uint32_t Lnz = plane_bytes_of(n32, Pnz, (uint32_t)W * n32);
  const uint32_t l2 = rze_encode<NT, W>(reinterpret_cast<const uint8_t*>(planes), W * n32, rzw, 0xffffffffu, w, Lnz);
  uint32_t len = 0xffffffffu;
  if (raw > 4) len = rze_encode<NT, 1>(rzw, l2, stage + 4, raw - 4, w);
  if (raw <= 4 || len + 4 >= raw) {  // nothing was staged; the words are read again
    store_raw_subbins<W_t>(reinterpret_cast<W_t*>(slot), s_glob, tb, g.nx, plane);
    if (threadIdx.x == 0) sizes[g.ntiles + tid] = raw | kRawFlag;
    return;
  }
  if (threadIdx.x == 0) *reinterpret_cast<uint32_t*>(stage) = l2;
  zero_tail16<NT>(stage, len + 4);
  __syncthreads();
  copy16<NT>(slot, stage, len + 4);
  if (threadIdx.x == 0) sizes[g.ntiles + tid] = len + 4;
}

// ------------------------------------------------------------- scan + pack

__device__ __forceinline__ uint64_t pad16(uint64_t v) { return (v + 15) & ~(uint64_t)15; }

// Exclusive scan of padded record sizes, one block per field: record c starts at
// base + the sum of pad16(size) of the records before it.
template <int NT>
__global__ void __launch_bounds__(NT) k_scan_sizes(const FieldInfo* __restrict__ F) {
  __shared__ uint64_t tmp[NT / 32 + 1];
  const FieldInfo& fi = F[blockIdx.x];
  Params* P = fi.P;
  if (P->constant) {
    if (threadIdx.x == 0) P->total = kHeaderBytes;
    return;
  }
  const int64_t m = 2 * fi.g.ntiles;
  const uint64_t base = kHeaderBytes + pad16((uint64_t)m * 4);
  const uint64_t end = record_offsets<NT>(fi.sizes, m, base, fi.offs, tmp);
  if (threadIdx.x == 0) P->total = end;
}

__device__ __forceinline__ void put_u64(uint8_t* p, uint64_t v) {
  for (int k = 0; k < 8; ++k) p[k] = (uint8_t)(v >> (8 * k));
}
__device__ __forceinline__ void put_u32(uint8_t* p, uint32_t v) {
  for (int k = 0; k < 4; ++k) p[k] = (uint8_t)(v >> (8 * k));
}

// Writes each field's header, size table and records at their offsets
// (blockIdx.y = field).
__global__ void k_pack(const FieldInfo* __restrict__ F) {
  const FieldInfo& fi = F[blockIdx.y];
  const Params* P = fi.P;
  if (P->status & (kErrNonfinite | kErrRange | kErrNotConverged)) return;
  const uint64_t total = P->total;
  if (total > fi.out_cap) return;
  const int constant = P->constant;
  const HeaderInfo& h = fi.hdr;
  uint8_t* __restrict__ out = fi.out;
  const int64_t ntiles = fi.g.ntiles;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    for (int k = 0; k < kHeaderBytes; ++k) out[k] = 0;
    put_u32(out + 0, kMagic);
    out[4] = LOPC_VERSION & 0xff;
    out[5] = 0;
    out[6] = (uint8_t)h.dtype;
    out[7] = (uint8_t)h.ndim;
    for (int k = 0; k < 3; ++k) put_u64(out + 8 + 8 * k, (uint64_t)h.dims[k]);
    out[32] = (uint8_t)h.mode;
    out[33] = (uint8_t)constant;
    for (int k = 0; k < 3; ++k) put_u32(out + 36 + 4 * k, (uint32_t)h.tile[k]);
    put_u64(out + 48, (uint64_t)__double_as_longlong(h.eb));
    put_u64(out + 56, (uint64_t)__double_as_longlong(constant ? 0.0 : P->eps));
    put_u64(out + 64, (uint64_t)__double_as_longlong(constant ? 0.0 : P->inv));
    put_u64(out + 72, constant ? P->const_bits : 0ULL);
    put_u64(out + 80, constant ? 0ULL : (uint64_t)ntiles);
    put_u64(out + 88, total);
  }
  if (constant) return;
  const int64_t m = 2 * ntiles;
  const uint32_t* __restrict__ sizes = fi.sizes;
  const uint64_t* __restrict__ offs = fi.offs;
  const uint8_t* __restrict__ slots = fi.slots;
  const uint64_t table_end = kHeaderBytes + pad16((uint64_t)m * 4);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (int64_t)(table_end - kHeaderBytes) / 4;
       i += (int64_t)gridDim.x * blockDim.x)
    reinterpret_cast<uint32_t*>(out + kHeaderBytes)[i] = i < m ? sizes[i] : 0u;
  // records: one warp per record, 16-byte copies, two in flight per lane; the bytes
  // that pad a record to 16 are written as zeros (a slot holds stale bytes there)
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t c = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c < m; c += warps) {
    const uint32_t len = sizes[c] & kSizeMask;
    const uint64_t n16 = pad16(len) / 16;
    const uint32_t rem = len & 15u;  // bytes of the record in its last 16-byte unit (0: all 16)
    const uint4* src = reinterpret_cast<const uint4*>(slots + (size_t)c * kSlotBytes);
    uint4* dst = reinterpret_cast<uint4*>(out + offs[c]);
    auto put = [&](uint64_t j, uint4 v) {
      if (rem && j + 1 == n16) {
        uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int keep = (int)rem - 4 * q;
          w[q] = keep >= 4 ? w[q] : keep <= 0 ? 0u : (w[q] & ((1u << (8 * keep)) - 1u));
        }
        v = make_uint4(w[0], w[1], w[2], w[3]);
      }
      dst[j] = v;
    };
    uint64_t j = lane;
    for (; j + 32 < n16; j += 64) {
      const uint4 a = src[j], b = src[j + 32];
      put(j, a);
      put(j + 32, b);
    }
    if (j < n16) put(j, src[j]);
  }
}

__device__ __forceinline__ int status_code(unsigned int st) {
  if (st & kErrNonfinite) return LOPC_ERR_NONFINITE;
  if (st & kErrRange) return LOPC_ERR_RANGE;
  if (st & kErrNotConverged) return LOPC_ERR_NOT_CONVERGED;
  if (st & kErrCorrupt) return LOPC_ERR_CORRUPT;
  if (st & kErrInternal) return LOPC_ERR_CUDA;
  return LOPC_OK;
}

// Per-field results for the caller: stream length and status.
__global__ void k_finalize(const FieldInfo* __restrict__ F, int nf) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= nf) return;
  const FieldInfo& fi = F[f];
  int st = status_code(fi.P->status);
  if (st == LOPC_OK && fi.P->total > fi.out_cap) st = LOPC_ERR_CAPACITY;
  if (fi.status_out) *fi.status_out = st;
  if (fi.size_out) *fi.size_out = st == LOPC_OK ? fi.P->total : 0ULL;
}

// Exports subbins (for stage-by-stage tests).
__global__ void k_export_subbins(int64_t n, const uint32_t* __restrict__ s_glob, uint64_t* __restrict__ subbins) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    subbins[i] = (uint64_t)s_glob[i];
}

}  // namespace lopc
