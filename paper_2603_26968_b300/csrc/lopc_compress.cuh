// lopc_compress.cuh -- compression kernels: value range (NOA), error-bound
// resolution, the tile pass (quantize, flags, tile-local least fixpoint), reruns of
// tiles whose halo changed, the chunk encoder, the size scan and the stream pack.
#pragma once
#include "lopc_device.cuh"

namespace lopc {

// Compile-time tile configuration (Sec. II-C chunk of 16 KiB of words, as a tile).
template <typename T, int ND>
struct TileCfg;
template <>
struct TileCfg<float, 3> {
  static constexpr int TZ = 16, TY = 16, TX = 16, HZ = 1, NT = 256;
};
template <>
struct TileCfg<double, 3> {
  static constexpr int TZ = 8, TY = 16, TX = 16, HZ = 1, NT = 128;
};
template <>
struct TileCfg<float, 2> {
  static constexpr int TZ = 1, TY = 64, TX = 64, HZ = 0, NT = 256;
};
template <>
struct TileCfg<double, 2> {
  static constexpr int TZ = 1, TY = 32, TX = 64, HZ = 0, NT = 128;
};

// Freudenthal neighbourhood (Sec. II): offsets +-d, d in {0,1}^3 \ {0}.  Direction
// k < 7 is -D[k] (lower linear index), k >= 7 is +D[k-7] (higher linear index).
__device__ __forceinline__ void dir3(int k, int& dz, int& dy, int& dx) {
  const int d = k % 7;
  const int s = k < 7 ? -1 : 1;
  // D = (0,0,1) (0,1,0) (0,1,1) (1,0,0) (1,0,1) (1,1,0) (1,1,1): bits of d+1 = (z,y,x)
  const int v = d + 1;
  dz = s * ((v >> 2) & 1);
  dy = s * ((v >> 1) & 1);
  dx = s * (v & 1);
}

template <int HZ>
__device__ __forceinline__ bool dir_valid(int k) {
  if (HZ) return true;
  int dz, dy, dx;
  dir3(k, dz, dy, dx);
  return dz == 0;
}

// ------------------------------------------------------------------ range

__global__ void k_init_params(Params* P, double eb, int mode) {
  P->kmin = ~0ULL;
  P->kmax = 0ULL;
  P->eb = eb;
  P->mode = mode;
  P->status = 0;
  P->constant = 0;
  P->dirty_count = 0;
  P->total = 0;
  P->rounds = 0;
}

template <typename T>
__device__ __forceinline__ unsigned long long biased(typename Traits<T>::Key k) {
  return (unsigned long long)((long long)k) ^ 0x8000000000000000ULL;
}

// Sec. III-A (NOA): x_min and x_max over the field, as order keys.
template <typename T>
__global__ void k_range(const T* __restrict__ x, int64_t n, Params* P) {
  using K = typename Traits<T>::Key;
  K lo = Traits<T>::kMaxKey, hi = -Traits<T>::kMaxKey;
  bool bad = false;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const T v = x[i];
    if (!is_finite_bits<T>(v)) {
      bad = true;
      continue;
    }
    const K k = order_key<T>(v);
    lo = min(lo, k);
    hi = max(hi, k);
  }
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
// inv = 1 / eps_q.  IEEE binary64, correctly rounded, no contraction.
template <typename T>
__global__ void k_resolve_eps(Params* P) {
  using K = typename Traits<T>::Key;
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
}

// ---------------------------------------------------------------- tile pass

template <typename T, int ND>
struct TileSmem {
  using C = TileCfg<T, ND>;
  using K = typename Traits<T>::Key;
  using B = typename Traits<T>::Bin;
  static constexpr int BZ = C::TZ + 2 * C::HZ, BY = C::TY + 2, BX = C::TX + 2;
  static constexpr int E = BZ * BY * BX;
  static constexpr int NP = C::TZ * C::TY * C::TX;
  static constexpr size_t bytes() { return (size_t)E * (sizeof(K) + sizeof(B) + 4) + (size_t)NP * 4 + 64; }
};

// Tile pass (mode 0) and rerun (mode 1) of one chunk-tile.
//   mode 0: halo subbins are taken as 0 (a lower bound); writes all subbins and bins.
//   mode 1: halo and own subbins come from the global array (current values).
// Then the tile-local least fixpoint of Alg. 2's update is computed in shared
// memory (chaotic relaxation; any schedule reaches the same least fixpoint,
// Sec. III-E), subbins that rose are written back, and every other tile holding a
// greater same-bin neighbour of a risen point is marked for the next round.
template <typename T, int ND, int MODE>
__global__ void __launch_bounds__(TileCfg<T, ND>::NT) k_tile(const T* __restrict__ x, Geometry g, Params* P,
                                                             uint32_t* __restrict__ s_glob,
                                                             typename Traits<T>::Bin* __restrict__ b_glob,
                                                             uint8_t* __restrict__ dirty,
                                                             const uint32_t* __restrict__ list) {
  using C = TileCfg<T, ND>;
  using S = TileSmem<T, ND>;
  using K = typename Traits<T>::Key;
  using B = typename Traits<T>::Bin;
  constexpr int NT = C::NT, BY = S::BY, BX = S::BX, E = S::E;
  if (P->status & kErrNonfinite) return;
  if (P->constant) return;
  extern __shared__ __align__(16) unsigned char smem[];
  K* key = reinterpret_cast<K*>(smem);
  B* bin = reinterpret_cast<B*>(key + E);
  uint32_t* sv = reinterpret_cast<uint32_t*>(bin + E);
  uint32_t* cm = sv + E;

  const int64_t tid = MODE == 0 ? (int64_t)blockIdx.x : (int64_t)list[blockIdx.x];
  const TileBox tb = tile_box(g, tid);
  const unsigned long long inv_m = P->inv_m;
  const int inv_e = P->inv_e;
  const int64_t plane = g.ny * g.nx;

  // load the tile and its halo: keys and bins (absent points get a bin no value has)
  bool range_bad = false;
  for (int e = threadIdx.x; e < E; e += NT) {
    const int lx = e % BX, ly = (e / BX) % BY, lz = e / (BX * BY);
    const int64_t gz = tb.z0 + lz - C::HZ, gy = tb.y0 + ly - 1, gx = tb.x0 + lx - 1;
    const bool in = gz >= 0 && gz < g.nz && gy >= 0 && gy < g.ny && gx >= 0 && gx < g.nx;
    B b = Traits<T>::kAbsent;
    K k = 0;
    uint32_t s0 = 0;
    if (in) {
      const int64_t gi = gz * plane + gy * g.nx + gx;
      const T v = x[gi];
      long long q;
      if (!is_finite_bits<T>(v)) {
        range_bad = true;  // only reachable in ABS mode; reported as non-finite below
      } else if (!quantize_exact<T>(v, inv_m, inv_e, q) || q >= Traits<T>::kBinLimit || q <= -Traits<T>::kBinLimit) {
        range_bad = true;
      } else {
        b = (B)q;
        k = order_key<T>(v);
      }
      if (MODE == 1) s0 = s_glob[gi];
    }
    key[e] = k;
    bin[e] = b;
    sv[e] = s0;
  }
  if (range_bad) {
    // tell the two cases apart once, off the fast path
    for (int e = threadIdx.x; e < E; e += NT) {
      const int lx = e % BX, ly = (e / BX) % BY, lz = e / (BX * BY);
      const int64_t gz = tb.z0 + lz - C::HZ, gy = tb.y0 + ly - 1, gx = tb.x0 + lx - 1;
      if (gz >= 0 && gz < g.nz && gy >= 0 && gy < g.ny && gx >= 0 && gx < g.nx) {
        const T v = x[gz * plane + gy * g.nx + gx];
        atomicOr(&P->status, is_finite_bits<T>(v) ? kErrRange : kErrNonfinite);
      }
    }
  }
  __syncthreads();

  // flags (Alg. 1): lower same-bin neighbours in bits 0..13, greater ones in 14..27
  const int p0 = threadIdx.x * kSegment;
  const int lz = p0 / (C::TX * C::TY), ly = (p0 / C::TX) % C::TY, lx0 = p0 % C::TX;
  const bool row_in = lz < tb.cz && ly < tb.cy;
  uint32_t sinit[kSegment];
#pragma unroll
  for (int j = 0; j < kSegment; ++j) {
    const int lx = lx0 + j;
    const int e = ((lz + C::HZ) * BY + ly + 1) * BX + lx + 1;
    uint32_t m = 0;
    if (row_in && lx < tb.cx) {
      const B bp = bin[e];
      const K kp = key[e];
#pragma unroll
      for (int k = 0; k < 14; ++k) {
        if (!dir_valid<C::HZ>(k)) continue;
        int dz, dy, dx;
        dir3(k, dz, dy, dx);
        const int e2 = e + (dz * BY + dy) * BX + dx;
        if (bin[e2] != bp) continue;
        const K kn = key[e2];
        const bool lower = kn < kp || (kn == kp && k < 7);
        m |= lower ? (1u << k) : (1u << (14 + k));
      }
    }
    cm[p0 + j] = m;
    sinit[j] = sv[e];
  }
  __syncthreads();

  // tile-local least fixpoint: s(p) = max(s(p), max over lower same-bin n of s(n) + [n after p])
  volatile uint32_t* vs = sv;
  int iter = 0;
  bool over = false;
  while (true) {
    int changed = 0;
    const bool fwd = (iter & 1) == 0;
#pragma unroll 1
    for (int jj = 0; jj < kSegment; ++jj) {
      const int j = fwd ? jj : kSegment - 1 - jj;
      const uint32_t m = cm[p0 + j] & 0x3fffu;
      if (!m) continue;
      const int e = ((lz + C::HZ) * BY + ly + 1) * BX + lx0 + j + 1;
      uint32_t best = vs[e];
      uint32_t mm = m;
      while (mm) {
        const int k = __ffs(mm) - 1;
        mm &= mm - 1;
        int dz, dy, dx;
        dir3(k, dz, dy, dx);
        const uint32_t c = vs[e + (dz * BY + dy) * BX + dx] + (k >= 7 ? 1u : 0u);
        best = c > best ? c : best;
      }
      if (best > vs[e]) {
        vs[e] = best;
        changed = 1;
      }
    }
    ++iter;
    if (!__syncthreads_or(changed)) break;
    if (iter > 4 * E + 64) {  // a chain inside the box has fewer than E links
      over = true;
      break;
    }
  }
  if (over && threadIdx.x == 0) atomicOr(&P->status, kErrNotConverged);

  // write back, mark tiles that hold greater same-bin neighbours of risen points
#pragma unroll 1
  for (int j = 0; j < kSegment; ++j) {
    const int lx = lx0 + j;
    if (!(row_in && lx < tb.cx)) continue;
    const int e = ((lz + C::HZ) * BY + ly + 1) * BX + lx + 1;
    const int64_t gz = tb.z0 + lz, gy = tb.y0 + ly, gx = tb.x0 + lx;
    const int64_t gi = gz * plane + gy * g.nx + gx;
    const uint32_t sf = sv[e];
    if (MODE == 0) {
      s_glob[gi] = sf;
      b_glob[gi] = bin[e];
    } else if (sf != sinit[j]) {
      s_glob[gi] = sf;
    }
    if (sf == sinit[j]) continue;
    uint32_t up = cm[p0 + j] >> 14;
    while (up) {
      const int k = __ffs(up) - 1;
      up &= up - 1;
      int dz, dy, dx;
      dir3(k, dz, dy, dx);
      const int nz = lz + dz, ny = ly + dy, nx = lx + dx;
      if (nz >= 0 && nz < C::TZ && ny >= 0 && ny < C::TY && nx >= 0 && nx < C::TX) continue;
      const int64_t qz = gz + dz, qy = gy + dy, qx = gx + dx;
      const int64_t t2 = ((qz / g.tz) * g.nty + qy / g.ty) * g.ntx + qx / g.tx;
      dirty[t2] = 1;
    }
  }
}

// Dirty flags -> list of tiles for the next round (flags are cleared).
__global__ void k_compact(uint8_t* dirty, int64_t ntiles, uint32_t* list, Params* P) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < ntiles; t += (int64_t)gridDim.x * blockDim.x) {
    if (dirty[t]) {
      dirty[t] = 0;
      const unsigned slot = atomicAdd(&P->dirty_count, 1u);
      list[slot] = (uint32_t)t;
    }
  }
}

// ----------------------------------------------------------------- encoder

constexpr uint32_t kSlotBytes = 16384;  // a record never exceeds the raw chunk (16 KiB)

template <typename T, int ND>
struct EncSmem {
  using C = TileCfg<T, ND>;
  static constexpr int NP = C::TZ * C::TY * C::TX;  // points of a full tile
  static constexpr int W = Traits<T>::W;
  static constexpr uint32_t L = (uint32_t)NP * W;   // BIT output bytes of a full tile
  static constexpr uint32_t LR = L + L / 8 + L / 64 + L / 512 + 16;  // RZE_w output bound
  static constexpr size_t bytes() {
    return (size_t)NP * 8 * 2 /*words*/ + L /*planes*/ + LR /*rze_w out*/ + (LR / 8 + 16) /*m0*/ +
           (LR / 64 + 16) /*m1*/ + (LR / 512 + 16) /*m2*/ + ((LR / 8 + 16) / 4 + 8) * 4 /*pre*/ + 64 * 4;
  }
};

// Chunk encoder (Sec. III-C): bins with DIFFNB_w, BIT_w, RZE_1; subbins with BIT_w,
// RZE_w, RZE_1 (record prefixed by the u32 RZE_w length).  A record that would not
// be shorter than the raw chunk is stored raw (size flag bit 31).
template <typename T, int ND>
__global__ void __launch_bounds__(TileCfg<T, ND>::NT) k_encode(Geometry g, const Params* P,
                                                               const uint32_t* __restrict__ s_glob,
                                                               const typename Traits<T>::Bin* __restrict__ b_glob,
                                                               uint8_t* __restrict__ slots, uint32_t* __restrict__ sizes) {
  using C = TileCfg<T, ND>;
  using ES = EncSmem<T, ND>;
  using W_t = typename Traits<T>::Bits;
  constexpr int NT = C::NT, W = Traits<T>::W;
  if (P->status & kErrNonfinite) return;
  if (P->constant) return;
  extern __shared__ __align__(16) unsigned char smem[];
  W_t* wb = reinterpret_cast<W_t*>(smem);
  W_t* ws = wb + ES::NP;
  uint32_t* planes = reinterpret_cast<uint32_t*>(ws + ES::NP);
  uint8_t* rzw = reinterpret_cast<uint8_t*>(planes) + ES::L;
  RzeScratch sc;
  sc.m0 = rzw + ES::LR;
  sc.m1 = sc.m0 + ES::LR / 8 + 16;
  sc.m2 = sc.m1 + ES::LR / 64 + 16;
  sc.pre = reinterpret_cast<uint32_t*>(((uintptr_t)(sc.m2 + ES::LR / 512 + 16) + 15) & ~(uintptr_t)15);
  sc.tmp = sc.pre + (ES::LR / 8 + 16) / 4 + 8;

  const int64_t tid = blockIdx.x;
  const TileBox tb = tile_box(g, tid);
  const int n = tb.n, n32 = (n + 31) & ~31;
  const int64_t plane = g.ny * g.nx;
  for (int i = threadIdx.x; i < n; i += NT) {
    const int lx = i % tb.cx, ly = (i / tb.cx) % tb.cy, lz = i / (tb.cx * tb.cy);
    const int64_t gi = (tb.z0 + lz) * plane + (tb.y0 + ly) * g.nx + tb.x0 + lx;
    wb[i] = (W_t)b_glob[gi];
    ws[i] = (W_t)s_glob[gi];
  }
  __syncthreads();
  const uint32_t raw = (uint32_t)n * W;
  uint8_t* slot_b = slots + (size_t)tid * kSlotBytes;
  uint8_t* slot_s = slots + ((size_t)g.ntiles + tid) * kSlotBytes;
  __shared__ uint32_t rec_len;

  // bins: DIFFNB_w on the fly, BIT_w, RZE_1
  constexpr W_t M = (W_t)0xAAAAAAAAAAAAAAAAULL;
  bit_transpose<NT, W>(n32, [&](int i) -> uint64_t {
    if (i >= n) return 0;
    const W_t d = wb[i] - (i ? wb[i - 1] : (W_t)0);
    return (uint64_t)((W_t)(d + M) ^ M);
  }, planes);
  __syncthreads();
  uint32_t len = rze_encode<NT>(reinterpret_cast<const uint8_t*>(planes), W * n32, 1, slot_b, raw, sc);
  if (len >= raw) {
    for (int i = threadIdx.x; i < n; i += NT) reinterpret_cast<W_t*>(slot_b)[i] = wb[i];
    len = raw | kRawFlag;
  }
  if (threadIdx.x == 0) rec_len = len;
  __syncthreads();
  len = rec_len;
  {
    const uint32_t l = len & ~kRawFlag, lp = (l + 15) & ~15u;
    for (uint32_t j = l + threadIdx.x; j < lp; j += NT) slot_b[j] = 0;
    if (threadIdx.x == 0) sizes[tid] = len;
  }
  __syncthreads();

  // subbins: BIT_w, RZE_w (to shared memory), RZE_1
  bit_transpose<NT, W>(n32, [&](int i) -> uint64_t { return i < n ? (uint64_t)ws[i] : 0ULL; }, planes);
  __syncthreads();
  const uint32_t l2 = rze_encode<NT>(reinterpret_cast<const uint8_t*>(planes), W * n32, W, rzw, 0xffffffffu, sc);
  __syncthreads();
  uint32_t len2 = 0;
  if (raw > 4) len2 = rze_encode<NT>(rzw, l2, 1, slot_s + 4, raw - 4, sc);
  if (raw <= 4 || len2 + 4 >= raw) {
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += NT) reinterpret_cast<W_t*>(slot_s)[i] = ws[i];
    len2 = raw | kRawFlag;
  } else {
    if (threadIdx.x == 0) {
      slot_s[0] = (uint8_t)l2;
      slot_s[1] = (uint8_t)(l2 >> 8);
      slot_s[2] = (uint8_t)(l2 >> 16);
      slot_s[3] = (uint8_t)(l2 >> 24);
    }
    len2 += 4;
  }
  if (threadIdx.x == 0) rec_len = len2;
  __syncthreads();
  len2 = rec_len;
  {
    const uint32_t l = len2 & ~kRawFlag, lp = (l + 15) & ~15u;
    for (uint32_t j = l + threadIdx.x; j < lp; j += NT) slot_s[j] = 0;
    if (threadIdx.x == 0) sizes[g.ntiles + tid] = len2;
  }
}

// ------------------------------------------------------------- scan + pack

__device__ __forceinline__ uint64_t pad16(uint64_t v) { return (v + 15) & ~(uint64_t)15; }

// Exclusive scan of padded record sizes (one block): record c starts at
// base + sum of pad16(size) of records before it.
template <int NT>
__global__ void __launch_bounds__(NT) k_scan_sizes(const uint32_t* __restrict__ sizes, int64_t m, uint64_t base,
                                                   uint64_t* __restrict__ offs, Params* P) {
  __shared__ uint64_t tmp[NT / 32 + 1];
  if (P->constant) {
    if (threadIdx.x == 0) P->total = kHeaderBytes;
    return;
  }
  const int64_t per = (m + NT - 1) / NT;
  const int64_t a = min(m, (int64_t)threadIdx.x * per), b = min(m, a + per);
  uint64_t c = 0;
  for (int64_t i = a; i < b; ++i) c += pad16(sizes[i] & ~kRawFlag);
  uint64_t total;
  uint64_t run = block_exclusive_scan<NT, uint64_t>(c, tmp, &total) + base;
  for (int64_t i = a; i < b; ++i) {
    offs[i] = run;
    run += pad16(sizes[i] & ~kRawFlag);
  }
  if (threadIdx.x == 0) P->total = base + total;
}

struct HeaderInfo {
  int32_t dtype, ndim, mode;
  int64_t dims[3];
  int32_t tile[3];
  double eb;
};

__device__ __forceinline__ void put_u64(uint8_t* p, uint64_t v) {
  for (int k = 0; k < 8; ++k) p[k] = (uint8_t)(v >> (8 * k));
}
__device__ __forceinline__ void put_u32(uint8_t* p, uint32_t v) {
  for (int k = 0; k < 4; ++k) p[k] = (uint8_t)(v >> (8 * k));
}

// Writes the header, the size table and the records at their offsets.
__global__ void k_pack(HeaderInfo h, int64_t ntiles, const uint32_t* __restrict__ sizes,
                       const uint64_t* __restrict__ offs, const uint8_t* __restrict__ slots, uint8_t* __restrict__ out,
                       uint64_t cap, const Params* P) {
  if (P->status & (kErrNonfinite | kErrRange | kErrNotConverged)) return;
  const uint64_t total = P->total;
  if (total > cap) return;
  const int constant = P->constant;
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
  const uint64_t table_end = kHeaderBytes + pad16((uint64_t)m * 4);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (int64_t)(table_end - kHeaderBytes) / 4;
       i += (int64_t)gridDim.x * blockDim.x)
    reinterpret_cast<uint32_t*>(out + kHeaderBytes)[i] = i < m ? sizes[i] : 0u;
  // records: one block per record, 16-byte copies
  for (int64_t c = blockIdx.x; c < m; c += gridDim.x) {
    const uint64_t n16 = pad16(sizes[c] & ~kRawFlag) / 16;
    const uint4* src = reinterpret_cast<const uint4*>(slots + (size_t)c * kSlotBytes);
    uint4* dst = reinterpret_cast<uint4*>(out + offs[c]);
    for (uint64_t j = threadIdx.x; j < n16; j += blockDim.x) dst[j] = src[j];
  }
}

// Exports bins and subbins (for stage-by-stage tests).
template <typename T>
__global__ void k_export(int64_t n, const uint32_t* __restrict__ s_glob, const typename Traits<T>::Bin* __restrict__ b_glob,
                         int64_t* __restrict__ bins, uint64_t* __restrict__ subbins) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    bins[i] = (int64_t)b_glob[i];
    subbins[i] = (uint64_t)s_glob[i];
  }
}

}  // namespace lopc
