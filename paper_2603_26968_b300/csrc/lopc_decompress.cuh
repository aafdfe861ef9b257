// lopc_decompress.cuh -- decompression kernels: record offsets from the size table,
// and one block per chunk that undoes RZE/BIT and the bin predictor (Lorenzo or 1D
// difference) for bins, RZE/RZE/BIT for subbins, and writes
// x_hat = succ^s(lowest value of bin b) (Sec. III-D, III-E).
#pragma once
#include "lopc_compress.cuh"
#include "lopc_codec.cuh"

namespace lopc {

// One stream of a decompression launch (a single stream is a batch of one).
struct DecField {
  Geometry g;
  const uint8_t* in;
  uint64_t in_size;
  void* x;                // output field
  uint64_t* offs;         // 2 x ntiles record offsets (workspace)
  unsigned int* status;   // kErr* bits (workspace)
  int* status_out;        // device: this stream's LOPC status (may be null)
  double eps_q;           // filled on the device from the header
  unsigned long long inv_m;
  int inv_e;
  int constant;
  int version;            // stream format, from the header
  unsigned long long const_bits;
  int64_t tile_base;
};

// Measurement aid: SM cycles per decode phase, summed over blocks, while enabled.
__device__ unsigned long long g_dec_phase[8];
__device__ int g_dec_phase_on;

__device__ __forceinline__ void dec_mark(int k, long long& t0) {
  if (threadIdx.x == 0 && g_dec_phase_on) {
    const long long t = clock64();
    atomicAdd(&g_dec_phase[k], (unsigned long long)(t - t0));
    t0 = t;
  }
}

// Reads each stream's header on the device: the decoder's parameters, and a check
// that the header (dtype, ndim, dims, chunk count) matches the descriptor the launch
// was planned for.
__global__ void k_dec_setup(DecField* F, int nf) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= nf) return;
  DecField& d = F[f];
  *d.status = 0;
  const uint8_t* h = d.in;
  auto rd = [&](int o, int nb) {
    uint64_t v = 0;
    for (int k = 0; k < nb; ++k) v |= (uint64_t)h[o + k] << (8 * k);
    return v;
  };
  bool ok = d.in_size >= (uint64_t)kHeaderBytes && rd(0, 4) == kMagic && rd(4, 2) >= 1 && rd(4, 2) <= LOPC_VERSION &&
            h[6] == (uint8_t)d.g.dtype && h[7] == (uint8_t)d.g.ndim;
  // the dims too: a descriptor with other dims but as many tiles would decode garbage
  if (d.g.ndim == 3)
    ok = ok && rd(8, 8) == (uint64_t)d.g.nz && rd(16, 8) == (uint64_t)d.g.ny && rd(24, 8) == (uint64_t)d.g.nx;
  else
    ok = ok && rd(8, 8) == (uint64_t)d.g.ny && rd(16, 8) == (uint64_t)d.g.nx && rd(24, 8) == 0;
  const uint64_t total = ok ? rd(88, 8) : 0;
  ok = ok && total <= d.in_size && total >= (uint64_t)kHeaderBytes;
  d.constant = ok ? h[33] : 0;
  const uint64_t iu = ok ? rd(64, 8) : 0;
  const double inv = __longlong_as_double((long long)iu);
  if (ok && !d.constant) ok = inv > 0.0 && inv <= 1.79e308 && rd(80, 8) == (uint64_t)d.g.ntiles;
  if (ok && d.constant) ok = rd(80, 8) == 0 && total == (uint64_t)kHeaderBytes;
  if (!ok) {
    *d.status = kErrCorrupt;
    return;
  }
  d.version = (int)rd(4, 2);
  d.const_bits = rd(72, 8);
  const int ex = (int)((iu >> 52) & 0x7ff);
  d.inv_m = (iu & 0xfffffffffffffULL) | (ex ? 0x10000000000000ULL : 0ULL);
  d.inv_e = ex ? ex - 1075 : -1074;
  d.eps_q = d.constant ? 0.0 : __ddiv_rn(1.0, inv);  // only seeds the search for a bin's lowest value
}

// Offsets of the records, one block per stream; flags a table that does not add up
// to the stream length.
template <int NT>
__global__ void __launch_bounds__(NT) k_dec_offsets(const DecField* __restrict__ F) {
  __shared__ uint64_t tmp[NT / 32 + 1];
  const DecField& d = F[blockIdx.x];
  if (*d.status || d.constant) return;
  const int64_t m = 2 * d.g.ntiles;
  const uint64_t total = (uint64_t)d.in[88] | ((uint64_t)d.in[89] << 8) | ((uint64_t)d.in[90] << 16) |
                         ((uint64_t)d.in[91] << 24) | ((uint64_t)d.in[92] << 32) | ((uint64_t)d.in[93] << 40) |
                         ((uint64_t)d.in[94] << 48) | ((uint64_t)d.in[95] << 56);
  const uint64_t base = kHeaderBytes + pad16((uint64_t)m * 4);
  if (base > total) {
    if (threadIdx.x == 0) atomicOr(d.status, kErrCorrupt);
    return;
  }
  const uint32_t* tab = reinterpret_cast<const uint32_t*>(d.in + kHeaderBytes);
  const uint64_t end = record_offsets<NT>(tab, m, base, d.offs, tmp);
  if (threadIdx.x == 0 && end != total) atomicOr(d.status, kErrCorrupt);
}

__global__ void k_dec_finalize(const DecField* __restrict__ F, int nf) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= nf) return;
  if (F[f].status_out) *F[f].status_out = *F[f].status ? LOPC_ERR_CORRUPT : LOPC_OK;
}

template <typename T, int ND>
struct DecSmem {
  using G = TileGeom<T, ND>;
  static constexpr int NP = G::NP;
  static constexpr int W = Traits<T>::W;
  static constexpr uint32_t L = (uint32_t)NP * W;                                   // planes of a full tile
  static constexpr uint32_t LR = (L + L / 8 + L / 64 + L / 512 + 16 + 15) & ~15u;  // largest legal RZE_w output
  static constexpr uint32_t CACHE = 16384;                                          // bytes of bin-lowest keys
  static constexpr uint32_t BB = LR > CACHE ? LR : CACHE;
  // A: staged record / subbin planes; B: RZE output, or the key cache between the two
  // halves; WB: bins, then each point's bin-lowest key
  static constexpr size_t bytes() { return (size_t)L + BB + (size_t)NP * W + RzeWork::bytes(LR) + 16; }
};

__device__ __forceinline__ uint32_t shfl_up_w(uint32_t v, int o) { return __shfl_up_sync(0xffffffffu, v, o); }
__device__ __forceinline__ uint64_t shfl_up_w(uint64_t v, int o) { return __shfl_up_sync(0xffffffffu, v, o); }
__device__ __forceinline__ uint32_t shfl_idx_w(uint32_t v, int l) { return __shfl_sync(0xffffffffu, v, l); }
__device__ __forceinline__ uint64_t shfl_idx_w(uint64_t v, int l) { return __shfl_sync(0xffffffffu, v, l); }

// Inverse of a chunk's Lorenzo residual (format 2 bin records): inclusive prefix sums
// of w[(z * cy + y) * cx + x] along x, then y, then z, modulo 2^(8 W).  Rows of 16
// or 32 words are scanned by warp shuffles in segments of a row, rows of 64 in two
// halves with a carry, other rows (clipped chunks) by one thread each; the y and z
// sums take one thread per line.
template <int NT, int ND, typename W_t>
__device__ __forceinline__ void undo_lorenzo(W_t* w, int cz, int cy, int cx) {
  constexpr int NWARP = NT / 32;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int rows = cz * cy;
  if (cx == 16 || cx == 32) {
    const int n = rows * cx;
    for (int base = wid * 32; base < n; base += NWARP * 32) {
      const int i = base + lane;
      W_t v = i < n ? w[i] : (W_t)0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const W_t y = __shfl_up_sync(0xffffffffu, v, o, cx);
        if (o < cx && (lane & (cx - 1)) >= o) v += y;
      }
      if (i < n) w[i] = v;
    }
  } else if (cx == 64) {
    for (int r = wid; r < rows; r += NWARP) {
      W_t* row = w + r * 64;
      W_t a = row[lane], b = row[32 + lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const W_t ya = __shfl_up_sync(0xffffffffu, a, o), yb = __shfl_up_sync(0xffffffffu, b, o);
        if (lane >= o) {
          a += ya;
          b += yb;
        }
      }
      b += __shfl_sync(0xffffffffu, a, 31);
      row[lane] = a;
      row[32 + lane] = b;
    }
  } else {
    for (int r = threadIdx.x; r < rows; r += NT) {
      W_t acc = 0;
      for (int x = 0; x < cx; ++x) {
        acc += w[r * cx + x];
        w[r * cx + x] = acc;
      }
    }
  }
  __syncthreads();
  // a strided line in batches of 8 independent loads, summed in registers
  auto scan_line = [&](W_t* p, int len, int stride) {
    W_t acc = 0;
    for (int a = 0; a < len; a += 8) {
      W_t v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = a + u < len ? p[(a + u) * stride] : (W_t)0;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        acc += v[u];
        if (a + u < len) p[(a + u) * stride] = acc;
      }
    }
  };
  for (int l = threadIdx.x; l < cz * cx; l += NT) {
    const int z = l / cx, x = l - z * cx;
    scan_line(w + z * cy * cx + x, cy, cx);
  }
  if (ND == 3) {
    __syncthreads();
    const int plane = cy * cx;
    for (int l = threadIdx.x; l < plane; l += NT) scan_line(w + l, cz, plane);
  }
}

// One block per chunk: bins (RZE_1, BIT_w and the predictor's inverses), then the lowest value
// of every bin of the tile's bin range (when it is small enough to cache), then
// subbins (RZE_1, RZE_w, BIT_w inverses) and x_hat = the subbin-th value above the
// bin's lowest value (Sec. III-E), written as the subbin words come out.
template <typename T, int ND>
__global__ void __launch_bounds__(TileCfg<T, ND>::NTC, 4) k_decode(const DecField* __restrict__ F, int f0, int nf,
                                                               int64_t tile0) {
  using G = TileGeom<T, ND>;
  using DS = DecSmem<T, ND>;
  using W_t = typename Traits<T>::Bits;
  using K = typename Traits<T>::Key;
  using B = typename Traits<T>::Bin;
  constexpr int NT = TileCfg<T, ND>::NTC, W = Traits<T>::W;
  constexpr int CAPN = DS::CACHE / sizeof(K);
  constexpr K kNone = (K)(-Traits<T>::kMaxKey - 1);  // never a valid key
  extern __shared__ __align__(16) unsigned char smem[];
  uint8_t* A = smem;
  uint8_t* Bf = smem + DS::L;
  K* cache = reinterpret_cast<K*>(Bf);  // between the halves, B holds the key cache
  W_t* wb = reinterpret_cast<W_t*>(smem + DS::L + DS::BB);
  const RzeWork w = rze_work_at(reinterpret_cast<uint8_t*>(wb + DS::NP), DS::LR);
  __shared__ int bad;
  __shared__ B red_min[NT / 32], red_max[NT / 32];
  const int64_t gt = tile0 + blockIdx.x;
  int lo_f = f0, hi_f = f0 + nf - 1;
  while (lo_f < hi_f) {
    const int mid = (lo_f + hi_f + 1) >> 1;
    if (F[mid].tile_base <= gt)
      lo_f = mid;
    else
      hi_f = mid - 1;
  }
  const DecField& df = F[lo_f];
  unsigned int* status = df.status;
  if (*status & kErrCorrupt) return;
  const Geometry g = df.g;
  const uint8_t* __restrict__ in = df.in;
  const uint64_t* __restrict__ offs = df.offs;
  T* __restrict__ xhat = reinterpret_cast<T*>(df.x);
  const int64_t tid = gt - df.tile_base;
  if (tid < 0 || tid >= g.ntiles) return;  // never for a consistent plan
  const TileBox tb = tile_box(g, tid);
  if (df.constant) {  // a constant field: every point is the stored value
    const T v = Traits<T>::from_bits((typename Traits<T>::Bits)df.const_bits);
    const int64_t plane = g.ny * g.nx;
    for (int i = threadIdx.x; i < tb.n; i += NT) {
      const int lx = i % tb.cx, ly = (i / tb.cx) % tb.cy, lz = i / (tb.cx * tb.cy);
      xhat[(tb.z0 + lz) * plane + (tb.y0 + ly) * g.nx + tb.x0 + lx] = v;
    }
    return;
  }
  struct {
    double eps_q;
    unsigned long long inv_m;
    int inv_e;
  } di = {df.eps_q, df.inv_m, df.inv_e};
  const int n = tb.n, n32 = (n + 31) & ~31;
  const uint32_t raw = (uint32_t)n * W;
  const bool full = n == G::NP;
  const uint32_t* tab = reinterpret_cast<const uint32_t*>(in + kHeaderBytes);
  const uint32_t sb = tab[tid], ss = tab[g.ntiles + tid];
  const uint8_t* rb = in + offs[tid];
  const uint8_t* rs = in + offs[g.ntiles + tid];
  if (threadIdx.x == 0) bad = 0;
  long long t0 = clock64();
  __syncthreads();

  // bins
  // the subbin record goes to A once A is free, behind the bins' work (raw bins never
  // use A); the subbin stage waits for it
  auto prefetch_sub = [&]() {
    if (!bad && !(ss & kRawFlag) && ss >= 4 && ss < raw) {
      const uint32_t n16 = (ss + 15) >> 4;
      for (uint32_t i = threadIdx.x; i < n16; i += NT) {
        const unsigned d = (unsigned)__cvta_generic_to_shared(A + 16 * i);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(rs + 16 * i) : "memory");
      }
    }
  };
  // format 2: bit 30 selects the 1D difference for an encoded bin record; format 1
  // has no other predictor
  if ((sb & kDiffFlag) && (df.version == 1 || (sb & kRawFlag))) bad = 1;
  const bool use_diff = df.version == 1 || (sb & kDiffFlag);
  const uint32_t sb_len = sb & kSizeMask;
  if (sb & kRawFlag) {
    prefetch_sub();
    if (sb_len != raw) bad = 1;
    for (int i = threadIdx.x; i < n; i += NT) wb[i] = reinterpret_cast<const W_t*>(rb)[i];
    __syncthreads();
  } else {
    if (sb_len >= raw) bad = 1;  // an encoded record is shorter than the raw chunk
    __syncthreads();
    uint32_t lw = 0;  // bytes of the bins' planes the decode wrote (the rest is zero)
    if (!bad) {
      copy16<NT>(A, rb, sb_len);
      __syncthreads();
      if (!rze_decode<NT, 1>(A, sb_len, (uint32_t)W * n32, Bf, w, &lw)) bad = 1;
      __syncthreads();
    }
    dec_mark(0, t0);
    prefetch_sub();  // A is free from here on
    if (!bad) {
      constexpr W_t M = (W_t)0xAAAAAAAAAAAAAAAAULL;
      // planes from P on are zero and not read; the rest of plane P - 1 is zeroed
      const int P = planes_in(lw, n32);
      zero_after_decode<NT>(Bf, lw, planes_zero_end(P, n32, (uint32_t)W * n32));
      bit_untranspose<NT, W>(
          n32, reinterpret_cast<const uint32_t*>(Bf),
          [&](int i, uint64_t u) {
            if (i < n)
              wb[i] = (W_t)(((W_t)u ^ M) - M);
            else if (u != 0)
              bad = 1;
          },
          P);
      __syncthreads();
    }
    if (!bad && !use_diff) undo_lorenzo<NT, ND>(wb, tb.cz, tb.cy, tb.cx);
    if (!bad && use_diff) {
      // prefix sum of the deltas (mod 2^(8W)): warp w scans words [w*per, (w+1)*per)
      // in rows of 32 (one word per lane, shuffle scan, running carry), then adds
      // the totals of the warps before it
      constexpr int NWARP = NT / 32;
      const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
      const int per = ((n + NWARP - 1) / NWARP + 31) & ~31;
      const int a = min(n, wid * per), b = min(n, a + per);
      W_t carry = 0;
      for (int r = a; r < b; r += 32) {
        const int i = r + lane;
        W_t v = i < b ? wb[i] : (W_t)0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const W_t y = shfl_up_w(v, o);
          if (lane >= o) v += y;
        }
        v += carry;
        if (i < b) wb[i] = v;
        carry = shfl_idx_w(v, 31);
      }
      __shared__ W_t warp_tot[NWARP];
      if (lane == 0) warp_tot[wid] = carry;
      __syncthreads();
      W_t before = 0;
      for (int k = 0; k < wid; ++k) before += warp_tot[k];
      if (before != (W_t)0)
        for (int i = a + lane; i < b; i += 32) wb[i] += before;
    }
    __syncthreads();
  }
  if (bad) {
    cp_async_wait_all();  // no copy may outlive the block
    if (threadIdx.x == 0) atomicOr(status, kErrCorrupt);
    return;
  }
  dec_mark(1, t0);

  // the lowest value of every bin in [bmin, bmax], when that range is small
  B lo_b = (B)(Traits<T>::kAbsent == INT32_MIN ? INT32_MAX : INT64_MAX), hi_b = (B)Traits<T>::kAbsent;
  for (int i = threadIdx.x; i < n; i += NT) {
    const B b = (B)wb[i];
    lo_b = b < lo_b ? b : lo_b;
    hi_b = b > hi_b ? b : hi_b;
  }
  for (int o = 16; o; o >>= 1) {
    const B a = __shfl_xor_sync(0xffffffffu, lo_b, o), c = __shfl_xor_sync(0xffffffffu, hi_b, o);
    lo_b = a < lo_b ? a : lo_b;
    hi_b = c > hi_b ? c : hi_b;
  }
  if ((threadIdx.x & 31) == 0) {
    red_min[threadIdx.x >> 5] = lo_b;
    red_max[threadIdx.x >> 5] = hi_b;
  }
  __syncthreads();
  B bmin = red_min[0], bmax = red_max[0];
  for (int k = 1; k < NT / 32; ++k) {
    bmin = red_min[k] < bmin ? red_min[k] : bmin;
    bmax = red_max[k] > bmax ? red_max[k] : bmax;
  }
  const bool cached = (unsigned long long)((long long)bmax - (long long)bmin) < (unsigned long long)CAPN;
  if (cached) {
    const int range = (int)((long long)bmax - (long long)bmin) + 1;
    for (int r = threadIdx.x; r < range; r += NT) {
      K k;
      cache[r] = lowest_key_in_bin<T>((long long)bmin + r, di.eps_q, di.inv_m, di.inv_e, k) ? k : kNone;
    }
  }
  __syncthreads();
  // every point's bin becomes its bin's lowest key, in place; the cache is then dead
  bool fail = false;
  for (int i = threadIdx.x; i < n; i += NT) {
    const long long b = (long long)(B)wb[i];
    K k;
    if (cached) {
      k = cache[b - (long long)bmin];
    } else if (!lowest_key_in_bin<T>(b, di.eps_q, di.inv_m, di.inv_e, k)) {
      k = kNone;
    }
    if (k == kNone) fail = true;
    wb[i] = (W_t)k;
  }
  __syncthreads();
  dec_mark(2, t0);

  const int64_t plane = g.ny * g.nx;
  auto put = [&](int i, uint64_t s) {
    const K k = (K)wb[i];
    if (s > (uint64_t)(long long)Traits<T>::kMaxKey - (uint64_t)(long long)k) {
      fail = true;
      return;
    }
    int lx, ly, lz;
    if (full) {
      lx = i % G::TX;
      ly = (i / G::TX) % G::TY;
      lz = i / (G::TX * G::TY);
    } else {
      lx = i % tb.cx;
      ly = (i / tb.cx) % tb.cy;
      lz = i / (tb.cx * tb.cy);
    }
    xhat[(tb.z0 + lz) * plane + (tb.y0 + ly) * g.nx + tb.x0 + lx] = value_of_key<T>((K)(k + (K)s));
  };

  // subbins, reconstructed as they are decoded
  if (ss & kRawFlag) {
    if ((ss & ~kRawFlag) != raw) fail = true;
    else
      for (int i = threadIdx.x; i < n; i += NT) put(i, (uint64_t)reinterpret_cast<const W_t*>(rs)[i]);
  } else {
    if (ss < 4 || ss >= raw) bad = 1;
    __syncthreads();
    uint32_t l2 = 0;
    if (!bad) {
      cp_async_wait_all();  // the record fetched after the bins' RZE stage
      __syncthreads();
      l2 = *reinterpret_cast<const uint32_t*>(A);
      if (l2 > DS::LR) bad = 1;  // uniform: every thread reads the same word
    }
    if (!bad && !rze_decode<NT, 1>(A + 4, ss - 4, l2, Bf, w)) bad = 1;
    __syncthreads();
    dec_mark(3, t0);
    uint32_t lws = 0;  // bytes of the subbins' planes the decode wrote (the rest is zero)
    if (!bad && !rze_decode<NT, W>(Bf, l2, (uint32_t)W * n32, A, w, &lws)) bad = 1;
    __syncthreads();
    dec_mark(4, t0);
    if (!bad) {
      const int P = planes_in(lws, n32);
      zero_after_decode<NT>(A, lws, planes_zero_end(P, n32, (uint32_t)W * n32));
      bit_untranspose<NT, W>(
          n32, reinterpret_cast<const uint32_t*>(A),
          [&](int i, uint64_t u) {
            if (i < n)
              put(i, (uint64_t)(W_t)u);
            else if (u != 0)
              fail = true;
          },
          P);
    }
  }
  cp_async_wait_all();  // no copy may outlive the block (a no-op once the record was consumed)
  if ((__syncthreads_or(fail) || bad) && threadIdx.x == 0) atomicOr(status, kErrCorrupt);
  dec_mark(5, t0);
}

}  // namespace lopc
