// lopc_decompress.cuh -- decompression kernels: record offsets from the size table,
// and one block per chunk that undoes RZE/BIT/DIFFNB for bins and subbins and writes
// x_hat = succ^s(lowest value of bin b) (Sec. III-D, III-E).
#pragma once
#include "lopc_compress.cuh"

namespace lopc {

struct DecodeInfo {
  double eps_q;  // quantizer width (only used for the first guess of a bin's lowest value)
  unsigned long long inv_m;
  int inv_e;
};

// Offsets of the records; flags a table that does not add up to the stream length.
template <int NT>
__global__ void __launch_bounds__(NT) k_dec_offsets(const uint8_t* __restrict__ in, uint64_t total, int64_t ntiles,
                                                     uint64_t* __restrict__ offs, unsigned int* status) {
  __shared__ uint64_t tmp[NT / 32 + 1];
  const int64_t m = 2 * ntiles;
  const uint32_t* tab = reinterpret_cast<const uint32_t*>(in + kHeaderBytes);
  const uint64_t base = kHeaderBytes + pad16((uint64_t)m * 4);
  const int64_t per = (m + NT - 1) / NT;
  const int64_t a = min(m, (int64_t)threadIdx.x * per), b = min(m, a + per);
  uint64_t c = 0;
  for (int64_t i = a; i < b; ++i) c += pad16(tab[i] & ~kRawFlag);
  uint64_t sum;
  uint64_t run = block_exclusive_scan<NT, uint64_t>(c, tmp, &sum) + base;
  for (int64_t i = a; i < b; ++i) {
    offs[i] = run;
    run += pad16(tab[i] & ~kRawFlag);
  }
  if (threadIdx.x == 0 && base + sum != total) atomicOr(status, kErrCorrupt);
}

template <typename T, int ND>
struct DecSmem {
  using C = TileCfg<T, ND>;
  static constexpr int NP = C::TZ * C::TY * C::TX;
  static constexpr int W = Traits<T>::W;
  static constexpr uint32_t L = (uint32_t)NP * W;
  static constexpr uint32_t LR = L + L / 8 + L / 64 + L / 512 + 16;  // largest legal RZE_w output
  static constexpr size_t bytes() {
    return (size_t)NP * W * 2 + L + LR + (LR / 8 + 16) + (LR / 64 + 16) + (LR / 512 + 16) +
           ((LR / 8 + 16) / 4 + 8) * 4 + 64 * 4 + 64;
  }
};

template <typename T, int ND>
__global__ void __launch_bounds__(TileCfg<T, ND>::NT) k_decode(const uint8_t* __restrict__ in, Geometry g,
                                                               DecodeInfo di, const uint64_t* __restrict__ offs,
                                                               T* __restrict__ xhat, unsigned int* status) {
  using C = TileCfg<T, ND>;
  using DS = DecSmem<T, ND>;
  using W_t = typename Traits<T>::Bits;
  using K = typename Traits<T>::Key;
  constexpr int NT = C::NT, W = Traits<T>::W;
  extern __shared__ __align__(16) unsigned char smem[];
  W_t* wb = reinterpret_cast<W_t*>(smem);
  W_t* ws = wb + DS::NP;
  uint32_t* planes = reinterpret_cast<uint32_t*>(ws + DS::NP);
  uint8_t* rz1 = reinterpret_cast<uint8_t*>(planes) + DS::L;
  RzeScratch sc;
  sc.m0 = rz1 + DS::LR;
  sc.m1 = sc.m0 + DS::LR / 8 + 16;
  sc.m2 = sc.m1 + DS::LR / 64 + 16;
  sc.pre = reinterpret_cast<uint32_t*>(((uintptr_t)(sc.m2 + DS::LR / 512 + 16) + 15) & ~(uintptr_t)15);
  sc.tmp = sc.pre + (DS::LR / 8 + 16) / 4 + 8;
  __shared__ int bad;
  if (*status & kErrCorrupt) return;

  const int64_t tid = blockIdx.x;
  const TileBox tb = tile_box(g, tid);
  const int n = tb.n, n32 = (n + 31) & ~31;
  const uint32_t raw = (uint32_t)n * W;
  const uint32_t* tab = reinterpret_cast<const uint32_t*>(in + kHeaderBytes);
  const uint32_t sb = tab[tid], ss = tab[g.ntiles + tid];
  const uint8_t* rb = in + offs[tid];
  const uint8_t* rs = in + offs[g.ntiles + tid];
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();

  // bins
  if (sb & kRawFlag) {
    if ((sb & ~kRawFlag) != raw) bad = 1;
    for (int i = threadIdx.x; i < n; i += NT) wb[i] = reinterpret_cast<const W_t*>(rb)[i];
    __syncthreads();
  } else {
    if (!rze_decode<NT>(rb, sb, (uint32_t)W * n32, 1, reinterpret_cast<uint8_t*>(planes), sc)) bad = 1;
    __syncthreads();
    if (!bad) {
      constexpr W_t M = (W_t)0xAAAAAAAAAAAAAAAAULL;
      bit_untranspose<NT, W>(n32, planes, [&](int i, uint64_t u) {
        if (i < n)
          wb[i] = (W_t)(((W_t)u ^ M) - M);
        else if (u != 0)
          bad = 1;
      });
      __syncthreads();
      // prefix sum of the deltas (mod 2^(8W)), contiguous ranges per thread
      const int per = (n + NT - 1) / NT;
      const int a = min(n, (int)threadIdx.x * per), b = min(n, a + per);
      W_t loc = 0;
      for (int i = a; i < b; ++i) loc += wb[i];
      __shared__ W_t scan_tmp[NT / 32 + 1];
      W_t run = block_exclusive_scan<NT, W_t>(loc, scan_tmp, (W_t*)nullptr);
      for (int i = a; i < b; ++i) {
        run += wb[i];
        wb[i] = run;
      }
    }
    __syncthreads();
  }
  // subbins
  if (!bad) {
    if (ss & kRawFlag) {
      if ((ss & ~kRawFlag) != raw) bad = 1;
      for (int i = threadIdx.x; i < n; i += NT) ws[i] = reinterpret_cast<const W_t*>(rs)[i];
      __syncthreads();
    } else {
      const uint32_t len = ss;
      uint32_t l2 = 0;
      if (len < 4) {
        bad = 1;
      } else {
        l2 = (uint32_t)rs[0] | ((uint32_t)rs[1] << 8) | ((uint32_t)rs[2] << 16) | ((uint32_t)rs[3] << 24);
        if (l2 > DS::LR) bad = 1;
      }
      __syncthreads();
      if (!bad && !rze_decode<NT>(rs + 4, len - 4, l2, 1, rz1, sc)) bad = 1;
      __syncthreads();
      if (!bad && !rze_decode<NT>(rz1, l2, (uint32_t)W * n32, W, reinterpret_cast<uint8_t*>(planes), sc)) bad = 1;
      __syncthreads();
      if (!bad) {
        bit_untranspose<NT, W>(n32, planes, [&](int i, uint64_t u) {
          if (i < n)
            ws[i] = (W_t)u;
          else if (u != 0)
            bad = 1;
        });
      }
      __syncthreads();
    }
  }
  if (bad) {
    if (threadIdx.x == 0) atomicOr(status, kErrCorrupt);
    return;
  }
  // reconstruct
  const int64_t plane = g.ny * g.nx;
  bool fail = false;
  for (int i = threadIdx.x; i < n; i += NT) {
    const long long b = (long long)(typename Traits<T>::Bin)wb[i];
    K k;
    if (!lowest_key_in_bin<T>(b, di.eps_q, di.inv_m, di.inv_e, k)) {
      fail = true;
      continue;
    }
    const uint64_t s = (uint64_t)ws[i];
    if (s > (uint64_t)(Traits<T>::kMaxKey - k)) {
      fail = true;
      continue;
    }
    const int lx = i % tb.cx, ly = (i / tb.cx) % tb.cy, lz = i / (tb.cx * tb.cy);
    xhat[(tb.z0 + lz) * plane + (tb.y0 + ly) * g.nx + tb.x0 + lx] = value_of_key<T>((K)(k + (K)s));
  }
  if (__syncthreads_or(fail) && threadIdx.x == 0) atomicOr(status, kErrCorrupt);
}

template <typename T>
__global__ void k_fill(T* __restrict__ x, int64_t n, unsigned long long bits) {
  const T v = Traits<T>::from_bits((typename Traits<T>::Bits)bits);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = v;
}

}  // namespace lopc
