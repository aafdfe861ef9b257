// lopc_verify.cuh -- the verifier: one pass over a field x and a reconstruction y
// that counts the neighbour pairs whose order differs (the local order of Sec. II,
// ties broken by index), classifies every point of both fields as minimum, maximum,
// saddle or regular from the connected pieces of its lower and upper links (Sec. II),
// counts Table III's false positives, false negatives and false types, and takes the
// value range, the largest absolute error and the sum of squared errors for the
// error bound (Sec. III-A) and the PSNR.
#pragma once
#include "lopc.h"
#include "lopc_compress.cuh"

namespace lopc {

// per-block counters of the verifier
enum {
  kVOrder = 0,
  kVClsX = 1,   // 4 counters: minima, maxima, saddles, regular points of x
  kVClsY = 5,   // the same for y
  kVFalsePos = 9,
  kVFalseNeg,
  kVFalseType,
  kVLink,
  kVNonfinite,
  kVCounters
};

struct VerifyPartial {
  unsigned long long c[kVCounters];
  double max_err, sumsq, xmin, xmax;
};

// Neighbours a and b of a point are joined in its link when b - a is itself a
// neighbour offset: in the Freudenthal triangulation {p, p + a, p + b} is then a
// triangle, and the triangulation is a flag complex, so these edges make the link.
__host__ __device__ constexpr uint32_t link_adjacent(int a) {
  uint32_t r = 0;
  for (int b = 0; b < 14; ++b) {
    const int dz = dz_of(b) - dz_of(a), dy = dy_of(b) - dy_of(a), dx = dx_of(b) - dx_of(a);
    const bool up = dz >= 0 && dz <= 1 && dy >= 0 && dy <= 1 && dx >= 0 && dx <= 1;
    const bool down = dz <= 0 && dz >= -1 && dy <= 0 && dy >= -1 && dx <= 0 && dx >= -1;
    if ((dz != 0 || dy != 0 || dx != 0) && (up || down)) r |= 1u << b;
  }
  return r;
}

// Number of connected pieces of the link vertices in the 14-bit set m (flood fill
// from the lowest vertex left, at most 14 growths per piece).
__device__ inline int link_pieces(uint32_t m) {
  uint32_t rem = m;
  int pieces = 0;
  while (rem) {
    uint32_t piece = rem & (0u - rem), prev = 0;
    while (piece != prev) {
      prev = piece;
      uint32_t grown = piece;
#pragma unroll
      for (int k = 0; k < 14; ++k)
        if (piece & (1u << k)) grown |= link_adjacent(k);
      piece = grown & m;
    }
    rem &= ~piece;
    ++pieces;
  }
  return pieces;
}

template <int ND>
__host__ __device__ constexpr uint32_t all_dirs() {
  uint32_t r = 0;
  for (int k = 0; k < 14; ++k)
    if (ND == 3 || dz_of(k) == 0) r |= 1u << k;
  return r;
}

// Link tables, one thread per 14-bit set m of lower neighbours: cc[m], the pieces of
// m; full3[m] and full2[m], the pieces of m and (<< 4) of the rest of a whole 3D or
// 2D link (an interior point's lower and upper pieces in one lookup).
__global__ void k_link_table(uint8_t* __restrict__ cc, uint8_t* __restrict__ full3, uint8_t* __restrict__ full2) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= (1 << 14)) return;
  const int lo = link_pieces((uint32_t)m);
  cc[m] = (uint8_t)lo;
  full3[m] = (uint8_t)(lo | (link_pieces(all_dirs<3>() & ~(uint32_t)m) << 4));
  full2[m] = (uint8_t)(link_pieces((uint32_t)m & all_dirs<2>()) | (link_pieces(all_dirs<2>() & ~(uint32_t)m) << 4));
}

// Sec. II's classes from a point's (lower pieces | upper pieces << 4): 0 minimum (no
// lower neighbour), 1 maximum (no upper one), 3 regular (one piece each), 2 saddle
__device__ __forceinline__ int cp_class(uint32_t pair) {
  return (pair & 15u) == 0 ? 0 : (pair >> 4) == 0 ? 1 : pair == 0x11u ? 3 : 2;
}

// Lower-neighbour bits of the point at entry e of a box: neighbour k is lower when
// its value is smaller, or equal with a smaller index (k < 7).
template <typename G, typename T>
__device__ __forceinline__ uint32_t lower_bits(const T* v, int e) {
  const T vp = v[e];
  uint32_t m = 0;
#pragma unroll
  for (int k = 0; k < 14; ++k) {
    if (!G::HZ && dz_of(k) != 0) continue;
    const T vn = v[e + G::off(dz_of(k), dy_of(k), dx_of(k))];
    if (k < 7 ? vn <= vp : vn < vp) m |= 1u << k;
  }
  return m;
}

template <typename T, int ND>
struct VerifySmem {
  using G = TileGeom<T, ND, true>;
  static constexpr size_t up16(size_t v) { return (v + 15) & ~(size_t)15; }
  static constexpr size_t box = up16((size_t)G::E * sizeof(T));
  static constexpr size_t bytes() { return 2 * box; }
};

// A persistent block walks tiles blockIdx.x, + gridDim.x, ...: both boxes (tile and
// halo) staged with asynchronous copies, then one thread per y-segment of a column
// classifies its points.  Partial sums go to part[blockIdx.x] in a fixed order, so
// the result does not depend on scheduling.  With types_x (and types_y) given, each
// point's link piece counts, lower | upper << 4, are written in C order.
template <typename T, int ND>
__global__ void __launch_bounds__(TileCfg<T, ND>::NT, 3) k_verify(Geometry g, const T* __restrict__ x,
                                                              const T* __restrict__ y,
                                                              const uint8_t* __restrict__ cc,
                                                              const uint8_t* __restrict__ full,
                                                              uint8_t* __restrict__ types_x,
                                                              uint8_t* __restrict__ types_y,
                                                              VerifyPartial* __restrict__ part) {
  using G = TileGeom<T, ND, true>;
  using VS = VerifySmem<T, ND>;
  using Raw = typename Traits<T>::Bits;
  constexpr int NT = G::NT, NWARP = NT / 32;
  constexpr uint32_t kUpper = 0x3F80u;  // directions 7..13: each neighbour pair once
  extern __shared__ __align__(16) unsigned char smem[];
  T* xs = reinterpret_cast<T*>(smem);
  T* ys = reinterpret_cast<T*>(smem + VS::box);
  const SegPos sp = seg_pos<G>();

  unsigned cnt[kVCounters];
#pragma unroll
  for (int i = 0; i < kVCounters; ++i) cnt[i] = 0;
  // largest error: for float fields the f32 difference (rounded, monotone in the
  // exact one) picks the candidates and only those take the binary64 difference
  float m32 = -1.0f;
  double m64 = 0.0, sumsq = 0.0;
  T vmin = (T)INFINITY, vmax = (T)-INFINITY;
  constexpr uint32_t FULL = all_dirs<ND>();
  constexpr uint32_t YL = dir_mask(1, -1), YH = dir_mask(1, 1);

  for (int64_t tid = blockIdx.x; tid < g.ntiles; tid += gridDim.x) {
    const TileBox tb = tile_box(g, tid);
    load_box_async<G, Raw>(reinterpret_cast<Raw*>(xs), reinterpret_cast<const Raw*>(x), g, tb);
    load_box_async<G, Raw>(reinterpret_cast<Raw*>(ys), reinterpret_cast<const Raw*>(y), g, tb);
    cp_async_wait_all();
    __syncthreads();
    if (sp.lz < tb.cz && sp.lx < tb.cx) {
      const int64_t gz = tb.z0 + sp.lz, gx = tb.x0 + sp.lx;
      // neighbours outside the field: x and z faces per column, y faces per point
      uint32_t col = FULL & ~((gx == 0 ? dir_mask(2, -1) : 0u) | (gx == g.nx - 1 ? dir_mask(2, 1) : 0u));
      if (ND == 3) col &= ~((gz == 0 ? dir_mask(0, -1) : 0u) | (gz == g.nz - 1 ? dir_mask(0, 1) : 0u));
      const int yfirst = tb.y0 == 0 ? 0 : -1;
      const int ylast = tb.y0 + tb.cy == g.ny ? tb.cy - 1 : -1;
      // (class of x, class of y) counts of this tile, one byte each: lo holds x
      // classes 0-1, hi classes 2-3
      unsigned long long conf_lo = 0, conf_hi = 0;
      float s32 = 0.0f;
#pragma unroll 2
      for (int j = 0; j < G::SEG; ++j) {
        const int ly = sp.ly0 + j;
        if (ly >= tb.cy) break;
        const int e = sp.e0 + j * G::BXP;
        const uint32_t pres = col & ~((ly == yfirst ? YL : 0u) | (ly == ylast ? YH : 0u));
        const uint32_t lx_ = lower_bits<G>(xs, e) & pres;
        const uint32_t ly_ = lower_bits<G>(ys, e) & pres;
        cnt[kVOrder] += __popc((lx_ ^ ly_) & kUpper);
        uint32_t px, py;
        if (pres == FULL) {
          px = __ldg(&full[lx_]);
          py = __ldg(&full[ly_]);
        } else {
          px = __ldg(&cc[lx_]) | ((uint32_t)__ldg(&cc[pres & ~lx_]) << 4);
          py = __ldg(&cc[ly_]) | ((uint32_t)__ldg(&cc[pres & ~ly_]) << 4);
        }
        if (types_x) {
          const int64_t gi = (gz * g.ny + tb.y0 + ly) * g.nx + gx;
          types_x[gi] = (uint8_t)px;
          if (types_y) types_y[gi] = (uint8_t)py;
        }
        cnt[kVLink] += px != py;
        const int cell = cp_class(px) * 4 + cp_class(py);
        const unsigned long long inc = 1ull << (8 * (cell & 7));
        conf_lo += cell < 8 ? inc : 0ull;
        conf_hi += cell < 8 ? 0ull : inc;
        const T xv = xs[e], yv = ys[e];
        cnt[kVNonfinite] += !(fabs(xv) <= Traits<T>::kMaxFinite && fabs(yv) <= Traits<T>::kMaxFinite);
        vmin = xv < vmin ? xv : vmin;
        vmax = xv > vmax ? xv : vmax;
        if (sizeof(T) == 4) {
          const float d = fabsf((float)xv - (float)yv);
          s32 = fmaf(d, d, s32);
          if (d >= m32) {
            const double d64 = fabs((double)xv - (double)yv);
            m64 = d > m32 ? d64 : fmax(m64, d64);
            m32 = d;
          }
        } else {
          const double d = fabs((double)xv - (double)yv);
          sumsq = fma(d, d, sumsq);
          m64 = fmax(m64, d);
        }
      }
      // the tile's (x class, y class) counts into the class and Table III counters
#pragma unroll
      for (int cx = 0; cx < 4; ++cx) {
#pragma unroll
        for (int cy = 0; cy < 4; ++cy) {
          const int cell = cx * 4 + cy;
          const unsigned v = (unsigned)(((cell < 8 ? conf_lo : conf_hi) >> (8 * (cell & 7))) & 0xFFu);
          cnt[kVClsX + cx] += v;
          cnt[kVClsY + cy] += v;
          if (cx == 3 && cy != 3) cnt[kVFalsePos] += v;
          if (cx != 3 && cy == 3) cnt[kVFalseNeg] += v;
          if (cx != 3 && cy != 3 && cx != cy) cnt[kVFalseType] += v;
        }
      }
      sumsq += (double)s32;
    }
    __syncthreads();  // the boxes are reloaded for the next tile
  }

  // block reduction in a fixed order: warps by shuffles, then warp 0 over the warps
  __shared__ unsigned wc[NWARP][kVCounters];
  __shared__ double wd[NWARP][4];
  __shared__ int wm[NWARP];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < kVCounters; ++i) {
    const unsigned s = __reduce_add_sync(0xffffffffu, cnt[i]);
    if (lane == 0) wc[warp][i] = s;
  }
  // the largest f32 difference of the block; only threads that hold it keep m64
  int mb = __reduce_max_sync(0xffffffffu, __float_as_int(m32));
  if (lane == 0) wm[warp] = mb;
  __syncthreads();
  mb = wm[0];
  for (int w = 1; w < NWARP; ++w) mb = max(mb, wm[w]);
  double cand = (sizeof(T) == 8 || __float_as_int(m32) == mb) ? m64 : 0.0;
  double xmn = (double)vmin, xmx = (double)vmax, ss = sumsq;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    cand = fmax(cand, __shfl_xor_sync(0xffffffffu, cand, o));
    xmn = fmin(xmn, __shfl_xor_sync(0xffffffffu, xmn, o));
    xmx = fmax(xmx, __shfl_xor_sync(0xffffffffu, xmx, o));
    ss += __shfl_xor_sync(0xffffffffu, ss, o);
  }
  if (lane == 0) {
    wd[warp][0] = cand;
    wd[warp][1] = ss;
    wd[warp][2] = xmn;
    wd[warp][3] = xmx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    VerifyPartial p;
    for (int i = 0; i < kVCounters; ++i) {
      unsigned long long s = 0;
      for (int w = 0; w < NWARP; ++w) s += wc[w][i];
      p.c[i] = s;
    }
    p.max_err = wd[0][0];
    p.sumsq = wd[0][1];
    p.xmin = wd[0][2];
    p.xmax = wd[0][3];
    for (int w = 1; w < NWARP; ++w) {
      p.max_err = fmax(p.max_err, wd[w][0]);
      p.sumsq += wd[w][1];
      p.xmin = fmin(p.xmin, wd[w][2]);
      p.xmax = fmax(p.xmax, wd[w][3]);
    }
    part[blockIdx.x] = p;
  }
}

// The report from the blocks' partial sums (one block; thread t takes partials t,
// t + NT, ..., then a fixed tree): counts, range, error bound and PSNR.
template <int NT>
__global__ void __launch_bounds__(NT) k_verify_finalize(const VerifyPartial* __restrict__ part, int nparts,
                                                        int64_t points, int mode, double eb,
                                                        lopc_verify_report* __restrict__ rep) {
  __shared__ unsigned long long sc[NT][kVCounters];
  __shared__ double sd[NT][4];
  unsigned long long c[kVCounters];
#pragma unroll
  for (int i = 0; i < kVCounters; ++i) c[i] = 0;
  double mx = 0.0, ss = 0.0, lo = INFINITY, hi = -INFINITY;
  for (int i = threadIdx.x; i < nparts; i += NT) {
    const VerifyPartial& p = part[i];
#pragma unroll
    for (int k = 0; k < kVCounters; ++k) c[k] += p.c[k];
    mx = fmax(mx, p.max_err);
    ss += p.sumsq;
    lo = fmin(lo, p.xmin);
    hi = fmax(hi, p.xmax);
  }
#pragma unroll
  for (int k = 0; k < kVCounters; ++k) sc[threadIdx.x][k] = c[k];
  sd[threadIdx.x][0] = mx;
  sd[threadIdx.x][1] = ss;
  sd[threadIdx.x][2] = lo;
  sd[threadIdx.x][3] = hi;
  __syncthreads();
  for (int h = NT / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      const int o = threadIdx.x + h;
      for (int k = 0; k < kVCounters; ++k) sc[threadIdx.x][k] += sc[o][k];
      sd[threadIdx.x][0] = fmax(sd[threadIdx.x][0], sd[o][0]);
      sd[threadIdx.x][1] += sd[o][1];
      sd[threadIdx.x][2] = fmin(sd[threadIdx.x][2], sd[o][2]);
      sd[threadIdx.x][3] = fmax(sd[threadIdx.x][3], sd[o][3]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    lopc_verify_report r;
    r.points = points;
    r.order_violations = (int64_t)sc[0][kVOrder];
    for (int k = 0; k < 4; ++k) {
      r.cp_x[k] = (int64_t)sc[0][kVClsX + k];
      r.cp_y[k] = (int64_t)sc[0][kVClsY + k];
    }
    r.false_positives = (int64_t)sc[0][kVFalsePos];
    r.false_negatives = (int64_t)sc[0][kVFalseNeg];
    r.false_types = (int64_t)sc[0][kVFalseType];
    r.link_mismatches = (int64_t)sc[0][kVLink];
    r.nonfinite = (int64_t)sc[0][kVNonfinite];
    r.x_min = sd[0][2];
    r.x_max = sd[0][3];
    r.max_abs_err = sd[0][0];
    r.mse = points ? sd[0][1] / (double)points : 0.0;
    const double range = r.x_max - r.x_min;
    r.psnr = r.mse == 0.0 ? INFINITY : range == 0.0 ? -INFINITY : 20.0 * log10(range) - 10.0 * log10(r.mse);
    r.eps = mode == LOPC_ABS ? eb : eb * range;
    r.bound_ok = r.max_abs_err <= r.eps ? 1 : 0;
    r.reserved = 0;
    *rep = r;
  }
}

}  // namespace lopc
