// lopc_worklist.cuh -- the paper's own GPU repair schedule (Sec. III-D, Alg. 1's
// main loop around Alg. 2), kept as an alternate repair mode beside the tile design:
// one thread per worklist item p evaluates
//   n_max = max over same-bin lower neighbours n of s(n) + [idx_n > idx_p]
// and raises s(p) with atomicMax; a point whose subbin rose puts its greater
// same-bin neighbours on the next worklist, each point at most once per iteration
// (an atomically raised iteration stamp, Sec. III-D).  Subbins start at 0 and the
// first iteration takes every point.  Raised subbins are visible to the rest of the
// iteration (neighbours are read through L2), so the schedule is chaotic relaxation
// from lower bounds and reaches the unique least fixpoint (Sec. III-E), the same
// subbins as the tile design.  The iterations run in a CUDA-graph while-node whose
// condition the one-thread swap kernel sets, instead of a host loop reading the
// worklist size after every iteration.
#pragma once
#include "lopc_compress.cuh"

namespace lopc {

struct WorklistState {
  unsigned int n[2];  // items on the two worklists; iteration i reads n[i & 1]
  unsigned int iter;  // iterations done
  unsigned int go;    // the loop continues (for the host-driven loop)
  unsigned long long evals, raises;
};

// Linear offset of neighbour direction k in a field of g's extents.
__device__ __forceinline__ int64_t lin_offset(const Geometry& g, int k) {
  return ((int64_t)dz_of(k) * g.ny + dy_of(k)) * g.nx + dx_of(k);
}

// One iteration over the current worklist (all != 0: every point of the field, the
// first iteration).  wl holds two lists of a field's point count each.
__global__ void __launch_bounds__(256) k_wl_iter(const FieldInfo* __restrict__ F, WorklistState* __restrict__ W,
                                                 uint32_t* __restrict__ wl, uint32_t* __restrict__ stamp, int all) {
  const FieldInfo& f = F[0];
  if (f.P->status || f.P->constant) return;  // no flags or subbins were written
  const Geometry g = f.g;
  const int64_t npts = g.nz * g.ny * g.nx;
  const unsigned iter = W->iter;
  const uint32_t* in = wl + (size_t)(iter & 1) * (size_t)npts;
  uint32_t* out = wl + (size_t)((iter + 1) & 1) * (size_t)npts;
  unsigned int* nout = &W->n[(iter + 1) & 1];
  const int64_t n = all ? npts : (int64_t)W->n[iter & 1];
  const unsigned next = iter + 1;  // the stamp of the next worklist
  uint32_t* s = f.s;
  const uint32_t* __restrict__ cm = f.cm;
  const int lane = threadIdx.x & 31;
  unsigned evals = 0, raises = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // a uniform trip count per warp: every lane takes part in the append
  for (int64_t b0 = (int64_t)blockIdx.x * blockDim.x; b0 < n; b0 += stride) {
    const int64_t i = b0 + threadIdx.x;
    uint32_t push = 0;
    int64_t p = 0;
    if (i < n) {
      p = all ? i : (int64_t)in[i];
      const uint32_t m = cm[p];
      const uint32_t lower = m & 0x3FFFu;
      if (lower) {
        ++evals;
        uint32_t nmax = 0;
#pragma unroll
        for (int k = 0; k < 14; ++k) {
          if (lower & (1u << k)) {
            const uint32_t v = __ldcg(&s[p + lin_offset(g, k)]) + (k >= 7 ? 1u : 0u);
            nmax = v > nmax ? v : nmax;
          }
        }
        if (atomicMax(&s[p], nmax) < nmax) {
          ++raises;
          const uint32_t upper = (m >> 16) & ~lower & 0x3FFFu;
#pragma unroll
          for (int k = 0; k < 14; ++k) {
            if (upper & (1u << k)) {
              if (atomicMax(&stamp[p + lin_offset(g, k)], next) < next) push |= 1u << k;
            }
          }
        }
      }
    }
    // warp-aggregated append of the pushed neighbours
    const unsigned c = __popc(push);
    unsigned incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const unsigned wt = __shfl_sync(0xffffffffu, incl, 31);
    unsigned pos = 0;
    if (lane == 31 && wt) pos = atomicAdd(nout, wt);
    pos = __shfl_sync(0xffffffffu, pos, 31) + incl - c;
#pragma unroll
    for (int k = 0; k < 14; ++k)
      if (push & (1u << k)) out[pos++] = (uint32_t)(p + lin_offset(g, k));
  }
  block_add2(evals, raises, &W->evals);
}

// After an iteration: clear the list just read (it is written two iterations later),
// count the iteration, stop at an empty worklist or past the field's round cap
// (status NOT_CONVERGED), and publish the counters.  One thread.
__global__ void k_wl_next(const FieldInfo* __restrict__ F, WorklistState* __restrict__ W, BatchState* __restrict__ B,
                          cudaGraphConditionalHandle handle, int use_handle) {
  const FieldInfo& f = F[0];
  const unsigned it = W->iter;
  W->n[it & 1] = 0u;
  W->iter = it + 1;
  const unsigned nn = W->n[(it + 1) & 1];
  f.P->rounds += 1;
  unsigned go = nn ? 1u : 0u;
  if (go && (long long)f.P->rounds > f.round_cap) {
    atomicOr(&f.P->status, kErrNotConverged);
    B->cap_hit = 1u;
    go = 0u;
  }
  if (f.P->status) go = 0u;
  W->go = go;
  B->count[0] = go ? nn : 0u;
  B->rounds += 1;
  f.P->work[2] = W->evals;
  f.P->work[3] = W->raises;
  if (use_handle) cudaGraphSetConditional(handle, go);
}

}  // namespace lopc
