// lopc_capi.cu -- host side of the C ABI (include/lopc.h): argument checks, the
// workspace layout, and the launch sequences of compression and decompression.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <mutex>

#include "lopc.h"
#include "lopc_decompress.cuh"

using namespace lopc;

namespace {

thread_local int64_t g_round_cap = 0;  // 0 = default

// ---------------------------------------------------------------- profiling
// Event pairs around each launch while profiling is on; resolved at the end of
// every API call, after its final synchronisation.
struct ProfEntry {
  const char* name;
  int64_t launches;
  double ms;
};
struct Pending {
  int entry;
  cudaEvent_t a, b;
};
struct Profiler {
  bool on = false;
  ProfEntry entries[64];
  int n = 0;
  Pending pend[4096];
  int npend = 0;
  cudaEvent_t pool[8192];
  int npool = 0, used = 0;
  int entry_of(const char* name) {
    for (int i = 0; i < n; ++i)
      if (entries[i].name == name) return i;
    if (n == 64) return -1;
    entries[n] = ProfEntry{name, 0, 0.0};
    return n++;
  }
  cudaEvent_t event() {
    if (used == npool) {
      if (npool == 8192) return nullptr;
      if (cudaEventCreate(&pool[npool]) != cudaSuccess) return nullptr;
      ++npool;
    }
    return pool[used++];
  }
  void before(const char* name, cudaStream_t st) {
    if (!on || npend == 4096) return;
    const int e = entry_of(name);
    cudaEvent_t a = event(), b = event();
    if (e < 0 || !a || !b) return;
    cudaEventRecord(a, st);
    pend[npend] = Pending{e, a, b};
  }
  void after(cudaStream_t st) {
    if (!on || npend == 4096) return;
    if (!pend[npend].a) return;
    cudaEventRecord(pend[npend].b, st);
    ++npend;
    pend[npend].a = nullptr;
  }
  void resolve() {
    for (int i = 0; i < npend; ++i) {
      float ms = 0.f;
      if (cudaEventSynchronize(pend[i].b) == cudaSuccess && cudaEventElapsedTime(&ms, pend[i].a, pend[i].b) == cudaSuccess) {
        entries[pend[i].entry].launches += 1;
        entries[pend[i].entry].ms += ms;
      }
    }
    npend = 0;
    used = 0;
    pend[0].a = nullptr;
  }
};
thread_local Profiler g_prof;

#define LAUNCH(name, st, ...)       \
  do {                              \
    g_prof.before(name, st);        \
    __VA_ARGS__;                    \
    g_prof.after(st);               \
  } while (0)
thread_local int64_t g_last_rounds = 0, g_last_tile_runs = 0, g_last_fix_iters = 0, g_last_fix_iters_max = 0;
thread_local int64_t g_last_phase[8] = {};

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }
int64_t imin64(int64_t a, int64_t b) { return a < b ? a : b; }

bool desc_valid(const lopc_field_desc* d) {
  if (!d) return false;
  if (d->dtype != LOPC_F32 && d->dtype != LOPC_F64) return false;
  if (d->ndim != 2 && d->ndim != 3) return false;
  if (d->mode != LOPC_ABS && d->mode != LOPC_NOA) return false;
  if (!(d->eb > 0.0) || !(d->eb <= 1.79e308)) return false;
  uint64_t n = 1;
  for (int k = 0; k < d->ndim; ++k) {
    if (d->dims[k] <= 0 || d->dims[k] > (int64_t(1) << 32)) return false;
    n *= (uint64_t)d->dims[k];
    if (n >= (uint64_t(1) << 32)) return false;
  }
  return true;
}

int word_bytes(int dtype) { return dtype == LOPC_F32 ? 4 : 8; }

Geometry geometry_of(const lopc_field_desc* d) {
  Geometry g;
  g.ndim = d->ndim;
  g.dtype = d->dtype;
  if (d->ndim == 2) {
    g.nz = 1;
    g.ny = d->dims[0];
    g.nx = d->dims[1];
    g.tz = 1;
    g.ty = d->dtype == LOPC_F32 ? 64 : 32;
    g.tx = 64;
  } else {
    g.nz = d->dims[0];
    g.ny = d->dims[1];
    g.nx = d->dims[2];
    g.tz = d->dtype == LOPC_F32 ? 16 : 8;
    g.ty = 16;
    g.tx = 16;
  }
  g.ntz = ceil_div(g.nz, g.tz);
  g.nty = ceil_div(g.ny, g.ty);
  g.ntx = ceil_div(g.nx, g.tx);
  g.ntiles = g.ntz * g.nty * g.ntx;
  return g;
}

struct CompressLayout {
  size_t params, dirty, done, list, s, cm, sizes, offs, slots, total;
};

CompressLayout compress_layout(const lopc_field_desc* d) {
  const Geometry g = geometry_of(d);
  const size_t n = (size_t)(g.nz * g.ny * g.nx);
  CompressLayout L;
  size_t o = 0;
  L.params = o;
  o = align256(o + sizeof(Params));
  L.dirty = o;
  o = align256(o + (size_t)g.ntiles);
  L.done = o;
  o = align256(o + (size_t)g.ntiles);
  L.list = o;
  o = align256(o + 4 * (size_t)g.ntiles);
  L.s = o;
  o = align256(o + 4 * n);
  L.cm = o;
  o = align256(o + 2 * n);
  L.sizes = o;
  o = align256(o + 8 * (size_t)g.ntiles);
  L.offs = o;
  o = align256(o + 16 * (size_t)g.ntiles);
  L.slots = o;
  o = align256(o + 2 * (size_t)g.ntiles * kSlotBytes);
  L.total = o;
  return L;
}

#define CK(call)                          \
  do {                                    \
    if ((call) != cudaSuccess) {          \
      (void)cudaGetLastError();           \
      return LOPC_ERR_CUDA;               \
    }                                     \
  } while (0)

int status_to_code(unsigned int st) {
  if (st & kErrNonfinite) return LOPC_ERR_NONFINITE;
  if (st & kErrRange) return LOPC_ERR_RANGE;
  if (st & kErrNotConverged) return LOPC_ERR_NOT_CONVERGED;
  if (st & kErrCorrupt) return LOPC_ERR_CORRUPT;
  if (st & kErrInternal) return LOPC_ERR_CUDA;
  return LOPC_OK;
}

template <typename T, int ND>
int run_repair(const lopc_field_desc* d, const Geometry& g, const T* x, uint8_t* ws, const CompressLayout& L,
               int64_t* bins_out, cudaStream_t st) {
  using C = TileCfg<T, ND>;
  Params* P = reinterpret_cast<Params*>(ws + L.params);
  uint8_t* dirty = ws + L.dirty;
  uint32_t* list = reinterpret_cast<uint32_t*>(ws + L.list);
  uint32_t* s = reinterpret_cast<uint32_t*>(ws + L.s);
  uint16_t* cm = reinterpret_cast<uint16_t*>(ws + L.cm);
  uint32_t* sizes = reinterpret_cast<uint32_t*>(ws + L.sizes);
  const int64_t n = g.nz * g.ny * g.nx;

  LAUNCH("init_params", st, k_init_params<<<1, 1, 0, st>>>(P, d->eb, d->mode));
  if (d->mode == LOPC_NOA) LAUNCH("range", st, k_range<T><<<148 * 8, 256, 0, st>>>(x, n, P));
  LAUNCH("resolve_eps", st, k_resolve_eps<T><<<1, 1, 0, st>>>(P));
  CK(cudaMemsetAsync(dirty, 0, (size_t)g.ntiles, st));
  const size_t psmem = PassSmem<T, ND>::bytes(), rsmem = RerunSmem<T, ND>::bytes();
  CK(cudaFuncSetAttribute(k_pass<T, ND>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psmem));
  CK(cudaFuncSetAttribute(k_rerun<T, ND>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsmem));
  LAUNCH("tile_pass", st,
         k_pass<T, ND><<<(unsigned)g.ntiles, C::NT, psmem, st>>>(x, g, P, s, cm, bins_out, ws + L.slots, sizes));
  CK(cudaGetLastError());
  // round 1 visits every tile: each one tests its own incoming cross-tile constraints
  LAUNCH("tile_rerun", st, k_rerun<T, ND><<<(unsigned)g.ntiles, C::NT, rsmem, st>>>(g, P, s, cm, dirty, nullptr));
  CK(cudaGetLastError());
  int64_t runs = 2 * g.ntiles, rounds = 1;
  const int64_t cap = g_round_cap > 0 ? g_round_cap : n + 16;  // a chain has fewer than n links
  const unsigned cgrid = (unsigned)imin64(ceil_div(g.ntiles, 256), 148 * 16);
  while (true) {
    CK(cudaMemsetAsync(&P->dirty_count, 0, sizeof(unsigned), st));
    LAUNCH("compact", st, k_compact<<<cgrid, 256, 0, st>>>(dirty, g.ntiles, list, P));
    unsigned cnt = 0, status = 0;
    CK(cudaMemcpyAsync(&cnt, &P->dirty_count, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&status, &P->status, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (status & (kErrNonfinite | kErrRange | kErrNotConverged)) break;
    if (cnt == 0) break;
    if (rounds >= cap) {
      unsigned bit = kErrNotConverged;
      CK(cudaMemcpyAsync(&P->status, &bit, sizeof(unsigned), cudaMemcpyHostToDevice, st));
      CK(cudaStreamSynchronize(st));
      break;
    }
    LAUNCH("tile_rerun", st, k_rerun<T, ND><<<cnt, C::NT, rsmem, st>>>(g, P, s, cm, dirty, list));
    CK(cudaGetLastError());
    runs += cnt;
    ++rounds;
  }
  g_last_rounds = rounds;
  g_last_tile_runs = runs;
  return LOPC_OK;
}

template <typename T, int ND>
int compress_impl(const lopc_field_desc* d, const void* d_x, void* d_out, size_t out_cap, size_t* out_size,
                  void* d_ws, cudaStream_t st) {
  using C = TileCfg<T, ND>;
  using B = typename Traits<T>::Bin;
  const Geometry g = geometry_of(d);
  const CompressLayout L = compress_layout(d);
  uint8_t* ws = reinterpret_cast<uint8_t*>(d_ws);
  Params* P = reinterpret_cast<Params*>(ws + L.params);
  int rc = run_repair<T, ND>(d, g, reinterpret_cast<const T*>(d_x), ws, L, nullptr, st);
  if (rc) return rc;
  const size_t esmem = EncSmem<T, ND>::bytes();
  CK(cudaFuncSetAttribute(k_encode_sub<T, ND>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)esmem));
  uint32_t* sizes = reinterpret_cast<uint32_t*>(ws + L.sizes);
  uint64_t* offs = reinterpret_cast<uint64_t*>(ws + L.offs);
  LAUNCH("encode_subbins", st,
         k_encode_sub<T, ND><<<(unsigned)g.ntiles, C::NT, esmem, st>>>(g, P, reinterpret_cast<const uint32_t*>(ws + L.s),
                                                                     ws + L.slots, sizes));
  CK(cudaGetLastError());
  const int64_t m = 2 * g.ntiles;
  const uint64_t base = kHeaderBytes + ((uint64_t)m * 4 + 15) / 16 * 16;
  LAUNCH("scan_sizes", st, k_scan_sizes<1024><<<1, 1024, 0, st>>>(sizes, m, base, offs, P));
  HeaderInfo h;
  h.dtype = d->dtype;
  h.ndim = d->ndim;
  h.mode = d->mode;
  for (int k = 0; k < 3; ++k) h.dims[k] = k < d->ndim ? d->dims[k] : 0;
  h.tile[0] = g.tz;
  h.tile[1] = g.ty;
  h.tile[2] = g.tx;
  h.eb = d->eb;
  const unsigned pgrid = (unsigned)imin64(m, 148 * 16);
  LAUNCH("pack", st, k_pack<<<pgrid, 256, 0, st>>>(h, g.ntiles, sizes, offs, ws + L.slots, reinterpret_cast<uint8_t*>(d_out),
                                (uint64_t)out_cap, P));
  CK(cudaGetLastError());
  Params hp;
  CK(cudaMemcpyAsync(&hp, P, sizeof(Params), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  g_last_fix_iters = (int64_t)hp.fix_iters;
  g_last_fix_iters_max = (int64_t)hp.fix_iters_max;
  for (int k = 0; k < 8; ++k) g_last_phase[k] = (int64_t)hp.phase[k];
  rc = status_to_code(hp.status);
  if (rc) return rc;
  if (hp.total > out_cap) return LOPC_ERR_CAPACITY;
  *out_size = (size_t)hp.total;
  return LOPC_OK;
}

template <typename T, int ND>
int quantize_repair_impl(const lopc_field_desc* d, const void* d_x, int64_t* bins, uint64_t* subbins, void* d_ws,
                         cudaStream_t st) {
  const Geometry g = geometry_of(d);
  const CompressLayout L = compress_layout(d);
  uint8_t* ws = reinterpret_cast<uint8_t*>(d_ws);
  int rc = run_repair<T, ND>(d, g, reinterpret_cast<const T*>(d_x), ws, L, bins, st);
  if (rc) return rc;
  const int64_t n = g.nz * g.ny * g.nx;
  LAUNCH("export", st, k_export_subbins<<<148 * 8, 256, 0, st>>>(n, reinterpret_cast<const uint32_t*>(ws + L.s), subbins));
  CK(cudaGetLastError());
  Params hp;
  CK(cudaMemcpyAsync(&hp, ws + L.params, sizeof(Params), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  g_last_fix_iters = (int64_t)hp.fix_iters;
  g_last_fix_iters_max = (int64_t)hp.fix_iters_max;
  return status_to_code(hp.status);
}

// ------------------------------------------------------------ header parsing

uint64_t rd(const uint8_t* p, int nb) {
  uint64_t v = 0;
  for (int k = 0; k < nb; ++k) v |= (uint64_t)p[k] << (8 * k);
  return v;
}

struct Header {
  lopc_field_desc d;
  int constant;
  double eps, inv;
  uint64_t const_bits, nchunks, total;
};

int parse_header(const uint8_t* h, size_t n, Header* H) {
  if (!h || n < (size_t)kHeaderBytes) return LOPC_ERR_CORRUPT;
  if (rd(h, 4) != kMagic || rd(h + 4, 2) != LOPC_VERSION) return LOPC_ERR_CORRUPT;
  memset(H, 0, sizeof(*H));
  H->d.dtype = h[6];
  H->d.ndim = h[7];
  H->d.mode = h[32];
  H->constant = h[33];
  for (int k = 0; k < 3; ++k) H->d.dims[k] = (int64_t)rd(h + 8 + 8 * k, 8);
  uint64_t ebu = rd(h + 48, 8);
  memcpy(&H->d.eb, &ebu, 8);
  if (H->d.ndim == 2 && H->d.dims[2] != 0) return LOPC_ERR_CORRUPT;
  if (H->constant > 1 || !desc_valid(&H->d)) return LOPC_ERR_CORRUPT;
  const Geometry g = geometry_of(&H->d);
  if (rd(h + 36, 4) != (uint64_t)g.tz || rd(h + 40, 4) != (uint64_t)g.ty || rd(h + 44, 4) != (uint64_t)g.tx)
    return LOPC_ERR_CORRUPT;
  uint64_t u = rd(h + 56, 8);
  memcpy(&H->eps, &u, 8);
  u = rd(h + 64, 8);
  memcpy(&H->inv, &u, 8);
  H->const_bits = rd(h + 72, 8);
  H->nchunks = rd(h + 80, 8);
  H->total = rd(h + 88, 8);
  if (H->total < (uint64_t)kHeaderBytes) return LOPC_ERR_CORRUPT;
  if (H->constant ? (H->nchunks != 0 || H->total != (uint64_t)kHeaderBytes) : H->nchunks != (uint64_t)g.ntiles)
    return LOPC_ERR_CORRUPT;
  if (!H->constant && !(H->inv > 0.0 && H->inv <= 1.79e308)) return LOPC_ERR_CORRUPT;
  return LOPC_OK;
}

template <typename T, int ND>
int decompress_impl(const Header& H, const uint8_t* in, size_t in_size, void* d_x, uint8_t* ws, cudaStream_t st) {
  using C = TileCfg<T, ND>;
  const Geometry g = geometry_of(&H.d);
  const int64_t n = g.nz * g.ny * g.nx;
  unsigned int* status = reinterpret_cast<unsigned int*>(ws);
  uint64_t* offs = reinterpret_cast<uint64_t*>(ws + 256);
  CK(cudaMemsetAsync(status, 0, sizeof(unsigned), st));
  if (H.constant) {
    LAUNCH("fill", st, k_fill<T><<<148 * 8, 256, 0, st>>>(reinterpret_cast<T*>(d_x), n, H.const_bits));
  } else {
    if ((uint64_t)kHeaderBytes + ((uint64_t)g.ntiles * 8 + 15) / 16 * 16 > H.total) return LOPC_ERR_CORRUPT;
    LAUNCH("dec_offsets", st, k_dec_offsets<1024><<<1, 1024, 0, st>>>(in, H.total, g.ntiles, offs, status));
    const size_t smem = DecSmem<T, ND>::bytes();
    CK(cudaFuncSetAttribute(k_decode<T, ND>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    DecodeInfo di;
    di.eps_q = 1.0 / H.inv;  // only seeds the search for a bin's lowest value
    const uint64_t iu = [&] {
      uint64_t v;
      memcpy(&v, &H.inv, 8);
      return v;
    }();
    const int ex = (int)((iu >> 52) & 0x7ff);
    di.inv_m = (iu & 0xfffffffffffffULL) | (ex ? 0x10000000000000ULL : 0ULL);
    di.inv_e = ex ? ex - 1075 : -1074;
    LAUNCH("decode", st, k_decode<T, ND><<<(unsigned)g.ntiles, C::NT, smem, st>>>(in, g, di, offs, reinterpret_cast<T*>(d_x), status));
  }
  CK(cudaGetLastError());
  unsigned hs = 0;
  CK(cudaMemcpyAsync(&hs, status, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  (void)in_size;
  return hs ? LOPC_ERR_CORRUPT : LOPC_OK;
}

}  // namespace

// ================================================================ C ABI

extern "C" {

size_t lopc_compress_bound(const lopc_field_desc* d) {
  if (!desc_valid(d)) return 0;
  const Geometry g = geometry_of(d);
  const size_t n = (size_t)(g.nz * g.ny * g.nx);
  return kHeaderBytes + ((size_t)g.ntiles * 8 + 15) / 16 * 16 + 2 * (n * word_bytes(d->dtype) + 16 * (size_t)g.ntiles);
}

size_t lopc_compress_workspace_size(const lopc_field_desc* d) {
  if (!desc_valid(d)) return 0;
  return compress_layout(d).total;
}

size_t lopc_decompress_workspace_size(const lopc_field_desc* d) {
  if (!desc_valid(d)) return 0;
  const Geometry g = geometry_of(d);
  return 256 + align256(16 * (size_t)g.ntiles);
}

static int compress_entry(const lopc_field_desc* d, const void* d_x, void* d_out, size_t out_cap, size_t* out_size,
                          void* d_ws, size_t ws_size, void* stream);
int lopc_compress(const lopc_field_desc* d, const void* d_x, void* d_out, size_t out_cap, size_t* out_size, void* d_ws,
                  size_t ws_size, void* stream) {
  const int rc = compress_entry(d, d_x, d_out, out_cap, out_size, d_ws, ws_size, stream);
  g_prof.resolve();
  return rc;
}

static int compress_entry(const lopc_field_desc* d, const void* d_x, void* d_out, size_t out_cap, size_t* out_size,
                          void* d_ws, size_t ws_size, void* stream) {
  if (!desc_valid(d) || !d_x || !d_out || !out_size) return LOPC_ERR_INVALID_ARG;
  if (!d_ws || ws_size < lopc_compress_workspace_size(d)) return LOPC_ERR_WORKSPACE;
  if (out_cap < (size_t)kHeaderBytes) return LOPC_ERR_CAPACITY;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int nd = d->ndim;
  if (d->dtype == LOPC_F32)
    return nd == 2 ? compress_impl<float, 2>(d, d_x, d_out, out_cap, out_size, d_ws, st)
                   : compress_impl<float, 3>(d, d_x, d_out, out_cap, out_size, d_ws, st);
  return nd == 2 ? compress_impl<double, 2>(d, d_x, d_out, out_cap, out_size, d_ws, st)
                 : compress_impl<double, 3>(d, d_x, d_out, out_cap, out_size, d_ws, st);
}

static int quantize_repair_entry(const lopc_field_desc* d, const void* d_x, int64_t* d_bins, uint64_t* d_subbins,
                                 void* d_ws, size_t ws_size, void* stream);
int lopc_quantize_repair(const lopc_field_desc* d, const void* d_x, int64_t* d_bins, uint64_t* d_subbins, void* d_ws,
                         size_t ws_size, void* stream) {
  const int rc = quantize_repair_entry(d, d_x, d_bins, d_subbins, d_ws, ws_size, stream);
  g_prof.resolve();
  return rc;
}

static int quantize_repair_entry(const lopc_field_desc* d, const void* d_x, int64_t* d_bins, uint64_t* d_subbins,
                                 void* d_ws, size_t ws_size, void* stream) {
  if (!desc_valid(d) || !d_x || !d_bins || !d_subbins) return LOPC_ERR_INVALID_ARG;
  if (!d_ws || ws_size < lopc_compress_workspace_size(d)) return LOPC_ERR_WORKSPACE;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int nd = d->ndim;
  if (d->dtype == LOPC_F32)
    return nd == 2 ? quantize_repair_impl<float, 2>(d, d_x, d_bins, d_subbins, d_ws, st)
                   : quantize_repair_impl<float, 3>(d, d_x, d_bins, d_subbins, d_ws, st);
  return nd == 2 ? quantize_repair_impl<double, 2>(d, d_x, d_bins, d_subbins, d_ws, st)
                 : quantize_repair_impl<double, 3>(d, d_x, d_bins, d_subbins, d_ws, st);
}

int lopc_peek(const void* h_stream, size_t n, lopc_field_desc* out) {
  if (!h_stream || !out) return LOPC_ERR_INVALID_ARG;
  Header H;
  const int rc = parse_header(reinterpret_cast<const uint8_t*>(h_stream), n, &H);
  if (rc) return rc;
  *out = H.d;
  return LOPC_OK;
}

static int decompress_entry(const void* d_in, size_t in_size, void* d_x, size_t x_cap, void* d_ws, size_t ws_size,
                            void* stream);
int lopc_decompress(const void* d_in, size_t in_size, void* d_x, size_t x_cap, void* d_ws, size_t ws_size,
                    void* stream) {
  const int rc = decompress_entry(d_in, in_size, d_x, x_cap, d_ws, ws_size, stream);
  g_prof.resolve();
  return rc;
}

static int decompress_entry(const void* d_in, size_t in_size, void* d_x, size_t x_cap, void* d_ws, size_t ws_size,
                            void* stream) {
  if (!d_in || !d_x) return LOPC_ERR_INVALID_ARG;
  if (in_size < (size_t)kHeaderBytes) return LOPC_ERR_CORRUPT;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  uint8_t hb[kHeaderBytes];
  CK(cudaMemcpyAsync(hb, d_in, kHeaderBytes, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  Header H;
  int rc = parse_header(hb, in_size, &H);
  if (rc) return rc;
  if (H.total > in_size) return LOPC_ERR_CORRUPT;
  const Geometry g = geometry_of(&H.d);
  const size_t need = (size_t)(g.nz * g.ny * g.nx) * word_bytes(H.d.dtype);
  if (x_cap < need) return LOPC_ERR_CAPACITY;
  if (!d_ws || ws_size < lopc_decompress_workspace_size(&H.d)) return LOPC_ERR_WORKSPACE;
  const uint8_t* in = reinterpret_cast<const uint8_t*>(d_in);
  uint8_t* ws = reinterpret_cast<uint8_t*>(d_ws);
  if (H.d.dtype == LOPC_F32)
    return H.d.ndim == 2 ? decompress_impl<float, 2>(H, in, in_size, d_x, ws, st)
                         : decompress_impl<float, 3>(H, in, in_size, d_x, ws, st);
  return H.d.ndim == 2 ? decompress_impl<double, 2>(H, in, in_size, d_x, ws, st)
                       : decompress_impl<double, 3>(H, in, in_size, d_x, ws, st);
}

// ------------------------------------------------- decompression without allocation
// For callers that cannot allocate device memory: code running where cudaMalloc is
// off limits (inside a caching allocator's own callbacks, in a process whose memory
// is reserved up front by a host framework, or on a path that must not take the
// driver's allocation locks).  The decompressor's scratch, a status word and two
// 64-bit record offsets per chunk, lives in this fixed device array instead of a
// caller workspace.  Every GPU that loads the library holds it until the process
// exits.
constexpr int64_t kNoAllocMaxChunks = 65536;
constexpr size_t kNoAllocScratchBytes = 256 + 16 * (size_t)kNoAllocMaxChunks;  // 1 MiB + 256 B
static __device__ __align__(256) uint8_t g_noalloc_scratch[kNoAllocScratchBytes];

namespace {
constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_addr[kNoAllocMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once per
// device.  In host code the array's name is only a stand-in, so the address must
// come from cudaGetSymbolAddress with that device current.
int noalloc_scratch(uint8_t** out) {
  int dev = -1;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoAllocMaxDevices) return LOPC_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    CK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_noalloc_addr[dev] = p;
  }
  *out = reinterpret_cast<uint8_t*>(g_noalloc_addr[dev]);
  return LOPC_OK;
}
}  // namespace

int lopc_decompress_noalloc(const void* d_in, size_t in_size, void* d_x, size_t x_cap, void* stream) {
  if (!d_in || !d_x) return LOPC_ERR_INVALID_ARG;
  if (in_size < (size_t)kHeaderBytes) return LOPC_ERR_CORRUPT;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  uint8_t* ws = nullptr;
  int rc = noalloc_scratch(&ws);
  if (rc) return rc;
  uint8_t hb[kHeaderBytes];
  CK(cudaMemcpyAsync(hb, d_in, kHeaderBytes, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  Header H;
  rc = parse_header(hb, in_size, &H);
  if (rc) return rc;
  const Geometry g = geometry_of(&H.d);
  if (g.ntiles > kNoAllocMaxChunks) return LOPC_ERR_WORKSPACE;  // beyond the fixed scratch
  if (H.total > in_size) return LOPC_ERR_CORRUPT;
  const size_t need = (size_t)(g.nz * g.ny * g.nx) * word_bytes(H.d.dtype);
  if (x_cap < need) return LOPC_ERR_CAPACITY;
  const uint8_t* in = reinterpret_cast<const uint8_t*>(d_in);
  // decompress_impl zeroes the status word and rewrites every offset it reads
  if (H.d.dtype == LOPC_F32)
    rc = H.d.ndim == 2 ? decompress_impl<float, 2>(H, in, in_size, d_x, ws, st)
                       : decompress_impl<float, 3>(H, in, in_size, d_x, ws, st);
  else
    rc = H.d.ndim == 2 ? decompress_impl<double, 2>(H, in, in_size, d_x, ws, st)
                       : decompress_impl<double, 3>(H, in, in_size, d_x, ws, st);
  g_prof.resolve();
  return rc;
}

int64_t lopc_noalloc_max_chunks(void) { return kNoAllocMaxChunks; }

int64_t lopc_set_round_cap(int64_t cap) {
  const int64_t old = g_round_cap;
  g_round_cap = cap < 0 ? 0 : cap;
  return old;
}

void lopc_last_stats(int64_t* rounds, int64_t* tile_runs) {
  if (rounds) *rounds = g_last_rounds;
  if (tile_runs) *tile_runs = g_last_tile_runs;
}

void lopc_last_fixpoint_stats(int64_t* sweeps_total, int64_t* sweeps_max) {
  if (sweeps_total) *sweeps_total = g_last_fix_iters;
  if (sweeps_max) *sweeps_max = g_last_fix_iters_max;
}

int lopc_last_phase_cycles(int64_t* cycles, int n) {
  for (int k = 0; k < n && k < 8; ++k) cycles[k] = g_last_phase[k];
  return 8;
}

void lopc_profile_enable(int on) {
  g_prof.resolve();
  g_prof.on = on != 0;
}

void lopc_profile_reset(void) {
  g_prof.resolve();
  g_prof.n = 0;
}

int lopc_profile_read(const char** names, int64_t* launches, double* total_ms, int cap) {
  g_prof.resolve();
  for (int i = 0; i < g_prof.n && i < cap; ++i) {
    if (names) names[i] = g_prof.entries[i].name;
    if (launches) launches[i] = g_prof.entries[i].launches;
    if (total_ms) total_ms[i] = g_prof.entries[i].ms;
  }
  return g_prof.n;
}

const char* lopc_strerror(int s) {
  switch (s) {
    case LOPC_OK: return "ok";
    case LOPC_ERR_INVALID_ARG: return "invalid argument";
    case LOPC_ERR_NONFINITE: return "field holds NaN or infinity";
    case LOPC_ERR_RANGE: return "value range too large for the error bound";
    case LOPC_ERR_CAPACITY: return "output buffer too small";
    case LOPC_ERR_CORRUPT: return "corrupt stream";
    case LOPC_ERR_NOT_CONVERGED: return "repair round cap reached";
    case LOPC_ERR_CUDA: return "CUDA runtime error";
    case LOPC_ERR_WORKSPACE: return "workspace missing or too small";
    default: return "unknown status";
  }
}

}  // extern "C"
