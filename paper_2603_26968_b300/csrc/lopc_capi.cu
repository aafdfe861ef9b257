// lopc_capi.cu -- host side of the C ABI (include/lopc.h): argument checks, the
// workspace layout, and the launch sequences of compression and decompression.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <deque>
#include <vector>

#include "lopc.h"
#include "lopc_decompress.cuh"
#include "lopc_verify.cuh"
#include "lopc_worklist.cuh"

using namespace lopc;

namespace {

thread_local int64_t g_round_cap = 0;  // 0 = default
// Repair schedule of single-field compressions (lopc_set_repair_mode).
thread_local int g_repair_mode = LOPC_REPAIR_TILES;

// ---------------------------------------------------------------- profiling
// Event pairs around each launch while profiling is on; resolved at the end of
// every API call, after its final synchronisation.
struct ProfEntry {
  const char* name;
  int64_t launches;
  double ms;
  std::vector<float> each;  // every launch's time, in order
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
    entries[n].name = name;
    entries[n].launches = 0;
    entries[n].ms = 0.0;
    entries[n].each.clear();
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
        if (entries[pend[i].entry].each.size() < 100000) entries[pend[i].entry].each.push_back(ms);
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
thread_local int64_t g_last_phase[9] = {};
thread_local int64_t g_last_work[7] = {};
thread_local std::vector<int64_t> g_round_tiles;  // tiles listed per round (host-driven loop only)

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

#define CK(call)                          \
  do {                                    \
    if ((call) != cudaSuccess) {          \
      (void)cudaGetLastError();           \
      return LOPC_ERR_CUDA;               \
    }                                     \
  } while (0)

// Field classes: one kernel instantiation each.
//   0 = float32 2D, 1 = float32 3D, 2 = float64 2D, 3 = float64 3D
int class_of(int dtype, int ndim) { return (dtype == LOPC_F64 ? 2 : 0) + (ndim == 3 ? 1 : 0); }

HeaderInfo header_info(const lopc_field_desc* d, const Geometry& g) {
  HeaderInfo h;
  h.dtype = d->dtype;
  h.ndim = d->ndim;
  h.mode = d->mode;
  for (int k = 0; k < 3; ++k) h.dims[k] = k < d->ndim ? d->dims[k] : 0;
  h.tile[0] = g.tz;
  h.tile[1] = g.ty;
  h.tile[2] = g.tx;
  h.eb = d->eb;
  return h;
}

// ------------------------------------------------------------ launch tables

// A table of fields for one set of launches: sorted by class, every field's tiles
// and dirty-bitmap words numbered consecutively.  A single field is a table of
// one; a batch, a serving round and a set of fields being finished are others.
struct Table {
  std::vector<FieldInfo> F;
  int cls_f0[4] = {0, 0, 0, 0}, cls_nf[4] = {0, 0, 0, 0};
  int64_t cls_t0[4] = {0, 0, 0, 0}, cls_nt[4] = {0, 0, 0, 0};
  int64_t total_tiles = 0, total_words = 0, max_words = 0;
  int n() const { return (int)F.size(); }
};

// Numbers the tiles and dirty words of t.F, which is already sorted by class.
void layout_table(Table& t) {
  for (int c = 0; c < 4; ++c) {
    t.cls_f0[c] = t.cls_nf[c] = 0;
    t.cls_t0[c] = t.cls_nt[c] = 0;
  }
  int64_t tiles = 0, words = 0, maxw = 0;
  for (int k = 0; k < t.n(); ++k) {
    FieldInfo& f = t.F[k];
    const int c = class_of_geometry(f.g);
    if (t.cls_nf[c] == 0) {
      t.cls_f0[c] = k;
      t.cls_t0[c] = tiles;
    }
    ++t.cls_nf[c];
    t.cls_nt[c] += f.g.ntiles;
    f.tile_base = tiles;
    tiles += f.g.ntiles;
    f.word_base = words;
    words += dirty_words(f.g.ntiles);
    maxw = std::max<int64_t>(maxw, dirty_words(f.g.ntiles));
  }
  t.total_tiles = tiles;
  t.total_words = words;
  t.max_words = maxw;
}

// Per-field part of a compression workspace: state, subbins, lower masks, record
// sizes and offsets, the dirty bitmap and the record slots.
struct FieldPart {
  size_t params, s, cm, sizes, offs, dirty, tkey, order, rank, slots, total;
};

FieldPart field_part(const Geometry& g) {
  const size_t n = (size_t)(g.nz * g.ny * g.nx);
  FieldPart L;
  size_t o = 0;
  L.params = o;
  o = align256(o + sizeof(Params));
  L.s = o;
  o = align256(o + 4 * n);
  L.cm = o;
  o = align256(o + 4 * n);
  L.sizes = o;
  o = align256(o + 8 * (size_t)g.ntiles);
  L.offs = o;
  o = align256(o + 16 * (size_t)g.ntiles);
  L.dirty = o;
  o = align256(o + 4 * (size_t)dirty_words(g.ntiles));
  L.tkey = o;
  o = align256(o + 4 * (size_t)g.ntiles);
  L.order = o;
  o = align256(o + 4 * (size_t)g.ntiles);
  L.rank = o;
  o = align256(o + 4 * (size_t)g.ntiles);
  L.slots = o;
  o = align256(o + 2 * (size_t)g.ntiles * kSlotBytes);
  L.total = o;
  return L;
}

// The default round cap of a field: a chain of constraints has fewer links than
// the field has points, so reaching it means a fault, not a slow field.
int64_t default_round_cap(const Geometry& g) {
  if (g_round_cap > 0) return g_round_cap;
  return std::max<int64_t>(16, g.nz * g.ny * g.nx + 16);
}

// A table entry for one field whose state lives at `base` (a FieldPart layout).
FieldInfo field_entry(const lopc_field_desc* d, const void* x, void* out, size_t cap, uint64_t* size_out,
                      int* status_out, int64_t* bins_out, uint8_t* base) {
  FieldInfo f{};
  f.g = geometry_of(d);
  f.hdr = header_info(d, f.g);
  f.round_cap = default_round_cap(f.g);
  if (!base) return f;
  const FieldPart L = field_part(f.g);
  f.x = x;
  f.out = reinterpret_cast<uint8_t*>(out);
  f.out_cap = (uint64_t)cap;
  f.P = reinterpret_cast<Params*>(base + L.params);
  f.s = reinterpret_cast<uint32_t*>(base + L.s);
  f.cm = reinterpret_cast<uint32_t*>(base + L.cm);
  f.sizes = reinterpret_cast<uint32_t*>(base + L.sizes);
  f.offs = reinterpret_cast<uint64_t*>(base + L.offs);
  f.dirty = reinterpret_cast<uint32_t*>(base + L.dirty);
  f.tkey = reinterpret_cast<uint32_t*>(base + L.tkey);
  f.order = reinterpret_cast<uint32_t*>(base + L.order);
  f.rank = reinterpret_cast<uint32_t*>(base + L.rank);
  f.slots = base + L.slots;
  f.bins_out = bins_out;
  f.size_out = size_out;
  f.status_out = status_out;
  return f;
}

// ------------------------------------------------------------ launch sequences

// Library-owned stream for capturing the body of the repair loop.
cudaStream_t side_stream() {
  thread_local cudaStream_t s = nullptr;
  if (!s) cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  return s;
}

template <typename T, int ND>
int set_smem_attrs() {
  // per instantiation and thread: one bit per device (attributes are per function and device)
  thread_local uint64_t done = 0;
  int dev = 0;
  CK(cudaGetDevice(&dev));
  const uint64_t bit = 1ull << (dev & 63);
  if (done & bit) return LOPC_OK;
  CK(cudaFuncSetAttribute(k_pass<T, ND>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PassSmem<T, ND>::bytes()));
  CK(cudaFuncSetAttribute(k_rerun<T, ND>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)RerunSmem<T, ND>::bytes()));
  CK(cudaFuncSetAttribute(k_encode_sub<T, ND>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)EncSmem<T, ND>::bytes()));
  CK(cudaFuncSetAttribute(k_decode<T, ND>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)DecSmem<T, ND>::bytes()));
  done |= bit;
  return LOPC_OK;
}

int sm_count() {
  thread_local int v[64] = {};  // per device
  int dev = 0;
  cudaGetDevice(&dev);
  int& c = v[dev & 63];
  if (!c) {
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    c = sms;
  }
  return c;
}

// Persistent rerun blocks per SM, per class (set by lopc_tune_set).
thread_local int g_rerun_per_sm[4] = {4, 4, 6, 6};
// Frontier evaluations of a tile pass before it switches to the topological order,
// in sixteenths of the tile's points, per class (set by lopc_tune_set_budget).
thread_local int g_pass_budget16[4] = {64, 64, 64, 64};
// Same-bin neighbour pairs, in sixteenths of a full tile's pairs, above which a tile
// pass goes straight to the topological order (set by lopc_tune_set_dense; 17 = never).
thread_local int g_pass_dense16[4] = {8, 8, 8, 8};
// Order of the tile pass, per class: 0 by the field's sample span, 1 tile index, 2 tile
// key (set by lopc_tune_set_pass_order).
thread_local int g_pass_order[4] = {0, 0, 0, 0};

// Launch settings of one compression: the caller's lopc_plan (lopc_batch_compress),
// else this thread's lopc_tune_* values.  Output bytes never depend on them.
struct Tune {
  int rerun_per_sm[4], budget16[4], dense16[4], order[4];
};

int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

Tune current_tune() {
  Tune u;
  for (int c = 0; c < 4; ++c) {
    u.rerun_per_sm[c] = g_rerun_per_sm[c];
    u.budget16[c] = g_pass_budget16[c];
    u.dense16[c] = g_pass_dense16[c];
    u.order[c] = g_pass_order[c];
  }
  return u;
}

Tune tune_of_plan(const lopc_plan& pl) {
  Tune u;
  for (int c = 0; c < 4; ++c) {
    u.rerun_per_sm[c] = clampi(pl.rerun_blocks_per_sm[c], 1, 16);
    u.budget16[c] = clampi(pl.pass_budget16[c], 1, 4096);
    u.dense16[c] = clampi(pl.pass_dense16[c], 0, 17);
    u.order[c] = clampi(pl.pass_order[c], 0, 2);
  }
  return u;
}

int rerun_blocks(const Tune& tu, int c) { return sm_count() * tu.rerun_per_sm[c]; }

int launch_init(const Table& t, const FieldInfo* dF, cudaStream_t st) {
  const unsigned gx = (unsigned)std::max<int64_t>(1, std::min<int64_t>(64, (t.max_words + 255) / 256));
  LAUNCH("init_params", st, k_init_params<<<dim3(gx, (unsigned)t.n()), 256, 0, st>>>(dF, t.n()));
  CK(cudaGetLastError());
  return LOPC_OK;
}

// Range, eps and tile keys of one class's fields.
template <typename T, int ND>
int launch_class_range(const Table& t, int c, const FieldInfo* dF, cudaStream_t st) {
  if (!t.cls_nf[c]) return LOPC_OK;
  int rc = set_smem_attrs<T, ND>();
  if (rc) return rc;
  LAUNCH("range", st, k_range<T><<<dim3(sm_count() * 4, t.cls_nf[c]), 256, 0, st>>>(dF, t.cls_f0[c]));
  LAUNCH("resolve_eps", st, k_resolve_eps<T><<<(t.cls_nf[c] + 63) / 64, 64, 0, st>>>(dF, t.cls_f0[c], t.cls_nf[c]));
  LAUNCH("tile_keys", st, k_tile_keys<T, ND><<<(unsigned)t.cls_nt[c], 64, 0, st>>>(dF, t.cls_f0[c], t.cls_nf[c], t.cls_t0[c]));
  CK(cudaGetLastError());
  return LOPC_OK;
}

// The tile pass of one class's fields.
template <typename T, int ND>
int launch_class_pre(const Table& t, int c, const FieldInfo* dF, const Tune& tu, int fix, cudaStream_t st) {
  using C = TileCfg<T, ND>;
  if (!t.cls_nf[c]) return LOPC_OK;
  LAUNCH("tile_pass", st,
         k_pass<T, ND><<<(unsigned)t.cls_nt[c], C::NT, PassSmem<T, ND>::bytes(), st>>>(
             dF, t.cls_f0[c], t.cls_nf[c], t.cls_t0[c], (unsigned)tu.budget16[c], (unsigned)tu.dense16[c], fix));
  CK(cudaGetLastError());
  return LOPC_OK;
}

template <typename T, int ND>
int launch_class_rerun(const Table& t, int c, const FieldInfo* dF, const Tune& tu, BatchState* dB,
                       const uint32_t* list, uint32_t* app, cudaStream_t st) {
  using C = TileCfg<T, ND>;
  if (!t.cls_nf[c]) return LOPC_OK;
  const unsigned grid = (unsigned)imin64(t.cls_nt[c], rerun_blocks(tu, c));
  LAUNCH(list ? "tile_rerun" : "tile_rerun_all", st,
         k_rerun<T, ND><<<grid, C::NT, RerunSmem<T, ND>::bytes(), st>>>(dF, t.cls_f0[c], t.cls_nf[c], t.cls_t0[c],
                                                                       t.cls_nt[c], c, dB, list, app));
  CK(cudaGetLastError());
  return LOPC_OK;
}

template <typename T, int ND>
int launch_class_encode(const Table& t, int c, const FieldInfo* dF, cudaStream_t st) {
  using C = TileCfg<T, ND>;
  if (!t.cls_nf[c]) return LOPC_OK;
  LAUNCH("encode_subbins", st,
         k_encode_sub<T, ND><<<(unsigned)t.cls_nt[c], C::NTC, EncSmem<T, ND>::bytes(), st>>>(dF, t.cls_f0[c],
                                                                                           t.cls_nf[c], t.cls_t0[c]));
  CK(cudaGetLastError());
  return LOPC_OK;
}

// State reset, range, eps, tile keys and order, cleared subbins (ordered passes only)
// and the tile pass of every field of the table (fix = 0: the pass leaves every subbin
// at 0, for the worklist schedule).  The reruns visit each field's tiles in ascending
// tile key, and so does the pass of a field whose tiles span few bins.
int launch_pre(const Table& t, const FieldInfo* dF, const Tune& tu, cudaStream_t st, int fix = 1) {
  int rc;
  if ((rc = launch_init(t, dF, st))) return rc;
  if ((rc = launch_class_range<float, 2>(t, 0, dF, st))) return rc;
  if ((rc = launch_class_range<float, 3>(t, 1, dF, st))) return rc;
  if ((rc = launch_class_range<double, 2>(t, 2, dF, st))) return rc;
  if ((rc = launch_class_range<double, 3>(t, 3, dF, st))) return rc;
  unsigned pass_order = 0;
  for (int c = 0; c < 4; ++c) pass_order |= (unsigned)tu.order[c] << (2 * c);
  LAUNCH("order", st, k_order<1024><<<t.n(), 1024, 0, st>>>(dF, pass_order));
  LAUNCH("clear_subbins", st, k_clear_subbins<<<dim3(sm_count() * 2, t.n()), 256, 0, st>>>(dF));
  CK(cudaGetLastError());
  if ((rc = launch_class_pre<float, 2>(t, 0, dF, tu, fix, st))) return rc;
  if ((rc = launch_class_pre<float, 3>(t, 1, dF, tu, fix, st))) return rc;
  if ((rc = launch_class_pre<double, 2>(t, 2, dF, tu, fix, st))) return rc;
  return launch_class_pre<double, 3>(t, 3, dF, tu, fix, st);
}

// One rerun round: of every tile (list == null, the first round) or of the listed ones.
// app (total_tiles entries, or null: no appends) receives the tiles reruns mark, for
// the round in progress to take.
int launch_reruns(const Table& t, const FieldInfo* dF, const Tune& tu, BatchState* dB, const uint32_t* list,
                  uint32_t* app, cudaStream_t st) {
  int rc;
  if (!list) CK(cudaMemsetAsync(dB->next_all, 0, sizeof(dB->next_all), st));  // the all-tile round's counters
  if (!list && app) CK(cudaMemsetAsync(dB->app, 0, sizeof(dB->app), st));
  if ((rc = launch_class_rerun<float, 2>(t, 0, dF, tu, dB, list, app, st))) return rc;
  if ((rc = launch_class_rerun<float, 3>(t, 1, dF, tu, dB, list, app, st))) return rc;
  if ((rc = launch_class_rerun<double, 2>(t, 2, dF, tu, dB, list, app, st))) return rc;
  return launch_class_rerun<double, 3>(t, 3, dF, tu, dB, list, app, st);
}

int launch_compact(const Table& t, FieldInfo* dF, uint32_t* list, BatchState* dB, unsigned int* field_counts,
                   cudaGraphConditionalHandle h, int use_h, cudaStream_t st) {
  LAUNCH("compact", st,
         k_compact<1024><<<1, 1024, 0, st>>>(dF, t.n(), t.total_words, list, dB, field_counts, h, use_h));
  CK(cudaGetLastError());
  return LOPC_OK;
}

// Subbin records, size scan, pack and per-field results of every field of the table.
int launch_epilogue(const Table& t, const FieldInfo* dF, cudaStream_t st) {
  int rc;
  if ((rc = launch_class_encode<float, 2>(t, 0, dF, st))) return rc;
  if ((rc = launch_class_encode<float, 3>(t, 1, dF, st))) return rc;
  if ((rc = launch_class_encode<double, 2>(t, 2, dF, st))) return rc;
  if ((rc = launch_class_encode<double, 3>(t, 3, dF, st))) return rc;
  LAUNCH("scan_sizes", st, k_scan_sizes<1024><<<t.n(), 1024, 0, st>>>(dF));
  LAUNCH("pack", st, k_pack<<<dim3(sm_count() * 8, t.n()), 256, 0, st>>>(dF));
  LAUNCH("finalize", st, k_finalize<<<(t.n() + 63) / 64, 64, 0, st>>>(dF, t.n()));
  CK(cudaGetLastError());
  return LOPC_OK;
}

// ------------------------------------------------------------ compress plan

// Workspace of a compression call: shared state, the field table, the results of a
// single-field call, the rerun list, then one FieldPart per field.
struct CompressPlan {
  Table t;
  std::vector<int> order;  // position in the table -> caller's index
  bool worklist = false;   // one field, repaired by the worklist schedule
  Tune tu;                 // launch settings (lopc_plan or this thread's tuning)
  size_t off_state = 0, off_table = 0, off_results = 0, off_list = 0, off_app = 0;
  size_t off_wl_state = 0, off_stamp = 0, off_wl = 0;
  std::vector<size_t> off_field;
  size_t ws_total = 0;
};

// Lays out a call over descs[0..n) (sorted by class); fills pointers when ws != null.
int plan_compress(int n, const lopc_field_desc* descs, const void* const* xs, void* const* outs, const size_t* caps,
                  uint64_t* d_sizes, int* d_status, int64_t* bins_out, uint8_t* ws, CompressPlan& p,
                  bool worklist = false) {
  p = CompressPlan{};  // planning twice (size, then pointers) must not accumulate
  p.worklist = worklist && n == 1;
  p.tu = current_tune();
  p.order.resize(n);
  for (int i = 0; i < n; ++i) p.order[i] = i;
  std::stable_sort(p.order.begin(), p.order.end(), [&](int a, int b) {
    return class_of(descs[a].dtype, descs[a].ndim) < class_of(descs[b].dtype, descs[b].ndim);
  });
  p.t.F.resize(n);
  for (int k = 0; k < n; ++k)
    p.t.F[k] = field_entry(&descs[p.order[k]], nullptr, nullptr, 0, nullptr, nullptr, nullptr, nullptr);
  layout_table(p.t);
  size_t o = 0;
  p.off_state = o;
  o = align256(o + sizeof(BatchState));
  p.off_table = o;
  o = align256(o + (size_t)n * sizeof(FieldInfo));
  p.off_results = o;
  o = align256(o + 16);
  p.off_list = o;
  o = align256(o + 4 * (size_t)p.t.total_tiles);
  p.off_app = o;
  o = align256(o + 4 * (size_t)p.t.total_tiles);
  p.off_field.resize(n);
  for (int k = 0; k < n; ++k) {
    p.off_field[k] = o;
    o += field_part(p.t.F[k].g).total;
  }
  if (p.worklist) {  // worklist state, one stamp per point, two worklists of a point each
    const size_t npts = (size_t)(p.t.F[0].g.nz * p.t.F[0].g.ny * p.t.F[0].g.nx);
    o = align256(o);
    p.off_wl_state = o;
    o = align256(o + sizeof(WorklistState));
    p.off_stamp = o;
    o = align256(o + 4 * npts);
    p.off_wl = o;
    o = align256(o + 8 * npts);
  }
  p.ws_total = o;
  if (!ws) return LOPC_OK;
  for (int k = 0; k < n; ++k) {
    const int i = p.order[k];
    FieldInfo f = field_entry(&descs[i], xs ? xs[i] : nullptr, outs ? outs[i] : nullptr, caps ? caps[i] : 0,
                              d_sizes ? d_sizes + i : nullptr, d_status ? d_status + i : nullptr, bins_out,
                              ws + p.off_field[k]);
    f.tile_base = p.t.F[k].tile_base;
    f.word_base = p.t.F[k].word_base;
    p.t.F[k] = f;
  }
  return LOPC_OK;
}

struct Ptrs {
  FieldInfo* F;
  BatchState* B;
  uint32_t* list;
  uint32_t* app;
};

Ptrs ptrs_of(const CompressPlan& p, uint8_t* ws) {
  Ptrs q;
  q.F = reinterpret_cast<FieldInfo*>(ws + p.off_table);
  q.B = reinterpret_cast<BatchState*>(ws + p.off_state);
  q.list = reinterpret_cast<uint32_t*>(ws + p.off_list);
  q.app = reinterpret_cast<uint32_t*>(ws + p.off_app);
  return q;
}

// The worklist schedule: launches of one iteration and of its swap.
int launch_wl(const CompressPlan& p, const Ptrs& q, uint8_t* ws, int all, cudaStream_t st,
              cudaGraphConditionalHandle h, int use_h) {
  WorklistState* W = reinterpret_cast<WorklistState*>(ws + p.off_wl_state);
  LAUNCH(all ? "wl_iter_all" : "wl_iter", st,
         k_wl_iter<<<sm_count() * 8, 256, 0, st>>>(q.F, W, reinterpret_cast<uint32_t*>(ws + p.off_wl),
                                                  reinterpret_cast<uint32_t*>(ws + p.off_stamp), all));
  LAUNCH("wl_next", st, k_wl_next<<<1, 1, 0, st>>>(q.F, W, q.B, h, use_h));
  CK(cudaGetLastError());
  return LOPC_OK;
}

// Everything before the repair loop: state reset, range, eps, tile pass, the first
// (all-tile) rerun round and its compaction.
int enqueue_prologue(const CompressPlan& p, const Ptrs& q, cudaStream_t st, cudaGraphConditionalHandle h, int use_h) {
  int rc;
  CK(cudaMemsetAsync(q.B, 0, sizeof(BatchState), st));
  if (p.worklist) {
    uint8_t* ws = reinterpret_cast<uint8_t*>(q.B) - p.off_state;
    const size_t npts = (size_t)(p.t.F[0].g.nz * p.t.F[0].g.ny * p.t.F[0].g.nx);
    CK(cudaMemsetAsync(ws + p.off_wl_state, 0, sizeof(WorklistState), st));
    CK(cudaMemsetAsync(ws + p.off_stamp, 0, 4 * npts, st));
    if ((rc = launch_pre(p.t, q.F, p.tu, st, 0))) return rc;
    return launch_wl(p, q, ws, 1, st, h, use_h);
  }
  if ((rc = launch_pre(p.t, q.F, p.tu, st))) return rc;
  if ((rc = launch_reruns(p.t, q.F, p.tu, q.B, nullptr, q.app, st))) return rc;
  return launch_compact(p.t, q.F, q.list, q.B, nullptr, h, use_h, st);
}

int enqueue_loop_body(const CompressPlan& p, const Ptrs& q, cudaStream_t st, cudaGraphConditionalHandle h, int use_h) {
  int rc;
  if (p.worklist) return launch_wl(p, q, reinterpret_cast<uint8_t*>(q.B) - p.off_state, 0, st, h, use_h);
  if ((rc = launch_reruns(p.t, q.F, p.tu, q.B, q.list, q.app, st))) return rc;
  return launch_compact(p.t, q.F, q.list, q.B, nullptr, h, use_h, st);
}

// Uploads the field table (not part of any graph).
int upload_plan(const CompressPlan& p, const Ptrs& q, cudaStream_t st) {
  CK(cudaMemcpyAsync(q.F, p.t.F.data(), (size_t)p.t.n() * sizeof(FieldInfo), cudaMemcpyHostToDevice, st));
  return LOPC_OK;
}

// Repair rounds driven by the host (one small read-back per round); used while
// per-kernel event timing is on, where every launch must be a direct launch.
int run_host_loop(const CompressPlan& p, const Ptrs& q, cudaStream_t st) {
  int rc = enqueue_prologue(p, q, st, cudaGraphConditionalHandle{}, 0);
  if (rc) return rc;
  g_round_tiles.clear();
  while (true) {
    BatchState hb;
    CK(cudaMemcpyAsync(&hb, q.B, sizeof(BatchState), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    const int64_t listed = (int64_t)hb.count[0] + hb.count[1] + hb.count[2] + hb.count[3];
    g_round_tiles.push_back(listed);
    if (listed == 0) break;
    if ((rc = enqueue_loop_body(p, q, st, cudaGraphConditionalHandle{}, 0))) return rc;
  }
  return launch_epilogue(p.t, q.F, st);
}

// The whole compression as one CUDA graph: the repair rounds run in a conditional
// while-node whose condition the compaction kernel sets on the device.
int capture_graph(const CompressPlan& p, const Ptrs& q, cudaStream_t st, cudaGraphExec_t* exec) {
  cudaGraph_t graph = nullptr;
  cudaStream_t cap = side_stream();
  if (!cap) return LOPC_ERR_CUDA;
  // capture on the library's own stream, so the caller's stream is never in capture mode
  CK(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
  cudaStreamCaptureStatus cs;
  cudaGraph_t cg = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  int rc = LOPC_OK;
  cudaGraphConditionalHandle h{};
  if (cudaStreamGetCaptureInfo(cap, &cs, nullptr, &cg, nullptr, nullptr, nullptr) != cudaSuccess ||
      cudaGraphConditionalHandleCreate(&h, cg, 0, cudaGraphCondAssignDefault) != cudaSuccess)
    rc = LOPC_ERR_CUDA;
  if (!rc) rc = enqueue_prologue(p, q, cap, h, 1);
  cudaGraphNode_t cnode = nullptr;
  cudaGraph_t body = nullptr;
  if (!rc) {
    if (cudaStreamGetCaptureInfo(cap, &cs, nullptr, &cg, &deps, nullptr, &ndeps) != cudaSuccess) rc = LOPC_ERR_CUDA;
  }
  if (!rc) {
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    if (cudaGraphAddNode(&cnode, cg, deps, nullptr, ndeps, &cp) != cudaSuccess ||
        cudaStreamUpdateCaptureDependencies(cap, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies) != cudaSuccess)
      rc = LOPC_ERR_CUDA;
    else
      body = cp.conditional.phGraph_out[0];
  }
  if (!rc) {
    // the body: reruns of the listed tiles, then the next compaction
    thread_local cudaStream_t bs = nullptr;
    if (!bs) cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking);
    if (!bs || cudaStreamBeginCaptureToGraph(bs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      rc = LOPC_ERR_CUDA;
    if (!rc) {
      rc = enqueue_loop_body(p, q, bs, h, 1);
      cudaGraph_t b2 = nullptr;
      if (cudaStreamEndCapture(bs, &b2) != cudaSuccess && !rc) rc = LOPC_ERR_CUDA;
    }
  }
  if (!rc) rc = launch_epilogue(p.t, q.F, cap);
  if (cudaStreamEndCapture(cap, &graph) != cudaSuccess && !rc) rc = LOPC_ERR_CUDA;
  if (!rc && cudaGraphInstantiate(exec, graph, 0) != cudaSuccess) rc = LOPC_ERR_CUDA;
  if (graph) cudaGraphDestroy(graph);
  (void)st;
  if (rc) (void)cudaGetLastError();
  return rc;
}

// Instantiated graphs keyed by everything the captured launches depend on.
struct GraphCache {
  struct Entry {
    std::vector<uint64_t> key;
    cudaGraphExec_t exec;
    uint64_t used;
  };
  std::vector<Entry> e;
  uint64_t tick = 0;
  cudaGraphExec_t* find(const std::vector<uint64_t>& key) {
    for (auto& x : e)
      if (x.key == key) {
        x.used = ++tick;
        return &x.exec;
      }
    return nullptr;
  }
  void put(std::vector<uint64_t> key, cudaGraphExec_t exec) {
    if (e.size() >= 128) {
      auto it = std::min_element(e.begin(), e.end(), [](const Entry& a, const Entry& b) { return a.used < b.used; });
      cudaGraphExecDestroy(it->exec);
      e.erase(it);
    }
    e.push_back(Entry{std::move(key), exec, ++tick});
  }
};
thread_local GraphCache g_graphs;

std::vector<uint64_t> plan_key(const CompressPlan& p, const uint8_t* ws) {
  std::vector<uint64_t> k;
  int dev = 0;
  cudaGetDevice(&dev);
  k.push_back((uint64_t)dev);
  k.push_back((uint64_t)(uintptr_t)ws);
  k.push_back((uint64_t)p.t.n() | ((uint64_t)p.worklist << 32));
  for (int c = 0; c < 4; ++c)
    k.push_back((uint64_t)rerun_blocks(p.tu, c) | ((uint64_t)p.tu.budget16[c] << 20) |
                ((uint64_t)p.tu.dense16[c] << 40) | ((uint64_t)p.tu.order[c] << 56));
  for (const FieldInfo& f : p.t.F) {
    const uint64_t* w = reinterpret_cast<const uint64_t*>(&f);
    for (size_t i = 0; i < sizeof(FieldInfo) / 8; ++i) k.push_back(w[i]);
  }
  return k;
}

// Enqueues a planned compression on `st`: as a cached graph, or as direct launches
// with a host-driven loop while per-kernel timing is on.
int run_compress(const CompressPlan& p, uint8_t* ws, cudaStream_t st) {
  const Ptrs q = ptrs_of(p, ws);
  int rc = upload_plan(p, q, st);
  if (rc) return rc;
  if (g_prof.on) return run_host_loop(p, q, st);
  std::vector<uint64_t> key = plan_key(p, ws);
  cudaGraphExec_t* ex = g_graphs.find(key);
  if (!ex) {
    cudaGraphExec_t e = nullptr;
    if ((rc = capture_graph(p, q, st, &e))) return rc;
    g_graphs.put(std::move(key), e);
    ex = g_graphs.find(plan_key(p, ws));
  }
  CK(cudaGraphLaunch(*ex, st));
  return LOPC_OK;
}

// Host staging of the small read-backs of a single-field call: pinned, one per host
// thread, so that the copies are plain DMA behind one synchronisation (pageable ones are
// staged by the driver one at a time).  Null when pinned memory cannot be had; the
// callers then use their stack.
struct Readback {
  struct {
    uint64_t size;
    int status;
    int pad;
  } res;
  Params hp;
  BatchState hb;
  uint8_t header[kHeaderBytes];
  unsigned status;
};
struct ReadbackHolder {
  Readback* p = nullptr;
  bool tried = false;
  ~ReadbackHolder() {
    if (p) (void)cudaFreeHost(p);
  }
};
Readback* readback() {
  thread_local ReadbackHolder h;
  if (!h.tried) {
    h.tried = true;
    if (cudaMallocHost(&h.p, sizeof(Readback)) != cudaSuccess) {
      h.p = nullptr;
      (void)cudaGetLastError();
    }
  }
  return h.p;
}

// Single field: plan, run, read back the size and status.
int compress_one(const lopc_field_desc* d, const void* d_x, void* d_out, size_t out_cap, size_t* out_size,
                 int64_t* bins_out, uint64_t* subbins_out, void* d_ws, size_t ws_size, cudaStream_t st) {
  CompressPlan p;
  const void* xs[1] = {d_x};
  void* outs[1] = {d_out};
  size_t caps[1] = {out_cap};
  const bool wl = g_repair_mode == LOPC_REPAIR_WORKLIST;
  plan_compress(1, d, xs, outs, caps, nullptr, nullptr, nullptr, nullptr, p, wl);
  if (!d_ws || ws_size < p.ws_total) return LOPC_ERR_WORKSPACE;
  uint8_t* ws = reinterpret_cast<uint8_t*>(d_ws);
  uint64_t* dsize = reinterpret_cast<uint64_t*>(ws + p.off_results);
  int* dstat = reinterpret_cast<int*>(ws + p.off_results + 8);
  plan_compress(1, d, xs, outs, caps, dsize, dstat, bins_out, ws, p, wl);
  int rc = run_compress(p, ws, st);
  if (rc) return rc;
  const FieldInfo& f = p.t.F[0];
  if (subbins_out)
    LAUNCH("export", st,
           k_export_subbins<<<148 * 8, 256, 0, st>>>(f.g.nz * f.g.ny * f.g.nx, f.s, subbins_out));
  Readback local;
  Readback* rbk = readback();
  if (!rbk) rbk = &local;
  auto& res = rbk->res;
  const Params& hp = rbk->hp;
  const BatchState& hb = rbk->hb;
  CK(cudaMemcpyAsync(&rbk->res, dsize, 16, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&rbk->hp, f.P, sizeof(Params), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&rbk->hb, ptrs_of(p, ws).B, sizeof(BatchState), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  g_last_rounds = (int64_t)hb.rounds;
  g_last_tile_runs = p.worklist ? f.g.ntiles : (int64_t)(2 * f.g.ntiles + hb.runs);
  g_last_fix_iters = (int64_t)hp.fix_iters;
  g_last_fix_iters_max = (int64_t)hp.fix_iters_max;
  for (int k = 0; k < 9; ++k) g_last_phase[k] = (int64_t)hp.phase[k];
  for (int k = 0; k < 6; ++k) g_last_work[k] = (int64_t)hp.work[k];
  g_last_work[6] = (int64_t)hp.pass_ordered;
  // the repair ran even if the output was too small: report the repair's status first
  if (res.status == LOPC_ERR_CAPACITY && subbins_out) res.status = LOPC_OK;
  if (res.status) return res.status;
  if (out_size) *out_size = (size_t)res.size;
  return LOPC_OK;
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
  if (rd(h, 4) != kMagic || rd(h + 4, 2) < 1 || rd(h + 4, 2) > LOPC_VERSION) return LOPC_ERR_CORRUPT;
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

// ------------------------------------------------------------ decompress plan

struct DecompressPlan {
  int n = 0;
  std::vector<int> order;
  std::vector<DecField> F;
  int cls_f0[4] = {0, 0, 0, 0}, cls_nf[4] = {0, 0, 0, 0};
  int64_t cls_t0[4] = {0, 0, 0, 0}, cls_nt[4] = {0, 0, 0, 0};
  size_t off_table = 0, off_status = 0;
  std::vector<size_t> off_offs;
  size_t ws_total = 0;
};

// Layout: the stream table and one status word per stream in the first aligned
// block, then each stream's record offsets.
int plan_decompress(int n, const lopc_field_desc* descs, const void* const* ins, const size_t* in_sizes,
                    void* const* xs, int* d_status, uint8_t* ws, DecompressPlan& p) {
  p = DecompressPlan{};  // planning twice (size, then pointers) must not accumulate
  p.n = n;
  p.order.resize(n);
  for (int i = 0; i < n; ++i) p.order[i] = i;
  std::stable_sort(p.order.begin(), p.order.end(), [&](int a, int b) {
    return class_of(descs[a].dtype, descs[a].ndim) < class_of(descs[b].dtype, descs[b].ndim);
  });
  p.F.assign(n, DecField{});
  int64_t tiles = 0;
  for (int k = 0; k < n; ++k) {
    const lopc_field_desc* d = &descs[p.order[k]];
    const int c = class_of(d->dtype, d->ndim);
    if (p.cls_nf[c] == 0) {
      p.cls_f0[c] = k;
      p.cls_t0[c] = tiles;
    }
    ++p.cls_nf[c];
    DecField& f = p.F[k];
    f.g = geometry_of(d);
    f.tile_base = tiles;
    tiles += f.g.ntiles;
    p.cls_nt[c] += f.g.ntiles;
  }
  size_t o = 0;
  p.off_table = o;
  o += (size_t)n * sizeof(DecField);
  p.off_status = o;
  o = align256(o + 4 * (size_t)n);
  p.off_offs.resize(n);
  for (int k = 0; k < n; ++k) {
    p.off_offs[k] = o;
    o = align256(o + 16 * (size_t)p.F[k].g.ntiles);
  }
  p.ws_total = o;
  if (!ws) return LOPC_OK;
  for (int k = 0; k < n; ++k) {
    const int i = p.order[k];
    DecField& f = p.F[k];
    f.in = reinterpret_cast<const uint8_t*>(ins[i]);
    f.in_size = (uint64_t)in_sizes[i];
    f.x = xs[i];
    f.offs = reinterpret_cast<uint64_t*>(ws + p.off_offs[k]);
    f.status = reinterpret_cast<unsigned int*>(ws + p.off_status) + k;
    f.status_out = d_status ? d_status + i : nullptr;
  }
  return LOPC_OK;
}
static_assert(sizeof(DecField) + 4 <= 256, "a one-stream table and its status fit the first 256 bytes");

template <typename T, int ND>
int launch_class_decode(const DecompressPlan& p, int c, const DecField* dF, cudaStream_t st) {
  using C = TileCfg<T, ND>;
  if (!p.cls_nf[c]) return LOPC_OK;
  int rc = set_smem_attrs<T, ND>();
  if (rc) return rc;
  LAUNCH("decode", st,
         k_decode<T, ND><<<(unsigned)p.cls_nt[c], C::NTC, DecSmem<T, ND>::bytes(), st>>>(dF, p.cls_f0[c], p.cls_nf[c],
                                                                                       p.cls_t0[c]));
  CK(cudaGetLastError());
  return LOPC_OK;
}

int run_decompress(const DecompressPlan& p, uint8_t* ws, cudaStream_t st) {
  DecField* dF = reinterpret_cast<DecField*>(ws + p.off_table);
  CK(cudaMemcpyAsync(dF, p.F.data(), (size_t)p.n * sizeof(DecField), cudaMemcpyHostToDevice, st));
  LAUNCH("dec_setup", st, k_dec_setup<<<(p.n + 63) / 64, 64, 0, st>>>(dF, p.n));
  LAUNCH("dec_offsets", st, k_dec_offsets<1024><<<p.n, 1024, 0, st>>>(dF));
  int rc;
  if ((rc = launch_class_decode<float, 2>(p, 0, dF, st))) return rc;
  if ((rc = launch_class_decode<float, 3>(p, 1, dF, st))) return rc;
  if ((rc = launch_class_decode<double, 2>(p, 2, dF, st))) return rc;
  if ((rc = launch_class_decode<double, 3>(p, 3, dF, st))) return rc;
  LAUNCH("dec_finalize", st, k_dec_finalize<<<(p.n + 63) / 64, 64, 0, st>>>(dF, p.n));
  CK(cudaGetLastError());
  return LOPC_OK;
}

// Single stream, decoded with the workspace `ws`: header to the host (the launch
// needs the field's class and shape), then the planned launch and its status.
int decompress_one(const void* d_in, size_t in_size, void* d_x, size_t x_cap, uint8_t* ws, size_t ws_size,
                   cudaStream_t st, size_t max_chunks) {
  if (!d_in || !d_x) return LOPC_ERR_INVALID_ARG;
  if (in_size < (size_t)kHeaderBytes) return LOPC_ERR_CORRUPT;
  // the pinned staging, except for the entry point that must allocate nothing
  Readback local;
  Readback* rbk = max_chunks ? nullptr : readback();
  if (!rbk) rbk = &local;
  uint8_t* hb = rbk->header;
  CK(cudaMemcpyAsync(hb, d_in, kHeaderBytes, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  Header H;
  int rc = parse_header(hb, in_size, &H);
  if (rc) return rc;
  const Geometry g = geometry_of(&H.d);
  if (H.total > in_size) return LOPC_ERR_CORRUPT;  // a truncated stream is corrupt, whatever it declares
  if (max_chunks && (size_t)g.ntiles > max_chunks) return LOPC_ERR_WORKSPACE;  // beyond a fixed scratch
  const size_t need = (size_t)(g.nz * g.ny * g.nx) * word_bytes(H.d.dtype);
  if (x_cap < need) return LOPC_ERR_CAPACITY;
  DecompressPlan p;
  plan_decompress(1, &H.d, nullptr, nullptr, nullptr, nullptr, nullptr, p);
  if (!ws || ws_size < p.ws_total) return LOPC_ERR_WORKSPACE;
  const void* ins[1] = {d_in};
  size_t sizes[1] = {in_size};
  void* xs[1] = {d_x};
  plan_decompress(1, &H.d, ins, sizes, xs, nullptr, ws, p);
  if ((rc = run_decompress(p, ws, st))) return rc;
  rbk->status = 0;
  CK(cudaMemcpyAsync(&rbk->status, ws + p.off_status, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return rbk->status ? LOPC_ERR_CORRUPT : LOPC_OK;
}

// ------------------------------------------------------------ serving engine
// Round-level continuous batching.  Every field admitted so far keeps its state
// (bins, subbins, lower masks, dirty bitmap) in its own workspace for its whole
// life.  One step runs a compaction and a rerun round over every field in repair
// on the rounds stream.  On the aux stream it runs the tile pass and first round
// of the fields submitted since the last step, and encodes and packs the fields
// whose last compaction listed no tile.  Fields join and leave between rounds, so
// a field that arrives while others are repairing is never held back by them.

struct EngineItem {
  FieldInfo f;
  uint64_t tag;
  int slot;
};

struct EngineBatch {
  std::vector<EngineItem> items;
  cudaEvent_t done;
};

}  // namespace

struct lopc_engine {
  int max_fields = 0;
  int64_t max_tiles = 0;
  cudaStream_t sm = nullptr, sa = nullptr;  // rounds; new and finishing fields
  cudaEvent_t ev_counts = nullptr, ev_pro = nullptr, ev_ready = nullptr;
  cudaEvent_t ev_stage[3] = {nullptr, nullptr, nullptr};
  FieldInfo* dT[3] = {nullptr, nullptr, nullptr};  // tables: 0 = in repair, 1 = new, 2 = finishing
  FieldInfo* hT[3] = {nullptr, nullptr, nullptr};  // their pinned staging copies
  BatchState* dB = nullptr;
  uint32_t* dlist = nullptr;
  uint32_t* dapp = nullptr;  // tiles the running fields' reruns append to their round
  unsigned int* dcounts = nullptr;
  unsigned int* hcounts = nullptr;  // pinned
  uint64_t* hsize = nullptr;        // pinned and mapped: k_finalize writes each field's result here
  int* hstatus = nullptr;
  uint64_t* dsize = nullptr;        // device aliases of hsize / hstatus
  int* dstatus = nullptr;
  std::vector<EngineItem> fresh, running, done;
  std::deque<EngineBatch> finishing;
  std::vector<cudaEvent_t> spare_events;
  std::vector<int> free_slots;
  bool pro_pending = false;
  int64_t tiles_held = 0;  // tiles of fresh + running fields (bounds the rerun list)
};

namespace {

void engine_free(lopc_engine* e) {
  if (e->sm) cudaStreamSynchronize(e->sm);
  if (e->sa) cudaStreamSynchronize(e->sa);
  for (auto& b : e->finishing) cudaEventDestroy(b.done);
  for (cudaEvent_t ev : e->spare_events) cudaEventDestroy(ev);
  cudaEvent_t evs[6] = {e->ev_counts, e->ev_pro, e->ev_ready, e->ev_stage[0], e->ev_stage[1], e->ev_stage[2]};
  for (cudaEvent_t ev : evs)
    if (ev) cudaEventDestroy(ev);
  for (int k = 0; k < 3; ++k) {
    if (e->dT[k]) cudaFree(e->dT[k]);
    if (e->hT[k]) cudaFreeHost(e->hT[k]);
  }
  if (e->dB) cudaFree(e->dB);
  if (e->dlist) cudaFree(e->dlist);
  if (e->dapp) cudaFree(e->dapp);
  if (e->dcounts) cudaFree(e->dcounts);
  if (e->hcounts) cudaFreeHost(e->hcounts);
  if (e->hsize) cudaFreeHost(e->hsize);
  if (e->hstatus) cudaFreeHost(e->hstatus);
  if (e->sm) cudaStreamDestroy(e->sm);
  if (e->sa) cudaStreamDestroy(e->sa);
  delete e;
}

int engine_init(lopc_engine* e) {
  const size_t tb = (size_t)e->max_fields * sizeof(FieldInfo);
  CK(cudaStreamCreateWithFlags(&e->sm, cudaStreamNonBlocking));
  CK(cudaStreamCreateWithFlags(&e->sa, cudaStreamNonBlocking));
  CK(cudaEventCreateWithFlags(&e->ev_counts, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&e->ev_pro, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&e->ev_ready, cudaEventDisableTiming));
  for (int k = 0; k < 3; ++k) {
    CK(cudaEventCreateWithFlags(&e->ev_stage[k], cudaEventDisableTiming));
    CK(cudaMalloc(&e->dT[k], tb));
    CK(cudaHostAlloc(&e->hT[k], tb, cudaHostAllocDefault));
  }
  CK(cudaMalloc(&e->dB, sizeof(BatchState)));
  CK(cudaMemset(e->dB, 0, sizeof(BatchState)));
  CK(cudaMalloc(&e->dlist, 4 * (size_t)std::max<int64_t>(1, e->max_tiles)));
  CK(cudaMalloc(&e->dapp, 4 * (size_t)std::max<int64_t>(1, e->max_tiles)));
  CK(cudaMalloc(&e->dcounts, 4 * (size_t)e->max_fields));
  CK(cudaHostAlloc(&e->hcounts, 4 * (size_t)e->max_fields, cudaHostAllocDefault));
  CK(cudaHostAlloc(&e->hsize, 8 * (size_t)e->max_fields, cudaHostAllocMapped));
  CK(cudaHostAlloc(&e->hstatus, 4 * (size_t)e->max_fields, cudaHostAllocMapped));
  CK(cudaHostGetDevicePointer(reinterpret_cast<void**>(&e->dsize), e->hsize, 0));
  CK(cudaHostGetDevicePointer(reinterpret_cast<void**>(&e->dstatus), e->hstatus, 0));
  for (int s = e->max_fields - 1; s >= 0; --s) e->free_slots.push_back(s);
  return LOPC_OK;
}

// Sorts items by class (stable) and builds their table with fresh numbering.
void engine_table(std::vector<EngineItem>& items, Table& t) {
  std::stable_sort(items.begin(), items.end(), [](const EngineItem& a, const EngineItem& b) {
    return class_of_geometry(a.f.g) < class_of_geometry(b.f.g);
  });
  t.F.resize(items.size());
  for (size_t k = 0; k < items.size(); ++k) t.F[k] = items[k].f;
  layout_table(t);
}

// Copies table t into device table `which` on stream st (staging reused once the
// previous copy from it has run).
int engine_upload(lopc_engine* e, int which, const Table& t, cudaStream_t st) {
  CK(cudaEventSynchronize(e->ev_stage[which]));
  memcpy(e->hT[which], t.F.data(), (size_t)t.n() * sizeof(FieldInfo));
  CK(cudaMemcpyAsync(e->dT[which], e->hT[which], (size_t)t.n() * sizeof(FieldInfo), cudaMemcpyHostToDevice, st));
  CK(cudaEventRecord(e->ev_stage[which], st));
  return LOPC_OK;
}

int engine_step(lopc_engine* e, int rounds, int* active) {
  int rc;
  const Tune tu = current_tune();
  const bool round = !e->running.empty();
  Table tr;
  if (round) {
    engine_table(e->running, tr);
    if ((rc = engine_upload(e, 0, tr, e->sm))) return rc;
    if (e->pro_pending) {
      CK(cudaStreamWaitEvent(e->sm, e->ev_pro, 0));
      e->pro_pending = false;
    }
    for (int r = 0; r < rounds; ++r) {
      const bool last = r + 1 == rounds;
      if ((rc = launch_compact(tr, e->dT[0], e->dlist, e->dB, last ? e->dcounts : nullptr, {}, 0, e->sm))) return rc;
      if (last) {
        CK(cudaMemcpyAsync(e->hcounts, e->dcounts, 4 * (size_t)tr.n(), cudaMemcpyDeviceToHost, e->sm));
        CK(cudaEventRecord(e->ev_counts, e->sm));
      }
      if ((rc = launch_reruns(tr, e->dT[0], tu, e->dB, e->dlist, e->dapp, e->sm))) return rc;
    }
  }
  if (!e->fresh.empty()) {
    Table ta;
    engine_table(e->fresh, ta);
    if ((rc = engine_upload(e, 1, ta, e->sa))) return rc;
    if ((rc = launch_pre(ta, e->dT[1], tu, e->sa))) return rc;
    // no appends here: this round runs beside the running fields' round, which owns
    // the append counters
    if ((rc = launch_reruns(ta, e->dT[1], tu, e->dB, nullptr, nullptr, e->sa))) return rc;
    CK(cudaEventRecord(e->ev_pro, e->sa));
    e->pro_pending = true;
  }
  if (round) {
    // the rerun round is still running on the device while the host sorts the fields
    CK(cudaEventSynchronize(e->ev_counts));
    std::vector<EngineItem> keep, fin;
    for (int k = 0; k < tr.n(); ++k) (e->hcounts[k] ? keep : fin).push_back(e->running[k]);
    e->running.swap(keep);
    if (!fin.empty()) {
      Table tc;
      engine_table(fin, tc);
      if ((rc = engine_upload(e, 2, tc, e->sa))) return rc;
      CK(cudaStreamWaitEvent(e->sa, e->ev_counts, 0));
      if ((rc = launch_epilogue(tc, e->dT[2], e->sa))) return rc;
      EngineBatch b;
      b.items = std::move(fin);
      if (e->spare_events.empty()) {
        CK(cudaEventCreateWithFlags(&b.done, cudaEventDisableTiming));
      } else {
        b.done = e->spare_events.back();
        e->spare_events.pop_back();
      }
      CK(cudaEventRecord(b.done, e->sa));
      for (const EngineItem& it : b.items) e->tiles_held -= it.f.g.ntiles;
      e->finishing.push_back(std::move(b));
    }
  }
  e->running.insert(e->running.end(), e->fresh.begin(), e->fresh.end());
  e->fresh.clear();
  if (active) {
    size_t n = e->running.size() + e->done.size();
    for (const auto& b : e->finishing) n += b.items.size();
    *active = (int)n;
  }
  return LOPC_OK;
}

// ---------------------------------------------------------------- verifier
// Workspace: the link table (one byte per 14-bit neighbour set), the blocks'
// partial sums and the report.
constexpr int64_t kVerifyMaxParts = 4096;
struct VerifyLayout {
  size_t table, parts, report, total;
};
VerifyLayout verify_layout() {
  VerifyLayout L;
  L.table = 0;
  L.parts = align256(3 << 14);  // cc, full3, full2; then one partial per block of the grid
  L.report = L.parts + align256(sizeof(VerifyPartial) * (size_t)kVerifyMaxParts);
  L.total = L.report + align256(sizeof(lopc_verify_report));
  return L;
}

template <typename T, int ND>
int launch_verify(const Geometry& g, const void* d_x, const void* d_y, uint8_t* tx, uint8_t* ty, uint8_t* ws,
                  const VerifyLayout& L, int64_t& nparts, cudaStream_t st) {
  using VS = VerifySmem<T, ND>;
  constexpr int NT = TileCfg<T, ND>::NT;
  thread_local int per_sm_dev[64] = {};  // resident blocks per SM, per instantiation and device
  int dev = 0;
  CK(cudaGetDevice(&dev));
  int& per_sm = per_sm_dev[dev & 63];
  if (!per_sm) {
    CK(cudaFuncSetAttribute(k_verify<T, ND>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)VS::bytes()));
    int occ = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_verify<T, ND>, NT, VS::bytes()));
    per_sm = std::max(1, occ);
  }
  nparts = std::min<int64_t>(std::min<int64_t>(g.ntiles, (int64_t)per_sm * sm_count()), kVerifyMaxParts);
  LAUNCH("verify", st,
         k_verify<T, ND><<<(unsigned)nparts, NT, VS::bytes(), st>>>(
             g, reinterpret_cast<const T*>(d_x), reinterpret_cast<const T*>(d_y), ws + L.table,
             ws + L.table + (ND == 3 ? 1 : 2) * (1 << 14), tx, ty,
             reinterpret_cast<VerifyPartial*>(ws + L.parts)));
  CK(cudaGetLastError());
  return LOPC_OK;
}

int verify_one(const lopc_field_desc* d, const void* d_x, const void* d_y, uint8_t* tx, uint8_t* ty,
               lopc_verify_report* h_report, uint8_t* ws, size_t ws_size, cudaStream_t st) {
  const Geometry g = geometry_of(d);
  const VerifyLayout L = verify_layout();
  if (!ws || ws_size < L.total || (reinterpret_cast<uintptr_t>(ws) & 255)) return LOPC_ERR_WORKSPACE;
  LAUNCH("link_table", st,
         k_link_table<<<(1 << 14) / 256, 256, 0, st>>>(ws + L.table, ws + L.table + (1 << 14), ws + L.table + (2 << 14)));
  CK(cudaGetLastError());
  int64_t nparts = 0;
  int rc;
  switch (class_of(d->dtype, d->ndim)) {
    case 0: rc = launch_verify<float, 2>(g, d_x, d_y, tx, ty, ws, L, nparts, st); break;
    case 1: rc = launch_verify<float, 3>(g, d_x, d_y, tx, ty, ws, L, nparts, st); break;
    case 2: rc = launch_verify<double, 2>(g, d_x, d_y, tx, ty, ws, L, nparts, st); break;
    default: rc = launch_verify<double, 3>(g, d_x, d_y, tx, ty, ws, L, nparts, st); break;
  }
  if (rc) return rc;
  const int64_t points = g.nz * g.ny * g.nx;
  lopc_verify_report* d_rep = reinterpret_cast<lopc_verify_report*>(ws + L.report);
  LAUNCH("verify_finalize", st,
         k_verify_finalize<256><<<1, 256, 0, st>>>(reinterpret_cast<const VerifyPartial*>(ws + L.parts),
                                                    (int)nparts, points, d->mode, d->eb, d_rep));
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(h_report, d_rep, sizeof(lopc_verify_report), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return h_report->nonfinite ? LOPC_ERR_NONFINITE : LOPC_OK;
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
  CompressPlan p;
  plan_compress(1, d, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, p,
                g_repair_mode == LOPC_REPAIR_WORKLIST);
  return p.ws_total;
}

int lopc_set_repair_mode(int mode) {
  if (mode != LOPC_REPAIR_TILES && mode != LOPC_REPAIR_WORKLIST) return LOPC_ERR_INVALID_ARG;
  const int prev = g_repair_mode;
  g_repair_mode = mode;
  return prev;
}

size_t lopc_batch_compress_workspace_size(int n, const lopc_field_desc* descs) {
  if (n <= 0 || n > LOPC_MAX_BATCH_FIELDS || !descs) return 0;
  for (int i = 0; i < n; ++i)
    if (!desc_valid(&descs[i])) return 0;
  CompressPlan p;
  plan_compress(n, descs, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, p);
  return p.ws_total;
}

size_t lopc_decompress_workspace_size(const lopc_field_desc* d) { return lopc_batch_decompress_workspace_size(1, d); }

size_t lopc_batch_decompress_workspace_size(int n, const lopc_field_desc* descs) {
  if (n <= 0 || !descs) return 0;
  for (int i = 0; i < n; ++i)
    if (!desc_valid(&descs[i])) return 0;
  DecompressPlan p;
  plan_decompress(n, descs, nullptr, nullptr, nullptr, nullptr, nullptr, p);
  return p.ws_total;
}

int lopc_compress(const lopc_field_desc* d, const void* d_x, void* d_out, size_t out_cap, size_t* out_size, void* d_ws,
                  size_t ws_size, void* stream) {
  int rc;
  if (!desc_valid(d) || !d_x || !d_out || !out_size) {
    rc = LOPC_ERR_INVALID_ARG;
  } else if (out_cap < (size_t)kHeaderBytes) {
    rc = LOPC_ERR_CAPACITY;
  } else {
    rc = compress_one(d, d_x, d_out, out_cap, out_size, nullptr, nullptr, d_ws, ws_size,
                      reinterpret_cast<cudaStream_t>(stream));
  }
  g_prof.resolve();
  return rc;
}

int lopc_batch_compress(int n, const lopc_field_desc* descs, const void* const* d_x, void* const* d_out,
                        const size_t* out_cap, uint64_t* d_out_size, int* d_status, const lopc_plan* plan,
                        void* d_ws, size_t ws_size, void* stream) {
  if (n <= 0 || n > LOPC_MAX_BATCH_FIELDS || !descs || !d_x || !d_out || !out_cap || !d_out_size || !d_status)
    return LOPC_ERR_INVALID_ARG;
  for (int i = 0; i < n; ++i)
    if (!desc_valid(&descs[i]) || !d_x[i] || !d_out[i]) return LOPC_ERR_INVALID_ARG;
  CompressPlan p;
  plan_compress(n, descs, d_x, d_out, out_cap, d_out_size, d_status, nullptr, nullptr, p);
  if (!d_ws || ws_size < p.ws_total) return LOPC_ERR_WORKSPACE;
  plan_compress(n, descs, d_x, d_out, out_cap, d_out_size, d_status, nullptr, reinterpret_cast<uint8_t*>(d_ws), p);
  if (plan) p.tu = tune_of_plan(*plan);
  const int rc = run_compress(p, reinterpret_cast<uint8_t*>(d_ws), reinterpret_cast<cudaStream_t>(stream));
  if (g_prof.on) {
    (void)cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream));
    g_prof.resolve();
  }
  return rc;
}

int lopc_quantize_repair(const lopc_field_desc* d, const void* d_x, int64_t* d_bins, uint64_t* d_subbins, void* d_ws,
                         size_t ws_size, void* stream) {
  int rc;
  if (!desc_valid(d) || !d_x || !d_bins || !d_subbins) {
    rc = LOPC_ERR_INVALID_ARG;
  } else {
    // the whole compression runs; with no output capacity the stream is not packed
    rc = compress_one(d, d_x, d_ws, 0, nullptr, d_bins, d_subbins, d_ws, ws_size, reinterpret_cast<cudaStream_t>(stream));
  }
  g_prof.resolve();
  return rc;
}

int lopc_peek(const void* h_stream, size_t n, lopc_field_desc* out) {
  if (!h_stream || !out) return LOPC_ERR_INVALID_ARG;
  Header H;
  const int rc = parse_header(reinterpret_cast<const uint8_t*>(h_stream), n, &H);
  if (rc) return rc;
  *out = H.d;
  return LOPC_OK;
}

int lopc_decompress(const void* d_in, size_t in_size, void* d_x, size_t x_cap, void* d_ws, size_t ws_size,
                    void* stream) {
  const int rc = decompress_one(d_in, in_size, d_x, x_cap, reinterpret_cast<uint8_t*>(d_ws), ws_size,
                                reinterpret_cast<cudaStream_t>(stream), 0);
  g_prof.resolve();
  return rc;
}

int lopc_batch_decompress(int n, const lopc_field_desc* descs, const void* const* d_in, const size_t* in_size,
                          void* const* d_x, int* d_status, void* d_ws, size_t ws_size, void* stream) {
  if (n <= 0 || !descs || !d_in || !in_size || !d_x || !d_status) return LOPC_ERR_INVALID_ARG;
  for (int i = 0; i < n; ++i)
    if (!desc_valid(&descs[i]) || !d_in[i] || !d_x[i]) return LOPC_ERR_INVALID_ARG;
  DecompressPlan p;
  plan_decompress(n, descs, d_in, in_size, d_x, d_status, nullptr, p);
  if (!d_ws || ws_size < p.ws_total) return LOPC_ERR_WORKSPACE;
  plan_decompress(n, descs, d_in, in_size, d_x, d_status, reinterpret_cast<uint8_t*>(d_ws), p);
  const int rc = run_decompress(p, reinterpret_cast<uint8_t*>(d_ws), reinterpret_cast<cudaStream_t>(stream));
  if (g_prof.on) {
    (void)cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream));
    g_prof.resolve();
  }
  return rc;
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
// Device address of the scratch array on the current device.  In host code the
// array's name is only a stand-in, so the address comes from cudaGetSymbolAddress
// with that device current.  It is looked up on every call (cheap next to the
// synchronous header read), so a device reset between calls cannot leave a stale
// address behind.
int noalloc_scratch(uint8_t** out) {
  void* p = nullptr;
  CK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
  *out = reinterpret_cast<uint8_t*>(p);
  return LOPC_OK;
}
}  // namespace

int lopc_decompress_noalloc(const void* d_in, size_t in_size, void* d_x, size_t x_cap, void* stream) {
  uint8_t* ws = nullptr;
  const cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int rc = noalloc_scratch(&ws);
  // every offset the decoder reads is rewritten and its status word zeroed first
  if (!rc) {
    rc = decompress_one(d_in, in_size, d_x, x_cap, ws, kNoAllocScratchBytes, st, (size_t)kNoAllocMaxChunks);
    // an error can come after work was queued on the shared scratch: wait for it, so
    // that every call returns with the scratch idle
    if (rc) (void)cudaStreamSynchronize(st);
  }
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
  for (int k = 0; k < n && k < 9; ++k) cycles[k] = g_last_phase[k];
  return 9;
}

int lopc_decode_phase_enable(int on) {
  const int v = on != 0;
  CK(cudaMemcpyToSymbol(g_dec_phase_on, &v, sizeof(int)));
  return LOPC_OK;
}

int lopc_decode_phase_read(int64_t* out, int n) {
  unsigned long long h[8] = {};
  CK(cudaDeviceSynchronize());
  CK(cudaMemcpyFromSymbol(h, g_dec_phase, sizeof(h)));
  for (int k = 0; k < n && k < 8; ++k) out[k] = (int64_t)h[k];
  const unsigned long long z[8] = {};
  CK(cudaMemcpyToSymbol(g_dec_phase, z, sizeof(z)));
  return 8;
}

int lopc_last_round_tiles(int64_t* out, int n) {
  const int m = (int)g_round_tiles.size();
  for (int k = 0; k < n && k < m; ++k) out[k] = g_round_tiles[k];
  return m;
}

int lopc_last_fixpoint_work(int64_t* out, int n) {
  for (int k = 0; k < n && k < 7; ++k) out[k] = g_last_work[k];
  return 7;
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

int lopc_profile_read_launches(const char* name, double* ms, int cap) {
  g_prof.resolve();
  for (int i = 0; i < g_prof.n; ++i) {
    if (!name || strcmp(g_prof.entries[i].name, name) != 0) continue;
    const std::vector<float>& v = g_prof.entries[i].each;
    for (int k = 0; k < cap && k < (int)v.size(); ++k) ms[k] = v[k];
    return (int)v.size();
  }
  return 0;
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
    case LOPC_ERR_BUSY: return "serving engine full";
    default: return "unknown status";
  }
}


void lopc_plan_get(lopc_plan* pl) {
  if (!pl) return;
  memset(pl, 0, sizeof(*pl));
  const Tune u = current_tune();
  for (int c = 0; c < 4; ++c) {
    pl->rerun_blocks_per_sm[c] = u.rerun_per_sm[c];
    pl->pass_budget16[c] = u.budget16[c];
    pl->pass_dense16[c] = u.dense16[c];
    pl->pass_order[c] = u.order[c];
  }
}

void lopc_plan_default(lopc_plan* pl) {
  if (!pl) return;
  memset(pl, 0, sizeof(*pl));
  for (int c = 0; c < 4; ++c) {
    pl->rerun_blocks_per_sm[c] = c < 2 ? 4 : 6;
    pl->pass_budget16[c] = 64;
    pl->pass_dense16[c] = 8;
    pl->pass_order[c] = 0;
  }
}

void lopc_tune_set(const int* v) {
  if (!v) return;
  for (int c = 0; c < 4; ++c) g_rerun_per_sm[c] = v[c] < 1 ? 1 : (v[c] > 16 ? 16 : v[c]);
}

void lopc_tune_get(int* v) {
  if (!v) return;
  for (int c = 0; c < 4; ++c) v[c] = g_rerun_per_sm[c];
}

void lopc_tune_set_budget(const int* v) {
  if (!v) return;
  for (int c = 0; c < 4; ++c) g_pass_budget16[c] = v[c] < 1 ? 1 : (v[c] > 4096 ? 4096 : v[c]);
}

void lopc_tune_get_budget(int* v) {
  if (!v) return;
  for (int c = 0; c < 4; ++c) v[c] = g_pass_budget16[c];
}

void lopc_tune_set_dense(const int* v) {
  if (!v) return;
  for (int c = 0; c < 4; ++c) g_pass_dense16[c] = v[c] < 0 ? 0 : (v[c] > 17 ? 17 : v[c]);
}

void lopc_tune_get_dense(int* v) {
  if (!v) return;
  for (int c = 0; c < 4; ++c) v[c] = g_pass_dense16[c];
}

void lopc_tune_set_pass_order(const int* v) {
  if (!v) return;
  for (int c = 0; c < 4; ++c) g_pass_order[c] = v[c] < 0 ? 0 : (v[c] > 2 ? 2 : v[c]);
}

void lopc_tune_get_pass_order(int* v) {
  if (!v) return;
  for (int c = 0; c < 4; ++c) v[c] = g_pass_order[c];
}

// ------------------------------------------------------------ serving engine ABI

int lopc_engine_create(int max_fields, int64_t max_tiles, lopc_engine** out) {
  if (!out || max_fields <= 0 || max_fields > 65535 || max_tiles <= 0 || max_tiles > (int64_t(1) << 32))
    return LOPC_ERR_INVALID_ARG;
  *out = nullptr;
  lopc_engine* e = new lopc_engine;
  e->max_fields = max_fields;
  e->max_tiles = max_tiles;
  const int rc = engine_init(e);
  if (rc) {
    engine_free(e);
    return rc;
  }
  *out = e;
  return LOPC_OK;
}

void lopc_engine_destroy(lopc_engine* e) {
  if (e) engine_free(e);
}

size_t lopc_engine_field_workspace_size(const lopc_field_desc* d) {
  if (!desc_valid(d)) return 0;
  return field_part(geometry_of(d)).total;
}

int lopc_engine_submit(lopc_engine* e, const lopc_field_desc* d, const void* d_x, void* d_out, size_t out_cap,
                       void* d_ws, size_t ws_size, uint64_t tag, void* ready_stream) {
  if (!e || !desc_valid(d) || !d_x || !d_out) return LOPC_ERR_INVALID_ARG;
  const Geometry g = geometry_of(d);
  if (!d_ws || ws_size < field_part(g).total || (reinterpret_cast<uintptr_t>(d_ws) & 255)) return LOPC_ERR_WORKSPACE;
  if (e->free_slots.empty() || e->tiles_held + g.ntiles > e->max_tiles) return LOPC_ERR_BUSY;
  // the engine's streams wait for the input to be ready on the caller's stream
  CK(cudaEventRecord(e->ev_ready, reinterpret_cast<cudaStream_t>(ready_stream)));
  CK(cudaStreamWaitEvent(e->sa, e->ev_ready, 0));
  EngineItem it;
  it.slot = e->free_slots.back();
  e->free_slots.pop_back();
  it.tag = tag;
  it.f = field_entry(d, d_x, d_out, out_cap, e->dsize + it.slot, e->dstatus + it.slot, nullptr,
                     reinterpret_cast<uint8_t*>(d_ws));
  e->hsize[it.slot] = 0;
  e->hstatus[it.slot] = LOPC_ERR_CUDA;
  e->tiles_held += g.ntiles;
  e->fresh.push_back(it);
  return LOPC_OK;
}

int lopc_engine_step(lopc_engine* e, int rounds, int* active) {
  if (!e || rounds <= 0) return LOPC_ERR_INVALID_ARG;
  return engine_step(e, rounds, active);
}

int lopc_engine_poll(lopc_engine* e, uint64_t* tags, uint64_t* sizes, int* statuses, int cap) {
  if (!e || cap < 0 || (cap > 0 && (!tags || !sizes || !statuses))) return LOPC_ERR_INVALID_ARG;
  while (!e->finishing.empty()) {
    const cudaError_t q = cudaEventQuery(e->finishing.front().done);
    if (q == cudaErrorNotReady) break;
    if (q != cudaSuccess) {
      (void)cudaGetLastError();
      return LOPC_ERR_CUDA;
    }
    EngineBatch& b = e->finishing.front();
    e->done.insert(e->done.end(), b.items.begin(), b.items.end());
    e->spare_events.push_back(b.done);
    e->finishing.pop_front();
  }
  const int n = (int)std::min<size_t>((size_t)cap, e->done.size());
  for (int k = 0; k < n; ++k) {
    const EngineItem& it = e->done[k];
    tags[k] = it.tag;
    sizes[k] = e->hsize[it.slot];
    statuses[k] = e->hstatus[it.slot];
    e->free_slots.push_back(it.slot);
  }
  e->done.erase(e->done.begin(), e->done.begin() + n);
  return n;
}

int lopc_engine_sync(lopc_engine* e) {
  if (!e) return LOPC_ERR_INVALID_ARG;
  CK(cudaStreamSynchronize(e->sm));
  CK(cudaStreamSynchronize(e->sa));
  return LOPC_OK;
}

size_t lopc_verify_workspace_size(const lopc_field_desc* d) {
  if (!desc_valid(d)) return 0;
  return verify_layout().total;
}

int lopc_verify(const lopc_field_desc* d, const void* d_x, const void* d_y, uint8_t* d_types_x,
                uint8_t* d_types_y, lopc_verify_report* h_report, void* d_ws, size_t ws_size, void* stream) {
  if (!desc_valid(d) || !d_x || !d_y || !h_report || (d_types_y && !d_types_x)) return LOPC_ERR_INVALID_ARG;
  const int rc = verify_one(d, d_x, d_y, d_types_x, d_types_y, h_report, reinterpret_cast<uint8_t*>(d_ws), ws_size,
                            reinterpret_cast<cudaStream_t>(stream));
  g_prof.resolve();
  return rc;
}

}  // extern "C"
