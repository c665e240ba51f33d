// Host side of the C ABI (include/ggeval.h): datasets, workspace, launch
// planning, CUDA-graph replay, the autotuner and argument validation.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <set>
#include <string>
#include <tuple>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "ggeval.h"
#include "gom.cuh"
#include "misc.cuh"

namespace {

// An NVTX range over a scope (a profiler's timeline shows where the host
// side of each call spends its time; without a tool attached it costs a
// load and a branch).
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range&) = delete;
  Range& operator=(const Range&) = delete;
};

thread_local std::string g_err = "no error";

ggeval_status fail(ggeval_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

#define GG_CU(call)                                                                          \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      return fail(e_ == cudaErrorMemoryAllocation ? GGEVAL_ERR_OOM : GGEVAL_ERR_CUDA,        \
                  "%s: %s", #call, cudaGetErrorString(e_));                                  \
  } while (0)

#define GG_TRY(expr)                  \
  do {                                        \
    ggeval_status s_ = (expr);                \
    if (s_ != GGEVAL_OK) return s_;           \
  } while (0)

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int d) {
    cudaGetDevice(&prev);
    if (prev != d) cudaSetDevice(d);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

inline int stride_of(int h) { return (1 << (h + 1)) - 1; }
// stack slots of a template of height h: Sethi-Ullman order with fused
// terminals needs at most h - 1 (the packer checks the bound)
inline int slots_of(int h) { return h > 2 ? h - 1 : 1; }
inline int lstride_of(int h) { return stride_of(h) + 1; }

const void* fwd_ptr(int variant, bool pow) {
  return pow ? gg::fwd_ptr_pow(variant) : gg::fwd_ptr_plain(variant);
}

// GGEVAL_F_POW selects the kernels that run pow instructions.
inline bool has_pow(uint32_t flags) { return (flags & GGEVAL_F_POW) != 0; }

// Raise the dynamic shared-memory limit of a kernel once per device.
ggeval_status prepare_kernel(int device, const void* fn) {
  static std::mutex mu;
  static std::set<std::pair<int, const void*>> done;
  std::lock_guard<std::mutex> lock(mu);
  if (done.count({device, fn})) return GGEVAL_OK;
  int optin = 0;
  GG_CU(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device));
  GG_CU(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
  done.insert({device, fn});
  return GGEVAL_OK;
}

struct Cfg {
  int variant = 0, tile_rows = 0, group = 0, warps = 0;
  bool operator==(const Cfg& o) const {
    return variant == o.variant && tile_rows == o.tile_rows && group == o.group &&
           warps == o.warps;
  }
};

struct Plan {
  Cfg cfg;
  bool pow = false;  // kernels with the pow instructions; the packer accepts pow
  bool fold = true;  // the packer folds constant subtrees (not GGEVAL_F_NO_FOLD)
  bool stall = false;  // GGEVAL_F_TEST_STALL
  int slots = 0, stride = 0, lstride = 0, n_tiles = 0, n_items = 0, grid = 0;
  size_t smem = 0;
  const void* fn = nullptr;
};

// the outputs of one evaluation call (any but smse may be null)
struct Outs {
  float* f[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};  // smse, a, b, mse, nmse
  int32_t* size = nullptr;
  int32_t* size_eval = nullptr;
};

Outs outs_of(float* smse, float* a, float* bb, float* mse) {
  Outs o;
  o.f[0] = smse;
  o.f[1] = a;
  o.f[2] = bb;
  o.f[3] = mse;
  return o;
}

struct GraphKey {
  ggeval_batch b;
  uint32_t flags;
  const void* mask;
  const void* out[7];
  const void* ws[8];  // workspace buffers the captured launches point at
  Cfg cfg;
  int kind;
};

bool same_key(const GraphKey& x, const GraphKey& y) {
  return std::memcmp(&x.b, &y.b, sizeof x.b) == 0 && x.flags == y.flags && x.mask == y.mask &&
         std::memcmp(x.out, y.out, sizeof x.out) == 0 && std::memcmp(x.ws, y.ws, sizeof x.ws) == 0 &&
         x.cfg == y.cfg && x.kind == y.kind;
}

}  // namespace

struct ggeval_dataset {
  int device = 0, sms = 0;
  char gpu_name[256] = {0};
  int64_t N = 0;
  int F = 0, ldx = 0;
  size_t smem_optin = 0;
  float* X = nullptr;        // [F + 1][ldx], row F = y - mean(y)
  float* ylo = nullptr;      // [ldx]: the FP32 rounding error of row F (adjoint residuals)
  float2* pref = nullptr;    // [N + 1] prefix sums of the stored centred target (hi, lo)
  double ybar = 0, syc = 0, sycyc = 0;
  cudaStream_t cap_stream = nullptr;
  // workspace (grown on demand)
  uint2* prog = nullptr;
  size_t cap_prog = 0;
  gg::Aux* aux = nullptr;
  size_t cap_aux = 0;
  int* len = nullptr;
  size_t cap_len = 0;
  float* part = nullptr;
  size_t cap_part = 0;
  double* ab = nullptr;
  size_t cap_ab = 0;
  double* gacc = nullptr;
  size_t cap_gacc = 0;
  int* counters = nullptr;
  size_t cap_counters = 0;
  int* adjbin = nullptr;  // adjoint: class counts and counters, then the class lists
  size_t cap_adjbin = 0;
  int* idx = nullptr;  // masked evaluation: the compacted trial indices
  size_t cap_idx = 0;
  unsigned* status = nullptr;
  // device staging of host-memory batches
  unsigned char* stage = nullptr;
  size_t cap_stage = 0;
  std::map<std::tuple<int, int, int, int>, Cfg> tuned;
  GraphKey gkey{};
  cudaGraphExec_t gexec = nullptr;
  // GGEVAL_F_PROFILE: event pairs around the batched forward kernel
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_ev;
  size_t prof_used = 0;
};

namespace {

template <class T>
ggeval_status grow(T*& p, size_t& cap, size_t need) {
  if (need <= cap) return GGEVAL_OK;
  if (p) cudaFree(p);
  p = nullptr;
  cap = 0;
  size_t n = need + need / 4 + 16;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&p), n * sizeof(T));
  if (e != cudaSuccess) {
    p = nullptr;
    return fail(GGEVAL_ERR_OOM, "cudaMalloc(%zu bytes): %s", n * sizeof(T), cudaGetErrorString(e));
  }
  cap = n;
  return GGEVAL_OK;
}

ggeval_status check_batch(const ggeval_dataset* ds, const ggeval_batch* b) {
  if (!ds) return fail(GGEVAL_ERR_ARG, "dataset is NULL");
  if (!b) return fail(GGEVAL_ERR_ARG, "batch is NULL");
  if (b->n < 0) return fail(GGEVAL_ERR_ARG, "batch n = %d < 0", b->n);
  if (b->max_height < 0) return fail(GGEVAL_ERR_ARG, "max_height %d < 0", b->max_height);
  if (b->max_height > GGEVAL_MAX_HEIGHT)
    return fail(GGEVAL_ERR_UNSUPPORTED, "max_height %d > %d", b->max_height, GGEVAL_MAX_HEIGHT);
  if (b->layout != GGEVAL_LAYOUT_HEAP && b->layout != GGEVAL_LAYOUT_PREFIX)
    return fail(GGEVAL_ERR_ARG, "unknown layout %d", b->layout);
  if (b->memory != GGEVAL_MEM_DEVICE && b->memory != GGEVAL_MEM_HOST)
    return fail(GGEVAL_ERR_ARG, "unknown memory kind %d", b->memory);
  if (b->n > 0 && (!b->op || !b->cval)) return fail(GGEVAL_ERR_ARG, "op or cval is NULL");
  if ((int64_t)b->n * stride_of(b->max_height) > (int64_t)1 << 31)
    return fail(GGEVAL_ERR_UNSUPPORTED, "batch of %d trials too large", b->n);
  return GGEVAL_OK;
}

// Trials per work item for row tiles of `tile` rows: about 32 work items per
// SM, and at least `warps` trials per item.
int group_for(const ggeval_dataset* ds, int n, int warps, int tile) {
  const double target = 16.0 * ds->sms * 2;
  const int n_tiles = (int)((ds->N + tile - 1) / tile);
  long long n_groups = (long long)std::ceil(target / n_tiles);
  const long long max_groups = (n + warps - 1) / warps;
  if (n_groups > max_groups) n_groups = max_groups;
  if (n_groups < 1) n_groups = 1;
  const int g = (int)((n + n_groups - 1) / n_groups);
  return g < 1 ? 1 : g;
}

// Default tile shape: enough work items for every SM several times over, X
// tiles as large as the work allows (each tile is reused by `group` trials).
Cfg default_cfg(const ggeval_dataset* ds, int n, int h_max, uint32_t flags) {
  Cfg c;
  const bool exact = (flags & GGEVAL_F_EXACT) || ds->N < 32768;
  c.variant = exact ? 2 : 0;
  c.warps = 8;
  const int rpp = 32 * gg::variant_rows(c.variant);
  const int lst = lstride_of(h_max);
  int max_tile = exact ? 2048 : 2048;
  while (max_tile > rpp &&
         gg::fwd_smem_bytes(ds->F, max_tile, c.warps, lst, slots_of(h_max),
                            gg::variant_rows(c.variant)) > ds->smem_optin / 2)
    max_tile /= 2;
  const double target = 16.0 * ds->sms * 2;
  double want = (double)ds->N * n / ((double)c.warps * target);
  int tile = rpp;
  while (tile < max_tile && tile < want && tile < ds->N) tile *= 2;
  c.tile_rows = tile;
  c.group = group_for(ds, n, c.warps, tile);
  return c;
}

ggeval_status make_plan(ggeval_dataset* ds, int n, int h_max, const Cfg& cfg, Plan* pl,
                        bool pow) {
  pl->cfg = cfg;
  pl->pow = pow;
  pl->slots = slots_of(h_max);
  pl->stride = stride_of(h_max);
  pl->lstride = lstride_of(h_max);
  pl->fn = fwd_ptr(cfg.variant, pow);
  if (!pl->fn) return fail(GGEVAL_ERR_ARG, "no kernel for variant %d", cfg.variant);
  const int rpp = 32 * gg::variant_rows(cfg.variant);
  if (cfg.tile_rows < rpp || cfg.tile_rows % rpp || cfg.group < 1 || cfg.warps < 1 ||
      cfg.warps > gg::variant_max_warps(cfg.variant))
    return fail(GGEVAL_ERR_ARG, "bad tile configuration");
  pl->smem = gg::fwd_smem_bytes(ds->F, cfg.tile_rows, cfg.warps, pl->lstride, pl->slots,
                                gg::variant_rows(cfg.variant));
  if (pl->smem > ds->smem_optin) return fail(GGEVAL_ERR_ARG, "tile needs too much shared memory");
  pl->n_tiles = (int)((ds->N + cfg.tile_rows - 1) / cfg.tile_rows);
  const long long n_groups = (n + cfg.group - 1) / cfg.group;
  if ((long long)pl->n_tiles * n_groups > (1ll << 31) - 1)
    return fail(GGEVAL_ERR_UNSUPPORTED, "too many work items");
  pl->n_items = (int)(pl->n_tiles * n_groups);
  GG_TRY(prepare_kernel(ds->device, pl->fn));
  int nb = 0;
  GG_CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, pl->fn, cfg.warps * 32, pl->smem));
  if (nb < 1) return fail(GGEVAL_ERR_ARG, "tile configuration does not fit on an SM");
  long long grid = (long long)nb * ds->sms;
  pl->grid = (int)(grid < pl->n_items ? grid : pl->n_items);
  if (pl->grid < 1) pl->grid = 1;
  return GGEVAL_OK;
}

Cfg pick_cfg(ggeval_dataset* ds, const ggeval_batch* b, uint32_t flags) {
  auto it = ds->tuned.find(
      {b->n, b->max_height, b->layout, (int)(flags & (GGEVAL_F_EXACT | GGEVAL_F_POW))});
  if (it != ds->tuned.end()) return it->second;
  return default_cfg(ds, b->n, b->max_height, flags);
}

struct DevBatch {
  const uint8_t* op;
  const float* cval;
  const int8_t* height;
};

// Copy a host batch into the staging area (on the stream) and return the
// device pointers; `extra` bytes after it are handed back in *scratch.
ggeval_status stage_batch(ggeval_dataset* ds, const ggeval_batch* b, size_t extra,
                          cudaStream_t st, DevBatch* db, unsigned char** scratch) {
  const size_t cnt = (size_t)b->n * stride_of(b->max_height);
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t o_op = 0, o_cv = al(cnt), o_h = o_cv + al(cnt * 4), o_x = o_h + al(b->n);
  GG_TRY(grow(ds->stage, ds->cap_stage, o_x + extra));
  if (b->memory == GGEVAL_MEM_HOST) {
    GG_CU(cudaMemcpyAsync(ds->stage + o_op, b->op, cnt, cudaMemcpyHostToDevice, st));
    GG_CU(cudaMemcpyAsync(ds->stage + o_cv, b->cval, cnt * 4, cudaMemcpyHostToDevice, st));
    if (b->height)
      GG_CU(cudaMemcpyAsync(ds->stage + o_h, b->height, b->n, cudaMemcpyHostToDevice, st));
    db->op = ds->stage + o_op;
    db->cval = reinterpret_cast<const float*>(ds->stage + o_cv);
    db->height = b->height ? reinterpret_cast<const int8_t*>(ds->stage + o_h) : nullptr;
  } else {
    db->op = b->op;
    db->cval = b->cval;
    db->height = b->height;
  }
  if (scratch) *scratch = ds->stage + o_x;
  return GGEVAL_OK;
}

ggeval_status ensure_ws(ggeval_dataset* ds, int n, const Plan& pl, bool grad) {
  GG_TRY(grow(ds->prog, ds->cap_prog, (size_t)n * pl.lstride));
  GG_TRY(grow(ds->len, ds->cap_len, (size_t)n + 1));
  GG_TRY(grow(ds->part, ds->cap_part, (size_t)n * pl.n_tiles * gg::NPART));
  GG_TRY(grow(ds->ab, ds->cap_ab, (size_t)n * 4 + 4));
  GG_TRY(grow(ds->counters, ds->cap_counters, (size_t)n + 8));
  GG_TRY(grow(ds->idx, ds->cap_idx, (size_t)n + 1));
  if (grad) {
    GG_TRY(grow(ds->aux, ds->cap_aux, (size_t)n * pl.lstride));
    GG_TRY(grow(ds->gacc, ds->cap_gacc, (size_t)n * pl.stride));
    GG_TRY(grow(ds->adjbin, ds->cap_adjbin, (size_t)gg::ADJ_NCLS_MAX * (2 + (size_t)n)));
  }
  return GGEVAL_OK;
}

ggeval_status launch(const void* fn, dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                     void* params) {
  void* args[] = {params};
  GG_CU(cudaLaunchKernel(fn, grid, block, args, smem, st));
  return GGEVAL_OK;
}

// A launch that may start before the kernel ahead of it in the stream has
// finished (programmatic dependent launch): the kernel waits for it with
// griddepcontrol.wait before it reads that kernel's output.
ggeval_status launch_overlapped(const void* fn, dim3 grid, dim3 block, size_t smem,
                                cudaStream_t st, void* params) {
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  void* args[] = {params};
  GG_CU(cudaLaunchKernelExC(&cfg, fn, args));
  return GGEVAL_OK;
}

ggeval_status enqueue_pack(ggeval_dataset* ds, const DevBatch& db, int n, int h_max, int layout,
                           const Plan& pl, bool with_aux, cudaStream_t st,
                           const int* count = nullptr, const int* idx = nullptr,
                           int32_t* size = nullptr, int32_t* size_eval = nullptr) {
  Range r("ggeval pack");
  gg::PackParams pp{};
  pp.op = db.op;
  pp.cval = db.cval;
  pp.height = db.height;
  pp.n = n;
  pp.h_max = h_max;
  pp.stride = pl.stride;
  pp.layout = layout;
  pp.n_features = ds->F;
  pp.max_slots = pl.slots;
  pp.lstride = pl.lstride;
  pp.prog = ds->prog;
  pp.aux = with_aux ? ds->aux : nullptr;
  pp.len = ds->len;
  pp.status = ds->status;
  pp.count = count;
  pp.idx = idx;
  pp.allow_pow = pl.pow ? 1 : 0;
  pp.fold = pl.fold ? 1 : 0;
  pp.size_active = size;
  pp.size_eval = size_eval;
  return launch(gg::pack_ptr(), dim3((n + gg::PACK_WARPS - 1) / gg::PACK_WARPS),
                dim3(32 * gg::PACK_WARPS), gg::PACK_WARPS * gg::pack_warp_bytes(pl.stride), st,
                &pp);
}

gg::FwdParams fwd_params(ggeval_dataset* ds, int n, const Plan& pl) {
  gg::FwdParams fp{};
  fp.X = ds->X;
  fp.N = (int)ds->N;
  fp.F = ds->F;
  fp.ldx = ds->ldx;
  fp.prog = ds->prog;
  fp.len = ds->len;
  fp.lstride = pl.lstride;
  fp.P = n;
  fp.tile_rows = pl.cfg.tile_rows;
  fp.n_tiles = pl.n_tiles;
  fp.group = pl.cfg.group;
  fp.n_items = pl.n_items;
  fp.slots = pl.slots;
  fp.part = ds->part;
  fp.counter = ds->counters;
  fp.status = ds->status;
  fp.rows_out = nullptr;
  fp.wait_limit = gg::WAIT_LIMIT;
  fp.stall = pl.stall ? 1 : 0;
  if (pl.stall) fp.wait_limit = 1u << 12;  // the test hook gives up soon
  return fp;
}

gg::FinParams fin_params(ggeval_dataset* ds, int n, const Plan& pl, float* smse, float* a,
                         float* b, float* mse) {
  gg::FinParams q{};
  q.part = ds->part;
  q.len = ds->len;
  q.P = n;
  q.n_tiles = pl.n_tiles;
  q.tile_rows = pl.cfg.tile_rows;
  q.N = ds->N;
  q.pref = ds->pref;
  q.ybar = ds->ybar;
  q.syc = ds->syc;
  q.sycyc = ds->sycyc;
  q.smse = smse;
  q.a = a;
  q.b = b;
  q.mse = mse;
  q.ab = ds->ab;
  return q;
}

constexpr size_t PROF_MAX = 4096;

// zero counters -> [compact the masked trials] -> pack -> batched forward ->
// finalise.  With a mask the changed trials are compacted into slots
// 0 .. count-1 on the device (counters[2] = count, ds->idx = their indices), so
// the forward kernel's work items cover only them.
ggeval_status enqueue_eval(ggeval_dataset* ds, const DevBatch& db, const ggeval_batch* b,
                           const Plan& pl, const Outs& o, bool with_aux, cudaStream_t st,
                           bool profile = false, const uint8_t* mask = nullptr) {
  Range r("ggeval enqueue evaluation");
  const int n = b->n;
  // counters[0]: the work counter; counters[2]: the compacted count;
  // counters[8 + slot]: the slot's trial found non-finite
  GG_CU(cudaMemsetAsync(ds->counters, 0, sizeof(int) * ((size_t)n + 8), st));
  const int* count = nullptr;
  const int* idx = nullptr;
  if (mask) {
    const int threads = n >= 1024 ? 1024 : ((n + 31) / 32) * 32;
    const uint8_t* m = mask;
    int nn = n;
    int* out_idx = ds->idx;
    int* out_count = ds->counters + 2;
    void* args[] = {&m, &nn, &out_idx, &out_count};
    GG_CU(cudaLaunchKernel(gg::compact_ptr(), dim3(1), dim3(threads), args, 0, st));
    count = ds->counters + 2;
    idx = ds->idx;
  }
  GG_TRY(enqueue_pack(ds, db, n, b->max_height, b->layout, pl, with_aux, st, count, idx,
                      o.size, o.size_eval));
  gg::FwdParams fp = fwd_params(ds, n, pl);
  fp.dead = ds->counters + 8;
  fp.count = count;
  std::pair<cudaEvent_t, cudaEvent_t>* ev = nullptr;
  if (profile && ds->prof_used < PROF_MAX) {
    if (ds->prof_used == ds->prof_ev.size()) {
      cudaEvent_t e0, e1;
      GG_CU(cudaEventCreate(&e0));
      GG_CU(cudaEventCreate(&e1));
      ds->prof_ev.push_back({e0, e1});
    }
    ev = &ds->prof_ev[ds->prof_used++];
    GG_CU(cudaEventRecord(ev->first, st));
  }
  // the forward kernel overlaps the packer's tail and the finaliser the
  // forward kernel's (not when a profiling event sits between them)
  if (ev) GG_TRY(launch(pl.fn, dim3(pl.grid), dim3(pl.cfg.warps * 32), pl.smem, st, &fp));
  else GG_TRY(launch_overlapped(pl.fn, dim3(pl.grid), dim3(pl.cfg.warps * 32), pl.smem, st, &fp));
  if (ev) GG_CU(cudaEventRecord(ev->second, st));
  gg::FinParams q = fin_params(ds, n, pl, o.f[0], o.f[1], o.f[2], o.f[3]);
  q.nmse = o.f[4];
  q.dead = fp.dead;
  q.count = count;
  q.idx = idx;
  GG_TRY(launch_overlapped(gg::fin_ptr(), dim3((n + gg::FIN_WARPS - 1) / gg::FIN_WARPS),
                           dim3(32 * gg::FIN_WARPS), 0, st, &q));
  return GGEVAL_OK;
}

// ------------------------------------------------------ tuning cache file
// One JSON object per line:
//   {"gpu": "NVIDIA GB300", "sms": 152, "rows": 100000, "features": 8,
//    "trials": 4096, "max_height": 4, "layout": 0, "flags": 0,
//    "variant": 0, "tile_rows": 2048, "group": 82, "warps": 24}
// A dataset takes the entries whose GPU name, SM count, rows and features
// match its own.
using TuneKey = std::tuple<int, int, int, int>;

bool json_int(const char* line, const char* key, long long* out) {
  char pat[64];
  std::snprintf(pat, sizeof pat, "\"%s\":", key);
  const char* p = std::strstr(line, pat);
  if (!p) return false;
  p += std::strlen(pat);
  char* end = nullptr;
  const long long v = std::strtoll(p, &end, 10);
  if (end == p) return false;
  *out = v;
  return true;
}

bool json_str(const char* line, const char* key, std::string* out) {
  char pat[64];
  std::snprintf(pat, sizeof pat, "\"%s\":", key);
  const char* p = std::strstr(line, pat);
  if (!p) return false;
  p = std::strchr(p + std::strlen(pat), '"');
  if (!p) return false;
  const char* q = std::strchr(p + 1, '"');
  if (!q) return false;
  out->assign(p + 1, q);
  return true;
}

// entries of `path` for this dataset (a missing file holds none)
ggeval_status load_tuning(ggeval_dataset* ds, const char* path, int* taken) {
  *taken = 0;
  FILE* f = std::fopen(path, "r");
  if (!f) return GGEVAL_OK;
  char line[1024];
  while (std::fgets(line, sizeof line, f)) {
    std::string gpu;
    long long sms, rows, feat, n, h, lay, fl, v, tile, group, warps;
    if (!json_str(line, "gpu", &gpu) || !json_int(line, "sms", &sms) ||
        !json_int(line, "rows", &rows) || !json_int(line, "features", &feat) ||
        !json_int(line, "trials", &n) || !json_int(line, "max_height", &h) ||
        !json_int(line, "layout", &lay) || !json_int(line, "flags", &fl) ||
        !json_int(line, "variant", &v) || !json_int(line, "tile_rows", &tile) ||
        !json_int(line, "group", &group) || !json_int(line, "warps", &warps))
      continue;  // not an entry
    if (gpu != ds->gpu_name || sms != ds->sms || rows != ds->N || feat != ds->F) continue;
    Cfg c;
    c.variant = (int)v;
    c.tile_rows = (int)tile;
    c.group = (int)group;
    c.warps = (int)warps;
    if (!gg::fitness_variant(c.variant)) continue;
    ds->tuned[TuneKey((int)n, (int)h, (int)lay, (int)fl)] = c;
    ++*taken;
  }
  std::fclose(f);
  return GGEVAL_OK;
}

ggeval_status append_tuning(const ggeval_dataset* ds, const char* path, const TuneKey& k,
                            const Cfg& c) {
  FILE* f = std::fopen(path, "a");
  if (!f) return fail(GGEVAL_ERR_ARG, "cannot open tuning cache %s", path);
  std::fprintf(f,
               "{\"gpu\": \"%s\", \"sms\": %d, \"rows\": %lld, \"features\": %d, "
               "\"trials\": %d, \"max_height\": %d, \"layout\": %d, \"flags\": %d, "
               "\"variant\": %d, \"tile_rows\": %d, \"group\": %d, \"warps\": %d}\n",
               ds->gpu_name, ds->sms, (long long)ds->N, ds->F, std::get<0>(k), std::get<1>(k),
               std::get<2>(k), std::get<3>(k), c.variant, c.tile_rows, c.group, c.warps);
  std::fclose(f);
  return GGEVAL_OK;
}

void drop_graph(ggeval_dataset* ds) {
  if (ds->gexec) cudaGraphExecDestroy(ds->gexec);
  ds->gexec = nullptr;
  std::memset(&ds->gkey, 0, sizeof ds->gkey);
}

}  // namespace

extern "C" {

const char* ggeval_last_error(void) { return g_err.c_str(); }

const char* ggeval_version(void) { return "ggeval 0.1 (sm_103a)"; }

ggeval_status ggeval_create_dataset(const float* X, const float* y, int64_t n_rows,
                                    int32_t n_features, int32_t x_row_major, int32_t device,
                                    void* stream, ggeval_dataset** out) {
  if (!out) return fail(GGEVAL_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!X || !y) return fail(GGEVAL_ERR_ARG, "X or y is NULL");
  if (n_rows < 1 || n_rows > (int64_t)1 << 30)
    return fail(GGEVAL_ERR_ARG, "n_rows = %lld out of range", (long long)n_rows);
  if (n_features < 1 || n_features > GGEVAL_MAX_FEATURES)
    return fail(GGEVAL_ERR_ARG, "n_features = %d out of range", n_features);
  int ndev = 0;
  GG_CU(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) return fail(GGEVAL_ERR_ARG, "no device %d", device);
  DeviceGuard guard(device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t N = n_rows;
  const int F = n_features;
  // target: centre in FP64, store as float
  std::vector<float> yh((size_t)N);
  GG_CU(cudaMemcpy(yh.data(), y, (size_t)N * 4, cudaMemcpyDefault));
  double sum = 0;
  for (int64_t i = 0; i < N; ++i) {
    const double v = yh[i];
    if (!std::isfinite(v) || std::fabs(v) > 1125899906842624.0)
      return fail(GGEVAL_ERR_ARG, "y[%lld] = %g is not finite or exceeds 2^50", (long long)i, v);
    sum += v;
  }
  auto* ds = new ggeval_dataset();
  ds->device = device;
  ds->N = N;
  ds->F = F;
  ds->ldx = (int)((N + 3) & ~(int64_t)3);
  ds->ybar = sum / (double)N;
  std::vector<double> pref((size_t)N + 1);
  pref[0] = 0;
  double s2 = 0;
  std::vector<float> ylo((size_t)N);
  for (int64_t i = 0; i < N; ++i) {
    const double yc = (double)yh[i] - ds->ybar;
    yh[i] = (float)yc;
    ylo[i] = (float)(yc - (double)yh[i]);
    pref[i + 1] = pref[i] + (double)yh[i];
    s2 += (double)yh[i] * (double)yh[i];
  }
  ds->syc = pref[N];
  ds->sycyc = s2;
  // the prefix sums as FP32 (hi, lo) pairs: the finaliser merges in FP32
  std::vector<float2> pref2((size_t)N + 1);
  for (size_t i = 0; i <= (size_t)N; ++i) {
    const float hi = (float)pref[i];
    pref2[i] = make_float2(hi, (float)(pref[i] - (double)hi));
  }
  auto cleanup = [&](ggeval_status s) {
    ggeval_destroy(ds);
    return s;
  };
  cudaError_t e;
  if ((e = cudaDeviceGetAttribute(&ds->sms, cudaDevAttrMultiProcessorCount, device)) ||
      (e = cudaStreamCreateWithFlags(&ds->cap_stream, cudaStreamNonBlocking))) {
    fail(GGEVAL_ERR_CUDA, "device query: %s", cudaGetErrorString(e));
    return cleanup(GGEVAL_ERR_CUDA);
  }
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  ds->smem_optin = (size_t)optin;
  {
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) == cudaSuccess)
      std::snprintf(ds->gpu_name, sizeof ds->gpu_name, "%s", prop.name);
  }
  const size_t xbytes = (size_t)(F + 1) * ds->ldx * 4;
  if ((e = cudaMalloc(&ds->X, xbytes)) || (e = cudaMalloc(&ds->pref, ((size_t)N + 1) * 8)) ||
      (e = cudaMalloc(&ds->ylo, (size_t)ds->ldx * 4)) ||
      (e = cudaMalloc(&ds->status, sizeof(unsigned)))) {
    fail(GGEVAL_ERR_OOM, "dataset allocation: %s", cudaGetErrorString(e));
    return cleanup(GGEVAL_ERR_OOM);
  }
  float* tmp = nullptr;
  do {
    if ((e = cudaMemsetAsync(ds->X, 0, xbytes, st))) break;
    if ((e = cudaMemsetAsync(ds->status, 0, sizeof(unsigned), st))) break;
    if (x_row_major) {
      if ((e = cudaMalloc(&tmp, (size_t)N * F * 4))) break;
      if ((e = cudaMemcpyAsync(tmp, X, (size_t)N * F * 4, cudaMemcpyDefault, st))) break;
      gg::TransposeParams tp{tmp, ds->X, (int)N, F, ds->ldx};
      void* args[] = {&tp};
      if ((e = cudaLaunchKernel(gg::transpose_ptr(), dim3((unsigned)((N + 31) / 32), (F + 31) / 32),
                                dim3(32, 8), args, 0, st)))
        break;
    } else {
      if ((e = cudaMemcpy2DAsync(ds->X, (size_t)ds->ldx * 4, X, (size_t)N * 4, (size_t)N * 4, F,
                                 cudaMemcpyDefault, st)))
        break;
    }
    if ((e = cudaMemcpyAsync(ds->X + (size_t)F * ds->ldx, yh.data(), (size_t)N * 4,
                             cudaMemcpyHostToDevice, st)))
      break;
    if ((e = cudaMemcpyAsync(ds->pref, pref2.data(), ((size_t)N + 1) * 8, cudaMemcpyHostToDevice,
                             st)))
      break;
    if ((e = cudaMemsetAsync(ds->ylo, 0, (size_t)ds->ldx * 4, st))) break;
    if ((e = cudaMemcpyAsync(ds->ylo, ylo.data(), (size_t)N * 4, cudaMemcpyHostToDevice, st)))
      break;
    e = cudaStreamSynchronize(st);
  } while (0);
  if (tmp) cudaFree(tmp);
  if (e) {
    fail(e == cudaErrorMemoryAllocation ? GGEVAL_ERR_OOM : GGEVAL_ERR_CUDA, "dataset upload: %s",
         cudaGetErrorString(e));
    return cleanup(e == cudaErrorMemoryAllocation ? GGEVAL_ERR_OOM : GGEVAL_ERR_CUDA);
  }
  *out = ds;
  return GGEVAL_OK;
}

void ggeval_destroy(ggeval_dataset* ds) {
  if (!ds) return;
  DeviceGuard guard(ds->device);
  cudaDeviceSynchronize();
  drop_graph(ds);
  cudaFree(ds->X);
  cudaFree(ds->pref);
  cudaFree(ds->ylo);
  cudaFree(ds->status);
  cudaFree(ds->prog);
  cudaFree(ds->aux);
  cudaFree(ds->len);
  cudaFree(ds->part);
  cudaFree(ds->ab);
  cudaFree(ds->gacc);
  cudaFree(ds->counters);
  cudaFree(ds->adjbin);
  cudaFree(ds->idx);
  cudaFree(ds->stage);
  for (auto& e : ds->prof_ev) {
    cudaEventDestroy(e.first);
    cudaEventDestroy(e.second);
  }
  if (ds->cap_stream) cudaStreamDestroy(ds->cap_stream);
  delete ds;
}

static ggeval_status eval_batch_impl(ggeval_dataset* ds, const ggeval_batch* b, uint32_t flags,
                                     const Outs& o, void* stream, const uint8_t* mask);

ggeval_status ggeval_eval_batch(ggeval_dataset* ds, const ggeval_batch* b, uint32_t flags,
                                float* smse, float* a, float* bb, float* mse, void* stream) {
  return eval_batch_impl(ds, b, flags, outs_of(smse, a, bb, mse), stream, nullptr);
}

ggeval_status ggeval_evaluate(ggeval_dataset* ds, const ggeval_batch* b, uint32_t flags,
                              const ggeval_outputs* out, void* stream) {
  if (!out) return fail(GGEVAL_ERR_ARG, "outputs is NULL");
  Outs o = outs_of(out->smse, out->a, out->b, out->mse);
  o.f[4] = out->nmse;
  o.size = out->size;
  o.size_eval = out->size_evaluated;
  return eval_batch_impl(ds, b, flags, o, stream, nullptr);
}

ggeval_status ggeval_eval_batch_masked(ggeval_dataset* ds, const ggeval_batch* b,
                                       const uint8_t* mask, uint32_t flags, float* smse, float* a,
                                       float* bb, float* mse, void* stream) {
  if (!mask) return fail(GGEVAL_ERR_ARG, "mask is NULL");
  if (b && b->memory != GGEVAL_MEM_DEVICE)
    return fail(GGEVAL_ERR_ARG, "eval_batch_masked needs a device batch");
  return eval_batch_impl(ds, b, flags, outs_of(smse, a, bb, mse), stream, mask);
}

static ggeval_status eval_batch_impl(ggeval_dataset* ds, const ggeval_batch* b, uint32_t flags,
                                     const Outs& o, void* stream, const uint8_t* mask) {
  Range range("ggeval_eval_batch");
  GG_TRY(check_batch(ds, b));
  if (b->n == 0) return GGEVAL_OK;
  if (!o.f[0]) return fail(GGEVAL_ERR_ARG, "smse is NULL");
  DeviceGuard guard(ds->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Plan pl;
  GG_TRY(make_plan(ds, b->n, b->max_height, pick_cfg(ds, b, flags), &pl, has_pow(flags)));
  pl.fold = (flags & GGEVAL_F_NO_FOLD) == 0;
  pl.stall = (flags & GGEVAL_F_TEST_STALL) != 0;
  GG_TRY(ensure_ws(ds, b->n, pl, false));
  const bool host = b->memory == GGEVAL_MEM_HOST;
  DevBatch db;
  unsigned char* scratch = nullptr;
  // a host batch's outputs are written to device staging first: 7 arrays of
  // n 4-byte values
  GG_TRY(stage_batch(ds, b, host ? (size_t)b->n * 4 * 7 : 0, st, &db, &scratch));
  Outs dev = o;
  if (host) {
    auto slot = [&](int i) { return scratch + (size_t)i * b->n * 4; };
    for (int i = 0; i < 5; ++i) dev.f[i] = o.f[i] ? reinterpret_cast<float*>(slot(i)) : nullptr;
    dev.size = o.size ? reinterpret_cast<int32_t*>(slot(5)) : nullptr;
    dev.size_eval = o.size_eval ? reinterpret_cast<int32_t*>(slot(6)) : nullptr;
  }

  if ((flags & GGEVAL_F_GRAPH) && !host) {
    GraphKey key;
    std::memset(&key, 0, sizeof key);
    key.b = *b;
    key.flags = flags;
    key.mask = mask;
    for (int i = 0; i < 5; ++i) key.out[i] = o.f[i];
    key.out[5] = o.size;
    key.out[6] = o.size_eval;
    const void* ws[8] = {ds->prog, ds->len,   ds->part,   ds->ab,
                         ds->counters, ds->stage, ds->status, ds->idx};
    std::memcpy(key.ws, ws, sizeof ws);
    key.cfg = pl.cfg;
    key.kind = 1;
    if (!ds->gexec || !same_key(key, ds->gkey)) {
      Range rc("ggeval graph capture");
      drop_graph(ds);
      cudaGraph_t g = nullptr;
      GG_CU(cudaStreamBeginCapture(ds->cap_stream, cudaStreamCaptureModeThreadLocal));
      ggeval_status s = enqueue_eval(ds, db, b, pl, dev, false, ds->cap_stream, false, mask);
      cudaError_t e = cudaStreamEndCapture(ds->cap_stream, &g);
      if (s != GGEVAL_OK) {
        if (g) cudaGraphDestroy(g);
        return s;
      }
      if (e != cudaSuccess) return fail(GGEVAL_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
      e = cudaGraphInstantiate(&ds->gexec, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) {
        ds->gexec = nullptr;
        return fail(GGEVAL_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
      }
      ds->gkey = key;
    }
    {
      Range rl("ggeval graph launch");
      GG_CU(cudaGraphLaunch(ds->gexec, st));
    }
    return GGEVAL_OK;
  }
  GG_TRY(enqueue_eval(ds, db, b, pl, dev, false, st, (flags & GGEVAL_F_PROFILE) != 0, mask));
  if (host) {
    for (int i = 0; i < 5; ++i)
      if (o.f[i])
        GG_CU(cudaMemcpyAsync(o.f[i], dev.f[i], (size_t)b->n * 4, cudaMemcpyDeviceToHost, st));
    if (o.size)
      GG_CU(cudaMemcpyAsync(o.size, dev.size, (size_t)b->n * 4, cudaMemcpyDeviceToHost, st));
    if (o.size_eval)
      GG_CU(cudaMemcpyAsync(o.size_eval, dev.size_eval, (size_t)b->n * 4,
                            cudaMemcpyDeviceToHost, st));
  }
  return GGEVAL_OK;
}

ggeval_status ggeval_eval_rows(ggeval_dataset* ds, const ggeval_batch* b, uint32_t flags,
                               float* f, void* stream) {
  GG_TRY(check_batch(ds, b));
  if (b->n == 0) return GGEVAL_OK;
  if (!f) return fail(GGEVAL_ERR_ARG, "f is NULL");
  DeviceGuard guard(ds->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // the configuration ggeval_eval_batch would run, in its per-row build
  Cfg c = pick_cfg(ds, b, flags);
  c.variant = gg::rows_variant(c.variant);
  Plan pl;
  GG_TRY(make_plan(ds, b->n, b->max_height, c, &pl, has_pow(flags)));
  pl.fold = (flags & GGEVAL_F_NO_FOLD) == 0;
  GG_TRY(ensure_ws(ds, b->n, pl, false));
  const bool host = b->memory == GGEVAL_MEM_HOST;
  const size_t fbytes = (size_t)b->n * ds->N * 4;
  DevBatch db;
  unsigned char* scratch = nullptr;
  GG_TRY(stage_batch(ds, b, host ? fbytes : 0, st, &db, &scratch));
  float* fd = host ? reinterpret_cast<float*>(scratch) : f;
  GG_TRY(enqueue_pack(ds, db, b->n, b->max_height, b->layout, pl, false, st));
  GG_CU(cudaMemsetAsync(ds->counters, 0, sizeof(int), st));
  gg::FwdParams fp = fwd_params(ds, b->n, pl);
  fp.rows_out = fd;
  GG_TRY(launch(pl.fn, dim3(pl.grid), dim3(pl.cfg.warps * 32), pl.smem, st, &fp));
  if (host) GG_CU(cudaMemcpyAsync(f, fd, fbytes, cudaMemcpyDeviceToHost, st));
  return GGEVAL_OK;
}

ggeval_status ggeval_eval_plain(ggeval_dataset* ds, const ggeval_batch* b, uint32_t flags,
                                float* smse, float* a, float* bb, float* mse, void* stream) {
  GG_TRY(check_batch(ds, b));
  if (b->n == 0) return GGEVAL_OK;
  if (!smse) return fail(GGEVAL_ERR_ARG, "smse is NULL");
  if (b->memory != GGEVAL_MEM_DEVICE) return fail(GGEVAL_ERR_ARG, "plain form needs a device batch");
  DeviceGuard guard(ds->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // one trial per launch: tiles only over rows, one pass per tile, two warps
  // per CTA (one per tile buffer)
  Cfg c = default_cfg(ds, 1, b->max_height, flags);
  c.group = 1;
  c.warps = 2;
  c.tile_rows = 32 * gg::variant_rows(c.variant);
  Plan pl;
  GG_TRY(make_plan(ds, 1, b->max_height, c, &pl, has_pow(flags)));
  pl.fold = (flags & GGEVAL_F_NO_FOLD) == 0;
  GG_TRY(ensure_ws(ds, b->n, pl, false));
  DevBatch db{b->op, b->cval, b->height};
  GG_TRY(enqueue_pack(ds, db, b->n, b->max_height, b->layout, pl, false, st));
  GG_CU(cudaMemsetAsync(ds->counters, 0, sizeof(int) * (size_t)b->n, st));
  for (int t = 0; t < b->n; ++t) {
    gg::FwdParams fp = fwd_params(ds, 1, pl);
    fp.prog = ds->prog + (size_t)t * pl.lstride;
    fp.len = ds->len + t;
    fp.part = ds->part + (size_t)t * pl.n_tiles * gg::NPART;
    fp.counter = ds->counters + t;
    GG_TRY(launch(pl.fn, dim3(pl.grid), dim3(pl.cfg.warps * 32), pl.smem, st, &fp));
    gg::FinParams q = fin_params(ds, 1, pl, smse + t, a ? a + t : nullptr, bb ? bb + t : nullptr,
                                 mse ? mse + t : nullptr);
    q.part = fp.part;
    q.len = fp.len;
    q.ab = nullptr;
    GG_TRY(launch(gg::fin_ptr(), dim3(1), dim3(32), 0, st, &q));  // one warp, one trial
  }
  return GGEVAL_OK;
}

ggeval_status ggeval_grad_batch(ggeval_dataset* ds, const ggeval_batch* b, uint32_t flags,
                                float* smse, float* dcval, void* stream) {
  Range range("ggeval_grad_batch");
  GG_TRY(check_batch(ds, b));
  if (b->n == 0) return GGEVAL_OK;
  if (!dcval) return fail(GGEVAL_ERR_ARG, "dcval is NULL");
  DeviceGuard guard(ds->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Plan pl;
  GG_TRY(make_plan(ds, b->n, b->max_height, pick_cfg(ds, b, flags), &pl, has_pow(flags)));
  pl.fold = (flags & GGEVAL_F_NO_FOLD) == 0;
  GG_TRY(ensure_ws(ds, b->n, pl, true));
  const bool host = b->memory == GGEVAL_MEM_HOST;
  const size_t gcount = (size_t)b->n * pl.stride;
  DevBatch db;
  unsigned char* scratch = nullptr;
  GG_TRY(stage_batch(ds, b, host ? gcount * 4 + (size_t)b->n * 4 : 0, st, &db, &scratch));
  float* dg = host ? reinterpret_cast<float*>(scratch) : dcval;
  float* ds_smse = smse ? (host ? dg + gcount : smse) : nullptr;
  GG_TRY(enqueue_eval(ds, db, b, pl, outs_of(ds_smse, nullptr, nullptr, nullptr), true, st));
  // adjoint, one launch per length class (programs of at most cap - 1
  // instructions).  Each warp holds its own copy of the program, R rows x
  // 32 lanes of values per instruction and its stack, so shared memory
  // bounds the resident warps.  For each R (rows per lane) take the CTA
  // size (1..8 warps) that keeps the most warps resident per SM, the larger
  // CTA on a tie; then the largest R that keeps at least 6 warps per SM
  // (more rows share each instruction's decode; fewer warps hide less
  // latency).  With at most ADJ_FTILE_MAX features, R = 4 is the staged
  // kernel, taken from 2 warps per SM on.  GGEVAL_ADJ_ROWS (1, 2 or 4)
  // fixes R.
  int caps[gg::ADJ_NCLS_MAX];
  int ncls = 0;
  for (int c : gg::ADJ_CAPS)
    if (c < pl.lstride && ncls < gg::ADJ_NCLS_MAX - 1) caps[ncls++] = c;
  caps[ncls++] = pl.lstride;
  int* cls_count = ds->adjbin;
  int* cls_counter = ds->adjbin + gg::ADJ_NCLS_MAX;
  int* cls_list = ds->adjbin + 2 * gg::ADJ_NCLS_MAX;
  GG_CU(cudaMemsetAsync(ds->adjbin, 0, sizeof(int) * 2 * gg::ADJ_NCLS_MAX, st));
  GG_CU(cudaMemsetAsync(ds->gacc, 0, gcount * 8, st));
  const int mse_mode = (flags & GGEVAL_F_GRAD_MSE) ? 1 : 0;
  gg::AdjBinParams bp{};
  bp.len = ds->len;
  bp.ab = ds->ab;
  bp.P = b->n;
  bp.mse_mode = mse_mode;
  bp.ncls = ncls;
  for (int c = 0; c < ncls; ++c) bp.caps[c] = caps[c];
  bp.count = cls_count;
  bp.list = cls_list;
  int force_rows = 0;
  if (const char* env = getenv("GGEVAL_ADJ_ROWS")) force_rows = atoi(env);
  const bool verbose = getenv("GGEVAL_VERBOSE") && getenv("GGEVAL_VERBOSE")[0] == '1';
  // GGEVAL_F_PROFILE: CUDA events around the adjoint's launches (read with
  // ggeval_profile_read, as the forward kernel's)
  std::pair<cudaEvent_t, cudaEvent_t>* ev = nullptr;
  if ((flags & GGEVAL_F_PROFILE) && !host && ds->prof_used < PROF_MAX) {
    if (ds->prof_used == ds->prof_ev.size()) {
      cudaEvent_t e0, e1;
      GG_CU(cudaEventCreate(&e0));
      GG_CU(cudaEventCreate(&e1));
      ds->prof_ev.push_back({e0, e1});
    }
    ev = &ds->prof_ev[ds->prof_used++];
    GG_CU(cudaEventRecord(ev->first, st));
  }
  GG_TRY(launch(gg::adj_bin_ptr(), dim3((unsigned)((b->n + 255) / 256)), dim3(256), 0, st, &bp));
  for (int c = 0; c < ncls; ++c) {
    const int lcap = caps[c];
    const int ecap = lcap < pl.lstride / 2 ? lcap : pl.lstride / 2;
    const void* afn = nullptr;
    int rows = 0, warps = 0, nb = 0;
    bool fast = false;
    gg::AdjLayout lay{};
    for (int R : {4, 2, 1}) {
      if (force_rows && R != force_rows) continue;
      const bool fs = R == 4 && ds->F <= gg::ADJ_FTILE_MAX;
      const void* fn = gg::adj_ptr(R, pl.pow, fs);
      GG_TRY(prepare_kernel(ds->device, fn));
      const gg::AdjLayout l = gg::adj_layout(lcap, ecap, pl.slots, R, fs, ds->F);
      int wR = 0, nR = 0;
      const int wmax = (int)((ds->smem_optin - 64) / l.total);
      for (int w = wmax < 8 ? wmax : 8; w >= 1; --w) {
        int n = 0;
        GG_CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, w * 32,
                                                            gg::adj_smem_bytes(w, l)));
        if (n * w > nR * wR) {
          wR = w;
          nR = n;
        }
      }
      if (wR < 1 || nR < 1) continue;
      // the staged kernel wins from 2 warps per SM on (measured on
      // 16,384 x h6 over 1,000,000 rows, classes of capacity 48 / 64 / 96:
      // 226 / 66 / 4.6 ms staged at 5 / 4 / 3 warps against 292 / 90 /
      // 6.6 ms with 2 rows per lane at 10 / 8 / 6 warps)
      const bool enough = fs ? nR * wR >= 2 : nR * wR >= 6;
      if (!afn || enough) {
        afn = fn;
        rows = R;
        warps = wR;
        nb = nR;
        fast = fs;
        lay = l;
        if (enough) break;
      }
    }
    if (!afn) return fail(GGEVAL_ERR_UNSUPPORTED, "template too large for the adjoint");
    if (verbose)
      fprintf(stderr, "ggeval adjoint class %d (cap %d): %d rows per lane%s, %d warps per CTA, "
              "%d CTAs per SM\n", c, lcap, rows, fast ? " (staged)" : "", warps, nb);
    gg::AdjParams ap{};
    ap.X = ds->X;
    ap.ylo = ds->ylo;
    ap.N = (int)ds->N;
    ap.F = ds->F;
    ap.ldx = ds->ldx;
    ap.prog = ds->prog;
    ap.aux = ds->aux;
    ap.len = ds->len;
    ap.lstride = pl.lstride;
    ap.P = b->n;
    ap.stride = pl.stride;
    ap.lcap = lcap;
    ap.ecap = ecap;
    ap.slots = pl.slots;
    ap.ab = ds->ab;
    ap.mse_mode = mse_mode;
    ap.ybar = ds->ybar;
    ap.list = cls_list + (size_t)c * b->n;
    ap.count = cls_count + c;
    const long long slots = (long long)nb * ds->sms * warps;
    ap.target_items = (int)(8 * slots);
    ap.counter = cls_counter + c;
    ap.gacc = ds->gacc;
    const long long agrid = (long long)nb * ds->sms;
    GG_TRY(launch(afn, dim3((unsigned)agrid), dim3(warps * 32), gg::adj_smem_bytes(warps, lay), st,
                  &ap));
  }
  if (ev) GG_CU(cudaEventRecord(ev->second, st));
  gg::GradOutParams gp{ds->gacc, ds->len, b->n, pl.stride, dg};
  GG_TRY(launch(gg::gradout_ptr(), dim3((unsigned)((gcount + 255) / 256)), dim3(256), 0, st, &gp));
  if (host) {
    GG_CU(cudaMemcpyAsync(dcval, dg, gcount * 4, cudaMemcpyDeviceToHost, st));
    if (smse) GG_CU(cudaMemcpyAsync(smse, ds_smse, (size_t)b->n * 4, cudaMemcpyDeviceToHost, st));
  }
  return GGEVAL_OK;
}

ggeval_status ggeval_adam_step(const ggeval_batch* b, float* cval, const float* grad, float* m,
                               float* v, int32_t t, float lr, float beta1, float beta2, float eps,
                               void* stream) {
  if (!b || !cval || !grad || !m || !v) return fail(GGEVAL_ERR_ARG, "NULL argument");
  if (b->memory != GGEVAL_MEM_DEVICE) return fail(GGEVAL_ERR_ARG, "adam needs device memory");
  if (b->max_height < 0 || b->max_height > GGEVAL_MAX_HEIGHT || b->n < 0 || t < 1)
    return fail(GGEVAL_ERR_ARG, "bad batch or step");
  if (b->n == 0) return GGEVAL_OK;
  gg::AdamParams p{};
  p.op = b->op;
  p.cval = cval;
  p.grad = grad;
  p.m = m;
  p.v = v;
  p.count = (long long)b->n * stride_of(b->max_height);
  p.lr = lr;
  p.b1 = beta1;
  p.b2 = beta2;
  p.eps = eps;
  p.c1 = (float)(1.0 / (1.0 - std::pow((double)beta1, (double)t)));
  p.c2 = (float)(1.0 / (1.0 - std::pow((double)beta2, (double)t)));
  return launch(gg::adam_ptr(), dim3((unsigned)((p.count + 255) / 256)), dim3(256), 0,
                static_cast<cudaStream_t>(stream), &p);
}

ggeval_status ggeval_autotune(ggeval_dataset* ds, const ggeval_batch* b, uint32_t flags,
                              void* stream) {
  Range range("ggeval_autotune");
  GG_TRY(check_batch(ds, b));
  if (b->n == 0) return GGEVAL_OK;
  if (b->memory != GGEVAL_MEM_DEVICE) return fail(GGEVAL_ERR_ARG, "autotune needs a device batch");
  DeviceGuard guard(ds->device);
  const TuneKey tkey(b->n, b->max_height, b->layout,
                     (int)(flags & (GGEVAL_F_EXACT | GGEVAL_F_POW)));
  const char* cache = getenv("GGEVAL_TUNE_CACHE");
  if (cache && cache[0]) {  // a cached choice for this GPU, dataset and batch shape
    int taken = 0;
    GG_TRY(load_tuning(ds, cache, &taken));
    if (ds->tuned.count(tkey)) {
      drop_graph(ds);
      return GGEVAL_OK;
    }
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const Cfg base = default_cfg(ds, b->n, b->max_height, flags);
  std::vector<int> variants;
  if (base.variant == 2) variants = {2, 6};
  else if (flags & GGEVAL_F_POW) variants = {5, 1, 4, 0};
  else variants = {5, 1, 4, 0, 8, 9};  // 8, 9: the C++ interpreter
  std::vector<Cfg> cands;
  for (int v : variants)
    for (int warps : {8, 16, 20, 24, 28})
      for (int tmul : {2, 4, 8, 16})
        for (int gq : {1, 2, 4}) {  // items per SM: 16, 32, 64
          if (warps > gg::variant_max_warps(v)) continue;
          Cfg c;
          c.variant = v;
          c.warps = warps;
          c.tile_rows = 32 * gg::variant_rows(v) * tmul;
          if (c.tile_rows > 2 * ds->N + 256) continue;
          const int n_tiles = (int)((ds->N + c.tile_rows - 1) / c.tile_rows);
          const double target = 32.0 * ds->sms;
          long long ng = (long long)std::ceil(target * gq / 2 / n_tiles);
          if (ng < 1) ng = 1;
          if (ng > b->n) ng = b->n;
          c.group = (int)((b->n + ng - 1) / ng);
          cands.push_back(c);
        }
  cands.insert(cands.begin(), base);  // the default first: it sets the timing budget
  float* out = nullptr;
  GG_CU(cudaMalloc(&out, (size_t)b->n * 4));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  DevBatch db{b->op, b->cval, b->height};
  const char* env = getenv("GGEVAL_VERBOSE");
  const bool verbose = env && env[0] && env[0] != '0';
  float best_ms = 1e30f;
  Cfg best = base;
  ggeval_status result = GGEVAL_OK;
  for (const Cfg& c : cands) {
    Plan pl;
    if (make_plan(ds, b->n, b->max_height, c, &pl, has_pow(flags)) != GGEVAL_OK) continue;
    pl.fold = (flags & GGEVAL_F_NO_FOLD) == 0;
    if ((result = ensure_ws(ds, b->n, pl, false)) != GGEVAL_OK) break;
    if ((result = enqueue_eval(ds, db, b, pl, outs_of(out, nullptr, nullptr, nullptr), false,
                               st)) != GGEVAL_OK)
      break;
    const int reps = best_ms < 40.f ? 2 : 1;  // one timed run for slow batches
    cudaEventRecord(e0, st);
    for (int r = 0; r < reps; ++r)
      enqueue_eval(ds, db, b, pl, outs_of(out, nullptr, nullptr, nullptr), false, st);
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      result = fail(GGEVAL_ERR_CUDA, "autotune run failed: %s", cudaGetErrorString(cudaGetLastError()));
      break;
    }
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    ms = ms * 2 / reps;  // compare as the time of two runs
    if (verbose)
      fprintf(stderr, "ggeval autotune: variant %d tile %d group %d warps %d grid %d: %.4f ms\n",
              c.variant, c.tile_rows, c.group, c.warps, pl.grid, ms / 2);
    if (ms < best_ms) {
      best_ms = ms;
      best = c;
    }
  }
  if (verbose)
    fprintf(stderr, "ggeval autotune: chose variant %d tile %d group %d warps %d (%.4f ms)\n",
            best.variant, best.tile_rows, best.group, best.warps, best_ms / 2);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (result != GGEVAL_OK) return result;
  ds->tuned[tkey] = best;
  drop_graph(ds);
  if (cache && cache[0]) GG_TRY(append_tuning(ds, cache, tkey, best));
  return GGEVAL_OK;
}

ggeval_status ggeval_tuning_save(ggeval_dataset* ds, const char* path) {
  if (!ds || !path) return fail(GGEVAL_ERR_ARG, "NULL argument");
  FILE* f = std::fopen(path, "w");
  if (!f) return fail(GGEVAL_ERR_ARG, "cannot open %s", path);
  std::fclose(f);
  for (const auto& kv : ds->tuned) GG_TRY(append_tuning(ds, path, kv.first, kv.second));
  return GGEVAL_OK;
}

ggeval_status ggeval_tuning_load(ggeval_dataset* ds, const char* path, int32_t* n_loaded) {
  if (!ds || !path) return fail(GGEVAL_ERR_ARG, "NULL argument");
  int taken = 0;
  GG_TRY(load_tuning(ds, path, &taken));
  if (n_loaded) *n_loaded = taken;
  if (taken) drop_graph(ds);
  return GGEVAL_OK;
}

ggeval_status ggeval_tile_config(ggeval_dataset* ds, const ggeval_batch* b, uint32_t flags,
                                 const int32_t* set, int32_t* get) {
  GG_TRY(check_batch(ds, b));
  if (b->n == 0) return fail(GGEVAL_ERR_ARG, "empty batch");
  DeviceGuard guard(ds->device);
  const auto key = std::make_tuple(b->n, b->max_height, b->layout,
                                   (int)(flags & (GGEVAL_F_EXACT | GGEVAL_F_POW)));
  if (set) {
    Cfg c;
    c.variant = set[0];
    c.tile_rows = set[1];
    c.group = set[2];
    c.warps = set[3];
    if (!gg::fitness_variant(c.variant))
      return fail(GGEVAL_ERR_ARG, "variant %d is not a fitness variant", c.variant);
    Plan pl;
    GG_TRY(make_plan(ds, b->n, b->max_height, c, &pl, has_pow(flags)));
    ds->tuned[key] = c;
    drop_graph(ds);
  }
  if (get) {
    const Cfg c = pick_cfg(ds, b, flags);
    get[0] = c.variant;
    get[1] = c.tile_rows;
    get[2] = c.group;
    get[3] = c.warps;
  }
  return GGEVAL_OK;
}

ggeval_status ggeval_sync(ggeval_dataset* ds, void* stream) {
  if (!ds) return fail(GGEVAL_ERR_ARG, "dataset is NULL");
  DeviceGuard guard(ds->device);
  GG_CU(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
  GG_CU(cudaStreamSynchronize(ds->cap_stream));
  unsigned s = 0;
  GG_CU(cudaMemcpy(&s, ds->status, sizeof s, cudaMemcpyDeviceToHost));
  if (!s) return GGEVAL_OK;
  GG_CU(cudaMemset(ds->status, 0, sizeof(unsigned)));
  if (s & gg::ST_TIMEOUT) return fail(GGEVAL_ERR_TIMEOUT, "a bounded device wait gave up");
  if (s & gg::ST_CHECKED) return fail(GGEVAL_ERR_CHECKED, "a device bounds check failed");
  return fail(GGEVAL_ERR_TEMPLATE, "a trial's template is invalid (its outputs are NaN)");
}

ggeval_status ggeval_gom_donate(int32_t n, int32_t max_height, uint8_t* op, float* cval,
                                const uint8_t* pop_op, const float* pop_cval, int32_t n_pop,
                                const int32_t* donor, const int32_t* subset,
                                const int32_t* fos_offsets, const int32_t* fos_nodes,
                                int32_t n_fos, void* stream) {
  if (n < 0 || n_pop < 0 || n_fos < 0 || max_height < 0 || max_height > GGEVAL_MAX_HEIGHT)
    return fail(GGEVAL_ERR_ARG, "bad sizes");
  if (n == 0) return GGEVAL_OK;
  if (!op || !cval || !pop_op || !pop_cval || !donor || !subset || !fos_offsets ||
      (n_fos > 0 && !fos_nodes))
    return fail(GGEVAL_ERR_ARG, "NULL argument");
  gg::GomDonateParams p{n, stride_of(max_height), n_fos, n_pop, op, cval, pop_op, pop_cval,
                        donor, subset, fos_offsets, fos_nodes};
  return launch(gg::gom_donate_ptr(), dim3((unsigned)n), dim3(32), 0,
                static_cast<cudaStream_t>(stream), &p);
}

ggeval_status ggeval_gom_changed(const ggeval_batch* b, const uint8_t* backup_op,
                                 const float* backup_cval, int32_t n_features, uint8_t* changed,
                                 void* stream) {
  if (!b || !backup_op || !backup_cval || !changed) return fail(GGEVAL_ERR_ARG, "NULL argument");
  if (b->memory != GGEVAL_MEM_DEVICE) return fail(GGEVAL_ERR_ARG, "gom_changed needs device memory");
  if (b->n < 0 || b->max_height < 0 || b->max_height > GGEVAL_MAX_HEIGHT)
    return fail(GGEVAL_ERR_ARG, "bad batch");
  if (b->n == 0) return GGEVAL_OK;
  const int stride = stride_of(b->max_height);
  gg::GomChangedParams p{b->n, stride, b->max_height, b->layout, n_features, b->op, b->cval,
                         b->height, backup_op, backup_cval, changed};
  constexpr int W = 4;  // one warp per offspring
  return launch(gg::gom_changed_ptr(), dim3((unsigned)((b->n + W - 1) / W)), dim3(32 * W),
                (size_t)W * 2 * stride, static_cast<cudaStream_t>(stream), &p);
}

ggeval_status ggeval_gom_accept(int32_t n, int32_t max_height, uint8_t* op, float* cval,
                                uint8_t* backup_op, float* backup_cval, const uint8_t* changed,
                                const float* f_new, float* f_backup, uint8_t* accepted,
                                void* stream) {
  if (n < 0 || max_height < 0 || max_height > GGEVAL_MAX_HEIGHT)
    return fail(GGEVAL_ERR_ARG, "bad sizes");
  if (n == 0) return GGEVAL_OK;
  if (!op || !cval || !backup_op || !backup_cval || !f_new || !f_backup)
    return fail(GGEVAL_ERR_ARG, "NULL argument");
  gg::GomAcceptParams p{n, stride_of(max_height), op, cval, backup_op, backup_cval, changed,
                        f_new, f_backup, accepted};
  return launch(gg::gom_accept_ptr(), dim3((unsigned)n), dim3(64), 0,
                static_cast<cudaStream_t>(stream), &p);
}

ggeval_status ggeval_trial_sizes(const ggeval_batch* b, int32_t n_features, int32_t* size,
                                 void* stream) {
  if (!b || !size) return fail(GGEVAL_ERR_ARG, "NULL argument");
  if (b->memory != GGEVAL_MEM_DEVICE) return fail(GGEVAL_ERR_ARG, "trial_sizes needs device memory");
  if (b->n < 0 || b->max_height < 0 || b->max_height > GGEVAL_MAX_HEIGHT || (b->n > 0 && !b->op))
    return fail(GGEVAL_ERR_ARG, "bad batch");
  if (b->n == 0) return GGEVAL_OK;
  const int stride = stride_of(b->max_height);
  gg::TrialSizeParams p{b->n, stride, b->max_height, b->layout, n_features, b->op, b->height,
                        size};
  constexpr int W = 4;  // one warp per trial
  return launch(gg::trial_size_ptr(), dim3((unsigned)((b->n + W - 1) / W)), dim3(32 * W),
                (size_t)W * stride, static_cast<cudaStream_t>(stream), &p);
}

ggeval_status ggeval_dataset_info(const ggeval_dataset* ds, int64_t* n_rows, int32_t* n_features,
                                  double* y_mean, double* y_var) {
  if (!ds) return fail(GGEVAL_ERR_ARG, "dataset is NULL");
  const double N = (double)ds->N;
  if (n_rows) *n_rows = ds->N;
  if (n_features) *n_features = ds->F;
  if (y_mean) *y_mean = ds->ybar + ds->syc / N;
  if (y_var) *y_var = (ds->sycyc - ds->syc * ds->syc / N) / N;
  return GGEVAL_OK;
}

ggeval_status ggeval_profile_read(ggeval_dataset* ds, double* fwd_ms, int64_t* launches) {
  if (!ds || !fwd_ms || !launches) return fail(GGEVAL_ERR_ARG, "NULL argument");
  DeviceGuard guard(ds->device);
  double tot = 0;
  for (size_t i = 0; i < ds->prof_used; ++i) {
    GG_CU(cudaEventSynchronize(ds->prof_ev[i].second));
    float ms = 0;
    GG_CU(cudaEventElapsedTime(&ms, ds->prof_ev[i].first, ds->prof_ev[i].second));
    tot += ms;
  }
  *fwd_ms = tot;
  *launches = (int64_t)ds->prof_used;
  ds->prof_used = 0;
  return GGEVAL_OK;
}

// Folding structure without values: lengths and node counts of the folded
// program on the host (the device computes the folded constants).
struct ShapeFold {
  static constexpr bool on = true;
  float un(int, float) const { return 0.f; }
  float bin(int, float, float) const { return 0.f; }
};

ggeval_status ggeval_batch_stats(const ggeval_batch* b, int32_t n_features, int64_t* out) {
  if (!b || !out) return fail(GGEVAL_ERR_ARG, "NULL argument");
  if (b->memory != GGEVAL_MEM_HOST) return fail(GGEVAL_ERR_ARG, "batch_stats needs a host batch");
  if (b->n < 0 || b->max_height < 0 || b->max_height > GGEVAL_MAX_HEIGHT)
    return fail(GGEVAL_ERR_ARG, "bad batch");
  if (b->n > 0 && (!b->op || !b->cval)) return fail(GGEVAL_ERR_ARG, "op or cval is NULL");
  const int stride = stride_of(b->max_height);
  std::vector<uint32_t> w(stride + 1);
  std::vector<float> c(stride + 1), fv(stride);
  std::vector<uint8_t> d1(stride), nd(stride);
  for (int t = 0; t < b->n; ++t) {
    const int h = b->height ? b->height[t] : b->max_height;
    int64_t* o = out + (size_t)t * GGEVAL_NSTAT;
    for (int i = 0; i < GGEVAL_NSTAT; ++i) o[i] = 0;
    if (h < 0 || h > b->max_height) {
      o[0] = -1;
      continue;
    }
    const uint8_t* op = b->op + (size_t)t * stride;
    const float* cv = b->cval + (size_t)t * stride;
    const gg::PackResult r = gg::pack_tree(op, cv, h, b->layout, n_features, gg::MAX_SLOTS,
                                           w.data(), c.data(), 1, nullptr, stride, d1.data(),
                                           nd.data());
    if (r.status) {
      o[0] = -1;
      continue;
    }
    // the folded program's structure (its constants are not computed here)
    const gg::PackResult f = gg::pack_tree(op, cv, h, b->layout, n_features, gg::MAX_SLOTS,
                                           w.data(), c.data(), 1, nullptr, stride, d1.data(),
                                           nd.data(), true, ShapeFold(), fv.data());
    for (int i = 0; i < 10; ++i) o[i] = r.counts[i];
    o[10] = r.len;
    o[11] = r.slots;
    o[12] = r.counts[10];
    for (int i = 0; i < 11; ++i) o[13 + i] = f.exec[i];
    o[24] = f.len;
  }
  return GGEVAL_OK;
}

ggeval_status ggeval_pack_device(ggeval_dataset* ds, const ggeval_batch* b, uint32_t flags,
                                 uint32_t* words, float* consts, int32_t* len, int32_t cap,
                                 void* stream) {
  GG_TRY(check_batch(ds, b));
  if (b->memory != GGEVAL_MEM_DEVICE) return fail(GGEVAL_ERR_ARG, "pack_device needs a device batch");
  if (b->n == 0) return GGEVAL_OK;
  if (!words || !consts || !len || cap < 1) return fail(GGEVAL_ERR_ARG, "NULL output or cap < 1");
  DeviceGuard guard(ds->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Plan pl;
  GG_TRY(make_plan(ds, b->n, b->max_height, default_cfg(ds, b->n, b->max_height, flags), &pl,
                   has_pow(flags)));
  pl.fold = (flags & GGEVAL_F_NO_FOLD) == 0;
  GG_TRY(ensure_ws(ds, b->n, pl, false));
  DevBatch db{b->op, b->cval, b->height};
  GG_TRY(enqueue_pack(ds, db, b->n, b->max_height, b->layout, pl, false, st));
  std::vector<uint2> prog((size_t)b->n * pl.lstride);
  std::vector<int> ln(b->n);
  GG_CU(cudaMemcpyAsync(prog.data(), ds->prog, prog.size() * sizeof(uint2), cudaMemcpyDeviceToHost,
                        st));
  GG_CU(cudaMemcpyAsync(ln.data(), ds->len, ln.size() * sizeof(int), cudaMemcpyDeviceToHost, st));
  GG_CU(cudaStreamSynchronize(st));
  for (int t = 0; t < b->n; ++t) {
    len[t] = ln[t];
    for (int k = 0; k < ln[t] && k < cap; ++k) {
      const uint2 w = prog[(size_t)t * pl.lstride + k];
      words[(size_t)t * cap + k] = w.x;
      std::memcpy(&consts[(size_t)t * cap + k], &w.y, 4);
    }
  }
  return GGEVAL_OK;
}

ggeval_status ggeval_pack_host(const ggeval_batch* b, int32_t index, int32_t n_features,
                               uint32_t* words, float* consts, int32_t* tpos, int32_t cap,
                               int32_t* len) {
  if (!b || !words || !consts || !len) return fail(GGEVAL_ERR_ARG, "NULL argument");
  if (b->memory != GGEVAL_MEM_HOST) return fail(GGEVAL_ERR_ARG, "pack_host needs a host batch");
  if (index < 0 || index >= b->n) return fail(GGEVAL_ERR_ARG, "index out of range");
  if (b->max_height < 0 || b->max_height > GGEVAL_MAX_HEIGHT)
    return fail(GGEVAL_ERR_UNSUPPORTED, "max_height out of range");
  const int stride = stride_of(b->max_height);
  if (cap < stride) return fail(GGEVAL_ERR_ARG, "cap %d < %d", cap, stride);
  const int h = b->height ? b->height[index] : b->max_height;
  if (h < 0 || h > b->max_height) return fail(GGEVAL_ERR_TEMPLATE, "height out of range");
  std::vector<uint32_t> w(stride + 1);
  std::vector<float> c(stride + 1);
  std::vector<gg::Aux> ax(stride + 1);
  std::vector<uint8_t> d1(stride), nd(stride);
  const gg::PackResult r =
      gg::pack_tree(b->op + (size_t)index * stride, b->cval + (size_t)index * stride, h, b->layout,
                    n_features, gg::MAX_SLOTS, w.data(), c.data(), 1, ax.data(), stride,
                    d1.data(), nd.data());
  if (r.status) return fail(GGEVAL_ERR_TEMPLATE, "trial %d: invalid template", index);
  for (int k = 0; k < r.len; ++k) {
    words[k] = w[k];
    consts[k] = c[k];
    if (tpos) tpos[k] = ax[k].tpos;
  }
  *len = r.len;
  return GGEVAL_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// ggeval_eval_batch_noalloc: the batched evaluation with its scratch (packed
// programs, instruction counts, per-tile partial sums, work counter) in one
// file-scope device array instead of the dataset's growable workspace.
namespace {
constexpr size_t NA_PROG_BYTES =
    (size_t)GGEVAL_NOALLOC_MAX_TRIALS * ((1u << (GGEVAL_NOALLOC_MAX_HEIGHT + 1)) * 8u);
constexpr size_t NA_LEN_OFF = NA_PROG_BYTES;
constexpr size_t NA_PART_OFF = NA_LEN_OFF + (size_t)GGEVAL_NOALLOC_MAX_TRIALS * 4u;
constexpr size_t NA_CNT_OFF =
    NA_PART_OFF + (size_t)GGEVAL_NOALLOC_MAX_TRIALS * GGEVAL_NOALLOC_MAX_TILES * gg::NPART * 4u;
constexpr size_t NA_BYTES = NA_CNT_OFF + 256u;
static_assert(NA_BYTES == GGEVAL_NOALLOC_SCRATCH_BYTES, "scratch size mismatch");
static_assert(NA_LEN_OFF % 256 == 0 && NA_PART_OFF % 256 == 0 && NA_CNT_OFF % 256 == 0,
              "scratch sub-arrays must stay aligned");
}  // namespace

// The scratch itself.  In host code this name is only a host-side stand-in
// for the device array: its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

namespace {
// Device address of g_noalloc_scratch on `device` (current).  Outside a
// stream capture every call looks it up again, so the address of a context
// created after a device reset is the one used; during a capture the
// address from the device's last call outside a capture is used.
ggeval_status noalloc_scratch(int device, cudaStream_t st, unsigned char** out) {
  static std::mutex mu;
  static std::map<int, unsigned char*> addr;
  std::lock_guard<std::mutex> lock(mu);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) cs = cudaStreamCaptureStatusActive;
  if (cs != cudaStreamCaptureStatusNone) {
    auto it = addr.find(device);
    if (it == addr.end())
      return fail(GGEVAL_ERR_ARG,
                  "eval_batch_noalloc: the first call on device %d must come before any "
                  "stream capture", device);
    *out = it->second;
    return GGEVAL_OK;
  }
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p)
    return fail(GGEVAL_ERR_CUDA, "cudaGetSymbolAddress(noalloc scratch): %s",
                cudaGetErrorString(e));
  addr[device] = static_cast<unsigned char*>(p);
  *out = static_cast<unsigned char*>(p);
  return GGEVAL_OK;
}
}  // namespace

extern "C" ggeval_status ggeval_eval_batch_noalloc(ggeval_dataset* ds, const ggeval_batch* b,
                                                   float* smse, float* a, float* bb, float* mse,
                                                   void* stream) {
  GG_TRY(check_batch(ds, b));
  if (b->memory != GGEVAL_MEM_DEVICE)
    return fail(GGEVAL_ERR_ARG, "eval_batch_noalloc needs a device batch");
  if (b->n > GGEVAL_NOALLOC_MAX_TRIALS)
    return fail(GGEVAL_ERR_UNSUPPORTED, "eval_batch_noalloc: %d trials > the static limit %d",
                b->n, GGEVAL_NOALLOC_MAX_TRIALS);
  if (b->max_height > GGEVAL_NOALLOC_MAX_HEIGHT)
    return fail(GGEVAL_ERR_UNSUPPORTED, "eval_batch_noalloc: max_height %d > the static limit %d",
                b->max_height, GGEVAL_NOALLOC_MAX_HEIGHT);
  if (b->n == 0) return GGEVAL_OK;
  if (!smse) return fail(GGEVAL_ERR_ARG, "smse is NULL");
  DeviceGuard guard(ds->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  unsigned char* base = nullptr;
  GG_TRY(noalloc_scratch(ds->device, st, &base));
  Cfg c = default_cfg(ds, b->n, b->max_height, 0);
  if ((ds->N + c.tile_rows - 1) / c.tile_rows > GGEVAL_NOALLOC_MAX_TILES) {
    while ((ds->N + c.tile_rows - 1) / c.tile_rows > GGEVAL_NOALLOC_MAX_TILES) c.tile_rows *= 2;
    c.group = group_for(ds, b->n, c.warps, c.tile_rows);  // for the wider tiles
  }
  Plan pl;
  if (make_plan(ds, b->n, b->max_height, c, &pl, false) != GGEVAL_OK)
    return fail(GGEVAL_ERR_UNSUPPORTED,
                "eval_batch_noalloc: %lld rows need tiles of %d rows, which do not fit in "
                "shared memory (at most %d tiles)",
                (long long)ds->N, c.tile_rows, GGEVAL_NOALLOC_MAX_TILES);
  uint2* prog = reinterpret_cast<uint2*>(base);
  int* len = reinterpret_cast<int*>(base + NA_LEN_OFF);
  float* part = reinterpret_cast<float*>(base + NA_PART_OFF);
  int* counter = reinterpret_cast<int*>(base + NA_CNT_OFF);
  gg::PackParams pp{};
  pp.op = b->op;
  pp.cval = b->cval;
  pp.height = b->height;
  pp.n = b->n;
  pp.h_max = b->max_height;
  pp.stride = pl.stride;
  pp.layout = b->layout;
  pp.n_features = ds->F;
  pp.max_slots = pl.slots;
  pp.lstride = pl.lstride;
  pp.prog = prog;
  pp.aux = nullptr;
  pp.len = len;
  pp.status = ds->status;
  pp.fold = 1;
  GG_TRY(launch(gg::pack_ptr(), dim3((b->n + gg::PACK_WARPS - 1) / gg::PACK_WARPS),
                dim3(32 * gg::PACK_WARPS), gg::PACK_WARPS * gg::pack_warp_bytes(pl.stride),
                st, &pp));
  GG_CU(cudaMemsetAsync(counter, 0, sizeof(int), st));
  gg::FwdParams fp = fwd_params(ds, b->n, pl);
  fp.prog = prog;
  fp.len = len;
  fp.part = part;
  fp.counter = counter;
  GG_TRY(launch(pl.fn, dim3(pl.grid), dim3(pl.cfg.warps * 32), pl.smem, st, &fp));
  gg::FinParams q = fin_params(ds, b->n, pl, smse, a, bb, mse);
  q.part = part;
  q.len = len;
  q.ab = nullptr;
  GG_TRY(launch(gg::fin_ptr(), dim3((b->n + gg::FIN_WARPS - 1) / gg::FIN_WARPS),
                dim3(32 * gg::FIN_WARPS), 0, st, &q));
  return GGEVAL_OK;
}
