// lof_api.cu -- host side of the C ABI declared in include/lof.h.
//
// A context owns the history rings (Section 4.1: one ring of binary64 means
// per channel slot) and the scratch of the persistent kernel.  lof_flag_block
// validates the unit descriptors, splits every unit into items (runs of whole
// rows that fit one CTA's shared-memory tile), uploads the descriptor tables
// and launches ONE cooperative kernel for the whole block.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "lof.h"
#include "lof_internal.h"

using lofk::DevUnit;
using lofk::Task;
using lofk::KParams;
using lofk::UnitState;

namespace {

thread_local char g_create_error[512];

constexpr int kStageRing = 4;
constexpr int kHostChunks = 16;  // pipeline depth of lof_flag_block_host

int esize_of(int dtype) {
  switch (dtype) {
    case LOF_CI8: return 2;
    case LOF_CI16: return 4;
    case LOF_F32: return 4;
    case LOF_CF32: return 8;
    default: return 0;
  }
}
// the float path (one CTA per unit): Stokes I power or complex visibilities
bool is_float(int dtype) { return dtype == LOF_F32 || dtype == LOF_CF32; }
int64_t round_up64(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

}  // namespace

// lof_f32.cu, lof_sir.cu, lof_integ.cu
extern "C" int lofk_launch_f32x(const lofk::KParams* kp, int n_units, int n_sm, int smem_bytes,
                                void* stream, int cplx);
extern "C" int lofk_sir_max_time();
extern "C" int lofk_integ_max_time();
extern "C" int lofk_launch_integ(int dtype, const lofk::KParams* kp, int n_units, int n_sm, void* stream,
                                 int mode, int cell_chan, int cell_time);
extern "C" int lofk_launch_sir(const lofk::DevUnit* units, int n_units, int64_t n_chan, int max_chan,
                               int max_time, int percent, int es, void* stream);

struct lof_ctx {
  int device = 0;
  lof_params params{};
  int n_sm = 0;
  int smem_per_sm = 0, smem_optin = 0;
  lof_tuning tuning = lofk::default_tuning();
  // history
  int64_t n_slots = 0;
  int H = 0;
  lofk::HistoryDev hist{};
  // scratch
  DevUnit* d_units = nullptr;
  size_t cap_units = 0;
  Task* d_tasks = nullptr;
  size_t cap_tasks = 0;
  UnitState* d_ustate = nullptr;
  size_t cap_ustate = 0;
  unsigned long long* d_chanS = nullptr;
  uint8_t* d_chanFc = nullptr;
  size_t cap_chan = 0, cap_chanfc = 0;
  uint32_t* d_gen = nullptr;  // general time-pass rows (per CTA)
  size_t cap_gen = 0;
  int* d_ctrl = nullptr;  // [0] queue, [1] error, [2..3] error detail, [4..5] counters
  int* h_err = nullptr;   // pinned copy of d_ctrl[1..3]
  cudaEvent_t ev_err = nullptr;
  bool err_copy_pending = false;
  // descriptor staging (pinned, ring of buffers guarded by events)
  void* h_stage[kStageRing] = {};
  size_t cap_stage[kStageRing] = {};
  cudaEvent_t ev_stage[kStageRing] = {};
  int stage_next = 0;
  // device staging for lof_flag_block_host, its two copy streams and the
  // events that chain them with the caller's stream (created on first use)
  uint8_t* d_io = nullptr;
  size_t cap_io = 0;
  cudaStream_t s_up = nullptr, s_down = nullptr;
  cudaEvent_t ev_start = nullptr, ev_down_done = nullptr;
  cudaEvent_t ev_in[kHostChunks] = {}, ev_flag[kHostChunks] = {};
  std::string last_error;
};

namespace {

int fail(lof_ctx* c, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->last_error = buf;
  else snprintf(g_create_error, sizeof g_create_error, "%s", buf);
  return code;
}

int cuda_fail(lof_ctx* c, cudaError_t e, const char* what) {
  return fail(c, LOF_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    else prev = -1;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

template <class T>
int grow(lof_ctx* c, T** p, size_t* cap, size_t need, const char* what) {
  if (need <= *cap && *p) return LOF_OK;
  size_t n = std::max<size_t>(need, *cap ? *cap * 2 : 64);
  if (*p) {
    cudaError_t e = cudaDeviceSynchronize();  // scratch may still be in use
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaDeviceSynchronize");
    cudaFree(*p);
    *p = nullptr;
    *cap = 0;
  }
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), n * sizeof(T));
  if (e != cudaSuccess) return fail(c, LOF_ERR_NOMEM, "cudaMalloc(%s, %zu): %s", what, n * sizeof(T), cudaGetErrorString(e));
  *cap = n;
  return LOF_OK;
}

int pending_device_error(lof_ctx* c) {
  if (!c->err_copy_pending) return LOF_OK;
  if (cudaEventQuery(c->ev_err) != cudaSuccess) return LOF_OK;  // not known yet
  c->err_copy_pending = false;
  const int code = c->h_err[0];
  if (code == lofk::kErrNone) return LOF_OK;
  const int info0 = c->h_err[1], info1 = c->h_err[2];
  c->h_err[0] = 0;
  cudaMemset(c->d_ctrl + 1, 0, 3 * sizeof(int));
  if (code == lofk::kErrTimeout)
    return fail(c, LOF_ERR_TIMEOUT, "device wait timed out (round %d, block %d)", info0, info1);
  return fail(c, LOF_ERR_STATE, "device error %d (detail %d, block %d)", code, info0, info1);
}

int static_smem_bytes(int dtype, int threads) {
  // conservative bound of the kernel's static shared memory (Fixed<NT> + locals)
  (void)dtype;
  return 7 * 1024 + (threads / 32) * 32;
}

// words of the time-pass buffer per row: padded chunk-local prefixes of
// nch + 3 chunks (36 words each), chunk bases and chunk totals
int pfx_row_words(int dtype, int T) {
  (void)dtype;
  const int nch = (T + 31) / 32;
  return ((nch + 3) * 36 + 2 * (nch + 4) + 3) & ~3;  // 16-byte aligned rows
}


// Budget of dynamic shared memory per CTA (at most as many resident CTAs as
// the kernel's launch bounds allow: 4 of 128 threads, 2 of 256).
int dyn_budget(const lofk::HostCfg& h, int dtype, int threads, int ctas) {
  ctas = std::min(ctas, threads >= 256 ? 2 : 4);
  const int per = h.smem_per_sm / std::max(1, ctas) - 1024;
  return std::min(per, h.smem_optin) - static_smem_bytes(dtype, threads);
}


}  // namespace

extern "C" void lof_default_params(lof_params* p) {
  if (!p) return;
  p->p = 1.5;
  p->sensitivity = 1.0;
  p->start_threshold = 6.0;
  p->max_window = 64;
  p->history_len = 60;
  p->history_min = 8;
  p->history_k = 6.0;
  p->sigma_estimator = LOF_SIGMA_MAD;
  p->enable_freq = 1;
  p->enable_time = 1;
  p->enable_history = 1;
  p->sir_percent = 0;
  p->time_mode = LOF_TIME_PER_CHANNEL;
  p->stats_scope = LOF_SCOPE_POOLED;
  p->integ_chan = 1;
  p->integ_time = 1;
}

extern "C" const char* lof_last_error(const lof_ctx* c) {
  return c ? c->last_error.c_str() : g_create_error;
}

namespace lofk {

lof_tuning default_tuning() {
  return lof_tuning{256, 2, 0, 2048, 64, 262144,
                    LOF_SCHED_SET | LOF_SCHED_PACKED | LOF_SCHED_BOUND64 | LOF_SCHED_COALESCED |
                        LOF_SCHED_VALUE_WINDOW};
}

// Checks every field of a parameter set (shared by lof_create and the
// allocation-free entry point); 1 = valid, else 0 with the reason in *why.
int validate_params(const lof_params* p, char* why, int nwhy) {
  if (!(p->p > 0.0) || !(p->sensitivity > 0.0) || !(p->start_threshold > 0.0)) {
    snprintf(why, nwhy, "%s", "p, sensitivity and start_threshold must be positive");
    return 0;
  }
  if (p->max_window < 1 || p->max_window > 64 || (p->max_window & (p->max_window - 1))) {
    snprintf(why, nwhy, "max_window %d must be a power of two in [1, 64]", p->max_window);
    return 0;
  }
  if (p->history_len < 1 || p->history_len > 1024 || p->history_min < 0 || !(p->history_k >= 0.0)) {
    snprintf(why, nwhy, "%s", "history_len in [1, 1024], history_min >= 0, history_k >= 0 required");
    return 0;
  }
  if (p->sigma_estimator != LOF_SIGMA_MAD && p->sigma_estimator != LOF_SIGMA_STD &&
      p->sigma_estimator != LOF_SIGMA_WINSOR) {
    snprintf(why, nwhy, "%s", "unknown sigma_estimator");
    return 0;
  }
  if (p->sir_percent < 0 || p->sir_percent > 99) {
    snprintf(why, nwhy, "%s", "sir_percent in [0, 99] required");
    return 0;
  }
  if (p->time_mode != LOF_TIME_PER_CHANNEL && p->time_mode != LOF_TIME_INTEGRATED &&
      p->time_mode != LOF_TIME_2D) {
    snprintf(why, nwhy, "%s", "unknown time_mode");
    return 0;
  }
  if (p->stats_scope != LOF_SCOPE_POOLED && p->stats_scope != LOF_SCOPE_CHANNEL) {
    snprintf(why, nwhy, "%s", "unknown stats_scope");
    return 0;
  }
  if (p->stats_scope == LOF_SCOPE_CHANNEL && p->time_mode != LOF_TIME_PER_CHANNEL) {
    snprintf(why, nwhy, "%s", "stats_scope LOF_SCOPE_CHANNEL needs time_mode LOF_TIME_PER_CHANNEL");
    return 0;
  }
  if (p->integ_chan < 1 || p->integ_time < 1 ||
      static_cast<int64_t>(p->integ_chan) * p->integ_time > 65536) {
    snprintf(why, nwhy, "%s", "integ_chan, integ_time >= 1 with integ_chan * integ_time <= 65536 required");
    return 0;
  }
  return 1;
}

}  // namespace lofk

extern "C" int lof_create(const lof_params* params, int cuda_device, int64_t n_history_slots,
                          lof_ctx** out) {
  if (!out) return fail(nullptr, LOF_ERR_INVALID, "lof_create: out is NULL");
  *out = nullptr;
  lof_params p;
  if (params) p = *params;
  else lof_default_params(&p);
  char why[256];
  if (!lofk::validate_params(&p, why, sizeof why)) return fail(nullptr, LOF_ERR_INVALID, "lof_create: %s", why);
  if (n_history_slots < 0) return fail(nullptr, LOF_ERR_INVALID, "lof_create: negative history slots");
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || ndev == 0)
    return fail(nullptr, LOF_ERR_CUDA, "lof_create: no CUDA device (%s)", cudaGetErrorString(e));
  if (cuda_device < 0 || cuda_device >= ndev)
    return fail(nullptr, LOF_ERR_INVALID, "lof_create: device %d of %d", cuda_device, ndev);
  DeviceGuard g(cuda_device);
  e = cudaSetDevice(cuda_device);
  if (e != cudaSuccess) return fail(nullptr, LOF_ERR_CUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
  lof_ctx* c = new lof_ctx();
  c->device = cuda_device;
  c->params = p;
  cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, cuda_device);
  cudaDeviceGetAttribute(&c->smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, cuda_device);
  cudaDeviceGetAttribute(&c->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, cuda_device);
  int rc = LOF_OK;
  auto ck = [&](cudaError_t err, const char* what) {
    if (err != cudaSuccess && rc == LOF_OK) rc = fail(nullptr, LOF_ERR_NOMEM, "%s: %s", what, cudaGetErrorString(err));
  };
  c->n_slots = n_history_slots;
  c->H = p.history_len;
  const size_t ns = static_cast<size_t>(std::max<int64_t>(1, n_history_slots));
  ck(cudaMalloc(&c->hist.vals, ns * c->H * sizeof(double)), "history ring");
  ck(cudaMalloc(&c->hist.count, ns * sizeof(int32_t)), "history count");
  ck(cudaMalloc(&c->hist.head, ns * sizeof(int32_t)), "history head");
  ck(cudaMalloc(&c->hist.thr, ns * sizeof(double)), "history threshold");
  ck(cudaMalloc(&c->hist.pend, ns * sizeof(double)), "history pending");
  ck(cudaMalloc(&c->hist.pend_flag, ns), "history pending flag");
  ck(cudaMalloc(&c->hist.pend_seq, ns * sizeof(uint64_t)), "history pending seq");
  ck(cudaMalloc(&c->hist.hint, ns * 2 * sizeof(unsigned long long)), "statistics hints");
  ck(cudaMalloc(&c->d_ctrl, lofk::kCtrlWords * sizeof(int)), "control words");
  ck(cudaHostAlloc(&c->h_err, 4 * sizeof(int), cudaHostAllocDefault), "pinned error word");
  ck(cudaEventCreateWithFlags(&c->ev_err, cudaEventDisableTiming), "event");
  for (int i = 0; i < kStageRing; ++i)
    ck(cudaEventCreateWithFlags(&c->ev_stage[i], cudaEventDisableTiming), "event");
  if (rc == LOF_OK) {
    ck(cudaMemset(c->hist.vals, 0, ns * c->H * sizeof(double)), "memset");
    ck(cudaMemset(c->hist.count, 0, ns * sizeof(int32_t)), "memset");
    ck(cudaMemset(c->hist.head, 0, ns * sizeof(int32_t)), "memset");
    ck(cudaMemset(c->hist.thr, 0, ns * sizeof(double)), "memset");
    ck(cudaMemset(c->hist.pend_flag, 0, ns), "memset");
    ck(cudaMemset(c->hist.hint, 0xFF, ns * 2 * sizeof(unsigned long long)), "memset");
    ck(cudaMemset(c->d_ctrl, 0, lofk::kCtrlWords * sizeof(int)), "memset");
    ck(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
    memset(c->h_err, 0, 4 * sizeof(int));
  }
  c->hist.n_slots = n_history_slots;
  c->hist.H = c->H;
  if (rc != LOF_OK) {
    lof_destroy(c);
    return rc;
  }
  *out = c;
  return LOF_OK;
}

extern "C" int lof_destroy(lof_ctx* c) {
  if (!c) return LOF_OK;
  DeviceGuard g(c->device);
  cudaDeviceSynchronize();
  cudaFree(c->hist.vals);
  cudaFree(c->hist.count);
  cudaFree(c->hist.head);
  cudaFree(c->hist.thr);
  cudaFree(c->hist.pend);
  cudaFree(c->hist.pend_flag);
  cudaFree(c->hist.pend_seq);
  cudaFree(c->hist.hint);
  cudaFree(c->d_units);
  cudaFree(c->d_tasks);
  cudaFree(c->d_ustate);
  cudaFree(c->d_chanS);
  cudaFree(c->d_chanFc);
  cudaFree(c->d_gen);
  cudaFree(c->d_ctrl);
  cudaFree(c->d_io);
  if (c->s_up) cudaStreamDestroy(c->s_up);
  if (c->s_down) cudaStreamDestroy(c->s_down);
  if (c->ev_start) cudaEventDestroy(c->ev_start);
  if (c->ev_down_done) cudaEventDestroy(c->ev_down_done);
  for (int i = 0; i < kHostChunks; ++i) {
    if (c->ev_in[i]) cudaEventDestroy(c->ev_in[i]);
    if (c->ev_flag[i]) cudaEventDestroy(c->ev_flag[i]);
  }
  if (c->h_err) cudaFreeHost(c->h_err);
  for (int i = 0; i < kStageRing; ++i) {
    if (c->h_stage[i]) cudaFreeHost(c->h_stage[i]);
    if (c->ev_stage[i]) cudaEventDestroy(c->ev_stage[i]);
  }
  if (c->ev_err) cudaEventDestroy(c->ev_err);
  delete c;
  return LOF_OK;
}

extern "C" int lof_set_tuning(lof_ctx* c, const lof_tuning* t) {
  if (!c || !t) return fail(c, LOF_ERR_INVALID, "lof_set_tuning: NULL argument");
  lof_tuning n = c->tuning;
  if (t->threads) {
    if (t->threads != 128 && t->threads != 256)
      return fail(c, LOF_ERR_INVALID, "threads must be 128 or 256");
    n.threads = t->threads;
  }
  if (t->ctas_per_sm) {
    if (t->ctas_per_sm < 1 || t->ctas_per_sm > 4) return fail(c, LOF_ERR_INVALID, "ctas_per_sm in [1, 4]");
    n.ctas_per_sm = t->ctas_per_sm;
  }
  if (t->tile_bytes) {
    if (t->tile_bytes < 4096 || (t->tile_bytes % 128)) return fail(c, LOF_ERR_INVALID, "tile_bytes >= 4096, multiple of 128");
    n.tile_bytes = t->tile_bytes;
  }
  if (t->flag_rows) {
    if (t->flag_rows < 1 || t->flag_rows > lofk::kMaxRowsPerTask)
      return fail(c, LOF_ERR_INVALID, "flag_rows in [1, %d]", lofk::kMaxRowsPerTask);
    n.flag_rows = t->flag_rows;
  }
  if (t->stat_samples) {
    if (t->stat_samples < 1024) return fail(c, LOF_ERR_INVALID, "stat_samples >= 1024");
    n.stat_samples = t->stat_samples;
  }
  if (t->schedule) {
    if (!(t->schedule & LOF_SCHED_SET) ||
        (t->schedule & ~(LOF_SCHED_SET | LOF_SCHED_PACKED | LOF_SCHED_BOUND64 | LOF_SCHED_COALESCED |
                         LOF_SCHED_VALUE_WINDOW | LOF_SCHED_F32_CLUSTER)))
      return fail(c, LOF_ERR_INVALID, "schedule: LOF_SCHED_SET plus LOF_SCHED_* flags");
    n.schedule = t->schedule;
  }
  if (t->fine_bins) {
    if (t->fine_bins < 64 || t->fine_bins > lofk::kMaxFine)
      return fail(c, LOF_ERR_INVALID, "fine_bins in [64, %d]", lofk::kMaxFine);
    n.fine_bins = t->fine_bins;
  }
  c->tuning = n;
  return LOF_OK;
}

extern "C" int lof_get_tuning(const lof_ctx* c, lof_tuning* t) {
  if (!c || !t) return LOF_ERR_INVALID;
  *t = c->tuning;
  return LOF_OK;
}

namespace {

// Rows of one flag task: four per warp, fewer if the shared memory cannot
// hold their flag words and the warps' staging buffers of the time pass (two
// per warp, 32 rows of 32 samples + 16 bytes).
int flag_words_row(int T) { return (T + 31) / 32 + 4; }
int stage_bytes(int dtype, int threads) {
  const int es = dtype == LOF_CI8 ? 2 : 4;
  return (threads / 32) * 2 * 32 * (32 * es + 16);
}
int flag_bytes(int dtype, int T, int R, int threads) {
  return ((4 * R * flag_words_row(T) + 15) & ~15) + stage_bytes(dtype, threads);
}
int flag_rows(int dtype, int T, int budget_bytes, int threads, int cap = 0) {
  int R = std::min(lofk::kMaxRowsPerTask, cap > 0 ? cap : 4 * (threads / 32));
  while (R > 0 && flag_bytes(dtype, T, R, threads) > budget_bytes) --R;
  return R;
}

// Rows of one stats / fine task (streamed, ~64K samples per task).
int stat_rows(int T, int samples = 0) {
  return std::max(1, std::min(lofk::kMaxRowsPerTask, (samples > 0 ? samples : 65536) / std::max(1, T)));
}

// Shared-memory plan: the unit-wide workspace, the flag words of a flag
// task and as many rows of the general path as the budget allows.
bool make_plan(const lofk::HostCfg& h, int dtype, const int* Ts, int nT, lofk::Plan* pl,
               char* why, int nwhy) {
  pl->threads = h.tuning.threads;
  pl->ctas = h.tuning.ctas_per_sm;
  int budget = dyn_budget(h, dtype, pl->threads, pl->ctas);
  if (h.tuning.tile_bytes) budget = std::min(budget, h.tuning.tile_bytes);
  int need = lofk::kWorkspaceBytes, want = lofk::kWorkspaceBytes;
  for (int i = 0; i < nT; ++i) {
    const int R = flag_rows(dtype, Ts[i], budget, pl->threads, h.tuning.flag_rows);
    if (R < 1) {
      snprintf(why, nwhy, "n_time %d does not fit the shared-memory budget (%d bytes)", Ts[i], budget);
      return false;
    }
    need = std::max(need, flag_bytes(dtype, Ts[i], R, pl->threads));
    want = std::max(want, flag_bytes(dtype, Ts[i], R, pl->threads));
  }
  if (need > budget) {
    snprintf(why, nwhy, "the workspace (%d bytes) exceeds the shared-memory budget (%d)", need, budget);
    return false;
  }
  pl->smem = std::min(budget, want) & ~127;
  if (pl->smem < need) pl->smem = need;
  return true;
}

}  // namespace

namespace lofk {

int host_count_tasks(const HostCfg& h, int dtype, const lof_unit* units, int n_units,
                     int* n_tasks, char* why, int nwhy) {
  if (is_float(dtype)) {  // one CTA per unit, no task queue
    for (int i = 0; i < n_units; ++i)
      if (lofk_f32_smem(units[i].n_time) > h.smem_optin) {
        snprintf(why, nwhy, "n_time %d does not fit the shared-memory budget", units[i].n_time);
        return LOF_ERR_INVALID;
      }
    *n_tasks = 0;
    return LOF_OK;
  }
  int budget = dyn_budget(h, dtype, h.tuning.threads, h.tuning.ctas_per_sm);
  if (h.tuning.tile_bytes) budget = std::min(budget, h.tuning.tile_bytes);
  int64_t n = 0;
  for (int i = 0; i < n_units; ++i) {
    const int T = units[i].n_time, C = units[i].n_chan;
    const int Rc = flag_rows(dtype, T, budget, h.tuning.threads, h.tuning.flag_rows);
    if (Rc < 1) {
      snprintf(why, nwhy, "n_time %d does not fit the shared-memory budget (%d bytes)", T, budget);
      return LOF_ERR_INVALID;
    }
    const int Rs = stat_rows(T, h.tuning.stat_samples);
    n += (C + Rs - 1) / Rs + (C + Rc - 1) / Rc;
  }
  // room for the split queue tails (host_prepare): three more tasks for each
  // of up to one task per CTA in each of the two queues
  n += 6 * int64_t(h.n_sm) * std::max(1, h.tuning.ctas_per_sm);
  if (n > (int64_t(1) << 30)) {
    snprintf(why, nwhy, "too many tasks");
    return LOF_ERR_INVALID;
  }
  *n_tasks = static_cast<int>(n);
  return LOF_OK;
}

// Unit descriptors of a float32 block (one CTA per unit, no tasks).
int host_prepare_f32(const HostCfg& h, const lof_unit* units, int n_units, DevUnit* du, Prep* out) {
  int maxT = 1;
  out->max_C = 1;
  int64_t chan = 0;
  for (int i = 0; i < n_units; ++i) {
    const lof_unit& u = units[i];
    DevUnit& d = du[i];
    d = DevUnit{};
    d.in = u.in;
    d.out = u.out;
    d.mask = u.mask;
    d.stats = u.stats;
    d.in_stride = u.in_row_stride;
    d.out_stride = u.out ? u.out_row_stride : 0;
    d.mask_stride = u.mask ? u.mask_row_stride : 0;
    d.hist_slot = u.history_slot;
    d.C = u.n_chan;
    d.T = u.n_time;
    d.chan_off = static_cast<int32_t>(chan);
    chan += u.n_chan;
    int flags = 0;
    if ((reinterpret_cast<uintptr_t>(u.in) % 16) == 0 && ((u.in_row_stride * 4) % 16) == 0)
      flags |= kUnitInVec;
    if (u.out && u.out == u.in) flags |= kUnitInPlace;
    else if (u.out && (reinterpret_cast<uintptr_t>(u.out) % 16) == 0 && ((u.out_row_stride * 4) % 16) == 0)
      flags |= kUnitOutVec;
    if (u.mask && (reinterpret_cast<uintptr_t>(u.mask) % 16) == 0 && (u.mask_row_stride % 16) == 0)
      flags |= kUnitMaskVec;
    d.flags = flags;
    maxT = std::max(maxT, u.n_time);
    out->max_C = std::max(out->max_C, u.n_chan);
  }
  out->max_T = maxT;
  out->plan = Plan{256, 1, lofk_f32_smem(maxT)};
  out->n_tasks = 0;
  out->n_chan = chan;
  out->grid = std::min(n_units, h.n_sm * 4);
  return LOF_OK;
}

int host_prepare(const HostCfg& h, int dtype, const lof_unit* units, int n_units, DevUnit* du,
                 Task* tasks, int max_tasks, Prep* out, char* why, int nwhy) {
  if (is_float(dtype)) return host_prepare_f32(h, units, n_units, du, out);
  const int es = esize_of(dtype);
  // plan over the distinct row lengths (bounded scan; units share few shapes)
  int Ts[64];
  int nT = 0;
  for (int i = 0; i < n_units; ++i) {
    bool seen = false;
    for (int j = 0; j < nT; ++j) seen = seen || Ts[j] == units[i].n_time;
    if (!seen) {
      if (nT == 64) {
        snprintf(why, nwhy, "more than 64 distinct n_time values in one block");
        return LOF_ERR_INVALID;
      }
      Ts[nT++] = units[i].n_time;
    }
  }
  if (!make_plan(h, dtype, Ts, nT, &out->plan, why, nwhy)) return LOF_ERR_INVALID;
  const Plan& pl = out->plan;
  int occ = 0;
  const int krc = lofk_max_blocks_per_sm(dtype, pl.threads, pl.smem, &occ);
  if (krc != 0 || occ < 1) {
    snprintf(why, nwhy, "kernel does not fit (%d threads, %d B shared): rc %d occ %d", pl.threads,
             pl.smem, krc, occ);
    return LOF_ERR_CUDA;
  }
  const int ctas = std::min(pl.ctas, occ);
  int budget = dyn_budget(h, dtype, pl.threads, pl.ctas);
  if (h.tuning.tile_bytes) budget = std::min(budget, h.tuning.tile_bytes);
  int64_t chan = 0, per_step = 0;
  out->max_C = 1;
  out->max_T = 1;
  for (int i = 0; i < n_units; ++i) {
    const lof_unit& u = units[i];
    DevUnit& d = du[i];
    out->max_C = std::max(out->max_C, u.n_chan);
    out->max_T = std::max(out->max_T, u.n_time);
    d.in = u.in;
    d.out = u.out;
    d.mask = u.mask;
    d.stats = u.stats;
    d.in_stride = u.in_row_stride;
    d.out_stride = u.out ? u.out_row_stride : 0;
    d.mask_stride = u.mask ? u.mask_row_stride : 0;
    d.hist_slot = u.history_slot;
    d.C = u.n_chan;
    d.T = u.n_time;
    d.chan_off = static_cast<int32_t>(chan);
    chan += u.n_chan;
    int flags = 0;
    if ((reinterpret_cast<uintptr_t>(u.in) % 16) == 0 && ((u.in_row_stride * es) % 16) == 0)
      flags |= kUnitInVec;
    if (u.out && u.out == u.in) flags |= kUnitInPlace;
    else if (u.out && (reinterpret_cast<uintptr_t>(u.out) % 16) == 0 &&
             ((u.out_row_stride * es) % 16) == 0)
      flags |= kUnitOutVec;
    if (u.mask && (reinterpret_cast<uintptr_t>(u.mask) % 16) == 0 && (u.mask_row_stride % 16) == 0)
      flags |= kUnitMaskVec;
    d.flags = flags;
    const int Rs = stat_rows(u.n_time, h.tuning.stat_samples),
              Rc = flag_rows(dtype, u.n_time, budget, pl.threads, h.tuning.flag_rows);
    d.nS = (u.n_chan + Rs - 1) / Rs;
    d.nF = d.nS;
    d.nC = (u.n_chan + Rc - 1) / Rc;
    d.pad = 0;
    per_step += d.nS + d.nC;
  }
  // Two queues, one per launch of the persistent kernel: the statistics
  // launch takes every unit's stats tasks, the flag launch then every unit's
  // flag tasks, all of whose statistics are final, so no flag task waits.
  const int grid = static_cast<int>(std::min<int64_t>(int64_t(h.n_sm) * ctas, std::max<int64_t>(1, per_step)));
  const double avg = static_cast<double>(per_step) / std::max(1, n_units);
  const int inflight = static_cast<int>(std::ceil(grid / std::max(1.0, avg)));
  const int dF = inflight + 2;
  int n = 0;
  // The last `grid` tasks of each queue go in quarters (rows / 4): the CTAs
  // take tasks in queue order, so the large ones go first and the small ones
  // even out the CTAs' finishing times (a queue of 10.1 waves of equal tasks
  // would otherwise keep a tenth of the CTAs busy for a whole task at the
  // end).  Only when the quarters fit the task buffer.
  int64_t q_stats = 0, q_flag = 0;
  for (int ui = 0; ui < n_units; ++ui) {
    q_stats += du[ui].nS;
    q_flag += du[ui].nC;
  }
  const int64_t k_stats = std::min<int64_t>(q_stats, grid), k_flag = std::min<int64_t>(q_flag, grid);
  const bool split = q_stats + q_flag + 3 * (k_stats + k_flag) <= max_tasks;
  auto emit_queue = [&](int kind) -> bool {
    const int64_t q = kind == kTaskFlag ? q_flag : q_stats;
    const int64_t first_split = split ? q - (kind == kTaskFlag ? k_flag : k_stats) : q;
    int64_t idx = 0;
    for (int ui = 0; ui < n_units; ++ui) {
      DevUnit& d = du[ui];
      const int rows = kind == kTaskFlag ? (d.C + d.nC - 1) / d.nC : (d.C + d.nS - 1) / d.nS;
      int cnt = 0;
      for (int r0 = 0; r0 < d.C; r0 += rows, ++idx) {
        const int nr = std::min(rows, d.C - r0);
        const int sub = (idx >= first_split && nr >= 4) ? (nr + 3) / 4 : nr;
        for (int s0 = r0; s0 < r0 + nr; s0 += sub) {
          if (n >= max_tasks) return false;
          tasks[n++] = Task{ui, kind, s0, std::min(sub, r0 + nr - s0)};
          ++cnt;
        }
      }
      if (kind == kTaskStats) d.nS = cnt;  // the unit's stats tasks, counted on completion
      else d.nC = cnt;
    }
    return true;
  };
  // (Refinement rounds, needed when a unit's first counting pass leaves its
  // statistics open, run in the CTA that finishes that pass; no task waits.)
  (void)dF;
  bool ok = emit_queue(kTaskStats);
  const int n_stats = n;
  ok = ok && emit_queue(kTaskFlag);
  if (!ok) {
    snprintf(why, nwhy, "more than %d tasks in one block", max_tasks);
    return LOF_ERR_INVALID;
  }
  for (int i = 0; i < n_units; ++i) du[i].nF = 0;
  out->n_tasks = n;
  out->n_tasks_stats = n_stats;
  out->n_chan = chan;
  out->grid = std::min(grid, n_stats);
  out->grid_flag = std::min(grid, n - n_stats);
  // one row of the general (any-magnitude) time pass per CTA, in global scratch
  int gw = 0;
  for (int i = 0; i < nT; ++i) gw = std::max(gw, pfx_row_words(dtype, Ts[i]) + flag_words_row(Ts[i]));
  out->gen_words = (gw + 31) & ~31;
  return LOF_OK;
}

// Device-side steps of one block (no host memory touched): per-unit state
// and queue reset, the kernel launch.  Stream-capturable.
// The mode of the exact-statistics unit kernel an option set runs on (one CTA
// per unit): 0 the integrated time mode, 1 the per-channel statistics scope, 2
// the pooled per-channel pass with the winsorized estimator, 3 the
// two-dimensional mode; -1 the block kernel (or the float kernel) with its
// histogram statistics.
int exact_stats_mode(const lof_params& P) {
  if (P.time_mode == LOF_TIME_2D) return 3;
  if (P.time_mode == LOF_TIME_INTEGRATED) return 0;
  if (P.stats_scope == LOF_SCOPE_CHANNEL) return 1;
  if (P.sigma_estimator == LOF_SIGMA_WINSOR) return 2;
  return -1;
}

int host_launch_kernel(const lof_params& P, const HostCfg& h, int dtype, const Prep& pr,
                       const Scratch& sc, int n_units, uint64_t seq, void* stream, int cooperative,
                       char* why, int nwhy) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  if (!is_float(dtype) &&
      ((e = cudaMemset2DAsync(sc.ustate, sizeof(UnitState), 0, kUnitStateZeroBytes, n_units, st)) !=
           cudaSuccess ||
       (e = cudaMemsetAsync(sc.ctrl, 0, sizeof(int), st)) != cudaSuccess ||
       (e = cudaMemsetAsync(sc.ctrl + 4, 0, 3 * sizeof(int), st)) != cudaSuccess)) {
    snprintf(why, nwhy, "state reset: %s", cudaGetErrorString(e));
    return LOF_ERR_CUDA;
  }
  KParams kp{};
  kp.units = sc.units;
  kp.tasks = sc.tasks;
  kp.ustate = sc.ustate;
  kp.chan_S = sc.chanS;
  kp.chan_Fc = sc.chanFc;
  kp.queue = sc.ctrl;
  kp.err = sc.ctrl + 1;
  kp.err_info = sc.ctrl + 2;
  kp.counters = sc.ctrl + 4;
  kp.hist = sc.hist;
  kp.n_units = n_units;
  kp.n_tasks = pr.n_tasks;
  kp.fine_bins = h.tuning.fine_bins;
  for (int k = 0; k <= kMaxLogWindow; ++k) {
    // Section 2.1: factor_I = startThreshold * p^(log2 I) / I (p^k by k products)
    volatile double pk = 1.0;
    for (int i = 0; i < k; ++i) pk = pk * P.p;
    volatile double fk = P.start_threshold * pk;
    kp.factor[k] = fk / static_cast<double>(1 << k);
  }
  kp.sensitivity = P.sensitivity;
  kp.history_k = P.history_k;
  int mlw = 0;
  while ((2 << mlw) <= P.max_window) ++mlw;
  kp.max_log_window = mlw;
  kp.history_min = P.history_min;
  // 0 MAD, 1 stddev, 2 winsorized (the last only reaches the exact-statistics
  // kernel: integer units, routed there below; float units reject it)
  kp.sigma_std = P.sigma_estimator;
  kp.enable_freq = P.enable_freq;
  kp.enable_time = P.enable_time;
  kp.enable_history = P.enable_history;
  kp.block_seq = seq;
  kp.spin_limit = 2000000000ll;  // 2 s
  kp.dyn_smem = pr.plan.smem;
  kp.gen_scratch = sc.gen;
  kp.gen_words = pr.gen_words;
  kp.schedule = h.tuning.schedule;
  int krc;
  if (is_float(dtype)) {
    // Stokes I units in clusters where they fit, else one CTA per unit
    krc = (dtype == LOF_F32 && (h.tuning.schedule & LOF_SCHED_F32_CLUSTER))
              ? lofk_launch_f32c(&kp, n_units, pr.max_C, pr.max_T, stream)
              : 1;
    if (krc == 1) krc = lofk_launch_f32x(&kp, n_units, h.n_sm, pr.plan.smem, stream, dtype == LOF_CF32);
  } else if (exact_stats_mode(P) >= 0) {
    krc = lofk_launch_integ(dtype, &kp, n_units, h.n_sm, stream, exact_stats_mode(P), P.integ_chan,
                            P.integ_time);
  } else {
    // the statistics launch (stats and fine tasks), then the flag launch
    kp.n_tasks = pr.n_tasks_stats;
    krc = lofk_launch_block(dtype, &kp, pr.grid, pr.plan.threads, pr.plan.smem, stream, cooperative, 0);
    if (krc == 0 && pr.n_tasks > pr.n_tasks_stats) {
      KParams kf = kp;
      kf.tasks = sc.tasks + pr.n_tasks_stats;
      kf.n_tasks = pr.n_tasks - pr.n_tasks_stats;
      kf.queue = sc.ctrl + 6;
      krc = lofk_launch_block(dtype, &kf, pr.grid_flag, pr.plan.threads, pr.plan.smem, stream, cooperative, 1);
    }
  }
  if (krc != 0) {
    snprintf(why, nwhy, "kernel launch failed: %s (grid %d, %d threads, %d B)",
             cudaGetErrorString(static_cast<cudaError_t>(krc)), pr.grid, pr.plan.threads,
             pr.plan.smem);
    return LOF_ERR_CUDA;
  }
  if (P.sir_percent > 0) {
    // Section 2.2: the SIR operator on the final mask (time, then frequency)
    const int src = lofk_launch_sir(sc.units, n_units, pr.n_chan, pr.max_C, pr.max_T, P.sir_percent,
                                    esize_of(dtype), stream);
    if (src != 0) {
      snprintf(why, nwhy, "SIR launch failed: %d", src);
      return LOF_ERR_CUDA;
    }
  }
  return LOF_OK;
}

int host_launch(const lof_params& P, const HostCfg& h, int dtype, const Prep& pr,
                const Scratch& sc, const DevUnit* du_host, int n_units, const Task* tasks_host,
                uint64_t seq, void* stream, char* why, int nwhy) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  if ((e = cudaMemcpyAsync(sc.units, du_host, n_units * sizeof(DevUnit), cudaMemcpyHostToDevice,
                           st)) != cudaSuccess ||
      (pr.n_tasks > 0 && (e = cudaMemcpyAsync(sc.tasks, tasks_host, pr.n_tasks * sizeof(Task),
                                              cudaMemcpyHostToDevice, st)) != cudaSuccess)) {
    snprintf(why, nwhy, "descriptor upload: %s", cudaGetErrorString(e));
    return LOF_ERR_CUDA;
  }
  return host_launch_kernel(P, h, dtype, pr, sc, n_units, seq, stream, 1, why, nwhy);
}

// Options with limits of their own: the integrated time mode, the per-channel
// statistics scope and the winsorized estimator (integer units, rows up to
// lofk_integ_max_time() samples), the two-dimensional mode (integer units,
// cells that divide the unit, at most lofk_integ_max_time() cells) and the
// SIR pass (the mask output, rows up to lofk_sir_max_time() samples).
int host_validate_options(const lof_params& P, int dtype, const lof_unit& u, int i, char* why, int nwhy) {
  const int xm = exact_stats_mode(P);
  const char* what = xm == 3   ? "the two-dimensional mode"
                     : xm == 0 ? "the integrated time mode"
                     : xm == 1 ? "the per-channel statistics scope"
                               : "the winsorized sigma estimator";
  if (xm >= 0 && is_float(dtype))
    return snprintf(why, nwhy, "%s takes integer units only", what), LOF_ERR_INVALID;
  if (xm == 3) {
    if (u.n_chan % P.integ_chan || u.n_time % P.integ_time)
      return snprintf(why, nwhy, "unit %d: %d x %d cells do not divide %d x %d samples", i, P.integ_chan,
                      P.integ_time, u.n_chan, u.n_time),
             LOF_ERR_INVALID;
    const int64_t cells = static_cast<int64_t>(u.n_chan / P.integ_chan) * (u.n_time / P.integ_time);
    if (cells > lofk_integ_max_time())
      return snprintf(why, nwhy, "unit %d: %lld cells above the two-dimensional limit %d", i,
                      static_cast<long long>(cells), lofk_integ_max_time()),
             LOF_ERR_INVALID;
  } else if (xm >= 0 && u.n_time > lofk_integ_max_time()) {
    return snprintf(why, nwhy, "unit %d: n_time %d above the limit %d of %s", i, u.n_time,
                    lofk_integ_max_time(), what),
           LOF_ERR_INVALID;
  }
  if (P.sir_percent <= 0) return LOF_OK;
  if (!u.mask)
    return snprintf(why, nwhy, "unit %d: the SIR operator (sir_percent > 0) needs the mask output", i),
           LOF_ERR_INVALID;
  if (u.n_time > lofk_sir_max_time())
    return snprintf(why, nwhy, "unit %d: n_time %d above the SIR limit %d", i, u.n_time,
                    lofk_sir_max_time()),
           LOF_ERR_INVALID;
  return LOF_OK;
}

int host_validate_unit(int dtype, const lof_unit& u, int i, int64_t n_slots, char* why, int nwhy) {
  const int es = esize_of(dtype);
  if (!u.in) return snprintf(why, nwhy, "unit %d: in is NULL", i), LOF_ERR_INVALID;
  if (u.n_chan < 1 || u.n_chan > kMaxChan)
    return snprintf(why, nwhy, "unit %d: n_chan %d outside [1, %d]", i, u.n_chan, kMaxChan),
           LOF_ERR_INVALID;
  if (u.n_time < 1) return snprintf(why, nwhy, "unit %d: n_time %d < 1", i, u.n_time), LOF_ERR_INVALID;
  if (u.in_row_stride < u.n_time && u.n_chan > 1)
    return snprintf(why, nwhy, "unit %d: in_row_stride %lld < n_time", i,
                    static_cast<long long>(u.in_row_stride)),
           LOF_ERR_INVALID;
  if (u.out && u.out_row_stride < u.n_time && u.n_chan > 1)
    return snprintf(why, nwhy, "unit %d: out_row_stride < n_time", i), LOF_ERR_INVALID;
  if (u.mask && u.mask_row_stride < u.n_time && u.n_chan > 1)
    return snprintf(why, nwhy, "unit %d: mask_row_stride < n_time", i), LOF_ERR_INVALID;
  if (u.out == u.in && u.out_row_stride != u.in_row_stride)
    return snprintf(why, nwhy, "unit %d: in-place output needs equal strides", i), LOF_ERR_INVALID;
  if ((reinterpret_cast<uintptr_t>(u.in) % es) || (u.out && reinterpret_cast<uintptr_t>(u.out) % es))
    return snprintf(why, nwhy, "unit %d: data pointers must be aligned to %d bytes", i, es),
           LOF_ERR_INVALID;
  if (u.history_slot < -1 || (u.history_slot >= 0 && u.history_slot + u.n_chan > n_slots))
    return snprintf(why, nwhy, "unit %d: history slots [%lld, +%d) outside [0, %lld)", i,
                    static_cast<long long>(u.history_slot), u.n_chan,
                    static_cast<long long>(n_slots)),
           LOF_ERR_INVALID;
  return LOF_OK;
}

void host_set_error(const char* msg) {
  snprintf(g_create_error, sizeof g_create_error, "%s", msg);
}

int host_check_dtype(int dtype, char* why, int nwhy) {
  if (esize_of(dtype) == 0) return snprintf(why, nwhy, "unknown dtype %d", dtype), LOF_ERR_INVALID;
  return LOF_OK;
}

}  // namespace lofk

namespace {

lofk::HostCfg host_cfg(const lof_ctx* c) {
  return lofk::HostCfg{c->n_sm, c->smem_per_sm, c->smem_optin, c->tuning};
}

// Builds and launches one block for units already holding DEVICE pointers.
int flag_block_device(lof_ctx* c, int dtype, const lof_unit* units, int n_units, uint64_t seq,
                      void* stream, bool err_copy = true) {
  char why[512];
  const lofk::HostCfg h = host_cfg(c);
  int n_tasks = 0;
  int rc = lofk::host_count_tasks(h, dtype, units, n_units, &n_tasks, why, sizeof why);
  if (rc) return fail(c, rc, "lof_flag_block: %s", why);
  // stage descriptors (pinned ring): units then tasks
  const size_t bytes_units = n_units * sizeof(DevUnit);
  const size_t bytes = bytes_units + static_cast<size_t>(n_tasks) * sizeof(Task);
  const int si = c->stage_next;
  c->stage_next = (si + 1) % kStageRing;
  cudaError_t e = cudaEventSynchronize(c->ev_stage[si]);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaEventSynchronize");
  if (c->cap_stage[si] < bytes) {
    if (c->h_stage[si]) cudaFreeHost(c->h_stage[si]);
    c->h_stage[si] = nullptr;
    size_t n = std::max(bytes, 2 * c->cap_stage[si]);
    e = cudaHostAlloc(&c->h_stage[si], n, cudaHostAllocDefault);
    if (e != cudaSuccess) return fail(c, LOF_ERR_NOMEM, "pinned staging: %s", cudaGetErrorString(e));
    c->cap_stage[si] = n;
  }
  uint8_t* hs = static_cast<uint8_t*>(c->h_stage[si]);
  DevUnit* du = reinterpret_cast<DevUnit*>(hs);
  Task* tasks = reinterpret_cast<Task*>(hs + bytes_units);
  lofk::Prep pr{};
  rc = lofk::host_prepare(h, dtype, units, n_units, du, tasks, n_tasks, &pr, why, sizeof why);
  if (rc) return fail(c, rc, "lof_flag_block: %s", why);
  if ((rc = grow(c, &c->d_units, &c->cap_units, n_units, "units"))) return rc;
  if ((rc = grow(c, &c->d_tasks, &c->cap_tasks, pr.n_tasks, "tasks"))) return rc;
  if ((rc = grow(c, &c->d_ustate, &c->cap_ustate, is_float(dtype) ? 1 : n_units, "unit state")))
    return rc;
  if ((rc = grow(c, &c->d_chanS, &c->cap_chan, static_cast<size_t>(pr.n_chan), "spectrum"))) return rc;
  if ((rc = grow(c, &c->d_chanFc, &c->cap_chanfc, static_cast<size_t>(pr.n_chan), "channel flags")))
    return rc;
  if ((rc = grow(c, &c->d_gen, &c->cap_gen,
                 static_cast<size_t>(std::max(1, pr.grid)) * std::max(1, pr.gen_words), "general rows")))
    return rc;
  lofk::Scratch sc{};
  sc.units = c->d_units;
  sc.tasks = c->d_tasks;
  sc.ustate = c->d_ustate;
  sc.chanS = c->d_chanS;
  sc.chanFc = c->d_chanFc;
  sc.ctrl = c->d_ctrl;
  sc.hist = c->hist;
  sc.gen = c->d_gen;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  rc = lofk::host_launch(c->params, h, dtype, pr, sc, du, n_units, tasks, seq, stream, why, sizeof why);
  cudaEventRecord(c->ev_stage[si], st);
  if (rc) return fail(c, rc, "lof_flag_block: %s", why);
  if (!err_copy) return LOF_OK;  // a later call of the same host-path block copies it
  if ((e = cudaMemcpyAsync(c->h_err, c->d_ctrl + 1, 3 * sizeof(int), cudaMemcpyDeviceToHost, st)) !=
      cudaSuccess)
    return cuda_fail(c, e, "error word copy");
  cudaEventRecord(c->ev_err, st);
  c->err_copy_pending = true;
  return LOF_OK;
}

int validate_units(lof_ctx* c, int dtype, const lof_unit* units, int n_units) {
  char why[512];
  int rc = lofk::host_check_dtype(dtype, why, sizeof why);
  if (rc) return fail(c, rc, "%s", why);
  if (n_units < 0 || (n_units > 0 && !units)) return fail(c, LOF_ERR_INVALID, "bad unit array");
  for (int i = 0; i < n_units; ++i) {
    rc = lofk::host_validate_unit(dtype, units[i], i, c->n_slots, why, sizeof why);
    if (rc) return fail(c, rc, "%s", why);
    rc = lofk::host_validate_options(c->params, dtype, units[i], i, why, sizeof why);
    if (rc) return fail(c, rc, "%s", why);
  }
  return LOF_OK;
}

}  // namespace

extern "C" int lof_flag_block(lof_ctx* c, int dtype, const lof_unit* units, int n_units,
                              uint64_t block_seq, void* cuda_stream) {
  if (!c) return fail(nullptr, LOF_ERR_INVALID, "lof_flag_block: ctx is NULL");
  DeviceGuard g(c->device);
  int rc = pending_device_error(c);
  if (rc) return rc;
  if ((rc = validate_units(c, dtype, units, n_units))) return rc;
  if (n_units == 0) return LOF_OK;
  return flag_block_device(c, dtype, units, n_units, block_seq, cuda_stream);
}

namespace {

// One host<->device copy of a run of rows: 1-D when both sides are compact
// (consecutive units that are contiguous on both sides merge into one copy),
// else 2-D.
struct HostCopy {
  void* dst;
  const void* src;
  size_t dpitch, spitch, width, rows;
};

void add_copy(std::vector<HostCopy>& v, void* dst, size_t dpitch, const void* src, size_t spitch,
              size_t width, size_t rows) {
  if (dpitch == width && spitch == width) {  // compact: one run of rows * width bytes
    width *= rows;
    dpitch = spitch = width;
    rows = 1;
  }
  if (!v.empty() && rows == 1 && v.back().rows == 1 &&
      static_cast<const uint8_t*>(v.back().dst) + v.back().width == dst &&
      static_cast<const uint8_t*>(v.back().src) + v.back().width == src) {
    v.back().width += width;  // contiguous on both sides: extend the previous copy
    v.back().dpitch = v.back().spitch = v.back().width;
    return;
  }
  v.push_back(HostCopy{dst, src, dpitch, spitch, width, rows});
}

cudaError_t run_copies(const std::vector<HostCopy>& v, cudaMemcpyKind kind, cudaStream_t st) {
  for (const HostCopy& c : v) {
    const cudaError_t e = c.rows == 1 ? cudaMemcpyAsync(c.dst, c.src, c.width, kind, st)
                                      : cudaMemcpy2DAsync(c.dst, c.dpitch, c.src, c.spitch, c.width,
                                                          c.rows, kind, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

int host_path_streams(lof_ctx* c) {
  if (c->s_up) return LOF_OK;
  cudaError_t e = cudaStreamCreateWithFlags(&c->s_up, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->s_down, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_start, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_down_done, cudaEventDisableTiming);
  for (int i = 0; i < kHostChunks && e == cudaSuccess; ++i) {
    e = cudaEventCreateWithFlags(&c->ev_in[i], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_flag[i], cudaEventDisableTiming);
  }
  return e == cudaSuccess ? LOF_OK : cuda_fail(c, e, "host-path streams");
}

}  // namespace

extern "C" int lof_flag_block_host(lof_ctx* c, int dtype, const lof_unit* units, int n_units,
                                   uint64_t block_seq, void* cuda_stream) {
  if (!c) return fail(nullptr, LOF_ERR_INVALID, "lof_flag_block_host: ctx is NULL");
  DeviceGuard g(c->device);
  int rc = pending_device_error(c);
  if (rc) return rc;
  if ((rc = validate_units(c, dtype, units, n_units))) return rc;
  if (n_units == 0) return LOF_OK;
  if ((rc = host_path_streams(c))) return rc;
  const int es = esize_of(dtype);
  // device staging: compact [C][T] inputs of all units, then their outputs,
  // then their masks, then the stats (consecutive units whose host buffers
  // are contiguous then move with one copy per chunk and direction)
  size_t need = 0;
  std::vector<size_t> off_in(n_units), off_out(n_units), off_mask(n_units), off_st(n_units);
  for (int i = 0; i < n_units; ++i) {
    off_in[i] = need;
    need += round_up64(static_cast<size_t>(units[i].n_chan) * units[i].n_time * es, 256);
  }
  for (int i = 0; i < n_units; ++i) {
    off_out[i] = need;
    if (units[i].out && units[i].out != units[i].in)
      need += round_up64(static_cast<size_t>(units[i].n_chan) * units[i].n_time * es, 256);
  }
  for (int i = 0; i < n_units; ++i) {
    off_mask[i] = need;
    if (units[i].mask) need += round_up64(static_cast<size_t>(units[i].n_chan) * units[i].n_time, 256);
  }
  // statistics records of all units side by side (one download when the
  // caller's records are contiguous too)
  for (int i = 0; i < n_units; ++i) off_st[i] = need + static_cast<size_t>(i) * sizeof(lof_unit_stats);
  need += round_up64(static_cast<size_t>(n_units) * sizeof(lof_unit_stats), 256);
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  if (need > c->cap_io) {
    if (c->d_io) {
      cudaError_t e = cudaDeviceSynchronize();
      if (e != cudaSuccess) return cuda_fail(c, e, "cudaDeviceSynchronize");
      cudaFree(c->d_io);
      c->d_io = nullptr;
      c->cap_io = 0;
    }
    cudaError_t e = cudaMalloc(&c->d_io, need);
    if (e != cudaSuccess) return fail(c, LOF_ERR_NOMEM, "host-path staging %zu B: %s", need, cudaGetErrorString(e));
    c->cap_io = need;
  }
  std::vector<lof_unit> du(units, units + n_units);
  for (int i = 0; i < n_units; ++i) {
    const lof_unit& u = units[i];
    uint8_t* din = c->d_io + off_in[i];
    du[i].in = din;
    du[i].in_row_stride = u.n_time;
    if (u.out) {
      du[i].out = (u.out == u.in) ? din : c->d_io + off_out[i];
      du[i].out_row_stride = u.n_time;
    }
    if (u.mask) {
      du[i].mask = c->d_io + off_mask[i];
      du[i].mask_row_stride = u.n_time;
    }
    if (u.stats) du[i].stats = reinterpret_cast<lof_unit_stats*>(c->d_io + off_st[i]);
  }
  // Chunks of whole units by input bytes: chunk g's uploads (stream s_up),
  // its flag launch (the caller's stream, after the uploads) and its
  // downloads (stream s_down, after the launch) overlap with the neighbouring
  // chunks' steps.  The copy streams first wait for the caller's earlier work
  // (the staging may still be in use), and the caller's stream ends waiting
  // for the last download, so synchronising it covers the whole call.
  size_t total_in = 0;
  for (int i = 0; i < n_units; ++i) total_in += static_cast<size_t>(units[i].n_chan) * units[i].n_time * es;
  const size_t target = std::max<size_t>(size_t(64) << 20, (total_in + kHostChunks - 1) / kHostChunks);
  std::vector<int> cut{0};
  size_t acc = 0;
  for (int i = 0; i < n_units; ++i) {
    acc += static_cast<size_t>(units[i].n_chan) * units[i].n_time * es;
    if (acc >= target && i + 1 < n_units && static_cast<int>(cut.size()) < kHostChunks) {
      cut.push_back(i + 1);
      acc = 0;
    }
  }
  cut.push_back(n_units);
  const int nchunk = static_cast<int>(cut.size()) - 1;
  cudaError_t e = cudaEventRecord(c->ev_start, st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(c->s_up, c->ev_start, 0);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(c->s_down, c->ev_start, 0);
  if (e != cudaSuccess) return cuda_fail(c, e, "host path: stream order");
  // (Issued chunk by chunk: the launch's own small descriptor copies then
  // queue behind their chunk's upload only, not behind every chunk's.)
  auto upload = [&](int g) -> cudaError_t {
    std::vector<HostCopy> up;
    for (int i = cut[g]; i < cut[g + 1]; ++i) {
      const lof_unit& u = units[i];
      const size_t rowb = static_cast<size_t>(u.n_time) * es;
      add_copy(up, const_cast<void*>(du[i].in), rowb, u.in, static_cast<size_t>(u.in_row_stride) * es, rowb,
               u.n_chan);
    }
    cudaError_t ee = run_copies(up, cudaMemcpyHostToDevice, c->s_up);
    if (ee == cudaSuccess) ee = cudaEventRecord(c->ev_in[g], c->s_up);
    return ee;
  };
  if ((e = upload(0)) != cudaSuccess) return cuda_fail(c, e, "host input copy");
  for (int g = 0; g < nchunk; ++g) {
    if ((e = cudaStreamWaitEvent(st, c->ev_in[g], 0)) != cudaSuccess) return cuda_fail(c, e, "host path: stream order");
    // the device error word is read back once, after the last chunk (a copy
    // after every chunk would queue behind the previous chunk's downloads
    // and hold back the next launch)
    rc = flag_block_device(c, dtype, du.data() + cut[g], cut[g + 1] - cut[g], block_seq, cuda_stream,
                           g + 1 == nchunk);
    if (rc) return rc;
    if (g + 1 < nchunk && (e = upload(g + 1)) != cudaSuccess) return cuda_fail(c, e, "host input copy");
    if ((e = cudaEventRecord(c->ev_flag[g], st)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(c->s_down, c->ev_flag[g], 0)) != cudaSuccess)
      return cuda_fail(c, e, "host path: stream order");
    std::vector<HostCopy> down, down_mask, down_st;
    for (int i = cut[g]; i < cut[g + 1]; ++i) {
      const lof_unit& u = units[i];
      const size_t rowb = static_cast<size_t>(u.n_time) * es;
      if (u.out) add_copy(down, u.out, static_cast<size_t>(u.out_row_stride) * es, du[i].out, rowb, rowb, u.n_chan);
      if (u.mask)
        add_copy(down_mask, u.mask, static_cast<size_t>(u.mask_row_stride), du[i].mask, u.n_time, u.n_time,
                 u.n_chan);
      if (u.stats) add_copy(down_st, u.stats, sizeof(lof_unit_stats), du[i].stats, sizeof(lof_unit_stats),
                            sizeof(lof_unit_stats), 1);
    }
    if ((e = run_copies(down, cudaMemcpyDeviceToHost, c->s_down)) != cudaSuccess ||
        (e = run_copies(down_mask, cudaMemcpyDeviceToHost, c->s_down)) != cudaSuccess ||
        (e = run_copies(down_st, cudaMemcpyDeviceToHost, c->s_down)) != cudaSuccess)
      return cuda_fail(c, e, "host output copy");
  }
  if ((e = cudaEventRecord(c->ev_down_done, c->s_down)) != cudaSuccess ||
      (e = cudaStreamWaitEvent(st, c->ev_down_done, 0)) != cudaSuccess)
    return cuda_fail(c, e, "host path: stream order");
  return LOF_OK;
}

namespace {

int commit_like(lof_ctx* c, const lof_unit* units, int n_units, void* stream, bool refresh) {
  std::vector<DevUnit> du;
  du.reserve(n_units);
  int64_t chan = 0;
  for (int i = 0; i < n_units; ++i) {
    const lof_unit& u = units[i];
    if (u.history_slot < 0) continue;
    if (u.n_chan < 1 || u.history_slot + u.n_chan > c->n_slots)
      return fail(c, LOF_ERR_INVALID, "unit %d: history slots out of range", i);
    DevUnit d{};
    d.C = u.n_chan;
    d.T = u.n_time;
    d.hist_slot = u.history_slot;
    d.chan_off = static_cast<int32_t>(chan);
    chan += u.n_chan;
    du.push_back(d);
  }
  if (du.empty()) return LOF_OK;
  int rc;
  if ((rc = grow(c, &c->d_units, &c->cap_units, du.size(), "units"))) return rc;
  const int si = c->stage_next;
  c->stage_next = (si + 1) % kStageRing;
  cudaError_t e = cudaEventSynchronize(c->ev_stage[si]);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaEventSynchronize");
  const size_t bytes = du.size() * sizeof(DevUnit);
  if (c->cap_stage[si] < bytes) {
    if (c->h_stage[si]) cudaFreeHost(c->h_stage[si]);
    c->h_stage[si] = nullptr;
    e = cudaHostAlloc(&c->h_stage[si], bytes, cudaHostAllocDefault);
    if (e != cudaSuccess) return fail(c, LOF_ERR_NOMEM, "pinned staging: %s", cudaGetErrorString(e));
    c->cap_stage[si] = bytes;
  }
  memcpy(c->h_stage[si], du.data(), bytes);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if ((e = cudaMemcpyAsync(c->d_units, c->h_stage[si], bytes, cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return cuda_fail(c, e, "descriptor upload");
  cudaEventRecord(c->ev_stage[si], st);
  lofk::CommitParams cp{};
  cp.units = c->d_units;
  cp.n_units = static_cast<int>(du.size());
  cp.hist = c->hist;
  cp.history_k = c->params.history_k;
  cp.history_min = c->params.history_min;
  const int krc = refresh ? lofk_launch_refresh(&cp, static_cast<int>(chan), stream)
                          : lofk_launch_commit(&cp, static_cast<int>(chan), stream);
  if (krc != 0)
    return fail(c, LOF_ERR_CUDA, "history kernel: %s", cudaGetErrorString(static_cast<cudaError_t>(krc)));
  return LOF_OK;
}

}  // namespace

extern "C" int lof_history_update(lof_ctx* c, const lof_unit* units, int n_units, void* cuda_stream) {
  if (!c) return fail(nullptr, LOF_ERR_INVALID, "lof_history_update: ctx is NULL");
  if (n_units < 0 || (n_units > 0 && !units)) return fail(c, LOF_ERR_INVALID, "bad unit array");
  DeviceGuard g(c->device);
  int rc = pending_device_error(c);
  if (rc) return rc;
  return commit_like(c, units, n_units, cuda_stream, false);
}

extern "C" int lof_history_export(lof_ctx* c, int64_t slot0, int64_t n, double* values, int32_t* counts) {
  if (!c || !values || !counts || slot0 < 0 || n < 0 || slot0 + n > c->n_slots)
    return fail(c, LOF_ERR_INVALID, "lof_history_export: bad arguments");
  DeviceGuard g(c->device);
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaDeviceSynchronize");
  const int H = c->H;
  std::vector<double> v(static_cast<size_t>(n) * H);
  std::vector<int32_t> cnt(n), head(n);
  if (n == 0) return LOF_OK;
  if ((e = cudaMemcpy(v.data(), c->hist.vals + slot0 * H, v.size() * sizeof(double), cudaMemcpyDeviceToHost)) ||
      (e = cudaMemcpy(cnt.data(), c->hist.count + slot0, n * sizeof(int32_t), cudaMemcpyDeviceToHost)) ||
      (e = cudaMemcpy(head.data(), c->hist.head + slot0, n * sizeof(int32_t), cudaMemcpyDeviceToHost)))
    return cuda_fail(c, e, "history export");
  for (int64_t s = 0; s < n; ++s) {
    const int k = cnt[s];
    const int oldest = ((head[s] - k) % H + H) % H;
    for (int i = 0; i < H; ++i) values[s * H + i] = i < k ? v[s * H + (oldest + i) % H] : 0.0;
    counts[s] = k;
  }
  return LOF_OK;
}

extern "C" int lof_history_import(lof_ctx* c, int64_t slot0, int64_t n, const double* values,
                                  const int32_t* counts) {
  if (!c || !values || !counts || slot0 < 0 || n < 0 || slot0 + n > c->n_slots)
    return fail(c, LOF_ERR_INVALID, "lof_history_import: bad arguments");
  const int H = c->H;
  for (int64_t s = 0; s < n; ++s)
    if (counts[s] < 0 || counts[s] > H) return fail(c, LOF_ERR_INVALID, "history count out of range");
  if (n == 0) return LOF_OK;
  DeviceGuard g(c->device);
  std::vector<int32_t> head(n);
  for (int64_t s = 0; s < n; ++s) head[s] = counts[s] % H;
  cudaError_t e;
  if ((e = cudaDeviceSynchronize()) ||
      (e = cudaMemcpy(c->hist.vals + slot0 * H, values, static_cast<size_t>(n) * H * sizeof(double), cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(c->hist.count + slot0, counts, n * sizeof(int32_t), cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(c->hist.head + slot0, head.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice)) ||
      (e = cudaMemset(c->hist.pend_flag + slot0, 0, n)))
    return cuda_fail(c, e, "history import");
  // refresh the cached thresholds with the device arithmetic
  std::vector<lof_unit> us;
  for (int64_t s = 0; s < n; s += lofk::kMaxChan) {
    lof_unit u{};
    u.n_chan = static_cast<int32_t>(std::min<int64_t>(lofk::kMaxChan, n - s));
    u.n_time = 1;
    u.history_slot = slot0 + s;
    us.push_back(u);
  }
  int rc = commit_like(c, us.data(), static_cast<int>(us.size()), nullptr, true);
  if (rc) return rc;
  if ((e = cudaDeviceSynchronize())) return cuda_fail(c, e, "history refresh");
  return LOF_OK;
}

extern "C" int lof_status(lof_ctx* c, void* cuda_stream) {
  if (!c) return fail(nullptr, LOF_ERR_INVALID, "lof_status: ctx is NULL");
  DeviceGuard g(c->device);
  cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(cuda_stream));
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamSynchronize");
  if (c->err_copy_pending) {
    e = cudaEventSynchronize(c->ev_err);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaEventSynchronize");
  }
  return pending_device_error(c);
}

extern "C" int lof_block_counters(lof_ctx* c, void* cuda_stream, int64_t* counts) {
  if (!c || !counts) return fail(c, LOF_ERR_INVALID, "lof_block_counters: NULL argument");
  DeviceGuard g(c->device);
  cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(cuda_stream));
  int h[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpy(h, c->d_ctrl + 4, sizeof h, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(c, e, "lof_block_counters");
  counts[0] = h[0];
  counts[1] = h[1];
  return LOF_OK;
}

extern "C" int lof_max_time(const lof_ctx* c, int dtype) {
  if (!c || esize_of(dtype) == 0) return 0;
  int lo = 0, hi = 1 << 20;
  while (hi - lo > 1) {
    const int mid = (lo + hi) / 2;
    lofk::Plan pl;
    char why[256];
    if (make_plan(host_cfg(c), dtype, &mid, 1, &pl, why, sizeof why)) lo = mid;
    else hi = mid;
  }
  return lo;
}

// ------------------------------------------------------------------ graph form

struct lof_graph {
  lof_ctx* ctx = nullptr;
  int dtype = 0, n_units = 0;
  DevUnit* d_units = nullptr;
  Task* d_tasks = nullptr;
  UnitState* d_ustate = nullptr;
  unsigned long long* d_chanS = nullptr;
  uint8_t* d_chanFc = nullptr;
  uint32_t* d_gen = nullptr;
  int* d_ctrl = nullptr;  // [0] queue, [1] error, [2..3] detail
  int* h_err = nullptr;   // pinned copy of d_ctrl[1..3], written by the graph
  cudaEvent_t ev_err = nullptr;
  bool launched = false;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphNode_t knode = nullptr;
  cudaKernelNodeParams kparams{};
  cudaGraphNode_t knode2 = nullptr;  // the flag launch of the block kernel (its second launch)
  cudaKernelNodeParams kparams2{};
  lofk::KParams kp2{};
  void* kargs2[1] = {nullptr};
  lofk::KParams kp{};  // argument storage for parameter updates
  int2 cells{1, 1};    // second argument of the exact-statistics kernel
  void* kargs[2] = {nullptr, nullptr};
};

namespace {

void graph_free(lof_graph* g) {
  if (!g) return;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  cudaFree(g->d_units);
  cudaFree(g->d_tasks);
  cudaFree(g->d_ustate);
  cudaFree(g->d_chanS);
  cudaFree(g->d_chanFc);
  cudaFree(g->d_gen);
  cudaFree(g->d_ctrl);
  if (g->h_err) cudaFreeHost(g->h_err);
  if (g->ev_err) cudaEventDestroy(g->ev_err);
  delete g;
}

// Capture the device-side steps of a block into g->graph / g->exec.
int graph_capture(lof_graph* g, const lofk::HostCfg& h, const lofk::Prep& pr, int cooperative,
                  char* why, int nwhy) {
  cudaStream_t s = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e != cudaSuccess) return snprintf(why, nwhy, "stream: %s", cudaGetErrorString(e)), LOF_ERR_CUDA;
  lofk::Scratch sc{};
  sc.units = g->d_units;
  sc.tasks = g->d_tasks;
  sc.ustate = g->d_ustate;
  sc.chanS = g->d_chanS;
  sc.chanFc = g->d_chanFc;
  sc.ctrl = g->d_ctrl;
  sc.hist = g->ctx->hist;
  sc.gen = g->d_gen;
  int rc = LOF_OK;
  e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    rc = lofk::host_launch_kernel(g->ctx->params, h, g->dtype, pr, sc, g->n_units, 0, s, cooperative,
                                  why, nwhy);
    if (rc == LOF_OK) {
      e = cudaMemcpyAsync(g->h_err, g->d_ctrl + 1, 3 * sizeof(int), cudaMemcpyDeviceToHost, s);
      if (e != cudaSuccess) rc = LOF_ERR_CUDA, snprintf(why, nwhy, "error copy: %s", cudaGetErrorString(e));
    }
    cudaGraph_t gr = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(s, &gr);
    if (rc == LOF_OK && ee != cudaSuccess)
      rc = LOF_ERR_CUDA, snprintf(why, nwhy, "capture: %s", cudaGetErrorString(ee));
    if (rc == LOF_OK) g->graph = gr;
    else if (gr) cudaGraphDestroy(gr);
  } else {
    rc = LOF_ERR_CUDA;
    snprintf(why, nwhy, "begin capture: %s", cudaGetErrorString(e));
  }
  cudaGetLastError();  // a refused launch inside the capture leaves no sticky error
  cudaStreamDestroy(s);
  if (rc) return rc;
  size_t n = 0;
  cudaGraphGetNodes(g->graph, nullptr, &n);
  std::vector<cudaGraphNode_t> nodes(n);
  cudaGraphGetNodes(g->graph, nodes.data(), &n);
  // the flag kernel is the kernel node that follows no other kernel (the SIR
  // pass's kernels, when present, follow it)
  auto is_kernel = [](cudaGraphNode_t nd) {
    cudaGraphNodeType t;
    return cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel;
  };
  for (size_t i = 0; i < n && !g->knode; ++i) {
    if (!is_kernel(nodes[i])) continue;
    size_t nd = 0;
    cudaGraphNodeGetDependencies(nodes[i], nullptr, nullptr, &nd);
    std::vector<cudaGraphNode_t> deps(nd);
    if (nd) cudaGraphNodeGetDependencies(nodes[i], deps.data(), nullptr, &nd);
    bool after_kernel = false;
    for (size_t j = 0; j < nd; ++j) after_kernel = after_kernel || is_kernel(deps[j]);
    if (after_kernel) continue;
    g->knode = nodes[i];
    cudaGraphKernelNodeGetParams(nodes[i], &g->kparams);
    std::memcpy(&g->kp, g->kparams.kernelParams[0], sizeof(lofk::KParams));
    // the exact-statistics kernel takes (KParams, int2 cells); the others KParams alone
    if (lofk::exact_stats_mode(g->ctx->params) >= 0)
      std::memcpy(&g->cells, g->kparams.kernelParams[1], sizeof(int2));
  }
  if (!g->knode) return snprintf(why, nwhy, "no kernel node in the captured graph"), LOF_ERR_CUDA;
  // the block kernel's flag launch, right after its statistics launch
  for (size_t i = 0; i < n && !g->knode2; ++i) {
    if (!is_kernel(nodes[i]) || nodes[i] == g->knode) continue;
    size_t nd = 0;
    cudaGraphNodeGetDependencies(nodes[i], nullptr, nullptr, &nd);
    std::vector<cudaGraphNode_t> deps(nd);
    if (nd) cudaGraphNodeGetDependencies(nodes[i], deps.data(), nullptr, &nd);
    bool after_first = false;
    for (size_t j = 0; j < nd; ++j) after_first = after_first || deps[j] == g->knode;
    cudaKernelNodeParams kp2{};
    if (!after_first || cudaGraphKernelNodeGetParams(nodes[i], &kp2) != cudaSuccess ||
        kp2.func != lofk_block_kernel(g->dtype, h.tuning.threads, 1))
      continue;
    g->knode2 = nodes[i];
    g->kparams2 = kp2;
    std::memcpy(&g->kp2, kp2.kernelParams[0], sizeof(lofk::KParams));
  }
  e = cudaGraphInstantiate(&g->exec, g->graph, 0);
  if (e != cudaSuccess) return snprintf(why, nwhy, "instantiate: %s", cudaGetErrorString(e)), LOF_ERR_CUDA;
  return LOF_OK;
}

}  // namespace

extern "C" int lof_graph_create(lof_ctx* c, int dtype, const lof_unit* units, int n_units,
                                lof_graph** out) {
  if (!c || !out) return fail(c, LOF_ERR_INVALID, "lof_graph_create: NULL argument");
  *out = nullptr;
  DeviceGuard dg(c->device);
  int rc = validate_units(c, dtype, units, n_units);
  if (rc) return rc;
  if (n_units == 0) return fail(c, LOF_ERR_INVALID, "lof_graph_create: no units");
  char why[512];
  const lofk::HostCfg h = host_cfg(c);
  int n_tasks = 0;
  rc = lofk::host_count_tasks(h, dtype, units, n_units, &n_tasks, why, sizeof why);
  if (rc) return fail(c, rc, "lof_graph_create: %s", why);
  std::vector<DevUnit> du(n_units);
  std::vector<Task> tasks(std::max(1, n_tasks));
  lofk::Prep pr{};
  rc = lofk::host_prepare(h, dtype, units, n_units, du.data(), tasks.data(), n_tasks, &pr, why,
                          sizeof why);
  if (rc) return fail(c, rc, "lof_graph_create: %s", why);
  lof_graph* g = new lof_graph();
  g->ctx = c;
  g->dtype = dtype;
  g->n_units = n_units;
  cudaError_t e;
  const size_t nus = is_float(dtype) ? 1 : static_cast<size_t>(n_units);
  if ((e = cudaMalloc(&g->d_units, n_units * sizeof(DevUnit))) != cudaSuccess ||
      (e = cudaMalloc(&g->d_tasks, std::max(1, pr.n_tasks) * sizeof(Task))) != cudaSuccess ||
      (e = cudaMalloc(&g->d_ustate, nus * sizeof(UnitState))) != cudaSuccess ||
      (e = cudaMalloc(&g->d_chanS, std::max<int64_t>(1, pr.n_chan) * 8)) != cudaSuccess ||
      (e = cudaMalloc(&g->d_chanFc, std::max<int64_t>(1, pr.n_chan))) != cudaSuccess ||
      (e = cudaMalloc(&g->d_gen, static_cast<size_t>(std::max(1, pr.grid)) * std::max(1, pr.gen_words) * 4)) !=
          cudaSuccess ||
      (e = cudaMalloc(&g->d_ctrl, lofk::kCtrlWords * sizeof(int))) != cudaSuccess ||
      (e = cudaHostAlloc(&g->h_err, 3 * sizeof(int), cudaHostAllocDefault)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&g->ev_err, cudaEventDisableTiming)) != cudaSuccess) {
    graph_free(g);
    return fail(c, LOF_ERR_NOMEM, "lof_graph_create: %s", cudaGetErrorString(e));
  }
  if ((e = cudaMemcpy(g->d_units, du.data(), n_units * sizeof(DevUnit), cudaMemcpyHostToDevice)) !=
          cudaSuccess ||
      (pr.n_tasks > 0 && (e = cudaMemcpy(g->d_tasks, tasks.data(), pr.n_tasks * sizeof(Task),
                                         cudaMemcpyHostToDevice)) != cudaSuccess) ||
      (e = cudaMemset(g->d_ctrl, 0, lofk::kCtrlWords * sizeof(int))) != cudaSuccess) {
    graph_free(g);
    return cuda_fail(c, e, "lof_graph_create: upload");
  }
  std::memset(g->h_err, 0, 3 * sizeof(int));
  // the persistent kernel is launched cooperatively (every CTA resident);
  // where capture refuses that attribute, the grid is the resident capacity
  rc = graph_capture(g, h, pr, 1, why, sizeof why);
  if (rc) {
    if (g->graph) cudaGraphDestroy(g->graph), g->graph = nullptr;
    g->knode = nullptr;
    g->knode2 = nullptr;
    rc = graph_capture(g, h, pr, 0, why, sizeof why);
  }
  if (rc) {
    graph_free(g);
    return fail(c, rc, "lof_graph_create: %s", why);
  }
  *out = g;
  return LOF_OK;
}

extern "C" int lof_graph_launch(lof_graph* g, uint64_t block_seq, void* cuda_stream) {
  if (!g) return fail(nullptr, LOF_ERR_INVALID, "lof_graph_launch: graph is NULL");
  lof_ctx* c = g->ctx;
  DeviceGuard dg(c->device);
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  if (g->launched) {  // error of the previous replay, once it has finished
    const cudaError_t q = cudaEventQuery(g->ev_err);
    if (q == cudaSuccess && g->h_err[0] != lofk::kErrNone) {
      const int code = g->h_err[0], i0 = g->h_err[1], i1 = g->h_err[2];
      g->h_err[0] = 0;
      cudaMemset(g->d_ctrl + 1, 0, 3 * sizeof(int));
      if (code == lofk::kErrTimeout)
        return fail(c, LOF_ERR_TIMEOUT, "device wait timed out (round %d, block %d)", i0, i1);
      return fail(c, LOF_ERR_STATE, "device error %d (detail %d, block %d)", code, i0, i1);
    }
  }
  g->kp.block_seq = block_seq;
  cudaKernelNodeParams p = g->kparams;
  g->kargs[0] = &g->kp;
  g->kargs[1] = &g->cells;  // read only by a kernel with a second parameter
  p.kernelParams = g->kargs;
  cudaError_t e = cudaGraphExecKernelNodeSetParams(g->exec, g->knode, &p);
  if (e == cudaSuccess && g->knode2) {
    g->kp2.block_seq = block_seq;
    cudaKernelNodeParams p2 = g->kparams2;
    g->kargs2[0] = &g->kp2;
    p2.kernelParams = g->kargs2;
    e = cudaGraphExecKernelNodeSetParams(g->exec, g->knode2, &p2);
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "lof_graph_launch: parameter update");
  e = cudaGraphLaunch(g->exec, st);
  if (e != cudaSuccess) return cuda_fail(c, e, "lof_graph_launch");
  cudaEventRecord(g->ev_err, st);
  g->launched = true;
  return LOF_OK;
}

extern "C" int lof_graph_status(lof_graph* g, void* cuda_stream) {
  if (!g) return fail(nullptr, LOF_ERR_INVALID, "lof_graph_status: graph is NULL");
  DeviceGuard dg(g->ctx->device);
  cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(cuda_stream));
  if (e != cudaSuccess) return cuda_fail(g->ctx, e, "lof_graph_status");
  if (g->launched && cudaEventSynchronize(g->ev_err) == cudaSuccess && g->h_err[0] != lofk::kErrNone) {
    const int code = g->h_err[0], i0 = g->h_err[1], i1 = g->h_err[2];
    g->h_err[0] = 0;
    cudaMemset(g->d_ctrl + 1, 0, 3 * sizeof(int));
    if (code == lofk::kErrTimeout)
      return fail(g->ctx, LOF_ERR_TIMEOUT, "device wait timed out (round %d, block %d)", i0, i1);
    return fail(g->ctx, LOF_ERR_STATE, "device error %d (detail %d, block %d)", code, i0, i1);
  }
  return LOF_OK;
}

extern "C" int lof_graph_destroy(lof_graph* g) {
  if (!g) return LOF_OK;
  DeviceGuard dg(g->ctx->device);
  cudaDeviceSynchronize();
  graph_free(g);
  return LOF_OK;
}

// ------------------------------------------------------------------ autotuner

extern "C" int lof_autotune(lof_ctx* c, int dtype, const lof_unit* units, int n_units, int reps,
                            void* cuda_stream, lof_tuning* best, float* best_ms) {
  if (!c) return fail(nullptr, LOF_ERR_INVALID, "lof_autotune: ctx is NULL");
  DeviceGuard dg(c->device);
  int rc = validate_units(c, dtype, units, n_units);
  if (rc) return rc;
  if (n_units == 0) return fail(c, LOF_ERR_INVALID, "lof_autotune: no units");
  if (reps < 1) reps = 3;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const lof_tuning saved = c->tuning;
  std::vector<lof_tuning> cands;
  if (is_float(dtype)) {
    // no launch shape to choose: one CTA per unit, or (Stokes I) one cluster per unit
    cands.push_back(saved);
    lof_tuning t = saved;
    t.schedule = saved.schedule ^ LOF_SCHED_F32_CLUSTER;
    if (dtype == LOF_F32) cands.push_back(t);
  } else {
    for (int threads : {128, 256})
      for (int ctas : {1, 2, 3, 4}) {
        if (threads >= 256 && ctas > 2) continue;  // the launch bounds allow two
        for (int rows : {8, 16, 32, 64})
          for (int samples : {32768, 65536, 131072, 262144})
            cands.push_back(lof_tuning{threads, ctas, saved.tile_bytes, saved.fine_bins, rows, samples,
                                       saved.schedule});
      }
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best_t = 1e30f;
  lof_tuning best_c = saved;
  std::vector<float> ts(reps);
  // stage 1: the launch shapes with the current schedule; stage 2: every
  // window schedule with the fastest shape
  const int n_shapes = static_cast<int>(cands.size());
  for (int ci = 0; ci < static_cast<int>(cands.size()); ++ci) {
    if (ci == n_shapes && !is_float(dtype)) {
      for (int sc = 0; sc < 16; ++sc) {
        lof_tuning t = best_c;
        t.schedule = LOF_SCHED_SET | sc;
        if (t.schedule != best_c.schedule) cands.push_back(t);
      }
      if (ci == static_cast<int>(cands.size())) break;
    }
    const lof_tuning t = cands[ci];
    c->tuning = t;
    if (lof_flag_block(c, dtype, units, n_units, 0, st) != LOF_OK) continue;  // warm-up
    bool ok = true;
    for (int r = 0; r < reps && ok; ++r) {
      cudaEventRecord(e0, st);
      ok = lof_flag_block(c, dtype, units, n_units, 0, st) == LOF_OK;
      cudaEventRecord(e1, st);
      cudaEventSynchronize(e1);
      cudaEventElapsedTime(&ts[r], e0, e1);
    }
    if (!ok || lof_status(c, st) != LOF_OK) continue;
    std::vector<float> srt(ts);
    std::sort(srt.begin(), srt.end());
    const float med = srt[reps / 2];
    if (med < best_t) {
      best_t = med;
      best_c = t;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->tuning = best_c;
  c->last_error.clear();
  if (best) *best = best_c;
  if (best_ms) *best_ms = best_t;
  return best_t < 1e30f ? LOF_OK : fail(c, LOF_ERR_CUDA, "lof_autotune: no candidate ran");
}
