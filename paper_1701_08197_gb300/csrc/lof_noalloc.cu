// lof_noalloc.cu -- lof_flag_block_noalloc: the flagger for callers that may
// not allocate memory at run time.
//
// Real-time pipelines often forbid allocation on their processing threads:
// cudaMalloc / cudaFree can block for milliseconds and synchronise the device,
// a memory pool may not exist, or the process runs under an allocation
// budget fixed at start-up.  This entry point does the same work as
// lof_flag_block but keeps all of its scratch in one file-scope device array
// of fixed size (kScratchBytes), and its host-side descriptors in fixed static
// arrays, so a call allocates nothing.  The caller still owns the inputs and
// outputs.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "lof.h"
#include "lof_internal.h"

namespace {

constexpr size_t kScratchBytes = size_t(64) << 20;  // 64 MiB, held by every GPU that loads the library
constexpr int kMaxUnitsNA = 1024;
constexpr int kMaxTasksNA = 262144;
constexpr int kMaxDevicesNA = 64;

// The scratch.  In host code its name is only a host-side stand-in: the
// device address comes from cudaGetSymbolAddress, once per device.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;                        // one caller at a time (the arrays below are shared)
void* g_addr[kMaxDevicesNA] = {};       // device address of g_scratch, per device
lofk::DevUnit g_du[kMaxUnitsNA];
lofk::Task g_tasks[kMaxTasksNA];

size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

namespace lofk {
void host_set_error(const char* msg);
int host_validate_options(const lof_params& P, int dtype, const lof_unit& u, int i, char* why, int nwhy);
}

extern "C" int lof_flag_block_noalloc(const lof_params* params, int dtype, const lof_unit* units,
                                      int n_units, int* status, void* cuda_stream) {
  char why[512];
  std::lock_guard<std::mutex> lock(g_mu);
  auto fail = [&](int code) {
    lofk::host_set_error(why);
    return code;
  };
  lof_params P;
  if (params) P = *params;
  else lof_default_params(&P);
  // the same parameter checks as lof_create, before anything reads them
  char pwhy[256];
  if (!lofk::validate_params(&P, pwhy, sizeof pwhy)) {
    snprintf(why, sizeof why, "lof_flag_block_noalloc: %s", pwhy);
    return fail(LOF_ERR_INVALID);
  }
  int rc = lofk::host_check_dtype(dtype, why, sizeof why);
  if (rc) return fail(rc);
  if (n_units < 0 || (n_units > 0 && !units)) {
    snprintf(why, sizeof why, "lof_flag_block_noalloc: bad unit array");
    return fail(LOF_ERR_INVALID);
  }
  if (n_units > kMaxUnitsNA) {
    snprintf(why, sizeof why, "lof_flag_block_noalloc: %d units exceed the maximum of %d", n_units,
             kMaxUnitsNA);
    return fail(LOF_ERR_INVALID);
  }
  for (int i = 0; i < n_units; ++i) {
    rc = lofk::host_validate_unit(dtype, units[i], i, 0, why, sizeof why);
    if (rc) return fail(rc);
    rc = lofk::host_validate_options(P, dtype, units[i], i, why, sizeof why);
    if (rc) return fail(rc);
    if (units[i].history_slot != -1) {
      snprintf(why, sizeof why,
               "lof_flag_block_noalloc: unit %d asks for history; the history rings need a context",
               i);
      return fail(LOF_ERR_INVALID);
    }
  }
  if (n_units == 0) return LOF_OK;
  // The descriptors are uploaded from the static host arrays below, which the
  // next call overwrites: a captured copy would replay some later call's units.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(static_cast<cudaStream_t>(cuda_stream), &cap);
  if (e != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
    snprintf(why, sizeof why,
             "lof_flag_block_noalloc: cuda_stream is capturing (or its state is unknown: %s); "
             "nothing was enqueued",
             cudaGetErrorString(e));
    return fail(LOF_ERR_INVALID);
  }
  int dev = 0;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevicesNA) {
    snprintf(why, sizeof why, "lof_flag_block_noalloc: no usable current device (%s)",
             cudaGetErrorString(e));
    return fail(LOF_ERR_CUDA);
  }
  // set-up, once per device, with that device current
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p) {
      snprintf(why, sizeof why, "lof_flag_block_noalloc: cudaGetSymbolAddress: %s",
               cudaGetErrorString(e));
      return fail(LOF_ERR_CUDA);
    }
    g_addr[dev] = p;
  }
  lofk::HostCfg h{};
  cudaDeviceGetAttribute(&h.n_sm, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&h.smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&h.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  h.tuning = lofk::default_tuning();
  int n_tasks = 0;
  rc = lofk::host_count_tasks(h, dtype, units, n_units, &n_tasks, why, sizeof why);
  if (rc) return fail(rc);
  if (n_tasks > kMaxTasksNA) {
    snprintf(why, sizeof why,
             "lof_flag_block_noalloc: the block needs %d tasks, the maximum is %d", n_tasks,
             kMaxTasksNA);
    return fail(LOF_ERR_INVALID);
  }
  lofk::Prep pr{};
  rc = lofk::host_prepare(h, dtype, units, n_units, g_du, g_tasks, kMaxTasksNA, &pr, why,
                          sizeof why);
  if (rc) return fail(rc);
  // carve the scratch
  unsigned char* base = static_cast<unsigned char*>(g_addr[dev]);
  size_t off = 0;
  lofk::Scratch sc{};
  sc.ctrl = reinterpret_cast<int*>(base + off);
  off += 256;
  sc.units = reinterpret_cast<lofk::DevUnit*>(base + off);
  off += up256(n_units * sizeof(lofk::DevUnit));
  sc.tasks = reinterpret_cast<lofk::Task*>(base + off);
  off += up256(static_cast<size_t>(pr.n_tasks) * sizeof(lofk::Task));
  sc.chanS = reinterpret_cast<unsigned long long*>(base + off);
  off += up256(static_cast<size_t>(pr.n_chan) * 8);
  sc.chanFc = base + off;
  off += up256(static_cast<size_t>(pr.n_chan));
  sc.ustate = reinterpret_cast<lofk::UnitState*>(base + off);
  off += up256(static_cast<size_t>((dtype == LOF_F32 || dtype == LOF_CF32) ? 0 : n_units) * sizeof(lofk::UnitState));
  sc.gen = reinterpret_cast<uint32_t*>(base + off);
  off += static_cast<size_t>(std::max(1, pr.grid)) * std::max(1, pr.gen_words) * 4;
  if (off > kScratchBytes) {
    snprintf(why, sizeof why,
             "lof_flag_block_noalloc: the block needs %zu bytes of scratch, the static array holds %zu",
             off, kScratchBytes);
    return fail(LOF_ERR_INVALID);
  }
  sc.hist = lofk::HistoryDev{};
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  // the error word and detail start at zero on every call (the queue, the
  // launch counters and the per-unit counters, moments and histograms are
  // cleared by host_launch); every other part is written before it is read
  e = cudaMemsetAsync(sc.ctrl, 0, lofk::kCtrlWords * sizeof(int), st);
  if (e != cudaSuccess) {
    snprintf(why, sizeof why, "lof_flag_block_noalloc: %s", cudaGetErrorString(e));
    return fail(LOF_ERR_CUDA);
  }
  rc = lofk::host_launch(P, h, dtype, pr, sc, g_du, n_units, g_tasks, 0, cuda_stream, why,
                         sizeof why);
  if (rc) return fail(rc);
  if (status) {
    e = cudaMemcpyAsync(status, sc.ctrl + 1, sizeof(int), cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) {
      snprintf(why, sizeof why, "lof_flag_block_noalloc: status copy: %s", cudaGetErrorString(e));
      return fail(LOF_ERR_CUDA);
    }
  }
  return LOF_OK;
}
