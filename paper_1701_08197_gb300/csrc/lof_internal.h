// lof_internal.h -- definitions shared by the host side (lof_api.cu) and the
// kernels (lof_kernels.cu) of the CUDA flagger library.  Not part of the ABI.
#pragma once

#include <cstddef>
#include <cstdint>

#include "lof.h"

namespace lofk {

// Coarse histogram of 32-bit keys: the exponent and 5 mantissa bits of the
// value as binary32 (32 bins per octave, one per integer below 64).
constexpr int kCoarseBins = 1056;
constexpr int kMaxLogWindow = 6;             // windows 1 .. 64
constexpr int kKTable = 134;                 // sum_{k=0..6} (2^k + 1) threshold entries
constexpr int kMaxChan = 2048;               // channels per unit
constexpr int kMaxRowsPerTask = 64;          // rows of one unit in one task
constexpr int kMaxTargets = 128;             // bins refined per selection round (and hinted bins)
constexpr int kMaxFine = 4096;               // counters per refinement round (upper bound)
constexpr int kMaxSpec = 4096;               // exact counters near the previous block's statistics
constexpr int kSpecHalf = 682;               // largest half-width of one hinted window (3 fit kMaxSpec)
constexpr int kSelCap = 2048;                // bin-list capacity for exact selection
constexpr int kMaxRounds = 12;               // refinement rounds before giving up
constexpr int kWorkspaceBytes = 56 * 1024;   // last-arriver workspace (overlays the prefix buffer)
constexpr int kCtrlWords = 8;               // control words of a launch (see Scratch::ctrl)

// device error codes (written to the context's mapped error word)
enum : int {
  kErrNone = 0,
  kErrTimeout = 1,     // a bounded wait on another CTA gave up
  kErrSelect = 2,      // exact selection did not converge / bin list overflow
  kErrInternal = 3,    // consistency check failed
  kErrHistory = 4,     // history slot out of range
};

struct DevUnit {
  const void* in;
  void* out;
  uint8_t* mask;
  lof_unit_stats* stats;
  int64_t in_stride, out_stride, mask_stride;  // elements
  int64_t hist_slot;                           // first slot, or -1
  int32_t C, T;
  int32_t chan_off;                            // into per-channel scratch
  int32_t nS, nF, nC;                          // stats / fine / flag tasks of the unit
  int32_t flags;                               // kUnit* bits
  int32_t pad;
};
enum : int32_t {
  kUnitInVec = 1,       // input rows 16-byte aligned: vector loads
  kUnitOutVec = 2,      // output rows 16-byte aligned: vector stores
  kUnitInPlace = 4,     // out == in: write flagged samples only
  kUnitMaskVec = 8,     // mask rows 16-byte aligned
};

// One task of the persistent queue: a run of rows of one unit.
enum : int32_t {
  kTaskStats = 0,  // row sums + coarse histogram (reads the rows from HBM)
  kTaskFine = 1,   // exact counts in refined bins (only when round 1 did not resolve)
  kTaskFlag = 2,   // SumThreshold in time, history, mask and output
};
struct Task {
  int32_t unit, kind, row0, nrows;
};

// Refinement target: bin [lo, hi] split into sub-bins of width 2^shift
// starting at fine counter 'base'.
struct alignas(16) Target {
  uint32_t lo, hi, shift, base;
};

// Per-unit state of one launch.  The leading part (counters, moments, coarse
// histogram) is zeroed by the host before every launch; the rest is written
// before it is read.
struct UnitState {
  int done_S, done_F;        // completed stats / fine tasks
  int ready;                 // 0: statistics pending, 1: fine counts needed, 2: final
  int win_below;             // value-window statistics: kept samples below the window
  unsigned long long mom[4]; // sum x (lo, hi), sum x^2 (lo, hi) -- 128-bit each
  uint32_t coarse[kCoarseBins];
  uint32_t spec[kMaxSpec];   // exact counts in the bins around the previous block's statistics
                             // (value-window statistics: one counter per value of the window)
  // ---- end of the zeroed part
  double median_f, sigma_f;
  long long n_pool;          // samples in the time-pass pool
  int n_chan_freq;
  int state;                 // kState*
  int n_bins;                // entries in the bin list
  int n_targets, n_fine;
  int round;
  int mom_ready;             // moments accumulated
  int pad0;
  Target tgt[kMaxTargets];
  int tgt_bin[kMaxTargets];  // bin-list index each target refines
  uint32_t fine[kMaxFine];
  uint32_t blo[kSelCap], bhi[kSelCap], bcnt[kSelCap];
  double median_t, sigma_t;
  long long K[kKTable];
  int time_on;
  int pad2;
};
constexpr size_t kUnitStateZeroBytes = offsetof(UnitState, median_f);
enum : int {
  kStateCoarse = 0,   // next: coarse histogram
  kStateFine = 1,     // next: fine counts for the targets
  kStateMoments = 2,  // next: exact moments (std estimator / MAD = 0)
  kStateDone = 3,     // statistics ready
};

struct HistoryDev {
  double* vals;        // [slots][H] ring storage
  int32_t* count;      // entries held
  int32_t* head;       // next write position
  double* thr;         // cached mean + k*stddev (valid when count >= history_min)
  double* pend;        // staged value
  uint8_t* pend_flag;  // 1 = staged
  uint64_t* pend_seq;  // block_seq of the staged value
  unsigned long long* hint;  // [slots][2]: last exact 2*median and 4*MAD of the unit starting here
  int64_t n_slots;
  int32_t H;
};

struct KParams {
  const DevUnit* units;
  const Task* tasks;
  UnitState* ustate;
  unsigned long long* chan_S;   // per channel spectrum sums
  uint8_t* chan_Fc;             // per channel frequency flags
  int* queue;                   // [0] next task
  int* err;                     // first device-side error (0 = none)
  int* err_info;                // detail words of that error
  int* counters;                // [0] units whose statistics needed a refinement round,
                                // [1] fine-count tasks that ran (zeroed per launch)
  HistoryDev hist;
  int n_units, n_tasks;
  int fine_bins;                // counters per refinement round
  double factor[kMaxLogWindow + 1];
  double sensitivity;
  double history_k;
  int max_log_window;
  int history_min;
  int sigma_std;
  int enable_freq, enable_time, enable_history;
  uint64_t block_seq;
  long long spin_limit;         // bound of every device-side wait (ns)
  int dyn_smem;                 // dynamic shared memory of each CTA (bytes)
  uint32_t* gen_scratch;        // general time-pass rows, gen_words per CTA
  int gen_words;
  int schedule;                 // LOF_SCHED_* bits of the time pass
};

struct CommitParams {
  const DevUnit* units;
  int n_units;
  HistoryDev hist;
  double history_k;
  int history_min;
};

// ---------------------------------------------------------------- host side
struct HostCfg {
  int n_sm, smem_per_sm, smem_optin;
  lof_tuning tuning;
};
struct Plan {
  int threads, ctas;
  int smem;                     // dynamic shared memory per CTA (bytes)
};
struct Prep {
  Plan plan;
  int n_tasks, grid;             // all tasks; CTAs of the statistics launch
  int n_tasks_stats, grid_flag;  // tasks of the statistics launch (the first ones); CTAs of the flag launch
  int64_t n_chan;
  int gen_words;                 // per CTA, general time-pass rows
  int max_C, max_T;              // the largest unit's channels and samples
};
// Device memory one launch works in.
struct Scratch {
  DevUnit* units;
  Task* tasks;
  UnitState* ustate;
  unsigned long long* chanS;
  uint8_t* chanFc;
  int* ctrl;  // [0] queue of the statistics launch, [1] error, [2..3] detail, [4..5] counters,
             // [6] queue of the flag launch (kCtrlWords ints)
  HistoryDev hist;
  uint32_t* gen;  // general time-pass rows: grid x gen_words words
};
// lof_api.cu: heap-free steps shared by every entry point
lof_tuning default_tuning();  // the library's launch shape before any lof_set_tuning
int validate_params(const lof_params* p, char* why, int nwhy);  // 1 = valid
int host_check_dtype(int dtype, char* why, int nwhy);
int host_validate_unit(int dtype, const lof_unit& u, int i, int64_t n_slots, char* why, int nwhy);
int host_count_tasks(const HostCfg& h, int dtype, const lof_unit* units, int n_units,
                     int* n_tasks, char* why, int nwhy);
int host_prepare(const HostCfg& h, int dtype, const lof_unit* units, int n_units, DevUnit* du,
                 Task* tasks, int max_tasks, Prep* out, char* why, int nwhy);
int host_launch(const lof_params& P, const HostCfg& h, int dtype, const Prep& pr, const Scratch& sc,
                const DevUnit* du_host, int n_units, const Task* tasks_host, uint64_t seq,
                void* stream, char* why, int nwhy);
int host_launch_kernel(const lof_params& P, const HostCfg& h, int dtype, const Prep& pr,
                       const Scratch& sc, int n_units, uint64_t seq, void* stream, int cooperative,
                       char* why, int nwhy);

}  // namespace lofk

// Kernel launchers (lof_kernels.cu)
extern "C" int lofk_launch_block(int dtype, const lofk::KParams* kp, int grid, int threads,
                                 int smem_bytes, void* stream, int cooperative, int phase);
extern "C" void* lofk_block_kernel(int dtype, int threads, int phase);
extern "C" int lofk_launch_commit(const lofk::CommitParams* cp, int total_channels, void* stream);
extern "C" int lofk_launch_refresh(const lofk::CommitParams* cp, int total_channels, void* stream);
extern "C" int lofk_max_blocks_per_sm(int dtype, int threads, int smem_bytes, int* out);
extern "C" int lofk_set_smem_limit(int dtype, int smem_bytes);
extern "C" int lofk_f32_smem(int max_T);
extern "C" int lofk_launch_f32(const lofk::KParams* kp, int n_units, int n_sm, int smem_bytes,
                               void* stream);
extern "C" int lofk_launch_f32c(const lofk::KParams* kp, int n_units, int max_C, int max_T, void* stream);
