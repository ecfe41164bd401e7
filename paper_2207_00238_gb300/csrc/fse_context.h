// Context state behind the opaque fse_context_t handle.
#pragma once
#include <cstdarg>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/fse.h"
#include "fse_internal.h"

struct fse_context {
  int device = 0;
  int sm_count = 0;
  char* arena = nullptr;
  size_t arena_bytes = 0;
  bool owns_arena = true;
  char* host_buf = nullptr;  // pinned staging of the per-call tables
  size_t host_cap = 0;
  // host_buf is rewritten by the next call only after the copy that reads it
  // has run (the calls are asynchronous): ev_host_free follows that copy
  cudaEvent_t ev_host_free = nullptr;
  bool host_buf_busy = false;
  // the captured graph's copy node reads graph_host_buf, which stays unchanged
  // while the graph exists; ev_graph_done follows its last launch
  char* graph_host_buf = nullptr;
  size_t graph_host_cap = 0;
  cudaEvent_t ev_graph_done = nullptr;
  bool graph_launched = false;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev2 = nullptr, ev3 = nullptr;
  cudaStream_t cap_stream = nullptr;  // graph capture happens here, replay on the caller's stream
  // options
  int exec_mode = FSE_EXEC_DAG;
  int timeout_ms = 20000;
  int ctas_per_sm = 0;
  int use_graph = 0;
  int debug = 0;
  int kernel_timing = 0;
  int tma = 2;  // TMA staging of F = 32 supports: 0 off, 1 where the buffers allow it, 2 auto
  int capturing = 0;
  int dbg_tma_stall = 0;  // test only (FSE_OPT_DEBUG_TMA_STALL)
  int server_classes = 3;  // FSE_OPT_SERVER_CLASSES of servers made from this context
  int root_window = 2;     // FSE_OPT_ROOT_WINDOW: fed roots per consumer (0 = all at once)
  std::vector<cudaEvent_t> tev;  // pairs: start, end of the iteration kernels
  size_t tev_used = 0;
  fse::ExecCfg cfg;                    // executor variant per class (options, autotuner)
  int occupancy[fse::MAX_CLS] = {1, 1, 1};  // of cfg's variants
  int concurrent = 1;                  // work classes of one call run on forked streams
  int class_order = 0;                 // 0: F = 64 class launched first; 1: F = 32 first
  cudaStream_t cls_stream[fse::MAX_CLS] = {nullptr, nullptr, nullptr};
  cudaEvent_t ev_fork = nullptr, ev_join[fse::MAX_CLS] = {nullptr, nullptr, nullptr};
  // per timed call: start/end of the whole execution, then start/end per class
  std::vector<int> tev_cls_mask;
  std::string tune_path;
  int tuned_ctas[fse::MAX_CLS] = {0, 0, 0};
  // cached graph of the last job set
  cudaGraphExec_t graph_exec = nullptr;
  std::vector<fse_job_t> graph_jobs;
  int graph_mode = -1, graph_debug = -1, graph_launches = 0;
  // last call (for fse_debug_fetch / fse_context_check)
  int64_t last_cap[fse::MAX_CLS] = {0, 0, 0};
  fse::QueueDev* last_q = nullptr;
  int32_t* last_dbg_rec = nullptr;
  int32_t* last_dbg_useq = nullptr;
  int32_t last_dbg_cap = 0;
  int32_t last_K_max = 0;
};

namespace fse {
using Context = fse_context;
int fail(int code, const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);
int plan_tiles(int32_t W, int32_t H, int32_t N, int32_t d, fse_tile_t* out, int32_t cap,
               int32_t* n_out);
int plan_tiles_mode(int32_t mode, int32_t W, int32_t H, int32_t N, int32_t d, fse_tile_t* out,
                    int32_t cap, int32_t* n_out);
int plan_tiles_vertical(int32_t W, int32_t H, int32_t N, int32_t d, fse_tile_t* out, int32_t cap,
                        int32_t* n_out);
int check_job(const fse_job_t& j, int idx);
int context_create(Context** out, int device, size_t arena_bytes, const char* tune_path);
// A context on caller-owned device memory (not freed by context_destroy).
int context_create_alias(Context** out, int device, char* arena, size_t arena_bytes);
int enqueue_host(Context* c, const fse_job_t* jobs, int32_t n, cudaStream_t st, fse_stats_t* stats);
size_t job_device_bytes(const fse_job_t& j);
void context_destroy(Context* c);
int run_batch(Context* c, const fse_job_t* jobs, int32_t n, cudaStream_t st, fse_stats_t* stats,
              size_t arena_offset);
int exec_grid(Context* c, int cls);
void update_occupancy(Context* c);  // occupancy of the context's variants
void tune_load(Context* c);
int autotune(Context* c, const fse_job_t* jobs, int32_t n, cudaStream_t st, int reps, double* trace,
             int cap);
const char* last_error();
}  // namespace fse
