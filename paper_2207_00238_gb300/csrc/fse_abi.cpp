// extern "C" entry points declared in include/fse.h.
#include <algorithm>
#include <cmath>
#include <vector>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/fse.h"
#include "fse_context.h"
#include "fse_internal.h"

using fse::Context;

namespace fse {

// Autotuner cache: the GPU name on the first line, then one line per work
// class "cls ctas_per_sm layout" (layout: FSE_OPT_F32_LAYOUT for class 0,
// FSE_OPT_F64_WARPS for class 1).
// A missing or foreign file is ignored.
void tune_load(Context* c) {
  FILE* f = fopen(c->tune_path.c_str(), "r");
  if (!f) return;
  char name[256] = {0};
  cudaDeviceProp prop;
  cudaGetDeviceProperties(&prop, c->device);
  if (fgets(name, sizeof(name), f)) {
    name[strcspn(name, "\r\n")] = 0;
    if (strcmp(name, prop.name) == 0) {
      int k, v, lay;
      while (fscanf(f, "%d %d %d", &k, &v, &lay) == 3) {
        if (k < 0 || k >= MAX_CLS || v <= 0) continue;
        c->tuned_ctas[k] = v;
        if (k == CLS_F32_64 && (lay == 2 || lay == 4 || lay == 5 || lay == 6 || lay == 8)) set_f64_warps(lay);
        if (k == CLS_F32_32 && lay >= 1 && lay <= 3) set_f32_layout(lay);
      }
    }
  }
  fclose(f);
}

static void tune_save(Context* c) {
  if (c->tune_path.empty()) return;
  FILE* f = fopen(c->tune_path.c_str(), "w");
  if (!f) return;
  cudaDeviceProp prop;
  cudaGetDeviceProperties(&prop, c->device);
  fprintf(f, "%s\n", prop.name);
  for (int k = 0; k < MAX_CLS; ++k)
    if (c->tuned_ctas[k] > 0) fprintf(f, "%d %d %d\n", k, c->tuned_ctas[k], k == CLS_F32_64 ? get_f64_warps() : (k == CLS_F32_32 ? get_f32_layout() : 0));
  fclose(f);
}

static int occupancy_of(int cls) {
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, exec_kernel_ptr(cls), exec_threads(cls),
                                                exec_smem(cls));
  return nb > 0 ? nb : 1;
}

int autotune(Context* c, const fse_job_t* jobs, int32_t n, cudaStream_t st, int reps,
             double* trace, int cap) {
  if (!c || n <= 0 || !jobs || reps < 1) return fail(FSE_EINVAL, "autotune: bad arguments");
  bool present[MAX_CLS] = {false, false, false};
  for (int i = 0; i < n; ++i) {
    int rc = check_job(jobs[i], i);
    if (rc) return rc;
    const fse_params_t& p = jobs[i].p;
    present[p.precision == 64 ? CLS_F64 : (p.fft == 32 ? CLS_F32_32 : CLS_F32_64)] = true;
  }
  const int saved_mode = c->exec_mode, saved_graph = c->use_graph, saved_ctas = c->ctas_per_sm;
  c->exec_mode = FSE_EXEC_DAG;
  c->use_graph = 0;
  int ran = 0;
  auto time_cfg = [&](int cls, int layout, int ctas, double* ms_out) -> int {
    c->ctas_per_sm = ctas;
    std::vector<double> ms;
    for (int r = 0; r < reps + 1; ++r) {
      fse_stats_t stt;
      int rc = run_batch(c, jobs, n, st, &stt, 0);
      if (rc) return rc;
      if (r > 0) ms.push_back(stt.exec_ms);  // first run warms up
    }
    std::sort(ms.begin(), ms.end());
    *ms_out = ms[ms.size() / 2];
    if (trace && ran < cap) {
      trace[4 * ran] = cls;
      trace[4 * ran + 1] = layout;
      trace[4 * ran + 2] = ctas;
      trace[4 * ran + 3] = *ms_out;
    }
    ++ran;
    return FSE_OK;
  };
  int rc = FSE_OK;
  // F = 64: executor layout x CTAs per SM (only this class is timed; the
  // others run at their current setting and add a constant)
  if (present[CLS_F32_64]) {
    double best = 1e30;
    int best_lay = get_f64_warps(), best_ctas = 0;
    const int layouts[5] = {6, 4, 5, 2, 8};
    for (int li = 0; li < 5 && rc == FSE_OK; ++li) {
      set_f64_warps(layouts[li]);
      c->occupancy[CLS_F32_64] = occupancy_of(CLS_F32_64);
      const int occ = c->occupancy[CLS_F32_64];
      for (int k = occ; k >= 1 && k >= occ - 1 && rc == FSE_OK; --k) {
        double ms;
        rc = time_cfg(CLS_F32_64, layouts[li], k, &ms);
        if (rc == FSE_OK && ms < best) {
          best = ms;
          best_lay = layouts[li];
          best_ctas = k;
        }
      }
    }
    set_f64_warps(best_lay);
    c->occupancy[CLS_F32_64] = occupancy_of(CLS_F32_64);
    c->tuned_ctas[CLS_F32_64] = best_ctas;
  }
  if (present[CLS_F32_32] && rc == FSE_OK) {
    double best = 1e30;
    int best_lay = get_f32_layout(), best_ctas = 0;
    const int layouts[3] = {3, 1, 2};
    for (int li = 0; li < 3 && rc == FSE_OK; ++li) {
      set_f32_layout(layouts[li]);
      c->occupancy[CLS_F32_32] = occupancy_of(CLS_F32_32);
      const int occ = c->occupancy[CLS_F32_32];
      for (int k = occ; k >= 1 && k >= occ - 3 && rc == FSE_OK; --k) {
        double ms;
        rc = time_cfg(CLS_F32_32, layouts[li], k, &ms);
        if (rc == FSE_OK && ms < best) {
          best = ms;
          best_lay = layouts[li];
          best_ctas = k;
        }
      }
    }
    set_f32_layout(best_lay);
    c->occupancy[CLS_F32_32] = occupancy_of(CLS_F32_32);
    c->tuned_ctas[CLS_F32_32] = best_ctas;
  }
  c->exec_mode = saved_mode;
  c->use_graph = saved_graph;
  c->ctas_per_sm = saved_ctas;
  c->graph_jobs.clear();
  if (rc) return rc;
  tune_save(c);
  return ran;
}

// Copies host inputs into the arena front, runs the batch and copies the
// outputs back, all enqueued on st (asynchronous for pinned host memory).
int enqueue_host(Context* c, const fse_job_t* jobs, int32_t n, cudaStream_t st,
                 fse_stats_t* stats) {
  if (!c) return fail(FSE_EINVAL, "NULL ctx");
  if (n < 0 || (n > 0 && !jobs)) return fail(FSE_EINVAL, "bad job list");
  if (cudaSetDevice(c->device) != cudaSuccess) return fail(FSE_ECUDA, "cudaSetDevice");
  std::vector<fse_job_t> dj(jobs, jobs + n);
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t r = (off + 255) / 256 * 256; off = r + bytes; return r; };
  for (int i = 0; i < n; ++i) {
    int rc = check_job(jobs[i], i);
    if (rc) return rc;
    const size_t px = (size_t)jobs[i].W * jobs[i].H;
    const int dp = (jobs[i].W + 15) & ~15;  // device row pitch: 16-byte rows for the TMA staging
    const size_t dpx = (size_t)dp * jobs[i].H;
    dj[i].image = (const uint8_t*)(c->arena + take(dpx));
    dj[i].mask = (const uint8_t*)(c->arena + take(dpx));
    dj[i].out = (uint8_t*)(c->arena + take(dpx));
    dj[i].out_f32 = jobs[i].out_f32 ? (float*)(c->arena + take(px * 4)) : nullptr;
    dj[i].out_f64 = jobs[i].out_f64 ? (double*)(c->arena + take(px * 8)) : nullptr;
    dj[i].pitch = dp;
  }
  off = (off + 255) / 256 * 256;
  if (off >= c->arena_bytes) return fail(FSE_ENOMEM, "arena too small for the host path");
  for (int i = 0; i < n; ++i) {
    const fse_job_t& j = jobs[i];
    cudaError_t e = cudaMemcpy2DAsync((void*)dj[i].image, dj[i].pitch, j.image, j.pitch, j.W, j.H,
                                      cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync((void*)dj[i].mask, dj[i].pitch, j.mask, j.pitch, j.W, j.H,
                            cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "host-to-device copy");
  }
  int rc = run_batch(c, dj.data(), n, st, stats, off);
  if (rc) return rc;
  for (int i = 0; i < n; ++i) {
    const fse_job_t& j = jobs[i];
    cudaError_t e = cudaMemcpy2DAsync(j.out, j.pitch, dj[i].out, dj[i].pitch, j.W, j.H,
                                      cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && j.out_f32)
      e = cudaMemcpyAsync(j.out_f32, dj[i].out_f32, sizeof(float) * j.W * j.H,
                          cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && j.out_f64)
      e = cudaMemcpyAsync(j.out_f64, dj[i].out_f64, sizeof(double) * j.W * j.H,
                          cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_fail(e, "device-to-host copy");
  }
  return FSE_OK;
}

// Device bytes one job needs on the host-buffer path (inputs, outputs and the
// planner's state), an upper bound used for admission.
size_t job_device_bytes(const fse_job_t& j) {
  const fse_params_t& p = j.p;
  const size_t px = (size_t)j.W * j.H;
  const double grow = 1.0 + 4.0 * p.overlap * std::sqrt((double)std::max(p.n_tiles, 1)) /
                                std::max(1, std::min(j.W, j.H));
  const size_t ext_px = (size_t)(px * std::min(grow, (double)std::max(p.n_tiles, 1)) + 1);
  const size_t blocks = ext_px / ((size_t)p.block * p.block) + 4 * (size_t)p.n_tiles * (j.W + j.H) / p.block + 16;
  const size_t vbytes = p.precision == 64 ? 8 : 4;
  const size_t dpx = (size_t)((j.W + 15) & ~15) * j.H;         // 16-byte device rows
  const size_t vpad = (size_t)std::max(p.n_tiles, 1) * 3 * (j.H + 2 * (size_t)p.overlap) * vbytes;
  const size_t maps = 128 * (2 + (size_t)std::max(p.n_tiles, 1)) + 256;  // tensor maps
  return dpx * 3 + (j.out_f32 ? 4 * px : 0) + (j.out_f64 ? 8 * px : 0) + ext_px * vbytes + vpad + maps +
         blocks * (4 + 8 + 4 + 4 + 4 * MAX_CLS) + (size_t)(p.block + 2 * p.border) * (p.block + 2 * p.border) * 12 +
         (1 << 16);
}

}  // namespace fse

extern "C" {

int fse_plan_tiles(int32_t W, int32_t H, int32_t N, int32_t d, fse_tile_t* out, int32_t cap,
                   int32_t* n_out) {
  return fse::plan_tiles(W, H, N, d, out, cap, n_out);
}

int fse_plan_tiles_vertical(int32_t W, int32_t H, int32_t N, int32_t d, fse_tile_t* out,
                            int32_t cap, int32_t* n_out) {
  return fse::plan_tiles_vertical(W, H, N, d, out, cap, n_out);
}

int fse_context_create(fse_context_t** ctx, int device, size_t arena_bytes,
                       const char* tune_cache_path) {
  if (!ctx) return fse::fail(FSE_EINVAL, "NULL ctx");
  return fse::context_create(ctx, device, arena_bytes, tune_cache_path);
}

void fse_context_destroy(fse_context_t* ctx) { fse::context_destroy(ctx); }

int fse_context_set_option(fse_context_t* c, int32_t key, int64_t value) {
  if (!c) return fse::fail(FSE_EINVAL, "NULL ctx");
  switch (key) {
    case FSE_OPT_EXEC_MODE:
      if (value < FSE_EXEC_DAG || value > FSE_EXEC_PER_BLOCK) return fse::fail(FSE_EINVAL, "exec mode");
      c->exec_mode = (int)value;
      return FSE_OK;
    case FSE_OPT_TIMEOUT_MS:
      if (value < 1 || value > 3600 * 1000) return fse::fail(FSE_EINVAL, "timeout_ms");
      c->timeout_ms = (int)value;
      return FSE_OK;
    case FSE_OPT_CTAS_PER_SM:
      if (value < 0 || value > 64) return fse::fail(FSE_EINVAL, "ctas_per_sm");
      c->ctas_per_sm = (int)value;
      return FSE_OK;
    case FSE_OPT_USE_GRAPH:
      c->use_graph = value != 0;
      return FSE_OK;
    case FSE_OPT_DEBUG_CAPTURE:
      c->debug = value != 0;
      return FSE_OK;
    case FSE_OPT_TMA_STAGING:
      if (value < 0 || value > 2) return fse::fail(FSE_EINVAL, "tma staging");
      c->tma = (int)value;
      c->graph_jobs.clear();
      return FSE_OK;
    case FSE_OPT_F32_LAYOUT: {
      if (value < 0 || value > 3) return fse::fail(FSE_EINVAL, "f32 layout");
      fse::set_f32_layout(value == 0 ? 3 : (int)value);
      int nb = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fse::exec_kernel_ptr(fse::CLS_F32_32),
                                                    fse::exec_threads(fse::CLS_F32_32),
                                                    fse::exec_smem(fse::CLS_F32_32));
      c->occupancy[fse::CLS_F32_32] = nb > 0 ? nb : 1;
      c->graph_jobs.clear();
      return FSE_OK;
    }
    case FSE_OPT_F64_WARPS: {
      if (value != 0 && value != 2 && value != 4 && value != 5 && value != 6 && value != 8)
        return fse::fail(FSE_EINVAL, "f64 warps");
      fse::set_f64_warps(value == 0 ? 6 : (int)value);
      int nb = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fse::exec_kernel_ptr(fse::CLS_F32_64),
                                                    fse::exec_threads(fse::CLS_F32_64),
                                                    fse::exec_smem(fse::CLS_F32_64));
      c->occupancy[fse::CLS_F32_64] = nb > 0 ? nb : 1;
      c->graph_jobs.clear();
      return FSE_OK;
    }
    case FSE_OPT_DEBUG_TMA_STALL:
      c->dbg_tma_stall = value != 0;
      c->graph_jobs.clear();
      return FSE_OK;
    case FSE_OPT_KERNEL_TIMING:
      c->kernel_timing = value != 0;
      c->tev_used = 0;
      return FSE_OK;
    default:
      return fse::fail(FSE_EINVAL, "unknown option %d", key);
  }
}

int fse_extrapolate_batch(fse_context_t* ctx, const fse_job_t* jobs, int32_t n, void* cuda_stream,
                          fse_stats_t* stats) {
  return fse::run_batch(ctx, jobs, n, (cudaStream_t)cuda_stream, stats, 0);
}

int fse_extrapolate_host(fse_context_t* c, const fse_job_t* jobs, int32_t n, void* cuda_stream,
                         fse_stats_t* stats) {
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int rc = fse::enqueue_host(c, jobs, n, st, stats);
  if (rc) return rc;
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fse::cuda_fail(e, "cudaStreamSynchronize");
  return FSE_OK;
}

const char* fse_last_error(void) { return fse::last_error(); }

int32_t fse_autotune(fse_context_t* ctx, const fse_job_t* jobs, int32_t n, void* cuda_stream,
                     int32_t reps, double* trace, int32_t cap) {
  return fse::autotune(ctx, jobs, n, (cudaStream_t)cuda_stream, reps, trace, cap);
}

int32_t fse_context_kernel_times(fse_context_t* c, float* ms, int32_t cap) {
  if (!c || (!ms && cap > 0)) return fse::fail(FSE_EINVAL, "NULL argument");
  if (cudaSetDevice(c->device) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess)
    return fse::fail(FSE_ECUDA, "synchronize");
  int32_t n = 0;
  for (size_t i = 0; i + 1 < c->tev_used && n < cap; i += 2) {
    float v = 0;
    if (cudaEventElapsedTime(&v, c->tev[i], c->tev[i + 1]) != cudaSuccess)
      return fse::fail(FSE_ECUDA, "cudaEventElapsedTime");
    ms[n++] = v;
  }
  c->tev_used = 0;
  return n;
}

int32_t fse_debug_fetch(fse_context_t* c, int32_t* rec, int32_t* useq, int32_t cap,
                        int32_t* K_max) {
  if (!c || !rec || !useq || !K_max) return fse::fail(FSE_EINVAL, "NULL argument");
  if (!c->last_dbg_rec) return fse::fail(FSE_EINVAL, "no captured batch (FSE_OPT_DEBUG_CAPTURE)");
  if (cudaSetDevice(c->device) != cudaSuccess) return fse::fail(FSE_ECUDA, "cudaSetDevice");
  if (cudaDeviceSynchronize() != cudaSuccess) return fse::fail(FSE_ECUDA, "sync");
  const size_t n = (size_t)fse::MAX_CLS * c->last_dbg_cap;
  std::vector<int32_t> r(n * 4), u(n * fse::KMAX);
  if (cudaMemcpy(r.data(), c->last_dbg_rec, r.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(u.data(), c->last_dbg_useq, u.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
    return fse::fail(FSE_ECUDA, "debug copy");
  const int K = c->last_K_max;
  *K_max = K;
  int32_t m = 0;
  for (size_t i = 0; i < n && m < cap; ++i) {
    if (r[i * 4] < 0) continue;
    memcpy(rec + 4 * m, &r[i * 4], 16);
    for (int k = 0; k < K; ++k) useq[(size_t)m * K + k] = u[i * fse::KMAX + k];
    ++m;
  }
  return m;
}

int fse_debug_wait_probe(fse_context_t* c, int32_t timeout_us) {
  if (!c || timeout_us <= 0) return fse::fail(FSE_EINVAL, "bad arguments");
  if (cudaSetDevice(c->device) != cudaSuccess) return fse::fail(FSE_ECUDA, "cudaSetDevice");
  // a queue with one item whose producer never runs
  fse::QueueDev* q = reinterpret_cast<fse::QueueDev*>(c->arena);
  int32_t* slots = reinterpret_cast<int32_t*>(c->arena + 256);
  fse::QueueDev hq;
  memset(&hq, 0, sizeof(hq));
  hq.n_items = 1;
  if (cudaMemcpy(q, &hq, sizeof(hq), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(slots, 0xFF, 4) != cudaSuccess)
    return fse::fail(FSE_ECUDA, "probe setup");
  fse::ExecArgs a;
  memset(&a, 0, sizeof(a));
  a.c[0].q = q;
  a.c[0].slots = slots;
  a.c[0].cap = 1;
  a.single_item = -1;
  a.timeout_ns = (int64_t)timeout_us * 1000;
  cudaError_t e = fse::launch_probe(a, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return fse::cuda_fail(e, "probe");
  if (cudaMemcpy(&hq, q, sizeof(hq), cudaMemcpyDeviceToHost) != cudaSuccess)
    return fse::fail(FSE_ECUDA, "probe readback");
  c->graph_jobs.clear();  // the arena front was overwritten
  if (hq.error & fse::ERR_TIMEOUT) return fse::fail(FSE_ETIMEOUT, "wait ran out after %d us", timeout_us);
  return FSE_OK;
}

}  // extern "C"
