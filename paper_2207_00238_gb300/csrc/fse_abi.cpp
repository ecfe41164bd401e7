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
// class "cls ctas_per_sm layout unroll" and one line "order concurrent order"
// for the class launches.  A missing or foreign file is ignored.
void tune_load(Context* c) {
  FILE* f = fopen(c->tune_path.c_str(), "r");
  if (!f) return;
  char name[256] = {0};
  cudaDeviceProp prop;
  cudaGetDeviceProperties(&prop, c->device);
  if (fgets(name, sizeof(name), f)) {
    name[strcspn(name, "\r\n")] = 0;
    if (strcmp(name, prop.name) == 0) {
      char line[256];
      while (fgets(line, sizeof(line), f)) {
        int k, v, lay, un;
        if (sscanf(line, "order %d %d", &v, &lay) == 2) {
          c->concurrent = v != 0;
          c->class_order = lay == 1;
          continue;
        }
        if (sscanf(line, "%d %d %d %d", &k, &v, &lay, &un) != 4) continue;
        if (k < 0 || k >= MAX_CLS || v <= 0 || !exec_cfg_valid(k, k == CLS_F64 ? 0 : lay, un)) continue;
        c->tuned_ctas[k] = v;
        if (k == CLS_F32_32) { c->cfg.lay32 = lay; c->cfg.unroll32 = un; }
        if (k == CLS_F32_64) { c->cfg.lay64 = lay; c->cfg.unroll64 = un; }
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
    if (c->tuned_ctas[k] > 0)
      fprintf(f, "%d %d %d %d\n", k, c->tuned_ctas[k],
              k == CLS_F32_64 ? c->cfg.lay64 : (k == CLS_F32_32 ? c->cfg.lay32 : 0),
              k == CLS_F32_64 ? c->cfg.unroll64 : (k == CLS_F32_32 ? c->cfg.unroll32 : 1));
  fprintf(f, "order %d %d\n", c->concurrent, c->class_order);
  fclose(f);
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
  // median time of `reps` runs after one warm-up: of the class's own
  // persistent kernel when tuning a class (its start and end events, so the
  // other classes add no noise), of all iteration kernels for the class launch
  // order.  Trace rows: (class or -1 for the class launch order,
  // layout*10 + unroll or order code, ctas per SM, milliseconds)
  const int saved_timing = c->kernel_timing;
  c->kernel_timing = 1;
  auto time_cfg = [&](int cls, int code, int ctas, double* ms_out) -> int {
    constexpr size_t per_call = 2 + 2 * MAX_CLS;
    std::vector<double> ms;
    for (int r = 0; r < reps + 1; ++r) {
      fse_stats_t stt;
      const size_t used = c->tev_used;
      int rc = run_batch(c, jobs, n, st, &stt, 0);
      if (rc) return rc;
      double v = stt.exec_ms;
      if (cls >= 0 && c->tev_used == used + per_call) {
        float f = 0.f;
        if (cudaEventElapsedTime(&f, c->tev[used + 2 + 2 * cls], c->tev[used + 3 + 2 * cls]) == cudaSuccess)
          v = f;
      }
      if (c->tev_used == used + per_call) {  // keep the autotuner's runs out of the timing record
        c->tev_used = used;
        c->tev_cls_mask.pop_back();
      }
      if (r > 0) ms.push_back(v);
    }
    std::sort(ms.begin(), ms.end());
    *ms_out = ms[ms.size() / 2];
    if (trace && ran < cap) {
      trace[4 * ran] = cls;
      trace[4 * ran + 1] = code;
      trace[4 * ran + 2] = ctas;
      trace[4 * ran + 3] = *ms_out;
    }
    ++ran;
    return FSE_OK;
  };
  int rc = FSE_OK;
  // per class: executor layout x K-loop unroll x persistent CTAs per SM, with
  // the classes launched one after the other and the class timed alone
  const int saved_conc = c->concurrent;
  c->concurrent = 0;
  struct Cand { int lay, un, ctas_span; };
  const Cand cand64[] = {{6, 1, 1}, {6, 2, 1}, {4, 1, 1}, {5, 1, 1}, {2, 1, 1}, {8, 1, 1}};
  const Cand cand32[] = {{3, 1, 3}, {3, 2, 3}, {4, 1, 3}, {4, 2, 3}, {2, 1, 3}, {2, 2, 3}, {1, 1, 3}};
  for (int cls : {CLS_F32_64, CLS_F32_32}) {
    if (!present[cls] || rc != FSE_OK) continue;
    const Cand* cands = cls == CLS_F32_64 ? cand64 : cand32;
    const int ncand = cls == CLS_F32_64 ? 6 : 7;
    int& lay = cls == CLS_F32_64 ? c->cfg.lay64 : c->cfg.lay32;
    int& un = cls == CLS_F32_64 ? c->cfg.unroll64 : c->cfg.unroll32;
    double best = 1e30;
    int best_lay = lay, best_un = un, best_ctas = 0;
    for (int ci = 0; ci < ncand && rc == FSE_OK; ++ci) {
      lay = cands[ci].lay;
      un = cands[ci].un;
      update_occupancy(c);
      const int occ = c->occupancy[cls];
      for (int k = occ; k >= 1 && k >= occ - cands[ci].ctas_span && rc == FSE_OK; --k) {
        c->ctas_per_sm = k;
        double ms;
        rc = time_cfg(cls, lay * 10 + un, k, &ms);
        if (rc == FSE_OK && ms < best) {
          best = ms;
          best_lay = lay;
          best_un = un;
          best_ctas = k;
        }
      }
    }
    lay = best_lay;
    un = best_un;
    update_occupancy(c);
    c->tuned_ctas[cls] = best_ctas;
  }
  c->ctas_per_sm = saved_ctas;
  c->concurrent = saved_conc;
  // class launches of a mixed call: one after the other, or concurrent on
  // forked streams with either class first (order code 0: sequential,
  // 1: concurrent F = 64 first, 2: concurrent F = 32 first)
  if (rc == FSE_OK && present[CLS_F32_32] + present[CLS_F32_64] + present[CLS_F64] > 1) {
    double best = 1e30;
    int best_code = 0;
    for (int code = 0; code < 3 && rc == FSE_OK; ++code) {
      c->concurrent = code != 0;
      c->class_order = code == 2;
      double ms;
      rc = time_cfg(-1, code, 0, &ms);
      if (rc == FSE_OK && ms < best) {
        best = ms;
        best_code = code;
      }
    }
    c->concurrent = best_code != 0;
    c->class_order = best_code == 2;
  }
  c->exec_mode = saved_mode;
  c->use_graph = saved_graph;
  c->kernel_timing = saved_timing;
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
  // Copies move whole contiguous planes (a strided copy of short rows runs far
  // below the link's bandwidth): a job whose host rows are packed (pitch = W)
  // but whose device rows are padded goes through a packed area and a re-pitch
  // kernel.  The packed area lies where the call's plan will be built: the
  // re-pitch runs before the plan is uploaded, and the outputs are packed there
  // after the last kernel that reads the plan, all in stream order.
  size_t packed = 0;
  for (int i = 0; i < n; ++i)
    if (jobs[i].pitch == jobs[i].W && dj[i].pitch != jobs[i].W) packed += 2 * (size_t)jobs[i].W * jobs[i].H;
  // (not with debug capture, whose records live in the plan region and are read after the call)
  const bool use_packed = !c->debug && off + packed + 256 * (size_t)n <= c->arena_bytes;
  std::vector<size_t> pk(n, 0);
  {
    size_t o = off;
    for (int i = 0; i < n; ++i) {
      pk[i] = o;
      if (jobs[i].pitch == jobs[i].W && dj[i].pitch != jobs[i].W)
        o = (o + 2 * (size_t)jobs[i].W * jobs[i].H + 255) / 256 * 256;
    }
  }
  for (int i = 0; i < n; ++i) {
    const fse_job_t& j = jobs[i];
    const size_t px = (size_t)j.W * j.H;
    cudaError_t e;
    if (j.pitch == j.W && dj[i].pitch == j.W) {  // both packed: plain copies
      e = cudaMemcpyAsync((void*)dj[i].image, j.image, px, cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess) e = cudaMemcpyAsync((void*)dj[i].mask, j.mask, px, cudaMemcpyHostToDevice, st);
    } else if (j.pitch == j.W && use_packed) {
      // image then mask into the packed area, one re-pitch for both planes
      // (the device mask follows the image at a fixed distance)
      char* p = c->arena + pk[i];
      e = cudaMemcpyAsync(p, j.image, px, cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess) e = cudaMemcpyAsync(p + px, j.mask, px, cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess)
        e = launch_repitch((const uint8_t*)p, j.W, px, (uint8_t*)dj[i].image, dj[i].pitch,
                           (size_t)((const char*)dj[i].mask - (const char*)dj[i].image), j.W, j.H, 2, st);
    } else {
      e = cudaMemcpy2DAsync((void*)dj[i].image, dj[i].pitch, j.image, j.pitch, j.W, j.H,
                            cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess)
        e = cudaMemcpy2DAsync((void*)dj[i].mask, dj[i].pitch, j.mask, j.pitch, j.W, j.H,
                              cudaMemcpyHostToDevice, st);
    }
    if (e != cudaSuccess) return cuda_fail(e, "host-to-device copy");
  }
  int rc = run_batch(c, dj.data(), n, st, stats, off);
  if (rc) return rc;
  for (int i = 0; i < n; ++i) {
    const fse_job_t& j = jobs[i];
    const size_t px = (size_t)j.W * j.H;
    cudaError_t e;
    if (j.pitch == j.W && dj[i].pitch == j.W) {
      e = cudaMemcpyAsync(j.out, dj[i].out, px, cudaMemcpyDeviceToHost, st);
    } else if (j.pitch == j.W && use_packed) {
      char* p = c->arena + pk[i];
      e = launch_repitch(dj[i].out, dj[i].pitch, 0, (uint8_t*)p, j.W, 0, j.W, j.H, 1, st);
      if (e == cudaSuccess) e = cudaMemcpyAsync(j.out, p, px, cudaMemcpyDeviceToHost, st);
    } else {
      e = cudaMemcpy2DAsync(j.out, j.pitch, dj[i].out, dj[i].pitch, j.W, j.H, cudaMemcpyDeviceToHost, st);
    }
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
      c->graph_jobs.clear();  // the grid (and the root window) of a captured graph
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
      const int lay = value == 0 ? 4 : (int)value;
      if (value < 0 || value > 4) return fse::fail(FSE_EINVAL, "f32 layout");
      c->cfg.lay32 = lay;
      if (!fse::exec_cfg_valid(fse::CLS_F32_32, lay, c->cfg.unroll32)) c->cfg.unroll32 = 1;
      fse::update_occupancy(c);
      return FSE_OK;
    }
    case FSE_OPT_F64_WARPS: {
      const int lay = value == 0 ? 6 : (int)value;
      if (!fse::exec_cfg_valid(fse::CLS_F32_64, lay, 1)) return fse::fail(FSE_EINVAL, "f64 warps");
      c->cfg.lay64 = lay;
      if (!fse::exec_cfg_valid(fse::CLS_F32_64, lay, c->cfg.unroll64)) c->cfg.unroll64 = 1;
      fse::update_occupancy(c);
      return FSE_OK;
    }
    case FSE_OPT_F32_UNROLL:
    case FSE_OPT_F64_UNROLL: {
      const int cls = key == FSE_OPT_F32_UNROLL ? fse::CLS_F32_32 : fse::CLS_F32_64;
      const int un = value == 0 ? 1 : (int)value;
      const int lay = cls == fse::CLS_F32_32 ? c->cfg.lay32 : c->cfg.lay64;
      if (!fse::exec_cfg_valid(cls, lay, un)) return fse::fail(FSE_EINVAL, "unroll %d for layout %d", un, lay);
      (cls == fse::CLS_F32_32 ? c->cfg.unroll32 : c->cfg.unroll64) = un;
      fse::update_occupancy(c);
      return FSE_OK;
    }
    case FSE_OPT_SERVER_CLASSES:
      if (value < 1 || value > 3) return fse::fail(FSE_EINVAL, "server classes %d", (int)value);
      c->server_classes = (int)value;
      return FSE_OK;
    case FSE_OPT_ROOT_WINDOW:
      if (value < 0 || value > 64) return fse::fail(FSE_EINVAL, "root window %d", (int)value);
      c->root_window = (int)value;
      c->graph_jobs.clear();
      return FSE_OK;
    case FSE_OPT_CLASS_LAUNCH:
      if (value < 0 || value > 2) return fse::fail(FSE_EINVAL, "class launch %d", (int)value);
      c->concurrent = value != 0;
      c->class_order = value == 2;
      c->graph_jobs.clear();
      return FSE_OK;
    case FSE_OPT_DEBUG_TMA_STALL:
      c->dbg_tma_stall = value != 0;
      c->graph_jobs.clear();
      return FSE_OK;
    case FSE_OPT_KERNEL_TIMING:
      c->kernel_timing = value != 0;
      c->tev_used = 0;
      c->tev_cls_mask.clear();
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

// Timed calls store 2 + 2 * MAX_CLS events each: start and end of the whole
// execution, then start and end per class.
static constexpr size_t kEventsPerCall = 2 + 2 * fse::MAX_CLS;

int32_t fse_context_class_times(fse_context_t* c, float* ms, int32_t cap) {
  if (!c || (!ms && cap > 0)) return fse::fail(FSE_EINVAL, "NULL argument");
  if (cudaSetDevice(c->device) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess)
    return fse::fail(FSE_ECUDA, "synchronize");
  int32_t n = 0;
  for (size_t call = 0; (call + 1) * kEventsPerCall <= c->tev_used && n < cap; ++call, ++n) {
    const cudaEvent_t* e = &c->tev[call * kEventsPerCall];
    for (int k = 0; k < fse::MAX_CLS; ++k) {
      float v = 0;
      if ((c->tev_cls_mask[call] >> k) & 1)
        if (cudaEventElapsedTime(&v, e[2 + 2 * k], e[3 + 2 * k]) != cudaSuccess)
          return fse::fail(FSE_ECUDA, "cudaEventElapsedTime");
      ms[(size_t)n * fse::MAX_CLS + k] = v;
    }
  }
  return n;
}

int32_t fse_context_kernel_times(fse_context_t* c, float* ms, int32_t cap) {
  if (!c || (!ms && cap > 0)) return fse::fail(FSE_EINVAL, "NULL argument");
  if (cudaSetDevice(c->device) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess)
    return fse::fail(FSE_ECUDA, "synchronize");
  int32_t n = 0;
  for (size_t call = 0; (call + 1) * kEventsPerCall <= c->tev_used && n < cap; ++call) {
    float v = 0;
    if (cudaEventElapsedTime(&v, c->tev[call * kEventsPerCall], c->tev[call * kEventsPerCall + 1]) !=
        cudaSuccess)
      return fse::fail(FSE_ECUDA, "cudaEventElapsedTime");
    ms[n++] = v;
  }
  c->tev_used = 0;
  c->tev_cls_mask.clear();
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
