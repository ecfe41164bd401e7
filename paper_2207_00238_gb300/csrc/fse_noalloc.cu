// fse_extrapolate_noalloc: the batch pass without any allocation.
//
// Some callers cannot allocate device memory themselves: plug-ins whose host
// application owns the whole device-memory budget, code that must not call
// cudaMalloc because it can synchronize the device and stall a latency-bound
// loop, or environments where a per-call context and arena are not wanted.
// This entry point runs the same kernels as fse_extrapolate_batch, but every
// piece of scratch state lives in one fixed array of device memory that the
// library declares statically (loaded with the module, held by every GPU that
// loads the library until the process exits), and the job and tile tables are
// staged in static host arrays.  The call path makes no cudaMalloc, cudaFree,
// cudaMallocHost or other allocating call.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/fse.h"
#include "fse_context.h"
#include "fse_internal.h"

namespace fse {
namespace {

constexpr size_t kScratchBytes = size_t(64) << 20;  // FSE_NOALLOC_SCRATCH_BYTES
constexpr int kMaxJobs = 16;
constexpr int kMaxTiles = 1024;
constexpr int kMaxDevices = 64;
constexpr int kMaxWeights = kMaxJobs * 64 * 64;
const ExecCfg kCfg;  // the default executor of every class (no context to tune)

// The shared scratch.  In host code this name is only a stand-in for the
// device array, never a device address: the address comes from
// cudaGetSymbolAddress at set-up.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

struct DeviceSetup {
  bool done = false;
  unsigned char* scratch = nullptr;  // device address of g_scratch on this device
  int sm_count = 0;
};
DeviceSetup g_setup[kMaxDevices];

// Static host staging of the per-call tables (no heap).
JobDev g_jobs[kMaxJobs];
TileDev g_tiles[kMaxTiles];
float g_wf[kMaxWeights];
double g_wd[kMaxWeights];
fse_tile_t g_tl[kMaxTiles];
QueueDev g_q[MAX_CLS];
std::mutex g_lock;  // the scratch and the host tables serve one call at a time

// Once per device, with that device current.
int setup(int dev) {
  DeviceSetup& s = g_setup[dev];
  if (s.done) return FSE_OK;
  cudaError_t e = cudaGetSymbolAddress(reinterpret_cast<void**>(&s.scratch), g_scratch);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
  e = cudaDeviceGetAttribute(&s.sm_count, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
  float2 twf[64];
  double2 twd[64];
  const double two_pi = 6.283185307179586476925286766559;
  for (int q = 0; q < 64; ++q) {
    const double cs = std::cos(two_pi * q / 64.0), sn = std::sin(two_pi * q / 64.0);
    twd[q] = make_double2(cs, -sn);
    twf[q] = make_float2((float)cs, (float)-sn);
  }
  set_twiddles(twf, twd);
  e = exec_setup(dev);
  if (e != cudaSuccess) return cuda_fail(e, "kernel set-up");
  s.done = true;
  return FSE_OK;
}

inline size_t align_up(size_t v) { return (v + 255) / 256 * 256; }

int run(const fse_job_t* jobs, int32_t n, cudaStream_t st) {
  if (n < 0 || (n > 0 && !jobs)) return fail(FSE_EINVAL, "bad job list");
  if (n > kMaxJobs) return fail(FSE_EINVAL, "noalloc: %d jobs, at most %d per call", n, kMaxJobs);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return fail(FSE_EINVAL, "device %d", dev);
  int rc = setup(dev);
  if (rc) return rc;
  const DeviceSetup& S = g_setup[dev];
  if (n == 0) return FSE_OK;

  // ---- plan into the static host tables
  int nt = 0, nw = 0, max_pixels = 0, max_tile_blocks = 0;
  int w_off[kMaxJobs];
  int64_t total_blocks = 0, cap[MAX_CLS] = {0, 0, 0}, val_f = 0, val_d = 0;
  for (int i = 0; i < n; ++i) {
    const fse_job_t& j = jobs[i];
    rc = check_job(j, i);
    if (rc) return rc;
    const fse_params_t& p = j.p;
    if (nt + p.n_tiles > kMaxTiles)
      return fail(FSE_EINVAL, "noalloc: more than %d tiles in one call", kMaxTiles);
    int32_t got = 0;
    rc = plan_tiles_mode(p.tiling, j.W, j.H, p.n_tiles, p.overlap, g_tl + nt, p.n_tiles, &got);
    if (rc) return rc;
    JobDev& J = g_jobs[i];
    memset(&J, 0, sizeof(J));
    J.image = j.image;
    J.mask = j.mask;
    J.out = j.out;
    J.out_f32 = j.out_f32;
    J.out_f64 = j.out_f64;
    J.W = j.W;
    J.H = j.H;
    J.pitch = j.pitch;
    J.b = p.block;
    J.B = p.border;
    J.S = p.block + 2 * p.border;
    J.F = p.fft;
    J.K = p.K;
    J.order = p.order;
    J.P = (p.border + p.block - 1) / p.block + 1;
    J.D = (p.border + p.block - 1) / p.block;
    J.cls = p.precision == 64 ? CLS_F64 : (p.fft == 32 ? CLS_F32_32 : CLS_F32_64);
    J.rho = p.rho;
    J.delta = p.delta;
    J.gamma = p.gamma;
    J.rho_f = (float)p.rho;
    J.delta_f = (float)p.delta;
    J.gamma_f = (float)p.gamma;
    J.tm_mask = nullptr;  // no tensor maps here: the support is staged with plain loads
    J.tm_image = nullptr;
    J.tma = 0;
    J.bw = J.bv = 0;
    const double mc = p.border + (p.block - 1) / 2.0;
    w_off[i] = nw;  // the table's pointers are set once the layout is known
    for (int m = 0; m < J.S; ++m)
      for (int q = 0; q < J.S; ++q) {
        const double w = std::pow(p.rho, std::sqrt((m - mc) * (m - mc) + (q - mc) * (q - mc)));
        g_wd[nw] = w;
        g_wf[nw] = (float)w;
        ++nw;
      }
    max_pixels = j.W * j.H > max_pixels ? j.W * j.H : max_pixels;
    for (int t = 0; t < got; ++t) {
      const fse_tile_t& tl = g_tl[nt];
      TileDev& T = g_tiles[nt];
      T.job = i;
      T.x = tl.x; T.y = tl.y; T.w = tl.w; T.h = tl.h;
      T.ex = tl.ex; T.ey = tl.ey; T.ew = tl.ew; T.eh = tl.eh;
      T.nbx = (T.ew + J.b - 1) / J.b;
      T.nby = (T.eh + J.b - 1) / J.b;
      T.cls = J.cls;
      T.vp = T.ew;
      T.pad_ = 0;
      T.tm_val = nullptr;
      T.map_off = total_blocks;
      const int64_t nb = (int64_t)T.nbx * T.nby;
      total_blocks += nb;
      cap[J.cls] += nb;
      if (nb > max_tile_blocks) max_tile_blocks = (int)nb;
      if (J.cls == CLS_F64) {
        T.val_off = val_d;
        val_d += (int64_t)T.ew * T.eh;
      } else {
        T.val_off = val_f;
        val_f += (int64_t)T.ew * T.eh;
      }
      ++nt;
    }
  }

  // ---- layout inside the static scratch
  size_t o = 0;
  auto take = [&](size_t bytes) { const size_t r = align_up(o); o = r + bytes; return r; };
  const size_t o_jobs = take(sizeof(JobDev) * n), o_tiles = take(sizeof(TileDev) * nt);
  const size_t o_wf = take(sizeof(float) * nw), o_wd = take(sizeof(double) * nw);
  const size_t o_map = take(sizeof(int32_t) * total_blocks);
  size_t o_items[MAX_CLS], o_cnt[MAX_CLS], o_slots[MAX_CLS];
  for (int k = 0; k < MAX_CLS; ++k) {
    o_items[k] = take(sizeof(int2) * cap[k]);
    o_cnt[k] = take(sizeof(int32_t) * cap[k]);
  }
  const size_t ff_begin = align_up(o);
  o = ff_begin;
  for (int k = 0; k < MAX_CLS; ++k) o_slots[k] = take(sizeof(int32_t) * cap[k]);
  const size_t o_valf = take(sizeof(float) * val_f), o_vald = take(sizeof(double) * val_d);
  const size_t ff_end = align_up(o);
  o = ff_end;
  const size_t o_q = take(sizeof(QueueDev) * MAX_CLS);
  const size_t zero_end = align_up(o);
  if (zero_end > kScratchBytes)
    return fail(FSE_ENOMEM, "noalloc: the call needs %zu bytes of scratch, the static scratch holds %zu",
                zero_end, kScratchBytes);
  for (int k = 0; k < MAX_CLS; ++k)
    if (cap[k] >= (int64_t(1) << 31)) return fail(FSE_EINVAL, "too many blocks in one call");

  unsigned char* base = S.scratch;
  for (int i = 0; i < n; ++i) {
    g_jobs[i].wiso_f = reinterpret_cast<const float*>(base + o_wf) + w_off[i];
    g_jobs[i].wiso_d = reinterpret_cast<const double*>(base + o_wd) + w_off[i];
  }
  ExecArgs a;
  memset(&a, 0, sizeof(a));
  a.jobs = reinterpret_cast<const JobDev*>(base + o_jobs);
  a.tiles = reinterpret_cast<const TileDev*>(base + o_tiles);
  a.map = reinterpret_cast<int32_t*>(base + o_map);
  a.val_f = reinterpret_cast<float*>(base + o_valf);
  a.val_d = reinterpret_cast<double*>(base + o_vald);
  for (int k = 0; k < MAX_CLS; ++k) {
    a.c[k].items = reinterpret_cast<int2*>(base + o_items[k]);
    a.c[k].cnt = reinterpret_cast<int32_t*>(base + o_cnt[k]);
    a.c[k].slots = reinterpret_cast<int32_t*>(base + o_slots[k]);
    a.c[k].q = reinterpret_cast<QueueDev*>(base + o_q) + k;
    a.c[k].cap = (int32_t)cap[k];
  }
  a.timeout_ns = 20000ll * 1000000ll;
  a.single_item = -1;

  // ---- stream-ordered pass: tables up, state cleared (the scratch keeps the
  // previous call's contents), planner, one persistent launch per class
#define NOALLOC_CUDA(call)                              \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)
  NOALLOC_CUDA(cudaMemcpyAsync(base + o_jobs, g_jobs, sizeof(JobDev) * n, cudaMemcpyHostToDevice, st));
  NOALLOC_CUDA(cudaMemcpyAsync(base + o_tiles, g_tiles, sizeof(TileDev) * nt, cudaMemcpyHostToDevice, st));
  NOALLOC_CUDA(cudaMemcpyAsync(base + o_wf, g_wf, sizeof(float) * nw, cudaMemcpyHostToDevice, st));
  NOALLOC_CUDA(cudaMemcpyAsync(base + o_wd, g_wd, sizeof(double) * nw, cudaMemcpyHostToDevice, st));
  NOALLOC_CUDA(cudaMemsetAsync(base + ff_begin, 0xFF, ff_end - ff_begin, st));
  NOALLOC_CUDA(cudaMemsetAsync(base + ff_end, 0, zero_end - ff_end, st));
  NOALLOC_CUDA(launch_init_out(a.jobs, n, max_pixels, st));
  NOALLOC_CUDA(launch_mark(a, nt, max_tile_blocks, st));
  for (int k = 0; k < MAX_CLS; ++k)
    if (cap[k] > 0) NOALLOC_CUDA(launch_deps(a, k, (int)cap[k], st));
  for (int k = 0; k < MAX_CLS; ++k)
    if (cap[k] > 0) {
      int nb = 0;
      NOALLOC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, exec_kernel_ptr(k, kCfg),
                                                                 exec_threads(k, kCfg), exec_smem(k, kCfg)));
      NOALLOC_CUDA(launch_exec(a, k, (nb > 0 ? nb : 1) * S.sm_count, st, kCfg));
    }
  // the queue state comes back on the caller's stream: no device-wide sync
  NOALLOC_CUDA(cudaMemcpyAsync(g_q, base + o_q, sizeof(g_q), cudaMemcpyDeviceToHost, st));
  NOALLOC_CUDA(cudaStreamSynchronize(st));
#undef NOALLOC_CUDA
  int err = 0;
  for (int k = 0; k < MAX_CLS; ++k) err |= g_q[k].error;
  if (err & ERR_TIMEOUT) return fail(FSE_ETIMEOUT, "noalloc: a device wait ran out");
  if (err) return fail(FSE_ENOMEM, "noalloc: work-item capacity exceeded");
  for (int k = 0; k < MAX_CLS; ++k)
    if (g_q[k].n_done != (g_q[k].n_items < cap[k] ? g_q[k].n_items : cap[k]))
      return fail(FSE_ECUDA, "noalloc: class %d finished %d of %d blocks", k, g_q[k].n_done,
                  g_q[k].n_items);
  return FSE_OK;
}

}  // namespace
}  // namespace fse

extern "C" int fse_extrapolate_noalloc(const fse_job_t* jobs, int32_t n, void* cuda_stream) {
  std::lock_guard<std::mutex> lk(fse::g_lock);
  return fse::run(jobs, n, (cudaStream_t)cuda_stream);
}
