// Host side of the C ABI: tiling (Algorithm 1), the per-call planner and
// arena layout, the stream-ordered executor and CUDA-graph replay.
#include <algorithm>
#include <cstdarg>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <cuda.h>          // CUtensorMap and its enums (types only; libcuda is not linked)
#include <cudaTypedefs.h>  // PFN_cuTensorMapEncodeTiled
#include <cuda_runtime.h>

#include "../../include/fse.h"
#include "fse_context.h"
#include "fse_internal.h"

namespace fse {

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string g_err = "";
const char* last_error() { return g_err.c_str(); }

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(FSE_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define FSE_CUDA(call)                                   \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);  \
  } while (0)

// ---------------------------------------------------------------------------
// Algorithm 1 (Sec. III): tiles of about equal area, compact, in O(N).
// ---------------------------------------------------------------------------
int plan_tiles(int32_t W0, int32_t H0, int32_t N, int32_t d, fse_tile_t* out, int32_t cap,
               int32_t* n_out) {
  if (n_out) *n_out = 0;
  if (W0 <= 0 || H0 <= 0 || N <= 0 || d < 0 || out == nullptr || cap < N)
    return fail(FSE_EINVAL, "fse_plan_tiles: invalid arguments (W=%d H=%d N=%d d=%d cap=%d)", W0,
                H0, N, d, cap);
  // landscape orientation is assumed; a portrait image is tiled transposed
  const bool portrait = W0 < H0;
  const int64_t W = portrait ? H0 : W0, H = portrait ? W0 : H0;
  // Eq. (2): rows = max(1, round(sqrt(N / r))), r = W / H (Eq. 1), rounding
  // half up; sqrt(N H / W) >= n - 1/2  <=>  W (2n - 1)^2 <= 4 N H
  int64_t rows = 1;
  while (W * (2 * rows + 1) * (2 * rows + 1) <= 4 * (int64_t)N * H) ++rows;
  const int64_t extra = N % rows;  // rows with one tile more
  int64_t yT = 0;
  int32_t t = 0;
  for (int64_t i = 1; i <= rows; ++i) {
    const int64_t nC = N / rows + (i <= extra ? 1 : 0);                 // Eq. (3)
    int64_t hT = (H * nC) / N + ((H * nC) % N) / rows;                   // Eq. (4)
    if (i == rows) hT = H - yT;                                          // cover the image
    const int64_t wide = W % nC;  // tiles one pixel wider
    int64_t xT = 0;
    for (int64_t j = 1; j <= nC; ++j) {
      const int64_t wT = W / nC + (j <= wide ? 1 : 0);                   // Eq. (5)
      if (wT <= 0 || hT <= 0)
        return fail(FSE_EDEGENERATE,
                    "fse_plan_tiles: degenerate tile (row %lld: w=%lld h=%lld) for W=%d H=%d N=%d",
                    (long long)i, (long long)wT, (long long)hT, W0, H0, N);
      fse_tile_t tl;
      const int64_t x0 = std::max<int64_t>(0, xT - d), y0 = std::max<int64_t>(0, yT - d);
      const int64_t x1 = std::min<int64_t>(W, xT + wT + d), y1 = std::min<int64_t>(H, yT + hT + d);
      if (!portrait) {
        tl = {(int32_t)xT, (int32_t)yT, (int32_t)wT, (int32_t)hT,
              (int32_t)x0, (int32_t)y0, (int32_t)(x1 - x0), (int32_t)(y1 - y0)};
      } else {
        tl = {(int32_t)yT, (int32_t)xT, (int32_t)hT, (int32_t)wT,
              (int32_t)y0, (int32_t)x0, (int32_t)(y1 - y0), (int32_t)(x1 - x0)};
      }
      out[t++] = tl;
      xT += wT;
    }
    yT += hT;
  }
  if (n_out) *n_out = t;
  return FSE_OK;
}

// Vertical stripes (the paper's comparison tiling): N full-height tiles,
// widths W/N with the first W mod N one pixel wider.
int plan_tiles_vertical(int32_t W, int32_t H, int32_t N, int32_t d, fse_tile_t* out, int32_t cap,
                        int32_t* n_out) {
  if (n_out) *n_out = 0;
  if (W <= 0 || H <= 0 || N <= 0 || d < 0 || out == nullptr || cap < N)
    return fail(FSE_EINVAL, "fse_plan_tiles_vertical: invalid arguments");
  int64_t x = 0;
  for (int32_t j = 1; j <= N; ++j) {
    const int64_t w = W / N + (j <= W % N ? 1 : 0);
    if (w <= 0) return fail(FSE_EDEGENERATE, "fse_plan_tiles_vertical: %d stripes for width %d", N, W);
    const int64_t x0 = std::max<int64_t>(0, x - d), x1 = std::min<int64_t>(W, x + w + d);
    out[j - 1] = {(int32_t)x, 0, (int32_t)w, H, (int32_t)x0, 0, (int32_t)(x1 - x0), H};
    x += w;
  }
  if (n_out) *n_out = N;
  return FSE_OK;
}

int plan_tiles_mode(int32_t mode, int32_t W, int32_t H, int32_t N, int32_t d, fse_tile_t* out,
                    int32_t cap, int32_t* n_out) {
  return mode == FSE_TILING_VERTICAL ? plan_tiles_vertical(W, H, N, d, out, cap, n_out)
                                     : plan_tiles(W, H, N, d, out, cap, n_out);
}

// ---------------------------------------------------------------------------
// parameter checks
// ---------------------------------------------------------------------------
int check_job(const fse_job_t& j, int idx) {
  const fse_params_t& p = j.p;
  if (!j.image || !j.mask || !j.out) return fail(FSE_EINVAL, "job %d: NULL image/mask/out", idx);
  if (j.W <= 0 || j.H <= 0 || j.pitch < j.W)
    return fail(FSE_EINVAL, "job %d: bad size W=%d H=%d pitch=%d", idx, j.W, j.H, j.pitch);
  if (p.block < 1 || p.block > BMAX) return fail(FSE_EINVAL, "job %d: block %d not in 1..%d", idx, p.block, BMAX);
  if (p.border < 0) return fail(FSE_EINVAL, "job %d: border %d < 0", idx, p.border);
  if (p.fft != 32 && p.fft != 64) return fail(FSE_EINVAL, "job %d: fft %d must be 32 or 64", idx, p.fft);
  if (p.block + 2 * p.border > p.fft)
    return fail(FSE_EINVAL, "job %d: support %d larger than fft %d", idx, p.block + 2 * p.border, p.fft);
  if (p.K < 0 || p.K > KMAX) return fail(FSE_EINVAL, "job %d: K %d not in 0..%d", idx, p.K, KMAX);
  if (!(p.rho > 0 && p.rho <= 1)) return fail(FSE_EINVAL, "job %d: rho %g not in (0,1]", idx, p.rho);
  if (!(p.gamma > 0 && p.gamma < 2)) return fail(FSE_EINVAL, "job %d: gamma %g not in (0,2)", idx, p.gamma);
  if (!(p.delta >= 0)) return fail(FSE_EINVAL, "job %d: delta %g < 0", idx, p.delta);
  if (p.order < 0 || p.order > 2) return fail(FSE_EINVAL, "job %d: order %d", idx, p.order);
  if (p.n_tiles < 1 || p.overlap < 0) return fail(FSE_EINVAL, "job %d: n_tiles/overlap", idx);
  if (p.precision != 32 && p.precision != 64)
    return fail(FSE_EINVAL, "job %d: precision %d must be 32 or 64", idx, p.precision);
  if (p.tiling != FSE_TILING_ALG1 && p.tiling != FSE_TILING_VERTICAL)
    return fail(FSE_EINVAL, "job %d: tiling %d", idx, p.tiling);
  if ((j.W + p.block - 1) / p.block >= 32768 || (j.H + p.block - 1) / p.block >= 32768)
    return fail(FSE_EINVAL, "job %d: image too large for block %d", idx, p.block);
  return FSE_OK;
}

static inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
static int context_init(Context** out, int device, size_t arena_bytes, char* alias,
                        const char* tune_path) {
  *out = nullptr;
  int ndev = 0;
  FSE_CUDA(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) return fail(FSE_EINVAL, "device %d of %d", device, ndev);
  if (arena_bytes < (1u << 20)) return fail(FSE_EINVAL, "arena_bytes too small");
  FSE_CUDA(cudaSetDevice(device));
  Context* c = new Context();
  c->device = device;
  cudaDeviceProp prop;
  cudaError_t e = cudaGetDeviceProperties(&prop, device);
  if (e != cudaSuccess) { delete c; return cuda_fail(e, "cudaGetDeviceProperties"); }
  c->sm_count = prop.multiProcessorCount;
  if (alias) {
    c->arena = alias;
    c->owns_arena = false;
  } else {
    e = cudaMalloc(&c->arena, arena_bytes);
    if (e != cudaSuccess) {
      delete c;
      cudaGetLastError();
      return fail(FSE_ENOMEM, "cudaMalloc(%zu) for the arena failed", arena_bytes);
    }
  }
  c->arena_bytes = arena_bytes;
  float2 twf[64];
  double2 twd[64];
  const double two_pi = 6.283185307179586476925286766559;
  for (int q = 0; q < 64; ++q) {
    const double cs = std::cos(two_pi * q / 64.0), sn = std::sin(two_pi * q / 64.0);
    twd[q] = make_double2(cs, -sn);
    twf[q] = make_float2((float)cs, (float)-sn);
  }
  set_twiddles(twf, twd);
  e = exec_setup(device);
  if (e == cudaSuccess) e = cudaEventCreate(&c->ev0);
  if (e == cudaSuccess) e = cudaEventCreate(&c->ev1);
  if (e == cudaSuccess) e = cudaEventCreate(&c->ev2);
  if (e == cudaSuccess) e = cudaEventCreate(&c->ev3);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_host_free, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_graph_done, cudaEventDisableTiming);
  for (int k = 0; k < MAX_CLS && e == cudaSuccess; ++k) {
    e = cudaStreamCreateWithFlags(&c->cls_stream[k], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_join[k], cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    context_destroy(c);
    return cuda_fail(e, "context setup");
  }
  if (tune_path) {
    c->tune_path = tune_path;
    tune_load(c);
  }
  update_occupancy(c);
  *out = c;
  return FSE_OK;
}

void update_occupancy(Context* c) {
  for (int k = 0; k < MAX_CLS; ++k) {
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, exec_kernel_ptr(k, c->cfg), exec_threads(k, c->cfg),
                                                  exec_smem(k, c->cfg));
    c->occupancy[k] = std::max(1, nb);
  }
  c->graph_jobs.clear();  // a captured graph holds the old variants
}

int context_create(Context** out, int device, size_t arena_bytes, const char* tune_path) {
  return context_init(out, device, arena_bytes, nullptr, tune_path);
}

int context_create_alias(Context** out, int device, char* arena, size_t arena_bytes) {
  return context_init(out, device, arena_bytes, arena, nullptr);
}

void context_destroy(Context* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  cudaDeviceSynchronize();  // no queued copy may still read the staging buffers
  if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
  if (c->arena && c->owns_arena) cudaFree(c->arena);
  if (c->host_buf) cudaFreeHost(c->host_buf);
  if (c->graph_host_buf) cudaFreeHost(c->graph_host_buf);
  if (c->ev_host_free) cudaEventDestroy(c->ev_host_free);
  if (c->ev_graph_done) cudaEventDestroy(c->ev_graph_done);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  if (c->ev2) cudaEventDestroy(c->ev2);
  if (c->ev3) cudaEventDestroy(c->ev3);
  for (cudaEvent_t e : c->tev) cudaEventDestroy(e);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  for (int k = 0; k < MAX_CLS; ++k) {
    if (c->cls_stream[k]) cudaStreamDestroy(c->cls_stream[k]);
    if (c->ev_join[k]) cudaEventDestroy(c->ev_join[k]);
  }
  delete c;
}

// Grows a pinned staging buffer; the caller has made sure that no queued copy
// still reads it.
static int ensure_pinned(char** buf, size_t* cap_io, size_t bytes) {
  if (bytes <= *cap_io) return FSE_OK;
  if (*buf) cudaFreeHost(*buf);
  *buf = nullptr;
  *cap_io = 0;
  const size_t cap = align_up(std::max(bytes, (size_t)1 << 20), 1 << 16);
  cudaError_t e = cudaMallocHost(buf, cap);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(FSE_ENOMEM, "pinned host buffer of %zu bytes", cap);
  }
  *cap_io = cap;
  return FSE_OK;
}

// ---------------------------------------------------------------------------
// TMA tensor maps for the support staging.  The driver's encoder is reached
// through the runtime's entry-point query, so libcuda is not linked.
// ---------------------------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder() {
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  }();
  return fn;
}

// 2-D tiled map: W x H elements of `esize` bytes, row stride `stride` bytes,
// box bw x bh.  Out-of-range elements of a box read as zero.
static bool encode_map(CUtensorMap* m, const void* base, bool f32, int W, int H, size_t stride, int bw,
                       int bh) {
  const PFN_cuTensorMapEncodeTiled_v12000 enc = tmap_encoder();
  if (!enc) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)W, (cuuint64_t)H};
  const cuuint64_t strides[1] = {(cuuint64_t)stride};
  const cuuint32_t box[2] = {(cuuint32_t)bw, (cuuint32_t)bh};
  const cuuint32_t es[2] = {1, 1};
  return enc(m, f32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_UINT8, 2,
             const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// ---------------------------------------------------------------------------
// planning: tables for the device and the arena layout of one call
// ---------------------------------------------------------------------------
struct Plan {
  std::vector<JobDev> jobs;
  std::vector<TileDev> tiles;
  std::vector<float> wf;
  std::vector<double> wd;
  std::vector<size_t> w_off;  // per job offset into wf / wd
  std::vector<CUtensorMap> maps;  // per job: mask, image; then per tile: value plane
  int64_t total_blocks = 0;
  int64_t cap[MAX_CLS] = {0, 0, 0};
  int64_t val_f = 0, val_d = 0;  // elements
  int max_tile_blocks = 0, max_pixels = 0;
  int K_max = 0;
  int64_t pixels = 0;
  // arena offsets (bytes)
  size_t o_jobs, o_tiles, o_wf, o_wd, o_map, o_items[MAX_CLS], o_cnt[MAX_CLS], o_slots[MAX_CLS], o_roots[MAX_CLS], o_tcnt, o_tctr, o_tbase,
      o_valf, o_vald, o_q, o_level, o_dbg_rec, o_dbg_useq, o_tmap, upload_bytes, ff_begin, ff_end,
      zero_begin, zero_end, total;
};

static int build_plan(Context* c, const fse_job_t* jobs, int32_t n, size_t arena_offset, Plan& P) {
  P.jobs.resize(n);
  P.w_off.resize(n);
  std::vector<fse_tile_t> tl;
  for (int i = 0; i < n; ++i) {
    const fse_job_t& j = jobs[i];
    int rc = check_job(j, i);
    if (rc) return rc;
    const fse_params_t& p = j.p;
    tl.resize(p.n_tiles);
    int32_t nt = 0;
    rc = plan_tiles_mode(p.tiling, j.W, j.H, p.n_tiles, p.overlap, tl.data(), p.n_tiles, &nt);
    if (rc) return rc;
    JobDev& J = P.jobs[i];
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
    // TMA staging (F = 32 class): 16-byte aligned image and mask with a
    // 16-byte multiple row stride (the encoder's rules); the maps are filled
    // in once the arena layout is known
    J.bw = (J.S + 15 + 15) & ~15;
    J.bv = (J.S + 3 + 3) & ~3;
    // TMA staging exists in the F = 32 row-run layout 3 only
    J.tma = c->tma && J.cls == CLS_F32_32 && c->cfg.lay32 == 3 && ((uintptr_t)j.image & 15) == 0 &&
            ((uintptr_t)j.mask & 15) == 0 &&
            (j.pitch & 15) == 0 && J.bw <= 256 && J.S <= 256 && tmap_encoder() != nullptr;
    J.tm_mask = nullptr;
    J.tm_image = nullptr;
    J.pad_ = 0;
    // rho^dist about the block centre, dist from (B + (b-1)/2, B + (b-1)/2)
    P.w_off[i] = P.wf.size();
    const double mc = p.border + (p.block - 1) / 2.0;
    for (int m = 0; m < J.S; ++m)
      for (int q = 0; q < J.S; ++q) {
        const double w = std::pow(p.rho, std::sqrt((m - mc) * (m - mc) + (q - mc) * (q - mc)));
        P.wd.push_back(w);
        P.wf.push_back((float)w);
      }
    P.K_max = std::max(P.K_max, p.K);
    P.pixels += (int64_t)j.W * j.H;
    P.max_pixels = std::max(P.max_pixels, j.W * j.H);
    for (int t = 0; t < nt; ++t) {
      TileDev T;
      T.job = i;
      T.x = tl[t].x; T.y = tl[t].y; T.w = tl[t].w; T.h = tl[t].h;
      T.ex = tl[t].ex; T.ey = tl[t].ey; T.ew = tl[t].ew; T.eh = tl[t].eh;
      T.nbx = (T.ew + J.b - 1) / J.b;
      T.nby = (T.eh + J.b - 1) / J.b;
      T.cls = J.cls;
      T.vp = J.cls == CLS_F32_32 ? (T.ew + 3) & ~3 : T.ew;  // 16-byte rows for the TMA
      T.pad_ = 0;
      T.tm_val = nullptr;
      T.map_off = P.total_blocks;
      const int64_t nb = (int64_t)T.nbx * T.nby;
      P.total_blocks += nb;
      P.cap[J.cls] += nb;
      P.max_tile_blocks = (int)std::max<int64_t>(P.max_tile_blocks, nb);
      if (J.cls == CLS_F64) {
        T.val_off = P.val_d;
        P.val_d += (int64_t)T.vp * T.eh;
      } else {
        if (J.cls == CLS_F32_32) P.val_f = (P.val_f + 3) & ~(int64_t)3;  // 16-byte plane base for the TMA
        T.val_off = P.val_f;
        P.val_f += (int64_t)T.vp * T.eh;
      }
      P.tiles.push_back(T);
    }
  }
  for (int k = 0; k < MAX_CLS; ++k)
    if (P.cap[k] >= (1ll << 31)) return fail(FSE_EINVAL, "too many blocks in one call");
  // auto: the TMA copies take longer per block than plain loads but free the
  // load/store queue, which pays only when many blocks share each SM, so they
  // are used when the F = 32 class has at least four blocks per resident warp
  if (c->tma == 2 &&
      P.cap[CLS_F32_32] < 4ll * exec_grid(c, CLS_F32_32) * (exec_threads(CLS_F32_32, c->cfg) / 32))
    for (JobDev& J : P.jobs) J.tma = 0;
  // arena layout (bytes from the arena base + arena_offset)
  size_t o = arena_offset;
  auto take = [&](size_t bytes) { size_t r = align_up(o, 256); o = r + bytes; return r; };
  P.o_jobs = take(sizeof(JobDev) * n);
  P.o_tiles = take(sizeof(TileDev) * P.tiles.size());
  P.o_wf = take(sizeof(float) * P.wf.size());
  P.o_wd = take(sizeof(double) * P.wd.size());
  P.o_tmap = take(sizeof(CUtensorMap) * (2 * (size_t)n + P.tiles.size()));
  P.upload_bytes = o - P.o_jobs;
  P.o_map = take(sizeof(int32_t) * P.total_blocks);
  for (int k = 0; k < MAX_CLS; ++k) {
    P.o_items[k] = take(sizeof(int2) * P.cap[k]);
    P.o_cnt[k] = take(sizeof(int32_t) * P.cap[k]);
    P.o_roots[k] = take(sizeof(int32_t) * P.cap[k]);
    if (k == 0) P.o_tbase = take(sizeof(int32_t) * std::max<size_t>(1, P.tiles.size()));
  }
  int64_t capmax = std::max({P.cap[0], P.cap[1], P.cap[2]});
  P.o_level = take(c->exec_mode == FSE_EXEC_DAG ? 0 : sizeof(int32_t) * MAX_CLS * capmax);
  // region filled with 0xFF: ready slots (-1) and value planes (NaN = pending)
  o = align_up(o, 256);
  P.ff_begin = o;
  for (int k = 0; k < MAX_CLS; ++k) P.o_slots[k] = take(sizeof(int32_t) * P.cap[k]);
  P.o_valf = take(sizeof(float) * P.val_f);
  P.o_vald = take(sizeof(double) * P.val_d);
  P.o_dbg_rec = take(c->debug ? sizeof(int32_t) * 4 * MAX_CLS * capmax : 0);
  P.ff_end = align_up(o, 256);
  o = P.ff_end;
  P.zero_begin = o;
  P.o_q = take(sizeof(QueueDev) * MAX_CLS);
  P.o_tcnt = take(sizeof(int32_t) * std::max<size_t>(1, P.tiles.size()));
  P.o_tctr = take(sizeof(int32_t) * std::max<size_t>(1, P.tiles.size()));
  P.zero_end = align_up(o, 256);
  o = P.zero_end;
  P.o_dbg_useq = take(c->debug ? sizeof(int32_t) * KMAX * MAX_CLS * capmax : 0);
  P.total = align_up(o, 256);
  if (P.total > c->arena_bytes)
    return fail(FSE_ENOMEM, "call needs %zu arena bytes, context has %zu", P.total, c->arena_bytes);
  for (int i = 0; i < n; ++i) {
    P.jobs[i].wiso_f = reinterpret_cast<const float*>(c->arena + P.o_wf) + P.w_off[i];
    P.jobs[i].wiso_d = reinterpret_cast<const double*>(c->arena + P.o_wd) + P.w_off[i];
  }
  // tensor maps: device copies land at o_tmap with the rest of the upload
  P.maps.assign(2 * (size_t)n + P.tiles.size(), CUtensorMap{});
  const CUtensorMap* dmaps = reinterpret_cast<const CUtensorMap*>(c->arena + P.o_tmap);
  for (int i = 0; i < n; ++i) {
    JobDev& J = P.jobs[i];
    if (!J.tma) continue;
    const bool ok = encode_map(&P.maps[2 * i], J.mask, false, J.W, J.H, (size_t)J.pitch, J.bw, J.S) &&
                    encode_map(&P.maps[2 * i + 1], J.image, false, J.W, J.H, (size_t)J.pitch, J.bw, J.S);
    J.tma = ok;
    J.tm_mask = ok ? dmaps + 2 * i : nullptr;
    J.tm_image = ok ? dmaps + 2 * i + 1 : nullptr;
  }
  for (size_t t = 0; t < P.tiles.size(); ++t) {
    TileDev& T = P.tiles[t];
    const JobDev& J = P.jobs[T.job];
    if (!J.tma) continue;
    const float* plane = reinterpret_cast<const float*>(c->arena + P.o_valf) + T.val_off;
    if (encode_map(&P.maps[2 * n + t], plane, true, T.ew, T.eh, sizeof(float) * (size_t)T.vp, J.bv, J.S))
      T.tm_val = dmaps + 2 * n + t;
  }
  return FSE_OK;
}

static ExecArgs make_args(Context* c, const Plan& P) {
  ExecArgs a;
  memset(&a, 0, sizeof(a));
  char* base = c->arena;
  a.jobs = reinterpret_cast<const JobDev*>(base + P.o_jobs);
  a.tiles = reinterpret_cast<const TileDev*>(base + P.o_tiles);
  a.map = reinterpret_cast<int32_t*>(base + P.o_map);
  a.val_f = reinterpret_cast<float*>(base + P.o_valf);
  a.val_d = reinterpret_cast<double*>(base + P.o_vald);
  for (int k = 0; k < MAX_CLS; ++k) {
    a.c[k].items = reinterpret_cast<int2*>(base + P.o_items[k]);
    a.c[k].cnt = reinterpret_cast<int32_t*>(base + P.o_cnt[k]);
    a.c[k].slots = reinterpret_cast<int32_t*>(base + P.o_slots[k]);
    a.c[k].roots = reinterpret_cast<int32_t*>(base + P.o_roots[k]);
    if (k == 0) {  // ordered enumeration: each tile's items one contiguous id range
      a.tile_cnt = reinterpret_cast<int32_t*>(base + P.o_tcnt);
      a.tile_ctr = reinterpret_cast<int32_t*>(base + P.o_tctr);
      a.tile_base = reinterpret_cast<int32_t*>(base + P.o_tbase);
      a.n_tiles = (int32_t)P.tiles.size();
    }
    // fed roots in DAG mode: a window of root_window items per consumer
    // (a warp of the F = 32 executor, a CTA of the others)
    a.c[k].window = c->exec_mode == FSE_EXEC_DAG && c->root_window > 0
                        ? c->root_window * exec_grid(c, k) * (k == CLS_F32_32 ? exec_threads(k, c->cfg) / 32 : 1)
                        : 0;
    a.c[k].q = reinterpret_cast<QueueDev*>(base + P.o_q) + k;
    a.c[k].cap = (int32_t)P.cap[k];
  }
  a.timeout_ns = (int64_t)c->timeout_ms * 1000000ll;
  a.level_of = c->exec_mode == FSE_EXEC_DAG ? nullptr : reinterpret_cast<int32_t*>(base + P.o_level);
  a.level_stride = std::max({P.cap[0], P.cap[1], P.cap[2]});
  if (c->debug) {
    a.dbg_rec = reinterpret_cast<int32_t*>(base + P.o_dbg_rec);
    a.dbg_useq = reinterpret_cast<int32_t*>(base + P.o_dbg_useq);
    a.dbg_cap = (int32_t)std::max({P.cap[0], P.cap[1], P.cap[2]});
  }
  a.single_item = -1;
  a.dbg_tma_stall = c->dbg_tma_stall;
  return a;
}

int exec_grid(Context* c, int k) {
  int per_sm = c->occupancy[k];
  if (c->ctas_per_sm > 0) per_sm = std::min(c->ctas_per_sm, c->occupancy[k]);
  else if (c->tuned_ctas[k] > 0) per_sm = std::min(c->tuned_ctas[k], c->occupancy[k]);
  return std::max(1, per_sm * c->sm_count);
}

// Enqueues the whole pass on `st`.  Returns launches in *nl.
static int enqueue(Context* c, const Plan& P, const ExecArgs& a, cudaStream_t st, int* nl,
                   bool timed) {
  int launches = 0;
  const char* src = c->capturing ? c->graph_host_buf : c->host_buf;
  FSE_CUDA(cudaMemcpyAsync(c->arena + P.o_jobs, src, P.upload_bytes, cudaMemcpyHostToDevice, st));
  if (!c->capturing) {
    FSE_CUDA(cudaEventRecord(c->ev_host_free, st));
    c->host_buf_busy = true;
  }
  if (P.ff_end > P.ff_begin) FSE_CUDA(cudaMemsetAsync(c->arena + P.ff_begin, 0xFF, P.ff_end - P.ff_begin, st));
  FSE_CUDA(cudaMemsetAsync(c->arena + P.zero_begin, 0, P.zero_end - P.zero_begin, st));
  if (c->debug && P.o_dbg_useq < P.total)
    FSE_CUDA(cudaMemsetAsync(c->arena + P.o_dbg_useq, 0xFF, P.total - P.o_dbg_useq, st));
  FSE_CUDA(launch_init_out(a.jobs, (int)P.jobs.size(), P.max_pixels, st));
  FSE_CUDA(launch_mark(a, (int)P.tiles.size(), P.max_tile_blocks, st));
  launches += P.tiles.empty() ? 1 : 4;  // init_out; mark: count, scan, assign
  for (int k = 0; k < MAX_CLS; ++k)
    if (P.cap[k] > 0) {
      FSE_CUDA(launch_deps(a, k, (int)P.cap[k], st));
      ++launches;
    }
  if (timed) FSE_CUDA(cudaEventRecord(c->ev2, st));
  // kernel-timing events of this call: start, end, then start / end per class
  cudaEvent_t* kt = nullptr;
  if (c->kernel_timing && !c->capturing) {
    constexpr size_t per_call = 2 + 2 * MAX_CLS;
    while (c->tev_used + per_call > c->tev.size()) {
      cudaEvent_t e;
      FSE_CUDA(cudaEventCreate(&e));
      c->tev.push_back(e);
    }
    kt = &c->tev[c->tev_used];
    c->tev_used += per_call;
    int mask = 0;
    for (int k = 0; k < MAX_CLS; ++k) mask |= P.cap[k] > 0 ? 1 << k : 0;
    c->tev_cls_mask.push_back(mask);
    FSE_CUDA(cudaEventRecord(kt[0], st));
  }
  if (c->exec_mode == FSE_EXEC_DAG) {
    // One persistent launch per work class.  With several classes they run
    // concurrently on forked streams (joined back into st, so a captured graph
    // holds them as parallel nodes): the persistent CTAs of the class launched
    // first fill the GPU, and as they drain, the next class's CTAs take the
    // freed SMs, so each class's dependency tail overlaps the other's work.
    int order[MAX_CLS] = {CLS_F32_64, CLS_F32_32, CLS_F64};
    if (c->class_order == 1) std::swap(order[0], order[1]);
    int n_present = 0;
    for (int k = 0; k < MAX_CLS; ++k) n_present += P.cap[k] > 0;
    const bool fork = c->concurrent && n_present > 1;
    if (fork) FSE_CUDA(cudaEventRecord(c->ev_fork, st));
    bool forked[MAX_CLS] = {false, false, false};
    bool first = true;
    for (int oi = 0; oi < MAX_CLS; ++oi) {
      const int k = order[oi];
      if (P.cap[k] == 0) continue;
      forked[k] = fork && !first;  // the first class runs on st itself
      cudaStream_t sk = forked[k] ? c->cls_stream[k] : st;
      if (forked[k]) FSE_CUDA(cudaStreamWaitEvent(sk, c->ev_fork, 0));
      if (kt) FSE_CUDA(cudaEventRecord(kt[2 + 2 * k], sk));
      FSE_CUDA(launch_exec(a, k, exec_grid(c, k), sk, c->cfg));
      if (kt) FSE_CUDA(cudaEventRecord(kt[3 + 2 * k], sk));
      if (forked[k]) FSE_CUDA(cudaEventRecord(c->ev_join[k], sk));
      ++launches;
      first = false;
    }
    for (int k = 0; k < MAX_CLS; ++k)
      if (forked[k]) FSE_CUDA(cudaStreamWaitEvent(st, c->ev_join[k], 0));
  } else if (c->exec_mode == FSE_EXEC_LEVELS) {
    int max_levels = 1;
    for (const JobDev& J : P.jobs)
      if (J.order == ORDER_PHASED) max_levels = std::max(max_levels, J.P * J.P);
    for (int lv = 0; lv < max_levels; ++lv)
      for (int k = 0; k < MAX_CLS; ++k)
        if (P.cap[k] > 0) {
          ExecArgs b = a;
          b.level_mode = 1;
          b.level = lv;
          if (kt && lv == 0) FSE_CUDA(cudaEventRecord(kt[2 + 2 * k], st));
          FSE_CUDA(launch_exec(b, k, exec_grid(c, k), st, c->cfg));
          if (kt) FSE_CUDA(cudaEventRecord(kt[3 + 2 * k], st));
          ++launches;
        }
  }
  if (timed) FSE_CUDA(cudaEventRecord(c->ev3, st));
  if (kt) FSE_CUDA(cudaEventRecord(kt[1], st));
  *nl = launches;
  return FSE_OK;
}

// Per-block baseline: items read back, sorted by processing order, one launch each.
static int run_per_block(Context* c, const Plan& P, const ExecArgs& a, cudaStream_t st, int* nl) {
  QueueDev q[MAX_CLS];
  FSE_CUDA(cudaMemcpyAsync(q, a.c[0].q, sizeof(q), cudaMemcpyDeviceToHost, st));
  FSE_CUDA(cudaStreamSynchronize(st));
  struct Ent { int job, tile, phase, I, J, cls, id; };
  std::vector<Ent> ents;
  for (int k = 0; k < MAX_CLS; ++k) {
    const int n = std::min<int64_t>(q[k].n_items, P.cap[k]);
    if (n <= 0) continue;
    std::vector<int2> items(n);
    FSE_CUDA(cudaMemcpy(items.data(), a.c[k].items, sizeof(int2) * n, cudaMemcpyDeviceToHost));
    for (int id = 0; id < n; ++id) {
      const TileDev& T = P.tiles[items[id].x];
      const JobDev& J = P.jobs[T.job];
      const int I = items[id].y >> 16, Jb = items[id].y & 0xFFFF;
      const int ph = J.order == ORDER_PHASED ? (I % J.P) * J.P + (Jb % J.P) : 0;
      ents.push_back({T.job, items[id].x, ph, I, Jb, k, id});
    }
  }
  std::sort(ents.begin(), ents.end(), [](const Ent& x, const Ent& y) {
    if (x.job != y.job) return x.job < y.job;
    if (x.tile != y.tile) return x.tile < y.tile;
    if (x.phase != y.phase) return x.phase < y.phase;
    if (x.I != y.I) return x.I < y.I;
    return x.J < y.J;
  });
  for (const Ent& e : ents) {
    ExecArgs b = a;
    b.single_item = e.id;
    FSE_CUDA(launch_exec(b, e.cls, 1, st, c->cfg));
  }
  *nl += (int)ents.size();
  return FSE_OK;
}

static bool same_plan(const Context* c, const Plan& P, const fse_job_t* jobs, int32_t n) {
  if (!c->graph_exec || c->graph_jobs.size() != (size_t)n || c->graph_mode != c->exec_mode ||
      c->graph_debug != c->debug)
    return false;
  for (int i = 0; i < n; ++i)
    if (memcmp(&c->graph_jobs[i], &jobs[i], sizeof(fse_job_t)) != 0) return false;
  (void)P;
  return true;
}

int run_batch(Context* c, const fse_job_t* jobs, int32_t n, cudaStream_t st, fse_stats_t* stats,
              size_t arena_offset) {
  if (!c) return fail(FSE_EINVAL, "NULL context");
  if (n < 0 || (n > 0 && !jobs)) return fail(FSE_EINVAL, "bad job list");
  FSE_CUDA(cudaSetDevice(c->device));
  Plan P;
  int rc = build_plan(c, jobs, n, arena_offset, P);
  if (rc) return rc;
  if (stats) memset(stats, 0, sizeof(*stats));
  if (n == 0) return FSE_OK;
  const bool timed = stats != nullptr;
  const bool replay = c->exec_mode != FSE_EXEC_PER_BLOCK && c->use_graph && !timed && same_plan(c, P, jobs, n);
  if (!replay) {
    // host tables -> pinned staging buffer, once the previous call's copy out
    // of it has run (a replayed graph copies from its own buffer instead)
    if (c->host_buf_busy) {
      FSE_CUDA(cudaEventSynchronize(c->ev_host_free));
      c->host_buf_busy = false;
    }
    rc = ensure_pinned(&c->host_buf, &c->host_cap, P.upload_bytes);
    if (rc) return rc;
    memset(c->host_buf, 0, P.upload_bytes);
    memcpy(c->host_buf, P.jobs.data(), sizeof(JobDev) * n);
    memcpy(c->host_buf + (P.o_tiles - P.o_jobs), P.tiles.data(), sizeof(TileDev) * P.tiles.size());
    memcpy(c->host_buf + (P.o_wf - P.o_jobs), P.wf.data(), sizeof(float) * P.wf.size());
    memcpy(c->host_buf + (P.o_wd - P.o_jobs), P.wd.data(), sizeof(double) * P.wd.size());
    memcpy(c->host_buf + (P.o_tmap - P.o_jobs), P.maps.data(), sizeof(CUtensorMap) * P.maps.size());
  }
  const ExecArgs a = make_args(c, P);
  if (timed) FSE_CUDA(cudaEventRecord(c->ev0, st));
  int launches = 0;
  int replayed = 0;
  if (c->exec_mode == FSE_EXEC_PER_BLOCK) {
    rc = enqueue(c, P, a, st, &launches, false);
    if (rc) return rc;
    if (timed) FSE_CUDA(cudaEventRecord(c->ev2, st));
    rc = run_per_block(c, P, a, st, &launches);
    if (rc) return rc;
    if (timed) FSE_CUDA(cudaEventRecord(c->ev3, st));
  } else if (c->use_graph && !timed) {
    if (replay) {
      replayed = 1;
    } else {
      if (c->graph_exec) {
        // its copy node reads graph_host_buf, which is about to be rewritten
        if (c->graph_launched) FSE_CUDA(cudaEventSynchronize(c->ev_graph_done));
        cudaGraphExecDestroy(c->graph_exec);
      }
      c->graph_exec = nullptr;
      c->graph_launched = false;
      rc = ensure_pinned(&c->graph_host_buf, &c->graph_host_cap, P.upload_bytes);
      if (rc) return rc;
      memcpy(c->graph_host_buf, c->host_buf, P.upload_bytes);
      cudaGraph_t g;
      FSE_CUDA(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
      c->capturing = 1;
      rc = enqueue(c, P, a, c->cap_stream, &launches, false);
      c->capturing = 0;
      cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
      if (rc) return rc;
      if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
      e = cudaGraphInstantiate(&c->graph_exec, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
      c->graph_jobs.assign(jobs, jobs + n);
      c->graph_mode = c->exec_mode;
      c->graph_debug = c->debug;
      c->graph_launches = launches;
    }
    launches = c->graph_launches;
    FSE_CUDA(cudaGraphLaunch(c->graph_exec, st));
    FSE_CUDA(cudaEventRecord(c->ev_graph_done, st));
    c->graph_launched = true;
  } else {
    rc = enqueue(c, P, a, st, &launches, timed);
    if (rc) return rc;
  }
  if (timed) FSE_CUDA(cudaEventRecord(c->ev1, st));
  c->last_cap[0] = P.cap[0];
  c->last_cap[1] = P.cap[1];
  c->last_cap[2] = P.cap[2];
  c->last_q = reinterpret_cast<QueueDev*>(c->arena + P.o_q);
  c->last_dbg_rec = c->debug ? reinterpret_cast<int32_t*>(c->arena + P.o_dbg_rec) : nullptr;
  c->last_dbg_useq = c->debug ? reinterpret_cast<int32_t*>(c->arena + P.o_dbg_useq) : nullptr;
  c->last_dbg_cap = a.dbg_cap;
  c->last_K_max = P.K_max;
  if (!timed) return FSE_OK;
  FSE_CUDA(cudaStreamSynchronize(st));
  QueueDev q[MAX_CLS];
  FSE_CUDA(cudaMemcpy(q, c->last_q, sizeof(q), cudaMemcpyDeviceToHost));
  int err = 0;
  for (int k = 0; k < MAX_CLS; ++k) err |= q[k].error;
  stats->jobs = n;
  stats->tiles = (int32_t)P.tiles.size();
  stats->launches = launches;
  stats->graph_replayed = replayed;
  stats->pixels = P.pixels;
  for (int k = 0; k < MAX_CLS; ++k) {
    stats->lost_blocks += q[k].n_items;
    stats->empty_blocks += q[k].n_empty;
    stats->core_lost_blocks += q[k].n_core;
  }
  // bin-iterations: K * F^2 over modelled blocks, from per-class counts
  {
    int64_t per_cls[MAX_CLS] = {0, 0, 0};
    bool uniform[MAX_CLS] = {true, true, true};
    int64_t kf[MAX_CLS] = {-1, -1, -1};
    for (const JobDev& J : P.jobs) {
      const int64_t v = (int64_t)J.K * J.F * J.F;
      if (kf[J.cls] < 0) kf[J.cls] = v;
      else if (kf[J.cls] != v) uniform[J.cls] = false;
    }
    for (int k = 0; k < MAX_CLS; ++k) per_cls[k] = kf[k] < 0 ? 0 : kf[k];
    for (int k = 0; k < MAX_CLS; ++k) {
      stats->class_blocks[k] = q[k].n_items;
      stats->class_bin_iterations[k] = uniform[k] ? per_cls[k] * (q[k].n_items - q[k].n_empty) : -1;
      stats->bin_iterations += uniform[k] ? per_cls[k] * (q[k].n_items - q[k].n_empty) : -1;
    }
    if (stats->bin_iterations < 0) stats->bin_iterations = -1;
  }
  cudaEventElapsedTime(&stats->device_ms, c->ev0, c->ev1);
  cudaEventElapsedTime(&stats->exec_ms, c->ev2, c->ev3);
  if (err & ERR_TIMEOUT) return fail(FSE_ETIMEOUT, "a device wait exceeded %d ms", c->timeout_ms);
  if (err & ERR_BOUNDS) return fail(FSE_ENOMEM, "work-item capacity exceeded");
  for (int k = 0; k < MAX_CLS; ++k)
    if (c->exec_mode == FSE_EXEC_DAG && q[k].n_done != std::min<int64_t>(q[k].n_items, P.cap[k]))
      return fail(FSE_ECUDA, "class %d finished %d of %d blocks", k, q[k].n_done, q[k].n_items);
  return FSE_OK;
}

}  // namespace fse
