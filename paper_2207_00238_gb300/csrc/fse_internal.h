// Internal layout shared by the host executor (fse_api.cpp) and the kernels
// (fse_kernels.cu).  Plain structs only; every pointer is a device address.
#pragma once
#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace fse {

constexpr int KMAX = 256;       // iterations per block (coefficient list in smem)
constexpr int BMAX = 16;        // largest block size
constexpr int MAX_CLS = 3;      // work classes, one executor kernel each
constexpr double TAU_F64 = 1e-9;  // FP64 tie tolerance of the argmax

// Work classes: which executor kernel runs a job's blocks.
enum Cls : int32_t {
  CLS_F32_32 = 0,  // FP32, F = 32: one warp per block, spectrum in registers
  CLS_F32_64 = 1,  // FP32, F = 64: four warps per block
  CLS_F64 = 2,     // FP64 validation path, F = 32 or 64
};

enum Order : int32_t { ORDER_PHASED = 0, ORDER_RASTER = 1, ORDER_INDEPENDENT = 2 };

enum ErrBits : int32_t { ERR_TIMEOUT = 1, ERR_BOUNDS = 2 };

struct JobDev {
  const uint8_t* image;
  const uint8_t* mask;
  uint8_t* out;
  float* out_f32;  // may be null
  double* out_f64; // may be null
  int32_t W, H, pitch;
  int32_t b, B, S, F, K, order, P, D, cls;
  float rho_f, delta_f, gamma_f;
  double rho, delta, gamma;
  const float* wiso_f;   // S*S, rho^dist about the block centre
  const double* wiso_d;  // same in FP64
  // TMA staging of the support (F = 32 class): tensor maps of the mask and the
  // image (u8, W x H, row stride pitch) in device memory, or null; box widths
  // bw = roundup16(S + 15) (u8) and bv = roundup4(S + 3) (value plane, f32),
  // both S rows high
  const void* tm_mask;
  const void* tm_image;
  int32_t tma, bw, bv, pad_;
};

struct TileDev {
  int32_t job;
  int32_t x, y, w, h;      // core
  int32_t ex, ey, ew, eh;  // extended
  int32_t nbx, nby;        // tile-local block grid
  int32_t cls;
  int64_t map_off;  // first block of this tile in the block map
  int64_t val_off;  // first pixel of this tile's value plane (elements)
  const void* tm_val;  // tensor map of the value plane (f32, ew x eh, row stride vp), or null
  int32_t vp;          // row pitch of the value plane (elements): ew, rounded up to 4 for F = 32
  int32_t pad_;
};

// Per-class ready queue: an item is pushed once every block it depends on is
// done; a consumer reserves the next slot with one atomicAdd and waits
// (bounded by a progress watchdog) until that slot's item is pushed.  Slots
// are reserved in push order, so every pushed item has a consumer.
struct QueueDev {
  int32_t n_items;  // items of this class (written by the planner)
  int32_t head;     // next slot to reserve
  int32_t tail;     // next slot to push
  int32_t n_done;   // items finished (progress watchdog of waiting consumers)
  int32_t n_empty;
  int32_t n_core;   // lost blocks that touch their tile's core
  int32_t error;    // ErrBits
  int32_t error_info;
  int32_t n_roots;    // items without lost predecessors (fed roots, see ClassArgs::window)
  int32_t root_next;  // roots fed by finished blocks so far
  int32_t pad_[2];
};

struct ClassArgs {
  int2* items;      // (tile, I << 16 | J)
  int32_t* cnt;     // unfinished predecessors per item
  int32_t* slots;   // ready queue, -1 = not yet pushed
  QueueDev* q;
  int32_t cap;
  // Fed roots (batch calls, DAG mode): the first `window` items without lost
  // predecessors start in the queue, the others wait in `roots` (id order) and
  // a finished block pushes the next ones only while fewer than `window` items
  // wait, so released successors go first and the queue follows a few images
  // at a time (their supports stay in L2) instead of sweeping every processing
  // phase across the whole batch.  0 = every root at once.
  int32_t* roots;
  int32_t window;
};

constexpr int NW32 = 2;  // F = 32 executor: warps (independent workers) per CTA

// Continuous-batching server state (fse_server.cpp).  Work items of every
// resident request share one queue per class that lives as long as the
// server; a request joins by an "admit" command that the resident executor
// itself carries out (output init, lost-block enumeration, dependency counts,
// first pushes), so no other kernel needs SM resources while it runs.
constexpr int SRV_MAXJ = 256;      // job slots (resident requests)
constexpr int SRV_MAXT = 64;       // tiles per request
constexpr int SRV_CMD_RING = 1024; // posted, not yet taken admit commands per class
constexpr int32_t SRV_CMD_BIT = 0x40000000;  // queue entry = command index | SRV_CMD_BIT

struct ServerCmd {
  int32_t job, gen, n_tiles, pad_;
};

// Device-memory control block.  The host writes its fields with small
// stream-ordered copies (a record before the count that publishes it); the
// resident executor reads them with acquire loads.
struct ServerDevCtl {
  int32_t stop;       // host: 1 = exit once idle
  int32_t heartbeat;  // host: advanced by the server's worker; stale => host gone
  int32_t cmd_tail[MAX_CLS];  // host: admit commands posted per class
  int32_t cmd_taken[MAX_CLS]; // device: commands moved into the work queue
  int32_t pad_[3];
  ServerCmd cmd[MAX_CLS][SRV_CMD_RING];  // host
  int32_t cancel_gen[SRV_MAXJ];  // host: the slot's job of this generation is cancelled
  int32_t total[SRV_MAXJ];       // device: lost blocks of the slot's job (its admit)
  int32_t done[SRV_MAXJ];        // device: blocks of the slot's job finished
  int32_t gen[SRV_MAXJ];         // device: generation of the slot's current job
};

// Host-mapped block written by the device.
struct ServerHostCtl {
  int32_t done_gen[SRV_MAXJ];  // generation of the last job completed in the slot
  int32_t error;               // ErrBits
  int32_t pad_[3];
};

struct ExecArgs {
  const JobDev* jobs;
  const TileDev* tiles;
  int32_t* map;  // per tile block: item id within its class, -1 if not lost
  float* val_f;  // value planes of FP32 jobs (NaN = pending)
  double* val_d; // value planes of FP64 jobs
  ClassArgs c[MAX_CLS];
  int64_t timeout_ns;
  // optional per-item capture of the selected bins
  int32_t* dbg_rec;   // 4 per item and class: job, tile, I, J
  int32_t* dbg_useq;  // KMAX per item
  int32_t dbg_cap;
  // level-synchronous / per-block execution: only items of this level key
  int32_t level_mode;   // 0 = DAG, 1 = only items whose level == level
  int32_t level;
  int32_t single_item;  // >= 0: process exactly this item (per-block launch)
  int32_t dbg_tma_stall;  // test only: TMA stagings never complete their mbarrier phase
  // server mode (0 = one batch call): the resident executor of fse_server
  int32_t server;
  ServerDevCtl* srv;
  ServerHostCtl* host;  // device address of the host-mapped control block
  int32_t* level_of;    // per class item level (levels mode), class stride level_stride
  int64_t level_stride;
  // ordered enumeration (batch calls): per tile lost-block count, first item
  // id and assignment counter, so each tile's items get one contiguous id
  // range in tile (= job) order; null = ids in arrival order (one pass)
  int32_t* tile_cnt;
  int32_t* tile_base;
  int32_t* tile_ctr;
  int32_t n_tiles;
};

// Executor configuration of one context: which kernel variant runs each work
// class.  F = 32 layouts: 1 one spectrum column per lane, 2 paired bins, 3 row
// runs, 4 row runs with plain-load staging only (8 CTAs per SM); F = 64
// layouts: 2, 4, 8 warps per block, 5 four warps with a 96-row table, 6 four
// warps with paired bins.  unroll: K-loop unroll factor (1 or 2; 2 exists for
// F = 32 layouts 2, 3, 4 and F = 64 layout 6).
struct ExecCfg {
  int32_t lay32 = 4;
  int32_t lay64 = 6;
  int32_t unroll32 = 1;
  int32_t unroll64 = 1;
};

// Launch wrappers (fse_kernels.cu).  All are stream-ordered, none syncs.
void set_twiddles(const float2* tw_f, const double2* tw_d);  // 64 entries each
cudaError_t launch_init_out(const JobDev* jobs_dev, int n_jobs, int max_pixels,
                            cudaStream_t st);
cudaError_t launch_mark(const ExecArgs& a, int n_tiles, int max_tile_blocks, cudaStream_t st);
cudaError_t launch_deps(const ExecArgs& a, int cls, int cap, cudaStream_t st);
cudaError_t launch_exec(const ExecArgs& a, int cls, int grid, cudaStream_t st, const ExecCfg& cfg);
cudaError_t launch_probe(const ExecArgs& a, cudaStream_t st);
cudaError_t launch_repitch(const uint8_t* src, int src_pitch, size_t src_plane, uint8_t* dst, int dst_pitch,
                           size_t dst_plane, int W, int H, int planes, cudaStream_t st);
bool exec_cfg_valid(int cls, int layout, int unroll);  // a kernel variant exists
int exec_threads(int cls, const ExecCfg& cfg);
size_t exec_smem(int cls, const ExecCfg& cfg);
const void* exec_kernel_ptr(int cls, const ExecCfg& cfg);
cudaError_t exec_setup(int device);  // smem opt-in for every executor kernel

}  // namespace fse
