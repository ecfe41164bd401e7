/*
 * fse.h -- C ABI of a single-GPU (sm_103a) library for Frequency Selective
 * Extrapolation (FSE) on the overlapping tiles of Seiler & Kaup's tiling
 * algorithm ("Distributed Parallel Image Signal Extrapolation Framework using
 * Message Passing Interface").
 *
 * Method (paper Sec. II and Sec. III):
 *   - The image is cut into N compact tiles by Algorithm 1 (Eqs. 1-5); each
 *     tile is grown by a stripe of d pixels on every side and extrapolated as
 *     a standalone image; the cores are merged into the output.
 *   - Inside a tile, every b x b block holding a lost pixel is modelled from
 *     its (b+2B) x (b+2B) support as a sparse sum of F x F Fourier basis
 *     functions, chosen greedily over K iterations (Sec. II): weights
 *     rho^dist on known pixels, delta*rho^dist on pixels reconstructed by
 *     earlier blocks, 0 on still-lost pixels; per iteration the bin u with
 *     the largest weighted residual energy |R_w(u)|^2 is picked, its
 *     coefficient grows by gamma*R_w(u)/W(0), and the shifted weight spectrum
 *     gamma*R_w(u)/W(0) * W(k-u) is subtracted from R_w; the model's real part
 *     fills the block's lost pixels.
 *
 * Conventions for every call:
 *   - Return value: FSE_OK (0) or a negative FSE_E* status.  No call aborts,
 *     traps or exits the process.  fse_last_error() gives a thread-local text.
 *   - Images are 8-bit, row-major with a row pitch in bytes; mask != 0 marks a
 *     lost pixel.  Known pixels are copied to the output unchanged.
 *   - "Device pointer" means memory of the context's GPU (cudaMalloc, or a
 *     torch tensor's data_ptr()); "host pointer" means ordinary or pinned
 *     host memory.  The caller keeps ownership of every buffer it passes.
 *   - Handles are created and destroyed only by the library.
 */
#ifndef FSE_H
#define FSE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define FSE_OK 0
#define FSE_EINVAL (-1)      /* bad argument or parameter                     */
#define FSE_EDEGENERATE (-2) /* Algorithm 1 produced a tile with w<=0 or h<=0 */
#define FSE_ENOMEM (-3)      /* arena or host allocation too small            */
#define FSE_EBUSY (-4)       /* server queue full                             */
#define FSE_ETIMEOUT (-5)    /* a bounded device or host wait ran out         */
#define FSE_ECUDA (-6)       /* a CUDA runtime call failed                    */
#define FSE_ENOTFOUND (-7)   /* unknown server ticket                         */
#define FSE_ECANCELLED (-8)  /* request cancelled or server shut down         */

/* ---- processing order of the lost blocks inside one tile ----------------
 * The paper defers the order to an earlier FSE publication (Sec. II) and
 * does not define it; these are the library's readings.
 *   PHASED      : P = ceil(B/b)+1; blocks sorted by ((I mod P)*P + J mod P, I, J).
 *                 Two blocks of one phase never lie in each other's support,
 *                 so a phase runs in parallel with sequential semantics.
 *   RASTER      : blocks sorted by (I, J).
 *   INDEPENDENT : no block ever uses another block's reconstruction. */
#define FSE_ORDER_PHASED 0
#define FSE_ORDER_RASTER 1
#define FSE_ORDER_INDEPENDENT 2

/* ---- tiling (Algorithm 1, Eqs. 1-5; overlap stripe of Sec. III) ---------- */
typedef struct fse_tile_t {
    int32_t x, y, w, h;     /* core tile: offset and size (Algorithm 1)      */
    int32_t ex, ey, ew, eh; /* core grown by d on each side, clipped to image */
} fse_tile_t;

/*
 * fse_plan_tiles -- Algorithm 1 with the overlap stripe d.  Host only, pure,
 * thread-safe.
 *   W, H  : image width and height (> 0).  W < H is tiled with the axes
 *           swapped and swapped back ("landscape assumed", Sec. III).
 *   N     : number of tiles (> 0);  d : overlap stripe width (>= 0).
 *   out   : caller-owned array of cap entries; tiles come row by row.
 *   n_out : receives N on success.
 * Eq. (2) rounds half up, evaluated in exact integers.
 * Errors: FSE_EINVAL (non-positive sizes, d < 0, cap < N, NULL out),
 *         FSE_EDEGENERATE (a tile of width or height <= 0, e.g. 32x32, N=23).
 */
int fse_plan_tiles(int32_t W, int32_t H, int32_t N, int32_t d, fse_tile_t* out, int32_t cap,
                   int32_t* n_out);

/* ---- parameters of one extrapolation job -------------------------------- */
typedef struct fse_params_t {
    int32_t block;  /* b: block size (1..16)                                 */
    int32_t border; /* B: support border; support S = b + 2B                 */
    int32_t fft;    /* F: DFT size per axis, 32 or 64, F >= S                */
    int32_t K;      /* iterations (0..256)                                   */
    double rho;     /* weight decay, 0 < rho <= 1                            */
    double delta;   /* weight factor of reconstructed pixels, >= 0           */
    double gamma;   /* coefficient step, 0 < gamma < 2                       */
    int32_t order;  /* FSE_ORDER_*                                           */
    int32_t n_tiles;   /* N of Algorithm 1 (>= 1)                            */
    int32_t overlap;   /* d (>= 0)                                           */
    int32_t precision; /* 32: FP32 fast path; 64: FP64 validation path       */
    int32_t tiling;    /* FSE_TILING_ALG1 (0) or FSE_TILING_VERTICAL (1)      */
} fse_params_t;

/* Tilings.  ALG1: Algorithm 1 (Eqs. 1-5).  VERTICAL: the baseline the paper
 * compares against (Sec. III): N full-height stripes, widths distributed as in
 * Eq. 5 (the first W mod N stripes one pixel wider); it needs no landscape
 * swap.  Both are extended by the overlap stripe d. */
#define FSE_TILING_ALG1 0
#define FSE_TILING_VERTICAL 1

/* fse_plan_tiles_vertical -- the VERTICAL tiling with overlap d; arguments,
 * output layout and errors as for fse_plan_tiles. */
int fse_plan_tiles_vertical(int32_t W, int32_t H, int32_t N, int32_t d, fse_tile_t* out,
                            int32_t cap, int32_t* n_out);

typedef struct fse_job_t {
    const uint8_t* image; /* W x H, row pitch `pitch` bytes                   */
    const uint8_t* mask;  /* same layout; != 0 marks a lost pixel             */
    uint8_t* out;         /* same layout; receives the extrapolated image     */
    float* out_f32;       /* optional (NULL): W x H floats, row stride W; the
                             unrounded model at lost pixels, the input elsewhere */
    double* out_f64;      /* optional (NULL): as out_f32 in FP64 (exact model
                             values of the FP64 validation path)               */
    int32_t W, H, pitch;
    fse_params_t p;
} fse_job_t;

typedef struct fse_stats_t {
    int64_t lost_blocks;      /* block runs, overlap duplicates included     */
    int64_t core_lost_blocks; /* lost blocks counted once per image           */
    int64_t empty_blocks;     /* blocks whose support had sum(w) == 0        */
    int64_t pixels;           /* input pixels, sum of W*H                     */
    int64_t bin_iterations;   /* sum over modelled blocks of K*F*F            */
    int32_t jobs, tiles, launches, graph_replayed;
    float device_ms;          /* stream time of the whole call (events)       */
    float exec_ms;            /* stream time of the iteration kernels         */
    /* per work class (0: FP32 F = 32, 1: FP32 F = 64, 2: FP64): block runs,
       and K*F*F over its modelled blocks (-1 when K varies within the class) */
    int64_t class_blocks[3];
    int64_t class_bin_iterations[3];
} fse_stats_t;

/* ---- context: one GPU, one device arena ---------------------------------- */
typedef struct fse_context fse_context_t;

/*
 * fse_context_create -- binds the calling thread's work to `device`, reserves
 * `arena_bytes` of device memory (cudaMalloc, once) for all per-call state and
 * reads the autotuner cache `tune_cache_path` (may be NULL; a missing file is
 * not an error).  Errors: FSE_EINVAL, FSE_ENOMEM, FSE_ECUDA.
 */
int fse_context_create(fse_context_t** ctx, int device, size_t arena_bytes,
                       const char* tune_cache_path);
void fse_context_destroy(fse_context_t* ctx);

/* Options (fse_context_set_option). */
#define FSE_OPT_EXEC_MODE 1     /* FSE_EXEC_*                                  */
#define FSE_OPT_TIMEOUT_MS 2    /* bound of every device wait (default 20000)  */
#define FSE_OPT_CTAS_PER_SM 3   /* 0 = autotuned / occupancy-derived          */
#define FSE_OPT_USE_GRAPH 4     /* 1 = capture each batch in a CUDA graph and
                                   replay it while the job set is unchanged    */
#define FSE_OPT_DEBUG_CAPTURE 5 /* 1 = record each block's selected bins       */
#define FSE_OPT_F64_WARPS 7     /* layout of this context's F = 64 FP32 executor: warps per
                                   block 2 (64 bins per thread), 4 (32) or 8 (16);
                                   5 = 4 warps with a 96-row W table (4 blocks
                                   per SM); 6 = 4 warps, bins paired for the
                                   two-wide FP32 instructions (W table of
                                   16-byte slots, 67 KB); 0 = default (6)      */
#define FSE_OPT_F32_LAYOUT 8    /* layout of this context's F = 32 executor: 1 = one
                                   spectrum column per lane, 2 = bins paired
                                   for the two-wide FP32 instructions, 3 = one
                                   column per lane read in row runs (39-row W
                                   table, TMA staging, 6 blocks of 2 warps per
                                   SM); 4 = the same with plain-load staging
                                   only, 8 blocks per SM; 0 = default (4)      */
#define FSE_OPT_TMA_STAGING 9   /* layout 3 of the F = 32 executor:
                                   1 = it stages each block's
                                   support with TMA tensor copies where the
                                   job's image and mask are 16-byte aligned
                                   with a 16-byte multiple row pitch; 2
                                   (default) = the same when the call has at
                                   least four F = 32 blocks per resident warp;
                                   0 = plain loads (always so for F = 64, FP64) */
#define FSE_OPT_DEBUG_TMA_STALL 10 /* test only: 1 = the TMA staging of F = 32
                                   supports never signals completion, so its
                                   bounded wait runs out: the call returns
                                   FSE_ETIMEOUT and the context stays usable
                                   (exercises the failure path, no fault)     */
#define FSE_OPT_KERNEL_TIMING 6 /* 1 = bracket the iteration kernels of every
                                   call with CUDA events (no synchronisation);
                                   read with fse_context_class_times and
                                   fse_context_kernel_times                   */
#define FSE_OPT_F32_UNROLL 11   /* K-loop unroll factor of the F = 32 executor:
                                   1 (default) or 2 (layouts 2, 3 and 4)       */
#define FSE_OPT_F64_UNROLL 12   /* K-loop unroll factor of the F = 64 executor:
                                   1 (default) or 2 (layout 6)                 */
#define FSE_OPT_SERVER_CLASSES 14 /* work classes the resident executor of a
                                   server made from this context runs: 1 = FP32
                                   F = 32, 2 = FP32 F = 64, 3 (default) = both
                                   (the F = 64 executor one CTA per SM below its
                                   occupancy, the compact F = 32 layout beside) */
#define FSE_OPT_CLASS_LAUNCH 13 /* work classes of one call (F = 32, F = 64,
                                   FP64): 0 = launched one after the other;
                                   1 (default) = concurrently on forked streams,
                                   the F = 64 class first; 2 = concurrently,
                                   the F = 32 class first                      */
#define FSE_OPT_ROOT_WINDOW 15  /* batch calls (DAG mode): blocks without lost
                                   predecessors enter the ready queue as a
                                   window of n per consumer (a warp of the F = 32
                                   executor, a CTA of the others), one more
                                   whenever a block finishes, in job order, so
                                   a few images at a time are in flight and
                                   their supports stay in L2; 0 = all at once.
                                   Results do not depend on it.  Default 2.    */
#define FSE_EXEC_DAG 0       /* one persistent launch per work class, the classes
                                concurrent (FSE_OPT_CLASS_LAUNCH); blocks start
                                as soon as the blocks they depend on are done  */
#define FSE_EXEC_LEVELS 1    /* one launch per order level (phase)            */
#define FSE_EXEC_PER_BLOCK 2 /* one launch per lost block, in processing order */
int fse_context_set_option(fse_context_t* ctx, int32_t key, int64_t value);

/*
 * fse_context_kernel_times -- with FSE_OPT_KERNEL_TIMING = 1: synchronises the
 * context's GPU, writes the elapsed milliseconds of the iteration kernels of
 * each call since the option was set (oldest first, at most cap; from the
 * first class launch to the end of the last, concurrent classes included) and
 * forgets them.  Returns the count written.
 */
int32_t fse_context_kernel_times(fse_context_t* ctx, float* ms, int32_t cap);

/*
 * fse_context_class_times -- as fse_context_kernel_times, per work class and
 * without forgetting: for each timed call (oldest first, at most cap) three
 * floats, the milliseconds of the class's own launch (0: FP32 F = 32,
 * 1: FP32 F = 64, 2: FP64; 0 when the call had no such work).  ms holds
 * 3 * cap floats.  Returns the number of calls written.
 */
int32_t fse_context_class_times(fse_context_t* ctx, float* ms, int32_t cap);

/*
 * fse_autotune -- times the given job mix (device pointers, as for
 * fse_extrapolate_batch; the outputs are written) under candidate launch
 * configurations of each work class present: the executor layout
 * (FSE_OPT_F64_WARPS 6, 4, 5, 2, 8; FSE_OPT_F32_LAYOUT 3, 4, 2, 1), the K-loop
 * unroll factor (1, 2 where the layout has it) and the persistent CTAs per
 * SM; then, for a mix of classes, the class launch (FSE_OPT_CLASS_LAUNCH 0, 1,
 * 2).  Each candidate runs `reps` times (median of the iteration-kernel time);
 * the fastest is applied to this context only and, when the context has a tune
 * cache path, written there.  Writes up to cap results as quadruples into
 * `trace` (may be NULL): (class, layout * 10 + unroll, ctas_per_sm, ms) for the
 * class candidates and (-1, launch mode, 0, ms) for the class launches.
 * Returns how many candidates ran, or a negative status.
 */
int32_t fse_autotune(fse_context_t* ctx, const fse_job_t* jobs, int32_t n, void* cuda_stream,
                     int32_t reps, double* trace, int32_t cap);

/*
 * fse_extrapolate_batch -- extrapolates n jobs in one stream-ordered pass.
 *   jobs[i].image/mask/out/out_f32 are DEVICE pointers on the context's GPU,
 *   valid until the work on `cuda_stream` (a cudaStream_t; NULL = default
 *   stream) completes.  All tiles of all jobs share the launches.
 *   stats (may be NULL): when non-NULL the call synchronises the stream and
 *   fills it; when NULL the call returns without waiting.
 * Device state lives in the context's arena only; no other allocation.
 * Errors: FSE_EINVAL (a bad job or parameter; nothing is launched),
 *         FSE_EDEGENERATE, FSE_ENOMEM (arena too small), FSE_ETIMEOUT (a device
 *         wait ran out; outputs undefined), FSE_ECUDA.
 */
int fse_extrapolate_batch(fse_context_t* ctx, const fse_job_t* jobs, int32_t n, void* cuda_stream,
                          fse_stats_t* stats);

/*
 * fse_extrapolate_host -- as fse_extrapolate_batch, but image/mask/out/out_f32
 * are HOST pointers: inputs are copied to the arena, outputs copied back, and
 * the call returns after the copies finished.  Pinned host memory makes the
 * copies asynchronous DMA.  Jobs whose host rows are packed (pitch == W) move
 * as whole planes; where the device rows need padding to 16 bytes a device
 * kernel re-pitches them (inputs) and packs them again (outputs).  Strided
 * host rows (pitch > W) are copied row by row, which is slower.
 */
int fse_extrapolate_host(fse_context_t* ctx, const fse_job_t* jobs, int32_t n, void* cuda_stream,
                         fse_stats_t* stats);

/*
 * fse_extrapolate_noalloc -- the pass of fse_extrapolate_batch for callers that
 * cannot allocate device memory (the paper has no counterpart; this is a
 * library convenience).  Such callers include plug-ins whose host application
 * owns the device-memory budget and latency-bound loops that must not call
 * cudaMalloc, which can synchronize the device.  The call allocates nothing:
 * all scratch state lives in one array of FSE_NOALLOC_SCRATCH_BYTES of device
 * memory declared statically in the library (every GPU that loads the library
 * holds it until the process exits), the tables are staged in static host
 * arrays, and no context is needed.
 *   jobs[i].image/mask/out/out_f32/out_f64: DEVICE pointers of the current
 *   device (cudaSetDevice), as for fse_extrapolate_batch; at most 16 jobs and
 *   1024 tiles per call.
 *   cuda_stream: the stream the work is ordered on (NULL = default stream);
 *   the call returns after that work has finished.
 * The first call on a device sets that device up (looks up the scratch
 * array's device address, uploads constants, configures the kernels); make it
 * before any stream capture.  Every call shares the one scratch array and
 * clears what must start empty; calls that overlapped on the GPU would race,
 * so calls are serialized by a process-wide lock.
 * Errors: FSE_ENOMEM when the call needs more than FSE_NOALLOC_SCRATCH_BYTES of
 * scratch (the message says how much), FSE_EINVAL for bad jobs or more than
 * 16 jobs / 1024 tiles, FSE_EDEGENERATE, FSE_ETIMEOUT, FSE_ECUDA.
 */
#define FSE_NOALLOC_SCRATCH_BYTES ((size_t)64 << 20)
int fse_extrapolate_noalloc(const fse_job_t* jobs, int32_t n, void* cuda_stream);

/* ---- serving: continuous batching ---------------------------------------- */
typedef struct fse_server fse_server_t;
typedef struct fse_server_cfg_t {
    size_t arena_bytes;    /* device bytes for the server: its work queues (a
                              quarter at most) and the resident requests'
                              buffers                                          */
    int32_t max_queue;     /* pending requests before FSE_EBUSY (0 = 64)     */
    int32_t max_resident;  /* requests resident on the GPU at once (0 = 64,
                              at most 256)                                     */
    int32_t max_batch;     /* unused (kept for the layout of this struct)    */
} fse_server_cfg_t;

#define FSE_REQ_QUEUED 0
#define FSE_REQ_RUNNING 1
#define FSE_REQ_DONE 2
#define FSE_REQ_FAILED 3

/*
 * fse_server_create -- starts a continuous-batching server on the context's
 * GPU (the context supplies the device, the executor layouts and options,
 * FSE_OPT_SERVER_CLASSES; its arena is not used).  The server reserves
 * cfg->arena_bytes of device memory (FSE_ENOMEM if that much is not free) and
 * launches one resident persistent executor per served class, which runs
 * until the server is destroyed and drains one work queue per class shared by
 * all resident requests.  A worker thread admits queued requests in arrival
 * order whenever a resident slot and device memory are free: it copies the
 * request in and posts it to the running executor, whose next idle group
 * enumerates the request's lost blocks and queues the ready ones, so a new
 * request's blocks run beside those of the requests already on the GPU (no
 * launch per request or batch).  Every wait of the executor is bounded by a
 * heartbeat of the worker and by FSE_OPT_TIMEOUT_MS.  Every result equals the
 * result of the same job run alone.  Serves FP32 jobs; fse_server_destroy
 * finishes queued and running requests first.
 */
int fse_server_create(fse_server_t** srv, fse_context_t* ctx, const fse_server_cfg_t* cfg);
/*
 * fse_submit -- queues one job; image/mask/out/out_f32 are HOST pointers.
 * image and mask are copied before the call returns; out (and out_f32) must
 * stay valid until fse_wait returns for this ticket.  FSE_EBUSY when the queue
 * is full; FSE_EINVAL for an FP64 job, a class the server does not run, or
 * more than 64 tiles; FSE_ENOMEM when the job can never fit the server.
 */
int fse_submit(fse_server_t* srv, const fse_job_t* job, uint64_t* ticket);
int fse_poll(fse_server_t* srv, uint64_t ticket, int32_t* state);
/*
 * fse_cancel -- cancels a request: a queued one leaves the queue, a running
 * one has its remaining blocks skipped (they are only released, so other
 * requests are unaffected).  Either way fse_wait then returns FSE_ECANCELLED;
 * a request already done is not changed.  FSE_ENOTFOUND for an unknown ticket.
 */
int fse_cancel(fse_server_t* srv, uint64_t ticket);
/* Waits up to timeout_ms (< 0: no limit) for completion; st may be NULL.
 * Returns FSE_OK, the request's error status, FSE_ETIMEOUT or FSE_ENOTFOUND.
 * A completed ticket is forgotten after fse_wait returns FSE_OK for it.
 * For a server request st holds jobs = 1, pixels, device_ms = milliseconds
 * from admission to completion and exec_ms = milliseconds from fse_submit to
 * completion (the request's latency); the other fields are 0. */
int fse_wait(fse_server_t* srv, uint64_t ticket, int32_t timeout_ms, fse_stats_t* st);
/* Per-request latency record of the last completed tickets (seconds from
 * submit to done), newest last; returns how many were written. */
int32_t fse_server_latencies(fse_server_t* srv, double* out, int32_t cap);
void fse_server_destroy(fse_server_t* srv);

/* ---- diagnostics ---------------------------------------------------------- */
const char* fse_last_error(void);

/*
 * fse_debug_fetch -- after a batch run with FSE_OPT_DEBUG_CAPTURE = 1, copies
 * out one record per processed block: rec[4*i..] = job, tile, I, J (block row
 * and column in the tile-local grid) and useq[K_max*i..] = the selected bins
 * (flat k1*F+k2) of its iterations, -1 past its K.  Returns the record count
 * (or a negative status).  K_max is the largest K of the batch.
 */
int32_t fse_debug_fetch(fse_context_t* ctx, int32_t* rec, int32_t* useq, int32_t cap,
                        int32_t* K_max);

/*
 * fse_server_debug_state -- a snapshot of a server's state for diagnosis:
 * per FP32 class (F = 32, then F = 64) 8 values: items enumerated, queue
 * positions reserved, positions filled, blocks done, admit commands posted and
 * taken (device), commands posted and queue entries reserved (host); then per
 * job slot (256) 8 values: ticket (-1 free), generation (host), generation,
 * lost blocks and blocks done (device), completed generation (host-mapped),
 * cancelled generation (device), request state.  out holds cap >= 2064
 * values.  Returns the count written.
 */
int32_t fse_server_debug_state(fse_server_t* srv, int64_t* out, int32_t cap);

/*
 * fse_debug_wait_probe -- launches the work-queue consumer on an empty queue
 * whose producer never comes, with the given wait bound.  Returns
 * FSE_ETIMEOUT when the bounded wait ran out as designed (the context stays
 * usable), another status otherwise.  Exercises the failure path without
 * any device fault.
 */
int fse_debug_wait_probe(fse_context_t* ctx, int32_t timeout_us);

#ifdef __cplusplus
}
#endif
#endif /* FSE_H */
