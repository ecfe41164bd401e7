// FSE device kernels for sm_103a.
//
// Per lost block (paper Sec. II; the method's steps in order):
//   stage   : gather the S x S support (S = b + 2B) around the block from the
//             8-bit image, the loss mask and the tile's value plane; weight
//             w = rho^dist (known), delta*rho^dist (reconstructed), 0 (pending
//             or outside the extended tile); rbar = sum(w r) / sum(w).
//   DFT     : one packed complex F x F FFT of w + i*w*(r - rbar) (zero padded
//             S -> F), split by Hermitian symmetry into W = DFT(w) and
//             R' = DFT(w*(r - rbar)); R_w = rbar*W + R' (= DFT(w*r)).  FP64
//             path: R_w = DFT(w*r) directly.
//   iterate : K times: u = argmax_k |R_w(k)|^2; Delta = gamma R_w(u) / W(0);
//             record (u, Delta); R_w(k) -= Delta * W(k - u) for every bin k.
//   model   : g = Re sum Delta_nu exp(+2 pi i u_nu . x / F) at the block's
//             pending pixels; store g in the tile's value plane (now
//             "reconstructed"), write round-half-even(clip(g)) to the output
//             if the pixel lies in the tile's core (crop and merge, Sec. III).
//   release : blocks whose support holds this block and that come later in the
//             processing order lose one pending predecessor; at zero they are
//             queued.
//
// Work distribution: every lost block of every extended tile of every job is
// one work item; one persistent launch per work class drains a ready queue.
// Waits on the queue are bounded by a wall-clock limit (globaltimer) and end
// with an error flag that the host reads; nothing traps.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstddef>
#include <cstdint>
#include <type_traits>

#include "fse_internal.h"

namespace fse {

__constant__ float2 c_twf[64];   // exp(-2 pi i q / 64)
__constant__ double2 c_twd[64];

void set_twiddles(const float2* tw_f, const double2* tw_d) {
  cudaMemcpyToSymbol(c_twf, tw_f, sizeof(float2) * 64);
  cudaMemcpyToSymbol(c_twd, tw_d, sizeof(double2) * 64);
}

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_relaxed(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Reads of data that may be written while the kernel runs (the server's
// descriptors, items, block maps and request buffers, written by the host's
// copies or by other SMs) go to L2 (ld.global.cg): L1 and the read-only path
// are not coherent across SMs, and a resident server kernel outlives those
// writes.
template <typename T_>
__device__ __forceinline__ T_ ldcg_struct(const T_* p) {
  static_assert(sizeof(T_) % 4 == 0, "descriptor size");
  T_ v;
  int* d = reinterpret_cast<int*>(&v);
  const int* q = reinterpret_cast<const int*>(p);
#pragma unroll 4
  for (int i = 0; i < (int)(sizeof(T_) / 4); ++i) d[i] = __ldcg(q + i);
  return v;
}

// Read of job data: through the read-only cache in a batch call (everything
// was written before the launch), through L2 in server mode (coh).
template <typename T_>
__device__ __forceinline__ T_ ld_in(const T_* p, bool coh) {
  return coh ? __ldcg(p) : __ldg(p);
}

// Barrier of a block's thread group: the CTA, or one warp.
template <bool CTA>
__device__ __forceinline__ void bar() {
  if constexpr (CTA) __syncthreads(); else __syncwarp();
}

// Processing-order key (PHASED: phase, I, J; RASTER: I, J).
__device__ __forceinline__ int64_t order_key(const JobDev& J, int I, int Jb) {
  int64_t k = ((int64_t)I << 20) | (int64_t)Jb;
  if (J.order == ORDER_PHASED) k |= (int64_t)((I % J.P) * J.P + (Jb % J.P)) << 40;
  return k;
}

__device__ __forceinline__ void queue_push(const ClassArgs& C, int item) {
  const int pos = atomicAdd(&C.q->tail, 1);
  st_release(&C.slots[pos], item);
}

// Warp-cooperative pop (all 32 lanes call it): lane 0 reserves the next slot
// and waits for its item.  Returns the item id, -1 once every item has been
// reserved, -2 on error.  A waiting warp gives up with ERR_TIMEOUT when no
// item of the class finished for timeout_ns (progress watchdog, wall clock).
__device__ int queue_pop_warp(const ClassArgs& C, int64_t timeout_ns, int lane) {
  int item = -1;
  if (lane == 0) {
    QueueDev* q = C.q;
    const int n = min(ld_relaxed(&q->n_items), C.cap);
    const int pos = atomicAdd(&q->head, 1);
    if (pos < n) {
      int last_done = ld_relaxed(&q->n_done);
      uint64_t t_last = global_ns();
      unsigned sleep_ns = 32;
      while ((item = ld_acquire(&C.slots[pos])) < 0) {
        if (ld_relaxed(&q->error) != 0) {
          item = -2;
          break;
        }
        const int done = ld_relaxed(&q->n_done);
        const uint64_t now = global_ns();
        if (done != last_done) {
          last_done = done;
          t_last = now;
        } else if ((int64_t)(now - t_last) > timeout_ns) {
          atomicOr(&q->error, ERR_TIMEOUT);
          q->error_info = pos;
          item = -2;
          break;
        }
        __nanosleep(sleep_ns);
        if (sleep_ns < 1024) sleep_ns <<= 1;
      }
    }
  }
  return __shfl_sync(0xffffffffu, item, 0);
}

// Lost predecessors of block (I, Jb) inside its dependency window: under
// PHASED the window's lost blocks of lower phase, under RASTER the earlier
// ones, under INDEPENDENT none.
__device__ __forceinline__ int count_preds(const JobDev& J, const TileDev& T, const int32_t* map, int I, int Jb,
                                           bool coh) {
  if (J.order == ORDER_INDEPENDENT) return 0;
  const int D = J.D;
  const int64_t kx = order_key(J, I, Jb);
  int cnt = 0;
  for (int dI = -D; dI <= D; ++dI)
    for (int dJ = -D; dJ <= D; ++dJ) {
      const int I2 = I + dI, J2 = Jb + dJ;
      if (I2 < 0 || I2 >= T.nby || J2 < 0 || J2 >= T.nbx) continue;
      const int id2 = ld_in(map + I2 * T.nbx + J2, coh);
      if (id2 >= 0 && order_key(J, I2, J2) < kx) ++cnt;
    }
  return cnt;
}

// Fed roots (ClassArgs::window): while fewer than `window` items wait in the
// queue, a finished block pushes the next root (four when consumers are
// already waiting), so released successors keep the queue filled and new
// roots, in id (job) order, enter only as the queue runs low.
__device__ __forceinline__ void feed_root(const ClassArgs& C) {
  const int pending = ld_relaxed(&C.q->tail) - ld_relaxed(&C.q->head);
  const int n = pending < 0 ? 4 : (pending < C.window ? 1 : 0);
  const int n_roots = ld_relaxed(&C.q->n_roots);
  for (int i = 0; i < n; ++i) {
    const int idx = C.window + atomicAdd(&C.q->root_next, 1);
    if (idx >= n_roots) break;
    queue_push(C, __ldcg(C.roots + idx));
  }
}

// After a block's writes are globally visible: decrement the pending count
// of every later lost block in its dependency window, queue those reaching 0;
// with fed roots, also queue the next root.
__device__ __forceinline__ void release_successors(const ExecArgs& a, const ClassArgs& C, const TileDev& T,
                                   const JobDev& J, int I, int Jb, int t, int nthr) {
  if (C.window > 0 && t == 0 && !a.level_mode && a.single_item < 0) feed_root(C);
  if (J.order == ORDER_INDEPENDENT || a.level_mode || a.single_item >= 0) return;
  const int D = J.D, wd = 2 * D + 1;
  const int64_t kx = order_key(J, I, Jb);
  const int32_t* map = a.map + T.map_off;
  for (int pos = t; pos < wd * wd; pos += nthr) {
    const int I2 = I + pos / wd - D, J2 = Jb + pos % wd - D;
    if (I2 < 0 || I2 >= T.nby || J2 < 0 || J2 >= T.nbx) continue;
    const int id2 = ld_in(map + I2 * T.nbx + J2, a.server != 0);
    if (id2 < 0 || order_key(J, I2, J2) <= kx) continue;
    if (atomicSub(&C.cnt[id2], 1) == 1) {
      __threadfence();
      queue_push(C, id2);
    }
  }
}


// ---------------------------------------------------------------------------
// Server mode: the resident executor of the continuous-batching server.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void st_release_sys(int* p, int v) {
  asm volatile("st.release.sys.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Moves one posted admit command of class cls into the work queue (any
// consumer may do it; a CAS on the taken count gives each command to one).
__device__ __forceinline__ void server_take_command(const ExecArgs& a, const ClassArgs& C, int cls) {
  ServerDevCtl* d = a.srv;
  const int tail = ld_acquire(&d->cmd_tail[cls]);
  int taken = ld_relaxed(&d->cmd_taken[cls]);
  while (taken < tail) {
    const int got = atomicCAS(&d->cmd_taken[cls], taken, taken + 1);
    if (got == taken) {
      queue_push(C, SRV_CMD_BIT | taken);
      return;
    }
    taken = got;
  }
}

// Server pop (lane 0's result broadcast to the warp): reserves the next queue
// slot and waits for its entry, taking posted commands into the queue while
// it waits.  Returns an item id, a command (SRV_CMD_BIT | index), -1 when the
// server stops, -2 when the host's heartbeat has been stale for timeout_ns
// (the host is gone) or the queue's capacity ran out.
__device__ int server_pop_warp(const ExecArgs& a, const ClassArgs& C, int cls, int lane) {
  int item = -1;
  if (lane == 0) {
    ServerDevCtl* d = a.srv;
    const bool stop = ld_acquire(&d->stop) != 0;
    if (!stop) {
      // a posted admit command goes before the queue's items (and takes no
      // queue slot), so a new request joins as soon as a group finishes a
      // block, not once the queue has drained
      const int ctail = ld_acquire(&d->cmd_tail[cls]);
      int taken = ld_relaxed(&d->cmd_taken[cls]);
      while (taken < ctail) {
        const int got = atomicCAS(&d->cmd_taken[cls], taken, taken + 1);
        if (got == taken) {
          item = SRV_CMD_BIT | taken;
          break;
        }
        taken = got;
      }
    }
    if (stop || item != -1) {
      // stopping (-1), or an admit command
    } else {
      const int pos = atomicAdd(&C.q->head, 1);
      if (pos >= C.cap) {
        atomicOr(&a.host->error, ERR_BOUNDS);
        item = -2;
      } else {
        int hb = ld_relaxed(&d->heartbeat);
        uint64_t t_hb = global_ns();
        unsigned sleep_ns = 32;
        for (;;) {
          item = ld_acquire(&C.slots[pos]);
          if (item != -1) break;
          server_take_command(a, C, cls);
          if (ld_acquire(&d->stop)) {
            item = -1;
            break;
          }
          const int h = ld_relaxed(&d->heartbeat);
          const uint64_t now = global_ns();
          if (h != hb) {
            hb = h;
            t_hb = now;
          } else if ((int64_t)(now - t_hb) > a.timeout_ns) {
            atomicOr(&a.host->error, ERR_TIMEOUT);
            item = -2;
            break;
          }
          __nanosleep(sleep_ns);
          if (sleep_ns < 4096) sleep_ns <<= 1;
        }
      }
    }
  }
  return __shfl_sync(0xffffffffu, item, 0);
}

// One block of a job finished (or was skipped): the job completes with its
// last block, which publishes the job's generation to the host.
__device__ __forceinline__ void server_block_done(const ExecArgs& a, int job) {
  ServerDevCtl* d = a.srv;
  const int n = atomicAdd(&d->done[job], 1) + 1;
  if (n == ld_relaxed(&d->total[job])) {
    __threadfence_system();
    st_release_sys(&a.host->done_gen[job], ld_relaxed(&d->gen[job]));
  }
}

// Whether the item's job has been cancelled (its generation marked).
__device__ __forceinline__ bool server_cancelled(const ExecArgs& a, const ClassArgs& C, int id) {
  const int job = __ldcg(&a.tiles[__ldcg(C.items + id).x].job);
  return ld_relaxed(&a.srv->cancel_gen[job]) == ld_relaxed(&a.srv->gen[job]);
}

// Admit command: makes job `j` (its descriptors, tiles and buffers written by
// the host) resident in the running executor.  The group's t of nthr threads
// write its known pixels to the output, mark its value planes pending,
// enumerate its lost blocks into the
// class's items, set every item's pending-predecessor count, and only then
// push the items without predecessors (so no block of the job runs before all
// counts are set).  The pushes recount instead of reading cnt, which running
// blocks already decrement.
template <bool CTA>
__device__ void server_admit(const ExecArgs& a, const ClassArgs& C, int cls, int cmd, int t, int nthr) {
  const ServerCmd rc = ldcg_struct(&a.srv->cmd[cls][cmd % SRV_CMD_RING]);
  const int j = rc.job, gen = rc.gen, nt = rc.n_tiles;
  const JobDev J = ldcg_struct(a.jobs + j);
  ServerDevCtl* d = a.srv;
  if (t == 0) {
    d->done[j] = 0;
    d->total[j] = 0;
    d->gen[j] = gen;
  }
  const int64_t npx = (int64_t)J.W * J.H;
  for (int64_t p = t; p < npx; p += nthr) {
    const int y = (int)(p / J.W), x = (int)(p - (int64_t)y * J.W);
    const size_t gi = (size_t)y * J.pitch + x;
    const uint8_t v = __ldcg(J.mask + gi) ? 0 : __ldcg(J.image + gi);
    J.out[gi] = v;
    if (J.out_f32) J.out_f32[p] = (float)v;
  }
  for (int ti = 0; ti < nt; ++ti) {  // value planes: every pixel pending (NaN)
    const TileDev T = ldcg_struct(a.tiles + j * SRV_MAXT + ti);
    float* plane = a.val_f + T.val_off;
    const int64_t n = (int64_t)T.ew * T.eh;
    for (int64_t p = t; p < n; p += nthr) plane[p] = __int_as_float(-1);
  }
  bar<CTA>();
  int local = 0;
  for (int ti = 0; ti < nt; ++ti) {
    const int tile = j * SRV_MAXT + ti;
    const TileDev T = ldcg_struct(a.tiles + tile);
    const int nb = T.nbx * T.nby;
    for (int k = t; k < nb; k += nthr) {
      const int I = k / T.nbx, Jb = k - I * T.nbx;
      bool lost = false;
      const int y0 = I * J.b, x0 = Jb * J.b;
      for (int yy = y0; yy < min(y0 + J.b, T.eh) && !lost; ++yy)
        for (int xx = x0; xx < min(x0 + J.b, T.ew); ++xx)
          if (__ldcg(J.mask + (size_t)(T.ey + yy) * J.pitch + T.ex + xx)) {
            lost = true;
            break;
          }
      int id = -1;
      if (lost) {
        id = atomicAdd(&C.q->n_items, 1);
        if (id < C.cap) {
          C.items[id] = make_int2(tile, (I << 16) | Jb);
          ++local;
        } else {
          atomicOr(&a.host->error, ERR_BOUNDS);
          id = -1;
        }
      }
      a.map[T.map_off + k] = id;
    }
  }
  if (local) atomicAdd(&d->total[j], local);
  __threadfence();
  bar<CTA>();
  for (int ti = 0; ti < nt; ++ti) {
    const TileDev T = ldcg_struct(a.tiles + j * SRV_MAXT + ti);
    const int32_t* map = a.map + T.map_off;
    const int nb = T.nbx * T.nby;
    for (int k = t; k < nb; k += nthr) {
      const int id = __ldcg(map + k);
      if (id >= 0) C.cnt[id] = count_preds(J, T, map, k / T.nbx, k % T.nbx, true);
    }
  }
  __threadfence();
  bar<CTA>();
  if (t == 0 && ld_relaxed(&d->total[j]) == 0) {  // nothing lost: done at once
    __threadfence_system();
    st_release_sys(&a.host->done_gen[j], gen);
  }
  for (int ti = 0; ti < nt; ++ti) {
    const TileDev T = ldcg_struct(a.tiles + j * SRV_MAXT + ti);
    const int32_t* map = a.map + T.map_off;
    const int nb = T.nbx * T.nby;
    for (int k = t; k < nb; k += nthr) {
      const int id = __ldcg(map + k);
      if (id >= 0 && count_preds(J, T, map, k / T.nbx, k % T.nbx, true) == 0) queue_push(C, id);
    }
  }
  bar<CTA>();
}

__device__ __forceinline__ uint8_t to_u8(float g) {
  float c = fminf(fmaxf(g, 0.f), 255.f);
  return (uint8_t)__float2int_rn(c);  // round half to even
}
__device__ __forceinline__ uint8_t to_u8(double g) {
  double c = fmin(fmax(g, 0.0), 255.0);
  return (uint8_t)__double2int_rn(c);
}

// ---------------------------------------------------------------------------
// Support staging: z(m, n) = (w, r) for m, n < S into a swizzled F x F buffer
// (r = 0 where w = 0); element (m, n) lives at m*F + (n ^ (m & (F-1))) so that
// row-wise and column-wise walks of a warp hit distinct banks.  The row FFTs
// read (w, w (r - c)) from it, c the support's weighted mean (support_mean).
// ---------------------------------------------------------------------------
template <int F>
__device__ __forceinline__ int swz(int m, int n) {
  return m * F + (n ^ (m & (F - 1)));
}

template <int F, bool COH, typename real, typename real2>
__device__ __forceinline__ void stage_support_impl(const TileDev& T, const JobDev& J, const real* val,
                                              int I, int Jb, real2* zbuf, int t, int nthr) {
  const int S = J.S;
  const int oy = I * J.b - J.B, ox = Jb * J.b - J.B;
  const real* wiso;
  real delta;
  if constexpr (sizeof(real) == 4) {
    wiso = J.wiso_f;
    delta = J.delta_f;
  } else {
    wiso = J.wiso_d;
    delta = J.delta;
  }
  const bool use_done = J.order != ORDER_INDEPENDENT;
  // Thread t owns support column n = t mod F and the rows m0, m0 + mstep, ...
  // Out-of-tile pixels load from the tile's first pixel and are masked off,
  // so every load of a batch issues unconditionally, back to back.
  const int n = t & (F - 1), m0 = t / F, mstep = nthr / F;
  const int tx = ox + n;
  const bool col_in = n < S && tx >= 0 && tx < T.ew;
  const int eh = T.eh, vp = F == 32 ? T.vp : T.ew;  // F = 64 value planes are unpadded
  const size_t pitch = J.pitch, g0 = (size_t)T.ey * pitch + T.ex;
  const uint8_t* mask = J.mask;
  const uint8_t* image = J.image;
  constexpr int U = 8;  // rows whose loads are in flight together
  if (n >= S) return;
  for (int mb = m0; mb < S; mb += U * mstep) {
    uint8_t mk[U], px[U];
    real wi[U], v[U];
    bool in[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int m = mb + u * mstep, ty = oy + m;
      in[u] = col_in && m < S && ty >= 0 && ty < eh;
      const size_t gi = in[u] ? g0 + (size_t)ty * pitch + tx : g0;
      const size_t vi = in[u] ? (size_t)ty * vp + tx : 0;
      wi[u] = ld_in(wiso + (m < S ? m * S + n : n), COH);
      mk[u] = ld_in(mask + gi, COH);
      px[u] = ld_in(image + gi, COH);
      v[u] = __ldcg(val + vi);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int m = mb + u * mstep;
      if (m >= S) break;
      real wv = 0, rv = 0;
      if (in[u]) {
        if (mk[u] == 0) {
          wv = wi[u];
          rv = (real)px[u];
        } else if (use_done && !isnan(v[u])) {
          wv = delta * wi[u];
          rv = v[u];
        }
      }
      real2 z;
      z.x = wv;
      z.y = rv;
      zbuf[swz<F>(m, n)] = z;
    }
  }
}

// The staging loop in its batch form (read-only cache) or its server form
// (L2), chosen once per block.
template <int F, typename real, typename real2>
__device__ __forceinline__ void stage_support(const TileDev& T, const JobDev& J, const real* val, int I, int Jb,
                                              real2* zbuf, int t, int nthr, bool coh) {
  if (coh)
    stage_support_impl<F, true, real, real2>(T, J, val, I, Jb, zbuf, t, nthr);
  else
    stage_support_impl<F, false, real, real2>(T, J, val, I, Jb, zbuf, t, nthr);
}

// ---------------------------------------------------------------------------
// TMA support staging (F = 32 executor, where twelve warps per SM share the
// load/store queue with the iteration loops).  One thread issues three tensor
// copies per block (the mask and image boxes from the job's maps, the
// value-plane box from the tile's map) that complete on an mbarrier; every x
// coordinate is rounded down to a 16-byte multiple and the boxes are wide
// enough to cover the support from there (bw = roundup16(S + 15) bytes,
// bv = roundup4(S + 3) floats), so no copy starts off a 16-byte boundary.
// Elements outside the image or the tile read as zero and are masked by the
// same in-tile test as the plain loads.  The wait is bounded by the context's
// wall-clock limit.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* mbar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Support bytes the three boxes need in shared memory (each box 128-byte aligned).
__device__ __forceinline__ int tma_stage_bytes(const JobDev& J) {
  return 2 * ((J.S * J.bw + 127) & ~127) + J.S * J.bv * 4;
}

// Issues the copies (leader thread only).  The value plane was written with
// ordinary stores by the warps that reconstructed earlier blocks and published
// through the ready queue (release / acquire); the global proxy fence orders
// what this thread has thereby observed before its asynchronous-proxy reads,
// and the shared one orders earlier accesses of the buffer before the
// asynchronous writes.  stall (test only): expect the bytes without arriving,
// so the phase cannot complete until the waiter arrives itself.
__device__ __forceinline__ void tma_issue_support(const TileDev& T, const JobDev& J, int I, int Jb,
                                                  unsigned char* sbuf, uint64_t* mbar, bool stall) {
  const int S = J.S;
  const int oy = I * J.b - J.B, ox = Jb * J.b - J.B;
  const int x0 = (T.ex + ox) & ~15, vx0 = ox & ~3, gy = T.ey + oy;
  const int sz8 = (S * J.bw + 127) & ~127;
  const uint32_t mb = smem_u32(mbar);
  const uint32_t bytes = (uint32_t)(2 * S * J.bw + S * J.bv * 4);
  asm volatile("fence.proxy.async.global;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (stall)
    asm volatile("mbarrier.expect_tx.shared::cta.b64 [%0], %1;" ::"r"(mb), "r"(bytes) : "memory");
  else
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(bytes) : "memory");
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(sbuf)),
      "l"(J.tm_mask), "r"(x0), "r"(gy), "r"(mb)
      : "memory");
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(sbuf + sz8)),
      "l"(J.tm_image), "r"(x0), "r"(gy), "r"(mb)
      : "memory");
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(sbuf + 2 * sz8)),
      "l"(T.tm_val), "r"(vx0), "r"(oy), "r"(mb)
      : "memory");
}

// The arrival a stalled staging withheld (test only).
__device__ __forceinline__ void mbar_arrive(uint64_t* mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(mbar)) : "memory");
}

// Waits for phase `parity` of the mbarrier; false when the wall-clock limit passed.
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity, int64_t timeout_ns) {
  const uint32_t mb = smem_u32(mbar);
  const uint64_t t0 = global_ns();
  for (uint32_t i = 0;; ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred q;\n mbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n selp.u32 %0, 1, 0, q;\n}"
        : "=r"(done)
        : "r"(mb), "r"(parity)
        : "memory");
    if (done) return true;
    if ((i & 63) == 63 && (int64_t)(global_ns() - t0) > timeout_ns) return false;
  }
}

// Whether this block can be staged by TMA into `sbuf` (bytes available).
__device__ __forceinline__ bool tma_usable(const TileDev& T, const JobDev& J, const unsigned char* sbuf,
                                           int bytes) {
  return J.tma && T.tm_val != nullptr && sbuf != nullptr && (smem_u32(sbuf) & 127) == 0 &&
         tma_stage_bytes(J) <= bytes;
}

// z(m, n) = (w, r) from the landed boxes; same thread mapping and the same
// arithmetic as stage_support.
template <int F>
__device__ __forceinline__ void stage_from_boxes(const TileDev& T, const JobDev& J, int I, int Jb,
                                                 float2* zbuf, const unsigned char* sbuf, int t, int nthr) {
  const int S = J.S, bw = J.bw, bv = J.bv;
  const int oy = I * J.b - J.B, ox = Jb * J.b - J.B;
  const int gx = T.ex + ox;
  const int dx8 = gx - (gx & ~15), dxv = ox - (ox & ~3);
  const int sz8 = (S * bw + 127) & ~127;
  const unsigned char* smask = sbuf;
  const unsigned char* simg = sbuf + sz8;
  const float* sval = reinterpret_cast<const float*>(sbuf + 2 * sz8);
  const float* wiso = J.wiso_f;
  const float delta = J.delta_f;
  const bool use_done = J.order != ORDER_INDEPENDENT;
  const int n = t & (F - 1), m0 = t / F, mstep = nthr / F;
  if (n >= S) return;
  const int tx = ox + n;
  const bool col_in = tx >= 0 && tx < T.ew;
  for (int m = m0; m < S; m += mstep) {
    const int ty = oy + m;
    float wv = 0.f, rv = 0.f;
    if (col_in && ty >= 0 && ty < T.eh) {
      const float wi = __ldg(wiso + m * S + n);
      const int mk = smask[m * bw + dx8 + n];
      if (mk == 0) {
        wv = wi;
        rv = (float)simg[m * bw + dx8 + n];
      } else if (use_done) {
        const float v = sval[m * bv + dxv + n];
        if (!isnan(v)) {
          wv = delta * wi;
          rv = v;
        }
      }
    }
    zbuf[swz<F>(m, n)] = make_float2(wv, rv);
  }
}

// ---------------------------------------------------------------------------
// Weighted mean c = sum(w r) / sum(w) of a staged support (z = (w, r)).
// The FP32 executors transform w (r - c) instead of w r and then form
// R_w = c W + DFT(w (r - c)), which is DFT(w r) exactly in real arithmetic:
// the FFT's rounding error scales with the norm of its input, and the
// support's mean dominates that norm, so taking it out before the transform
// and adding it back through W (the spectrum the iteration subtracts from)
// keeps R_w consistent with W to the precision of the small remainder.
// Any c gives the same mathematics; the mean makes the remainder smallest.
// Every thread of the group sums in the same fixed order, so all get the same
// bits whichever staging path filled the buffer.  red: NT/32 floats (CTA).
// ---------------------------------------------------------------------------
template <int F, int NT>
__device__ __forceinline__ float support_mean(const float2* zbuf, int S, int t, float* red) {
  float sw = 0.f, swr = 0.f;
  const int n = t & (F - 1);
  if (n < S)
    for (int m = t / F; m < S; m += NT / F) {
      const float2 z = zbuf[swz<F>(m, n)];
      sw += z.x;
      swr = fmaf(z.x, z.y, swr);
    }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sw += __shfl_xor_sync(0xffffffffu, sw, o);
    swr += __shfl_xor_sync(0xffffffffu, swr, o);
  }
  if constexpr (NT > 32) {
    const int warp = t >> 5;
    __syncthreads();
    if ((t & 31) == 0) {
      red[2 * warp] = sw;
      red[2 * warp + 1] = swr;
    }
    __syncthreads();
    sw = red[0];
    swr = red[1];
#pragma unroll
    for (int w = 1; w < NT / 32; ++w) {
      sw += red[2 * w];
      swr += red[2 * w + 1];
    }
    __syncthreads();
  }
  return sw > 0.f ? swr / sw : 0.f;
}

// The row-FFT input w (r - c) from a staged pixel (w, r).
__device__ __forceinline__ float2 centred(float2 z, float c) { return make_float2(z.x, (z.y - c) * z.x); }

// ---------------------------------------------------------------------------
// Register FFT (radix-2 decimation in time, natural order in and out):
// X[k] = sum_n x[n] exp(-2 pi i k n / N), N = 32 or 64, fully unrolled.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int brev_c(int i, int bits) {
  int r = 0;
  for (int b = 0; b < bits; ++b) r |= ((i >> b) & 1) << (bits - 1 - b);
  return r;
}

// Bit-reversal permutation as compile-time register renaming.
template <int I, int N, int LOG>
struct BitRev {
  static __device__ __forceinline__ void run(float2 (&x)[N]) {
    constexpr int J = brev_c(I, LOG);
    if constexpr (I < J) {
      const float2 t = x[I];
      x[I] = x[J];
      x[J] = t;
    }
    BitRev<I + 1, N, LOG>::run(x);
  }
};
template <int N, int LOG>
struct BitRev<N, N, LOG> {
  static __device__ __forceinline__ void run(float2 (&)[N]) {}
};

// One radix-2 stage (butterfly span 2^S); twiddle exp(-2 pi i k / 2^(S+1)).
template <int S, int N, int LOG>
struct FftStage {
  static __device__ __forceinline__ void run(float2 (&x)[N]) {
    constexpr int half = 1 << S;
#pragma unroll
    for (int g = 0; g < N; g += 2 * half) {
#pragma unroll
      for (int k = 0; k < half; ++k) {
        const float2 a = x[g + k], b = x[g + k + half];
        float2 tt;
        if (k == 0) {
          tt = b;
        } else {
          const float2 w = c_twf[k * (32 >> S)];
          tt = make_float2(w.x * b.x - w.y * b.y, w.x * b.y + w.y * b.x);
        }
        x[g + k] = make_float2(a.x + tt.x, a.y + tt.y);
        x[g + k + half] = make_float2(a.x - tt.x, a.y - tt.y);
      }
    }
    FftStage<S + 1, N, LOG>::run(x);
  }
};
template <int N, int LOG>
struct FftStage<LOG, N, LOG> {
  static __device__ __forceinline__ void run(float2 (&)[N]) {}
};

template <int N>
__device__ __forceinline__ void fft_reg(float2 (&x)[N]) {
  constexpr int LOG = (N == 32) ? 5 : 6;
  BitRev<0, N, LOG>::run(x);
  FftStage<0, N, LOG>::run(x);
}

// Copies a descriptor into shared memory word by word (t of nthr threads).
template <typename T_>
__device__ __forceinline__ void copy_desc(T_* dst, const T_* src, int t, int nthr, bool coh) {
  static_assert(sizeof(T_) % 4 == 0, "descriptor size");
  const int* s = reinterpret_cast<const int*>(src);
  int* d = reinterpret_cast<int*>(dst);
  for (int i = t; i < (int)(sizeof(T_) / 4); i += nthr) d[i] = ld_in(s + i, coh);
}

// Second radix-2 step of a 64-point transform split over lanes l and l ^ 16:
// lane half h = 0 holds E = FFT32(even samples), h = 1 holds O = FFT32(odd
// samples); afterwards half h holds X[k + 32h], k = 0..31.
__device__ __forceinline__ void fft64_combine(float2 (&x)[32], int h) {
#pragma unroll
  for (int k = 0; k < 32; ++k) {
    const float2 w = c_twf[k];
    const float2 o = x[k];
    const float2 t = make_float2(w.x * o.x - w.y * o.y, w.x * o.y + w.y * o.x);
    const float2 own = h ? t : o;
    float2 rcv;
    rcv.x = __shfl_xor_sync(0xffffffffu, own.x, 16);
    rcv.y = __shfl_xor_sync(0xffffffffu, own.y, 16);
    x[k] = h ? make_float2(rcv.x - own.x, rcv.y - own.y) : make_float2(own.x + rcv.x, own.y + rcv.y);
  }
}


// Model evaluation at the block's b x b pixels and write-back (all executors).
// coef_u / coef_d hold the K selected (u, Delta) pairs; tw[q] = exp(+2 pi i q/64).
// Threads split the K terms when the block has fewer pixels than threads.
template <bool CTA, int C, typename real, typename real2>
__device__ __forceinline__ void eval_body(const TileDev& T, const JobDev& J, real* val, int I, int Jb,
                               const int* coef_u, const real2* coef_d, const real2* tw,
                               real* red, int t, int nthr, bool coh) {
  const int b = J.b, np = b * b, K = J.K, F = J.F, B = J.B;
  const int logF = F == 32 ? 5 : 6, tshift = 6 - logF;  // tw has 64 entries
  const int nsplit = np <= nthr ? nthr / np : 1;
  for (int p0 = 0; p0 < np; p0 += nthr / nsplit) {
    const int p = p0 + t % (nthr / nsplit), s = t / (nthr / nsplit);
    real g = 0;
    if (p < np && s < nsplit) {
      const int m = B + p / b, n = B + p % b;
      real acc[C];  // independent partial sums: the loads of C terms in flight
#pragma unroll
      for (int c = 0; c < C; ++c) acc[c] = 0;
      int nu = s;
      for (; nu + (C - 1) * nsplit < K; nu += C * nsplit) {
#pragma unroll
        for (int c = 0; c < C; ++c) {
          const int u = coef_u[nu + c * nsplit];
          const int q = ((((u >> logF) * m + (u & (F - 1)) * n) & (F - 1)) << tshift);
          const real2 d = coef_d[nu + c * nsplit], e = tw[q];
          acc[c] += d.x * e.x - d.y * e.y;
        }
      }
      for (int c = 0; nu < K; nu += nsplit, ++c) {
        const int u = coef_u[nu];
        const int q = ((((u >> logF) * m + (u & (F - 1)) * n) & (F - 1)) << tshift);
        const real2 d = coef_d[nu], e = tw[q];
        acc[0] += d.x * e.x - d.y * e.y;
      }
#pragma unroll
      for (int c = 0; c < C; ++c) g += acc[c];
    }
    red[t] = g;
    bar<CTA>();
    if (s == 0 && p < np) {
      for (int k = 1; k < nsplit; ++k) g += red[t + k * (nthr / nsplit)];
      const int ty = I * b + p / b, tx = Jb * b + p % b;
      if (ty < T.eh && tx < T.ew) {
        const int gy = T.ey + ty, gx = T.ex + tx;
        const size_t gi = (size_t)gy * J.pitch + gx;
        if (ld_in(J.mask + gi, coh) != 0) {
          val[(size_t)ty * (CTA ? T.ew : T.vp) + tx] = g;  // CTA-wide executors: unpadded planes
          if (gx >= T.x && gx < T.x + T.w && gy >= T.y && gy < T.y + T.h) {
            J.out[gi] = to_u8(g);
            if (J.out_f32) J.out_f32[(size_t)gy * J.W + gx] = (float)g;
            if (J.out_f64) J.out_f64[(size_t)gy * J.W + gx] = (double)g;
          }
        }
      }
    }
    bar<CTA>();
  }
}

// F = 32 (one warp per block): inline, two partial sums.
template <bool CTA, typename real, typename real2>
__device__ __forceinline__ void eval_and_write(const TileDev& T, const JobDev& J, real* val, int I, int Jb,
                                               const int* coef_u, const real2* coef_d, const real2* tw,
                                               real* red, int t, int nthr, bool coh) {
  eval_body<CTA, 2, real, real2>(T, J, val, I, Jb, coef_u, coef_d, tw, red, t, nthr, coh);
}

// CTA-wide executors: eight partial sums in a call of its own, so the
// evaluation's registers do not shape the allocation of the iteration loop.
template <bool CTA, typename real, typename real2>
__device__ __noinline__ void eval_and_write_call(const TileDev& T, const JobDev& J, real* val, int I,
                                                 int Jb, const int* coef_u, const real2* coef_d,
                                                 const real2* tw, real* red, int t, int nthr, bool coh) {
  eval_body<CTA, 8, real, real2>(T, J, val, I, Jb, coef_u, coef_d, tw, red, t, nthr, coh);
}

__device__ __forceinline__ void debug_record(const ExecArgs& a, int cls, int id, const TileDev& T,
                                             int tile, int I, int Jb) {
  if (a.dbg_rec == nullptr || id >= a.dbg_cap) return;
  int32_t* r = a.dbg_rec + ((size_t)cls * a.dbg_cap + id) * 4;
  r[0] = T.job; r[1] = tile; r[2] = I; r[3] = Jb;
}
__device__ __forceinline__ void debug_useq(const ExecArgs& a, int cls, int id, int it, int u) {
  if (a.dbg_useq == nullptr || id >= a.dbg_cap) return;
  a.dbg_useq[((size_t)cls * a.dbg_cap + id) * KMAX + it] = u;
}

// Register select v = R[i] for a warp-uniform i: one indirect branch through a
// jump table (brx.idx) to a pair of moves, so the spectrum stays in registers
// and the select costs one branch instead of a compare tree.
__device__ __forceinline__ float2 select_reg32(const float2 (&R)[32], int i) {
  float vx, vy;
  asm volatile(
      "{\n"
      "ts: .branchtargets L0, L1, L2, L3, L4, L5, L6, L7, L8, L9, L10, L11, L12, L13, L14, L15, L16, L17, L18, L19, L20, L21, L22, L23, L24, L25, L26, L27, L28, L29, L30, L31;\n"
      "brx.idx.uni %2, ts;\n"
      "L0: mov.b32 %0, %3; mov.b32 %1, %4; bra.uni LEND;\n"
      "L1: mov.b32 %0, %5; mov.b32 %1, %6; bra.uni LEND;\n"
      "L2: mov.b32 %0, %7; mov.b32 %1, %8; bra.uni LEND;\n"
      "L3: mov.b32 %0, %9; mov.b32 %1, %10; bra.uni LEND;\n"
      "L4: mov.b32 %0, %11; mov.b32 %1, %12; bra.uni LEND;\n"
      "L5: mov.b32 %0, %13; mov.b32 %1, %14; bra.uni LEND;\n"
      "L6: mov.b32 %0, %15; mov.b32 %1, %16; bra.uni LEND;\n"
      "L7: mov.b32 %0, %17; mov.b32 %1, %18; bra.uni LEND;\n"
      "L8: mov.b32 %0, %19; mov.b32 %1, %20; bra.uni LEND;\n"
      "L9: mov.b32 %0, %21; mov.b32 %1, %22; bra.uni LEND;\n"
      "L10: mov.b32 %0, %23; mov.b32 %1, %24; bra.uni LEND;\n"
      "L11: mov.b32 %0, %25; mov.b32 %1, %26; bra.uni LEND;\n"
      "L12: mov.b32 %0, %27; mov.b32 %1, %28; bra.uni LEND;\n"
      "L13: mov.b32 %0, %29; mov.b32 %1, %30; bra.uni LEND;\n"
      "L14: mov.b32 %0, %31; mov.b32 %1, %32; bra.uni LEND;\n"
      "L15: mov.b32 %0, %33; mov.b32 %1, %34; bra.uni LEND;\n"
      "L16: mov.b32 %0, %35; mov.b32 %1, %36; bra.uni LEND;\n"
      "L17: mov.b32 %0, %37; mov.b32 %1, %38; bra.uni LEND;\n"
      "L18: mov.b32 %0, %39; mov.b32 %1, %40; bra.uni LEND;\n"
      "L19: mov.b32 %0, %41; mov.b32 %1, %42; bra.uni LEND;\n"
      "L20: mov.b32 %0, %43; mov.b32 %1, %44; bra.uni LEND;\n"
      "L21: mov.b32 %0, %45; mov.b32 %1, %46; bra.uni LEND;\n"
      "L22: mov.b32 %0, %47; mov.b32 %1, %48; bra.uni LEND;\n"
      "L23: mov.b32 %0, %49; mov.b32 %1, %50; bra.uni LEND;\n"
      "L24: mov.b32 %0, %51; mov.b32 %1, %52; bra.uni LEND;\n"
      "L25: mov.b32 %0, %53; mov.b32 %1, %54; bra.uni LEND;\n"
      "L26: mov.b32 %0, %55; mov.b32 %1, %56; bra.uni LEND;\n"
      "L27: mov.b32 %0, %57; mov.b32 %1, %58; bra.uni LEND;\n"
      "L28: mov.b32 %0, %59; mov.b32 %1, %60; bra.uni LEND;\n"
      "L29: mov.b32 %0, %61; mov.b32 %1, %62; bra.uni LEND;\n"
      "L30: mov.b32 %0, %63; mov.b32 %1, %64; bra.uni LEND;\n"
      "L31: mov.b32 %0, %65; mov.b32 %1, %66; bra.uni LEND;\n"
      "LEND:\n}"
      : "=f"(vx), "=f"(vy)
      : "r"(i & 31),
        "f"(R[0].x), "f"(R[0].y), "f"(R[1].x), "f"(R[1].y), "f"(R[2].x), "f"(R[2].y), "f"(R[3].x), "f"(R[3].y),
        "f"(R[4].x), "f"(R[4].y), "f"(R[5].x), "f"(R[5].y), "f"(R[6].x), "f"(R[6].y), "f"(R[7].x), "f"(R[7].y),
        "f"(R[8].x), "f"(R[8].y), "f"(R[9].x), "f"(R[9].y), "f"(R[10].x), "f"(R[10].y), "f"(R[11].x), "f"(R[11].y),
        "f"(R[12].x), "f"(R[12].y), "f"(R[13].x), "f"(R[13].y), "f"(R[14].x), "f"(R[14].y), "f"(R[15].x), "f"(R[15].y),
        "f"(R[16].x), "f"(R[16].y), "f"(R[17].x), "f"(R[17].y), "f"(R[18].x), "f"(R[18].y), "f"(R[19].x), "f"(R[19].y),
        "f"(R[20].x), "f"(R[20].y), "f"(R[21].x), "f"(R[21].y), "f"(R[22].x), "f"(R[22].y), "f"(R[23].x), "f"(R[23].y),
        "f"(R[24].x), "f"(R[24].y), "f"(R[25].x), "f"(R[25].y), "f"(R[26].x), "f"(R[26].y), "f"(R[27].x), "f"(R[27].y),
        "f"(R[28].x), "f"(R[28].y), "f"(R[29].x), "f"(R[29].y), "f"(R[30].x), "f"(R[30].y), "f"(R[31].x), "f"(R[31].y));
  return make_float2(vx, vy);
}

__device__ __forceinline__ float2 select_reg16(const float2 (&R)[16], int i) {
  float vx, vy;
  asm volatile(
      "{\n"
      "ts: .branchtargets L0, L1, L2, L3, L4, L5, L6, L7, L8, L9, L10, L11, L12, L13, L14, L15;\n"
      "brx.idx.uni %2, ts;\n"
      "L0: mov.b32 %0, %3; mov.b32 %1, %4; bra.uni LEND;\n"
      "L1: mov.b32 %0, %5; mov.b32 %1, %6; bra.uni LEND;\n"
      "L2: mov.b32 %0, %7; mov.b32 %1, %8; bra.uni LEND;\n"
      "L3: mov.b32 %0, %9; mov.b32 %1, %10; bra.uni LEND;\n"
      "L4: mov.b32 %0, %11; mov.b32 %1, %12; bra.uni LEND;\n"
      "L5: mov.b32 %0, %13; mov.b32 %1, %14; bra.uni LEND;\n"
      "L6: mov.b32 %0, %15; mov.b32 %1, %16; bra.uni LEND;\n"
      "L7: mov.b32 %0, %17; mov.b32 %1, %18; bra.uni LEND;\n"
      "L8: mov.b32 %0, %19; mov.b32 %1, %20; bra.uni LEND;\n"
      "L9: mov.b32 %0, %21; mov.b32 %1, %22; bra.uni LEND;\n"
      "L10: mov.b32 %0, %23; mov.b32 %1, %24; bra.uni LEND;\n"
      "L11: mov.b32 %0, %25; mov.b32 %1, %26; bra.uni LEND;\n"
      "L12: mov.b32 %0, %27; mov.b32 %1, %28; bra.uni LEND;\n"
      "L13: mov.b32 %0, %29; mov.b32 %1, %30; bra.uni LEND;\n"
      "L14: mov.b32 %0, %31; mov.b32 %1, %32; bra.uni LEND;\n"
      "L15: mov.b32 %0, %33; mov.b32 %1, %34; bra.uni LEND;\n"
      "LEND:\n}"
      : "=f"(vx), "=f"(vy)
      : "r"(i & 15),
        "f"(R[0].x), "f"(R[0].y), "f"(R[1].x), "f"(R[1].y), "f"(R[2].x), "f"(R[2].y), "f"(R[3].x), "f"(R[3].y),
        "f"(R[4].x), "f"(R[4].y), "f"(R[5].x), "f"(R[5].y), "f"(R[6].x), "f"(R[6].y), "f"(R[7].x), "f"(R[7].y),
        "f"(R[8].x), "f"(R[8].y), "f"(R[9].x), "f"(R[9].y), "f"(R[10].x), "f"(R[10].y), "f"(R[11].x), "f"(R[11].y),
        "f"(R[12].x), "f"(R[12].y), "f"(R[13].x), "f"(R[13].y), "f"(R[14].x), "f"(R[14].y), "f"(R[15].x), "f"(R[15].y));
  return make_float2(vx, vy);
}

template <int N>
__device__ __forceinline__ float2 select_reg(const float2 (&R)[N], int i) {
  if constexpr (N == 64) {
    const float2(&lo)[32] = *reinterpret_cast<const float2(*)[32]>(&R[0]);
    const float2(&hi)[32] = *reinterpret_cast<const float2(*)[32]>(&R[32]);
    return i < 32 ? select_reg32(lo, i) : select_reg32(hi, i - 32);
  } else if constexpr (N == 32) {
    return select_reg32(R, i);
  } else {
    return select_reg16(R, i);
  }
}

// An opaque register copy of a constant.
__device__ __forceinline__ uint32_t opaque(uint32_t v) {
  uint32_t r;
  asm volatile("mov.b32 %0, %1;" : "=r"(r) : "r"(v));
  return r;
}

// Argmax key of one bin: (energy bits & mask) | index bits, as one three-input
// logic op with the index as the immediate operand (LUT 0xEC = (a & c) | b).
template <uint32_t IDX>
__device__ __forceinline__ uint32_t make_key(float e, uint32_t mask) {
  uint32_t k;
  asm("lop3.b32 %0, %1, %2, %3, 0xEC;" : "=r"(k) : "r"(__float_as_uint(e)), "n"(IDX), "r"(mask));
  return k;
}

// Stores to shared memory only where `pred` holds, as a predicated store
// (no branch, so the warp never splits around it).
__device__ __forceinline__ void st_shared_if(bool pred, void* p, float4 v) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("{\n .reg .pred q;\n setp.ne.u32 q, %0, 0;\n @q st.shared.v4.f32 [%1], {%2, %3, %4, %5};\n}"
               ::"r"((unsigned)pred), "r"(a), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w) : "memory");
}
__device__ __forceinline__ void st_shared_if(bool pred, void* p, float2 v) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("{\n .reg .pred q;\n setp.ne.u32 q, %0, 0;\n @q st.shared.v2.f32 [%1], {%2, %3};\n}"
               ::"r"((unsigned)pred), "r"(a), "f"(v.x), "f"(v.y) : "memory");
}
__device__ __forceinline__ void st_shared_if(bool pred, void* p, int v) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("{\n .reg .pred q;\n setp.ne.u32 q, %0, 0;\n @q st.shared.s32 [%1], %2;\n}"
               ::"r"((unsigned)pred), "r"(a), "r"(v) : "memory");
}

// Exchanges the halves of both pairs of a (re, re', im, im') slot.
__device__ __forceinline__ float4 swap_pair(float4 v) { return make_float4(v.y, v.x, v.w, v.z); }

// Three-input unsigned max.
__device__ __forceinline__ uint32_t max3u(uint32_t a, uint32_t b, uint32_t c) {
  return max(a, max(b, c));
}

// Static loop helper: f(std::integral_constant<int, I>) for I = 0..N-1.
template <int I, int N, typename Fn>
__device__ __forceinline__ void static_for(Fn&& f) {
  if constexpr (I < N) {
    f(std::integral_constant<int, I>{});
    static_for<I + 1, N>(f);
  }
}

// ===========================================================================
// Executor 1: FP32, F = 32.  One warp per lost block.  Lane l owns spectrum
// column k2 = l, bins (k1 = j, l) for j = 0..31 in registers.  W sits in
// shared memory with its 32 rows stored twice, so W(k - u) for row j is at a
// per-iteration base plus the compile-time offset j * 32.
// ===========================================================================
struct alignas(128) WarpSmem32 {
  float2 Wd[64 * 32];     // rows 0..63: W rows (r mod 32); 32..63 double as FFT buffer,
                          // 0..31 take the TMA support boxes during staging
  float2 coef_d[KMAX];
  int32_t coef_u[KMAX];
  float red[32];
  uint64_t mbar;          // completion of the TMA staging copies
  uint32_t tma_ph;        // stagings done (phase parity)
  TileDev T;              // descriptors of the current block's tile and job
  JobDev J;
};
constexpr size_t SMEM32 = 64 * sizeof(float2) + NW32 * sizeof(WarpSmem32);

// Prologue of one F = 32 block: descriptors into shared memory, the support
// staged into zbuf (32 x 32, swizzled), row FFTs in place, then the column
// FFTs into registers: x[k1] = Z(k1, lane).
// Returns false when the TMA staging's bounded wait ran out: the error is
// flagged, the copies in flight are waited for (bounded again), and the warp
// must stop (its buffer and mbarrier phase are no longer in a known state).
template <class WS>
__device__ __forceinline__ bool stage_fft32(const ExecArgs& a, int id, WS& sm, float2* zbuf, int lane,
                                            float2 (&x)[32], unsigned char* sbuf, int sbytes, float& rbar) {
  const ClassArgs& C = a.c[CLS_F32_32];
  const int2 it = ld_in(C.items + id, a.server != 0);
  copy_desc(&sm.T, a.tiles + it.x, lane, 32, a.server != 0);
  __syncwarp();
  copy_desc(&sm.J, a.jobs + sm.T.job, lane, 32, a.server != 0);
  __syncwarp();
  const TileDev& T = sm.T;
  const JobDev& J = sm.J;
  const int I = it.y >> 16, Jb = it.y & 0xFFFF;
  const int S = J.S;
  float* val = a.val_f + T.val_off;
  if (lane == 0) debug_record(a, CLS_F32_32, id, T, it.x, I, Jb);
  if (tma_usable(T, J, sbuf, sbytes)) {
    const uint32_t ph = sm.tma_ph;
    if (lane == 0) tma_issue_support(T, J, I, Jb, sbuf, &sm.mbar, a.dbg_tma_stall != 0);
    // every lane waits with its own clock; the warp agrees on the outcome
    if (!__all_sync(0xffffffffu, mbar_wait(&sm.mbar, ph & 1, a.timeout_ns))) {
      if (lane == 0) {
        atomicOr(&C.q->error, ERR_TIMEOUT);
        if (a.dbg_tma_stall) mbar_arrive(&sm.mbar);
      }
      __syncwarp();
      mbar_wait(&sm.mbar, ph & 1, a.timeout_ns);  // the copies in flight, bounded again
      __syncwarp();
      return false;
    }
    stage_from_boxes<32>(T, J, I, Jb, zbuf, sbuf, lane, 32);
    __syncwarp();
    if (lane == 0) sm.tma_ph = ph + 1;
  } else {
    stage_support<32, float, float2>(T, J, val, I, Jb, zbuf, lane, 32, a.server != 0);
  }
  __syncwarp();
  const float c = support_mean<32, 32>(zbuf, S, lane, nullptr);
  // row FFTs of w (r - c): lane m transforms support row m
  if (lane < S) {
#pragma unroll
    for (int n = 0; n < 32; ++n) x[n] = n < S ? centred(zbuf[swz<32>(lane, n)], c) : make_float2(0.f, 0.f);
    fft_reg<32>(x);
#pragma unroll
    for (int n = 0; n < 32; ++n) zbuf[swz<32>(lane, n)] = x[n];
  }
  __syncwarp();
  // column FFTs: lane l transforms column l
#pragma unroll
  for (int m = 0; m < 32; ++m) x[m] = m < S ? zbuf[swz<32>(m, lane)] : make_float2(0.f, 0.f);
  fft_reg<32>(x);
  __syncwarp();
  rbar = c;
  return true;
}

__device__ __forceinline__ bool item_f32_32(const ExecArgs& a, int id, WarpSmem32& sm, const float2* tw,
                            int lane) {
  const ClassArgs& C = a.c[CLS_F32_32];
  float2 x[32];
  // stage -> rows 32..63 (swizzled F x F buffer); TMA boxes in rows 0..31
  float rbar;
  if (!stage_fft32(a, id, sm, sm.Wd + 32 * 32, lane, x, reinterpret_cast<unsigned char*>(sm.Wd), 8192, rbar)) return false;
  const int2 it = ld_in(C.items + id, a.server != 0);
  const TileDev& T = sm.T;
  const JobDev& J = sm.J;
  const int I = it.y >> 16, Jb = it.y & 0xFFFF;
  const int K = J.K;
  float* val = a.val_f + T.val_off;
  // Hermitian split: W = (Z(k) + conj Z(-k))/2, R' = (Z(k) - conj Z(-k))/(2i),
  // R_w = rbar W + R'
  const int src = (32 - lane) & 31;
#pragma unroll
  for (int j = 0; j <= 16; ++j) {
    const int j2 = (32 - j) & 31;
    float2 zm, zm2;
    zm.x = __shfl_sync(0xffffffffu, x[j2].x, src);
    zm.y = __shfl_sync(0xffffffffu, x[j2].y, src);
    zm2.x = __shfl_sync(0xffffffffu, x[j].x, src);
    zm2.y = __shfl_sync(0xffffffffu, x[j].y, src);
    const float2 z = x[j], z2 = x[j2];
    const float2 w = make_float2(0.5f * (z.x + zm.x), 0.5f * (z.y - zm.y));
    sm.Wd[j * 32 + lane] = w;
    sm.Wd[(j + 32) * 32 + lane] = w;
    x[j] = make_float2(fmaf(rbar, w.x, 0.5f * (z.y + zm.y)), fmaf(rbar, w.y, 0.5f * (zm.x - z.x)));
    if (j2 != j) {
      const float2 w2 = make_float2(0.5f * (z2.x + zm2.x), 0.5f * (z2.y - zm2.y));
      sm.Wd[j2 * 32 + lane] = w2;
      sm.Wd[(j2 + 32) * 32 + lane] = w2;
      x[j2] = make_float2(fmaf(rbar, w2.x, 0.5f * (z2.y + zm2.y)), fmaf(rbar, w2.y, 0.5f * (zm2.x - z2.x)));
    }
  }
  __syncwarp();
  const float W0 = sm.Wd[0].x;
  if (!(W0 > 0.f)) {  // no usable pixel in the support
    if (lane == 0) atomicAdd(&C.q->n_empty, 1);
    return true;
  }
  const float gs = J.gamma_f / W0;
  float2(&R)[32] = x;

  // key: energy bits with the low 5 bits replaced by 31 - row; equal keys go
  // to the lowest lane, i.e. the lowest flat index
  const uint32_t kmask = opaque(0xFFFFFFE0u);
  uint32_t bq[4] = {0u, 0u, 0u, 0u};  // four independent max chains, three-input max
  static_for<0, 16>([&](auto h) {
    constexpr int j = 2 * decltype(h)::value;
    const float e0 = fmaf(R[j].y, R[j].y, R[j].x * R[j].x);
    const float e1 = fmaf(R[j + 1].y, R[j + 1].y, R[j + 1].x * R[j + 1].x);
    bq[(j >> 1) & 3] = max3u(bq[(j >> 1) & 3], make_key<31u - j>(e0, kmask),
                             make_key<30u - j>(e1, kmask));
  });
  uint32_t best = max3u(bq[0], bq[1], max(bq[2], bq[3]));
  for (int iter = 0; iter < K; ++iter) {
    const uint32_t wbest = __reduce_max_sync(0xffffffffu, best);
    const int u2 = __ffs(__ballot_sync(0xffffffffu, best == wbest)) - 1;
    const int u1 = 31 - (int)(wbest & 31u);
    const int flat = u1 * 32 + u2;
    const float2 v = select_reg<32>(R, u1);
    const float rux = __shfl_sync(0xffffffffu, v.x, u2);
    const float ruy = __shfl_sync(0xffffffffu, v.y, u2);
    const float dx = gs * rux, dy = gs * ruy;
    st_shared_if(lane == 0, &sm.coef_u[iter], flat);
    st_shared_if(lane == 0, &sm.coef_d[iter], make_float2(dx, dy));
    if (iter + 1 == K) break;
    const float2* wp = sm.Wd + (32 - u1) * 32 + ((lane - u2) & 31);
    const float ndx = -dx, ndy = -dy;
    bq[0] = bq[1] = bq[2] = bq[3] = 0u;
    static_for<0, 16>([&](auto h) {
      constexpr int j = 2 * decltype(h)::value;
      float e[2];
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const float2 w = wp[(j + k) * 32];
        float rx = fmaf(ndx, w.x, R[j + k].x);
        rx = fmaf(dy, w.y, rx);
        float ry = fmaf(ndx, w.y, R[j + k].y);
        ry = fmaf(ndy, w.x, ry);
        R[j + k] = make_float2(rx, ry);
        e[k] = fmaf(ry, ry, rx * rx);
      }
      bq[(j >> 1) & 3] = max3u(bq[(j >> 1) & 3], make_key<31u - j>(e[0], kmask),
                               make_key<30u - j>(e[1], kmask));
    });
    best = max3u(bq[0], bq[1], max(bq[2], bq[3]));
  }
  __syncwarp();
  if (a.dbg_useq)
    for (int k = lane; k < K; k += 32) debug_useq(a, CLS_F32_32, id, k, sm.coef_u[k]);
  eval_and_write<false, float, float2>(T, J, val, I, Jb, sm.coef_u, sm.coef_d, tw, sm.red, lane,
                                       32, a.server != 0);
  return true;
}

// ---------------------------------------------------------------------------
// Paired-bin layout of the F = 32 executor.  Lane L = 16 h + p owns the bins
// (k1, p) and (k1, p + 16) for the 16 rows k1 = 8 m + 4 h + j (m, j = 0..3),
// as pairs RX[4m + j] = (Re R(k1, p), Re R(k1, p + 16)), RY likewise.  W is a
// table of 16-byte slots (Re W(r, d), Re W(r, d ^ 16), Im W(r, d),
// Im W(r, d ^ 16)) with rows 0..2 repeated as rows 32..34; rows 0..15 double
// as the FFT buffer.  Equal keys name the same (m, j, column half), where the
// lower lane holds the lower row, then the lower column: the lowest lane is
// the lowest flat index.
// ---------------------------------------------------------------------------
struct alignas(128) WarpSmem32P {
  float4 Wt[35 * 32];  // rows 16..34 take the TMA support boxes during staging
  float2 coef_d[KMAX];
  int32_t coef_u[KMAX];
  float red[32];
  uint64_t mbar;
  uint32_t tma_ph;
  TileDev T;
  JobDev J;
};

template <int U>
__device__ __forceinline__ bool item_f32_32p(const ExecArgs& a, int id, WarpSmem32P& sm, const float2* tw,
                                             int lane) {
  const ClassArgs& C = a.c[CLS_F32_32];
  float2* zbuf = reinterpret_cast<float2*>(sm.Wt);
  float4* Wt = sm.Wt;
  float2 x[32];
  float rbar;
  if (!stage_fft32(a, id, sm, zbuf, lane, x, reinterpret_cast<unsigned char*>(sm.Wt) + 8192, 35 * 32 * 16 - 8192, rbar)) return false;
  const int2 it = ld_in(C.items + id, a.server != 0);
  const TileDev& T = sm.T;
  const JobDev& J = sm.J;
  const int I = it.y >> 16, Jb = it.y & 0xFFFF;
  const int K = J.K;
  float* val = a.val_f + T.val_off;
  // the column spectra back to the buffer, then the Hermitian split of the
  // pairs this lane owns
#pragma unroll
  for (int k1 = 0; k1 < 32; ++k1) zbuf[swz<32>(k1, lane)] = x[k1];
  __syncwarp();
  const int p = lane & 15, h = lane >> 4;
  float2 RX[16], RY[16];
  float4 wlo[8];
  static_for<0, 16>([&](auto P) {
    constexpr int pi = decltype(P)::value, m = pi >> 2, j = pi & 3;
    const int k1 = 8 * m + 4 * h + j, k1m = (32 - k1) & 31;
    float2 w[2], r[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int col = p + 16 * c, colm = (32 - col) & 31;
      const float2 z = zbuf[swz<32>(k1, col)], zm = zbuf[swz<32>(k1m, colm)];
      w[c] = make_float2(0.5f * (z.x + zm.x), 0.5f * (z.y - zm.y));
      r[c] = make_float2(fmaf(rbar, w[c].x, 0.5f * (z.y + zm.y)), fmaf(rbar, w[c].y, 0.5f * (zm.x - z.x)));
    }
    RX[pi] = make_float2(r[0].x, r[1].x);
    RY[pi] = make_float2(r[0].y, r[1].y);
    const float4 slot = make_float4(w[0].x, w[1].x, w[0].y, w[1].y);
    if constexpr (m >= 2) {  // rows 16..31: past the FFT buffer
      Wt[k1 * 32 + p] = slot;
      Wt[k1 * 32 + p + 16] = swap_pair(slot);
    } else {
      wlo[pi] = slot;
    }
  });
  __syncwarp();
  static_for<0, 8>([&](auto P) {
    constexpr int pi = decltype(P)::value, m = pi >> 2, j = pi & 3;
    const int k1 = 8 * m + 4 * h + j;
    Wt[k1 * 32 + p] = wlo[pi];
    Wt[k1 * 32 + p + 16] = swap_pair(wlo[pi]);
    if (m == 0 && j < 3 && h == 0) {
      Wt[(k1 + 32) * 32 + p] = wlo[pi];
      Wt[(k1 + 32) * 32 + p + 16] = swap_pair(wlo[pi]);
    }
  });
  __syncwarp();
  const float W0 = Wt[0].x;
  if (!(W0 > 0.f)) {  // no usable pixel in the support
    if (lane == 0) atomicAdd(&C.q->n_empty, 1);
    return true;
  }
  const float gs = J.gamma_f / W0;
  // key: energy bits with the low 5 bits replaced by 31 - l, l = 2 pi + c
  const uint32_t kmask = opaque(~31u);
  uint32_t bq[4] = {0u, 0u, 0u, 0u};
  static_for<0, 16>([&](auto P) {
    constexpr int pi = decltype(P)::value;
    float2 e = __fmul2_rn(RX[pi], RX[pi]);
    e = __ffma2_rn(RY[pi], RY[pi], e);
    bq[pi & 3] = max3u(bq[pi & 3], make_key<(uint32_t)(31 - 2 * pi)>(e.x, kmask),
                       make_key<(uint32_t)(30 - 2 * pi)>(e.y, kmask));
  });
  uint32_t best = max3u(bq[0], bq[1], max(bq[2], bq[3]));
#pragma unroll U  // K-loop unroll factor (autotuned)
  for (int iter = 0; iter < K; ++iter) {
    const uint32_t wbest = __reduce_max_sync(0xffffffffu, best);
    const int l_w = __ffs(__ballot_sync(0xffffffffu, best == wbest)) - 1;
    const int ell = 31 - (int)(wbest & 31u), pw = ell >> 1;
    const int u1 = 8 * (pw >> 2) + 4 * (l_w >> 4) + (pw & 3);
    const int u2 = (l_w & 15) + 16 * (ell & 1);
    float2 view[32];  // bin l as (Re, Im): register aliases, no copies
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      view[2 * k] = make_float2(RX[k].x, RY[k].x);
      view[2 * k + 1] = make_float2(RX[k].y, RY[k].y);
    }
    const float2 v = select_reg32(view, ell);
    const float rux = __shfl_sync(0xffffffffu, v.x, l_w);
    const float ruy = __shfl_sync(0xffffffffu, v.y, l_w);
    const float dx = gs * rux, dy = gs * ruy;
    st_shared_if(lane == 0, &sm.coef_u[iter], u1 * 32 + u2);
    st_shared_if(lane == 0, &sm.coef_d[iter], make_float2(dx, dy));
    if (iter + 1 == K) break;
    const int d = (p - u2) & 31;
    const float4* wp[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) wp[m] = Wt + ((8 * m + 4 * h - u1) & 31) * 32 + d;
    const float2 ndx2 = make_float2(-dx, -dx), dy2 = make_float2(dy, dy), ndy2 = make_float2(-dy, -dy);
    bq[0] = bq[1] = bq[2] = bq[3] = 0u;
    static_for<0, 16>([&](auto P) {
      constexpr int pi = decltype(P)::value, m = pi >> 2, j = pi & 3;
      const float4 w = wp[m][j * 32];
      const float2 wx = make_float2(w.x, w.y), wy = make_float2(w.z, w.w);
      float2 rx = __ffma2_rn(ndx2, wx, RX[pi]);
      rx = __ffma2_rn(dy2, wy, rx);
      float2 ry = __ffma2_rn(ndx2, wy, RY[pi]);
      ry = __ffma2_rn(ndy2, wx, ry);
      RX[pi] = rx;
      RY[pi] = ry;
      float2 e = __fmul2_rn(rx, rx);
      e = __ffma2_rn(ry, ry, e);
      bq[pi & 3] = max3u(bq[pi & 3], make_key<(uint32_t)(31 - 2 * pi)>(e.x, kmask),
                         make_key<(uint32_t)(30 - 2 * pi)>(e.y, kmask));
    });
    best = max3u(bq[0], bq[1], max(bq[2], bq[3]));
  }
  __syncwarp();
  if (a.dbg_useq)
    for (int k = lane; k < K; k += 32) debug_useq(a, CLS_F32_32, id, k, sm.coef_u[k]);
  eval_and_write<false, float, float2>(T, J, val, I, Jb, sm.coef_u, sm.coef_d, tw, sm.red, lane,
                                       32, a.server != 0);
  return true;
}
constexpr size_t SMEM32P = 64 * sizeof(float2) + NW32 * sizeof(WarpSmem32P);

// ---------------------------------------------------------------------------
// Run layout of the F = 32 executor: lane l owns column l and all 32 rows, as
// the column layout does, but reads its rows in four runs of eight, each from
// its own base row, so W needs only rows 0..6 repeated (39 rows, 9.75 KB per
// warp) and the table overlays the FFT buffer.  Same arithmetic and keys as
// the column layout; more warps fit on an SM.
// ---------------------------------------------------------------------------
// PAD = 2688: bytes 8192..15871 from Wd take the TMA support boxes.  The
// compact form (PAD = 16, layout 4) stages with plain loads only and fits
// 8 CTAs of 2 warps per SM at 128 registers per thread.
constexpr int RUN32 = 8;                // rows per run
constexpr int ROWS32 = 32 + RUN32 - 1;  // table rows: 0..31, then 0..RUN32-2 again
template <int PAD>
struct alignas(128) WarpSmem32RT {
  float2 Wd[ROWS32 * 32];  // W rows 0..31 and the repeated rows; rows 0..31 double as FFT buffer
  float2 coef_d[KMAX];
  int32_t coef_u[KMAX];
  float red[32];
  unsigned char stage_pad[PAD];
  uint64_t mbar;
  uint32_t tma_ph;
  TileDev T;
  JobDev J;
};
using WarpSmem32R = WarpSmem32RT<2688>;
using WarpSmem32C = WarpSmem32RT<16>;
static_assert(offsetof(WarpSmem32R, stage_pad) + 2688 >= 8192 + 7680, "TMA box area");

template <int U, class WS>
__device__ __forceinline__ bool item_f32_32r(const ExecArgs& a, int id, WS& sm, const float2* tw,
                                             int lane) {
  const ClassArgs& C = a.c[CLS_F32_32];
  float2 x[32];
  float rbar;
  constexpr bool kTma = std::is_same<WS, WarpSmem32R>::value;  // the compact form has no box space
  if (!stage_fft32(a, id, sm, sm.Wd, lane, x, kTma ? reinterpret_cast<unsigned char*>(sm.Wd) + 8192 : nullptr,
                   kTma ? 7680 : 0, rbar))
    return false;
  const int2 it = ld_in(C.items + id, a.server != 0);
  const TileDev& T = sm.T;
  const JobDev& J = sm.J;
  const int I = it.y >> 16, Jb = it.y & 0xFFFF;
  const int K = J.K;
  float* val = a.val_f + T.val_off;
  // Hermitian split from registers (the FFT buffer is no longer read),
  // R_w = rbar W + R'
  const int src = (32 - lane) & 31;
#pragma unroll
  for (int j = 0; j <= 16; ++j) {
    const int j2 = (32 - j) & 31;
    float2 zm, zm2;
    zm.x = __shfl_sync(0xffffffffu, x[j2].x, src);
    zm.y = __shfl_sync(0xffffffffu, x[j2].y, src);
    zm2.x = __shfl_sync(0xffffffffu, x[j].x, src);
    zm2.y = __shfl_sync(0xffffffffu, x[j].y, src);
    const float2 z = x[j], z2 = x[j2];
    const float2 w = make_float2(0.5f * (z.x + zm.x), 0.5f * (z.y - zm.y));
    sm.Wd[j * 32 + lane] = w;
    if (j < RUN32 - 1) sm.Wd[(j + 32) * 32 + lane] = w;
    x[j] = make_float2(fmaf(rbar, w.x, 0.5f * (z.y + zm.y)), fmaf(rbar, w.y, 0.5f * (zm.x - z.x)));
    if (j2 != j) {
      const float2 w2 = make_float2(0.5f * (z2.x + zm2.x), 0.5f * (z2.y - zm2.y));
      sm.Wd[j2 * 32 + lane] = w2;
      x[j2] = make_float2(fmaf(rbar, w2.x, 0.5f * (z2.y + zm2.y)), fmaf(rbar, w2.y, 0.5f * (zm2.x - z2.x)));
    }
  }
  __syncwarp();
  const float W0 = sm.Wd[0].x;
  if (!(W0 > 0.f)) {  // no usable pixel in the support
    if (lane == 0) atomicAdd(&C.q->n_empty, 1);
    return true;
  }
  const float gs = J.gamma_f / W0;
  float2(&R)[32] = x;
  // key: energy bits with the low 5 bits replaced by 31 - row; ties between
  // lanes (equal keys) go to the lowest lane, i.e. the lowest flat index
  const uint32_t kmask = opaque(0xFFFFFFE0u);
  uint32_t bq[4] = {0u, 0u, 0u, 0u};
  static_for<0, 16>([&](auto h) {
    constexpr int j = 2 * decltype(h)::value;
    const float e0 = fmaf(R[j].y, R[j].y, R[j].x * R[j].x);
    const float e1 = fmaf(R[j + 1].y, R[j + 1].y, R[j + 1].x * R[j + 1].x);
    bq[(j >> 1) & 3] = max3u(bq[(j >> 1) & 3], make_key<31u - j>(e0, kmask),
                             make_key<30u - j>(e1, kmask));
  });
  uint32_t best = max3u(bq[0], bq[1], max(bq[2], bq[3]));
#pragma unroll U  // K-loop unroll factor (autotuned)
  for (int iter = 0; iter < K; ++iter) {
    const uint32_t wbest = __reduce_max_sync(0xffffffffu, best);
    const int u2 = __ffs(__ballot_sync(0xffffffffu, best == wbest)) - 1;
    const int u1 = 31 - (int)(wbest & 31u);
    const int flat = u1 * 32 + u2;
    const float2 v = select_reg<32>(R, u1);
    const float rux = __shfl_sync(0xffffffffu, v.x, u2);
    const float ruy = __shfl_sync(0xffffffffu, v.y, u2);
    const float dx = gs * rux, dy = gs * ruy;
    st_shared_if(lane == 0, &sm.coef_u[iter], flat);
    st_shared_if(lane == 0, &sm.coef_d[iter], make_float2(dx, dy));
    if (iter + 1 == K) break;
    const int d = (lane - u2) & 31;
    const float2* wp[32 / RUN32];
#pragma unroll
    for (int q = 0; q < 32 / RUN32; ++q) wp[q] = sm.Wd + ((RUN32 * q - u1) & 31) * 32 + d;
    const float ndx = -dx, ndy = -dy;
    bq[0] = bq[1] = bq[2] = bq[3] = 0u;
    static_for<0, 16>([&](auto h) {
      constexpr int j = 2 * decltype(h)::value;
      float e[2];
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const float2 w = wp[(j + k) / RUN32][((j + k) % RUN32) * 32];
        float rx = fmaf(ndx, w.x, R[j + k].x);
        rx = fmaf(dy, w.y, rx);
        float ry = fmaf(ndx, w.y, R[j + k].y);
        ry = fmaf(ndy, w.x, ry);
        R[j + k] = make_float2(rx, ry);
        e[k] = fmaf(ry, ry, rx * rx);
      }
      bq[(j >> 1) & 3] = max3u(bq[(j >> 1) & 3], make_key<31u - j>(e[0], kmask),
                               make_key<30u - j>(e[1], kmask));
    });
    best = max3u(bq[0], bq[1], max(bq[2], bq[3]));
  }
  __syncwarp();
  if (a.dbg_useq)
    for (int k = lane; k < K; k += 32) debug_useq(a, CLS_F32_32, id, k, sm.coef_u[k]);
  eval_and_write<false, float, float2>(T, J, val, I, Jb, sm.coef_u, sm.coef_d, tw, sm.red, lane,
                                       32, a.server != 0);
  return true;
}
constexpr size_t SMEM32R = 64 * sizeof(float2) + NW32 * sizeof(WarpSmem32R);
constexpr size_t SMEM32C = 64 * sizeof(float2) + NW32 * sizeof(WarpSmem32C);
static_assert(8 * (SMEM32C + 1024) <= 228 * 1024, "layout 4: 8 CTAs per SM");

template <class WS, int U>
__device__ __forceinline__ bool run_item32(const ExecArgs& a, int id, WS& sm, const float2* tw, int lane) {
  if constexpr (std::is_same<WS, WarpSmem32P>::value) return item_f32_32p<U>(a, id, sm, tw, lane);
  else if constexpr (std::is_same<WS, WarpSmem32R>::value || std::is_same<WS, WarpSmem32C>::value)
    return item_f32_32r<U>(a, id, sm, tw, lane);
  else return item_f32_32(a, id, sm, tw, lane);
}

template <class WS, int U>
__global__ void __launch_bounds__(NW32 * 32, std::is_same<WS, WarpSmem32C>::value
                                                 ? 8
                                                 : (std::is_same<WS, WarpSmem32R>::value ? 6 : 5))
    k_exec_f32_32(const __grid_constant__ ExecArgs a) {
  extern __shared__ __align__(128) unsigned char smem32_raw[];
  float2* tw = reinterpret_cast<float2*>(smem32_raw);
  WS* wsm = reinterpret_cast<WS*>(smem32_raw + 64 * sizeof(float2));
  for (int q = threadIdx.x; q < 64; q += blockDim.x) tw[q] = make_float2(c_twf[q].x, -c_twf[q].y);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  WS& sm = wsm[warp];
  if (lane == 0) {
    mbar_init(&sm.mbar);
    sm.tma_ph = 0;
  }
  __syncwarp();
  const ClassArgs& C = a.c[CLS_F32_32];
  if (a.single_item >= 0) {
    if (blockIdx.x == 0 && warp == 0) run_item32<WS, U>(a, a.single_item, sm, tw, lane);
    return;
  }
  if (a.level_mode) {
    const int n = min(C.q->n_items, C.cap);
    for (int id = blockIdx.x * NW32 + warp; id < n; id += gridDim.x * NW32)
      if (a.level_of[(size_t)CLS_F32_32 * a.level_stride + id] == a.level)
        if (!run_item32<WS, U>(a, id, sm, tw, lane)) break;
    return;
  }
  for (;;) {
    const int id = a.server ? server_pop_warp(a, C, CLS_F32_32, lane) : queue_pop_warp(C, a.timeout_ns, lane);
    if (id < 0) break;
    if (id & SRV_CMD_BIT) {  // a request joins the running executor
      server_admit<false>(a, C, CLS_F32_32, id & ~SRV_CMD_BIT, lane, 32);
      continue;
    }
    // cancelled: release only (decided once, by lane 0, for the whole warp)
    const bool skip = a.server && __shfl_sync(0xffffffffu, lane == 0 ? (int)server_cancelled(a, C, id) : 0, 0);
    if (skip) {
      const int2 it = ld_in(C.items + id, a.server != 0);
      copy_desc(&sm.T, a.tiles + it.x, lane, 32, a.server != 0);
      __syncwarp();
      copy_desc(&sm.J, a.jobs + sm.T.job, lane, 32, a.server != 0);
      __syncwarp();
    } else if (!run_item32<WS, U>(a, id, sm, tw, lane)) {
      break;  // staging timed out: this warp stops
    }
    // value-plane stores before later blocks' TMA (asynchronous-proxy) reads
    asm volatile("fence.proxy.async.global;" ::: "memory");
    __threadfence();
    __syncwarp();
    const int2 it = ld_in(C.items + id, a.server != 0);
    release_successors(a, C, sm.T, sm.J, it.y >> 16, it.y & 0xFFFF, lane, 32);
    __syncwarp();
    if (lane == 0) {
      atomicAdd(&C.q->n_done, 1);
      if (a.server) server_block_done(a, sm.T.job);
    }
    __syncwarp();
  }
}

// ===========================================================================
// Executor 2: FP32, F = 64.  NWB warps (NT = 32*NWB threads) per lost block.
// Thread t owns spectrum column c = t & 63 and rows k1 = i + RPT*(t >> 6),
// i = 0..RPT-1 (RPT = 4096 / NT), in registers.  Per iteration: warp max
// (redux), then an NWB-way exchange through shared memory behind one
// barrier, double-buffered by iteration parity.
// ===========================================================================
template <int NWB, int ROWS = 128>
struct alignas(16) CtaSmem64 {
  float2 Wd[ROWS * 64];  // W rows (r mod 64); ROWS = 128: 64..127 double as FFT buffer,
                         // ROWS = 96: 0..63 are the FFT buffer, 64..95 copy rows 0..31
  float2 coef_d[KMAX];
  int32_t coef_u[KMAX];
  float2 tw[64];
  float red[NWB * 32];
  alignas(16) float4 xrec[2][NWB];  // per warp: (key bits, flat bits, Re R_u, Im R_u)
  int item;
  int skip;  // server mode: the popped block's request is cancelled
  TileDev T;
  JobDev J;
};

// Prologue of one F = 64 block: descriptors into shared memory, the support
// staged into zbuf (64 x 64, swizzled) and transformed in place by the 2-D FFT.
// Ends behind a barrier.
template <int NT, class Sm>
__device__ __forceinline__ float stage_fft64(const ExecArgs& a, int id, Sm& sm, float2* zbuf, int t) {
  const ClassArgs& C = a.c[CLS_F32_64];
  const int2 it = ld_in(C.items + id, a.server != 0);
  copy_desc(&sm.T, a.tiles + it.x, t, NT, a.server != 0);
  __syncthreads();
  copy_desc(&sm.J, a.jobs + sm.T.job, t, NT, a.server != 0);
  __syncthreads();
  const TileDev& T = sm.T;
  const JobDev& J = sm.J;
  const int I = it.y >> 16, Jb = it.y & 0xFFFF;
  const int S = J.S;
  float* val = a.val_f + T.val_off;
  if (t == 0) debug_record(a, CLS_F32_64, id, T, it.x, I, Jb);

  stage_support<64, float, float2>(T, J, val, I, Jb, zbuf, t, NT, a.server != 0);
  __syncthreads();
  const float c = support_mean<64, NT>(zbuf, S, t, sm.red);
  // rows of w (r - c), 64-point lines on lane pairs (l, l ^ 16): half h transforms the samples
  // 2n + h (32 points), then X[k + 32h] = E[k] +- exp(-2 pi i k/64) O[k].
  // NT/2 lines per pass.
  for (int lb = 0; lb < 64; lb += NT / 2) {
    const int h = (t >> 4) & 1, line = lb + (((t >> 5) << 4) | (t & 15));
    float2 x[32];
    // row FFTs (rows >= S are zero).  The branch is warp-uniform: the pair
    // combine shuffles across the whole warp, so every lane of a warp that
    // holds any row < S takes part; lanes past S only skip loads and stores.
    if (t < 128 && lb + ((t >> 5) << 4) < S) {
      const bool live = line < S;
#pragma unroll
      for (int n = 0; n < 32; ++n)
        x[n] = live && 2 * n + h < S ? centred(zbuf[swz<64>(live ? line : 0, 2 * n + h)], c)
                                     : make_float2(0.f, 0.f);
      fft_reg<32>(x);
      fft64_combine(x, h);
      if (live) {
#pragma unroll
        for (int k = 0; k < 32; ++k) zbuf[swz<64>(line, k + 32 * h)] = x[k];
      }
    }
  }
  __syncthreads();
  for (int lb = 0; lb < 64; lb += NT / 2) {
    if (t < 128) {
      // column FFTs: own column only
      const int h = (t >> 4) & 1, line = lb + (((t >> 5) << 4) | (t & 15));
      float2 x[32];
#pragma unroll
      for (int n = 0; n < 32; ++n)
        x[n] = 2 * n + h < S ? zbuf[swz<64>(2 * n + h, line)] : make_float2(0.f, 0.f);
      fft_reg<32>(x);
      fft64_combine(x, h);
#pragma unroll
      for (int k = 0; k < 32; ++k) zbuf[swz<64>(k + 32 * h, line)] = x[k];
    }
  }
  __syncthreads();
  return c;
}

template <int NWB, int ROWS>
__device__ __forceinline__ void item_f32_64(const ExecArgs& a, int id, CtaSmem64<NWB, ROWS>& sm, int t) {
  constexpr int NT = NWB * 32, RPT = 4096 / NT;
  const ClassArgs& C = a.c[CLS_F32_64];
  float2* zbuf = ROWS == 128 ? sm.Wd + 64 * 64 : sm.Wd;
  const float rbar = stage_fft64<NT>(a, id, sm, zbuf, t);
  const int2 it = ld_in(C.items + id, a.server != 0);
  const TileDev& T = sm.T;
  const JobDev& J = sm.J;
  const int I = it.y >> 16, Jb = it.y & 0xFFFF;
  const int K = J.K;
  float* val = a.val_f + T.val_off;
  const int c = t & 63, q = t >> 6, lane = t & 31, warp = t >> 5;
  float2 R[RPT];
  if constexpr (ROWS == 128) {
    const int cm = (64 - c) & 63;
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
      const int k1 = i + RPT * q, k1m = (64 - k1) & 63;
      const float2 z = zbuf[swz<64>(k1, c)], zm = zbuf[swz<64>(k1m, cm)];
      const float2 w = make_float2(0.5f * (z.x + zm.x), 0.5f * (z.y - zm.y));
      sm.Wd[k1 * 64 + c] = w;
      R[i] = make_float2(fmaf(rbar, w.x, 0.5f * (z.y + zm.y)), fmaf(rbar, w.y, 0.5f * (zm.x - z.x)));
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
      const int k1 = i + RPT * q;
      sm.Wd[(k1 + 64) * 64 + c] = sm.Wd[k1 * 64 + c];
    }
    __syncthreads();
  } else {
    // R = rbar W + (Z(k) - conj Z(-k)) / 2i into registers (reads only)
    const int cm = (64 - c) & 63;
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
      const int k1 = i + RPT * q, k1m = (64 - k1) & 63;
      const float2 z = zbuf[swz<64>(k1, c)], zm = zbuf[swz<64>(k1m, cm)];
      R[i] = make_float2(fmaf(rbar, 0.5f * (z.x + zm.x), 0.5f * (z.y + zm.y)),
                         fmaf(rbar, 0.5f * (z.y - zm.y), 0.5f * (zm.x - z.x)));
    }
    __syncthreads();
    // W = (Z(k) + conj Z(-k)) / 2 in place, unswizzled.  The swizzle permutes
    // within a row, so a warp that owns rows k1 and -k1 touches no other
    // warp's data; all its reads precede its writes.
    for (int rp = warp; rp <= 32; rp += NWB) {
      const int k1 = rp, k1m = (64 - rp) & 63;
      float2 wa[2], wb[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int cc = lane + 32 * h, ccm = (64 - cc) & 63;
        const float2 z = zbuf[swz<64>(k1, cc)], zm = zbuf[swz<64>(k1m, ccm)];
        wa[h] = make_float2(0.5f * (z.x + zm.x), 0.5f * (z.y - zm.y));  // W(k1, cc)
        wb[h] = make_float2(wa[h].x, -wa[h].y);                        // W(-k1, -cc)
      }
      __syncwarp();
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int cc = lane + 32 * h, ccm = (64 - cc) & 63;
        sm.Wd[k1 * 64 + cc] = wa[h];
        sm.Wd[k1m * 64 + ccm] = wb[h];
      }
      __syncwarp();
    }
    __syncthreads();
    for (int e = t; e < 32 * 64; e += NT) sm.Wd[64 * 64 + e] = sm.Wd[e];
    __syncthreads();
  }
  const float W0 = sm.Wd[0].x;
  if (!(W0 > 0.f)) {
    if (t == 0) atomicAdd(&C.q->n_empty, 1);
    return;
  }
  const float gs = J.gamma_f / W0;
  // key = energy bits, low 12 bits replaced by 4095 - flat; flat = k1*64 + c
  // key: energy bits with the low log2(RPT) bits replaced by RPT-1-row; equal
  // keys are resolved by the lowest flat index (lane ballot, then warps)
  const uint32_t kmask = opaque(~(uint32_t)(RPT - 1));

  uint32_t bq[2] = {0u, 0u};
  static_for<0, RPT / 2>([&](auto h) {
    constexpr int i = 2 * decltype(h)::value;
    const float e0 = fmaf(R[i].y, R[i].y, R[i].x * R[i].x);
    const float e1 = fmaf(R[i + 1].y, R[i + 1].y, R[i + 1].x * R[i + 1].x);
    bq[(i >> 1) & 1] = max3u(bq[(i >> 1) & 1], make_key<(uint32_t)(RPT - 1 - i)>(e0, kmask),
                             make_key<(uint32_t)(RPT - 2 - i)>(e1, kmask));
  });
  uint32_t best = max(bq[0], bq[1]);
  for (int iter = 0; iter < K; ++iter) {
    {
      const uint32_t wbest = __reduce_max_sync(0xffffffffu, best);
      const int l_w = __ffs(__ballot_sync(0xffffffffu, best == wbest)) - 1;
      const int i_w = RPT - 1 - (int)(wbest & (uint32_t)(RPT - 1));
      const int tw = (warp << 5) | l_w;  // the winning thread
      const int flat_w = (i_w + RPT * (tw >> 6)) * 64 + (tw & 63);
      const float2 v = select_reg<RPT>(R, i_w);  // meaningful in lane l_w only
      st_shared_if(lane == l_w, &sm.xrec[iter & 1][warp],
                   make_float4(__uint_as_float(wbest), __int_as_float(flat_w), v.x, v.y));
    }
    __syncthreads();
    // largest key over the warps (lowest flat index on equal keys), carrying R_u
    float4 rb = sm.xrec[iter & 1][0];
#pragma unroll
    for (int w = 1; w < NWB; ++w) {
      const float4 rw = sm.xrec[iter & 1][w];
      const uint32_t kw = __float_as_uint(rw.x), kb0 = __float_as_uint(rb.x);
      if (kw > kb0 || (kw == kb0 && __float_as_int(rw.y) < __float_as_int(rb.y))) rb = rw;
    }
    const int flat = __float_as_int(rb.y);
    const int u1 = flat >> 6, u2 = flat & 63;
    const float2 ru = make_float2(rb.z, rb.w);
    const float dx = gs * ru.x, dy = gs * ru.y;
    st_shared_if(t == 0, &sm.coef_u[iter], flat);
    st_shared_if(t == 0, &sm.coef_d[iter], make_float2(dx, dy));
    if (iter + 1 == K) break;
    const int r0 = RPT * q - u1;  // first W row of this thread, mod 64
    const float2* wp =
        sm.Wd + (ROWS == 128 ? r0 + 64 : (r0 < 0 ? r0 + 64 : r0)) * 64 + ((c - u2) & 63);
    const float ndx = -dx, ndy = -dy;
    bq[0] = bq[1] = 0u;
    static_for<0, RPT / 2>([&](auto h) {
      constexpr int i = 2 * decltype(h)::value;
      float e[2];
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const float2 w = wp[(i + k) * 64];
        float rx = fmaf(ndx, w.x, R[i + k].x);
        rx = fmaf(dy, w.y, rx);
        float ry = fmaf(ndx, w.y, R[i + k].y);
        ry = fmaf(ndy, w.x, ry);
        R[i + k] = make_float2(rx, ry);
        e[k] = fmaf(ry, ry, rx * rx);
      }
      bq[(i >> 1) & 1] = max3u(bq[(i >> 1) & 1], make_key<(uint32_t)(RPT - 1 - i)>(e[0], kmask),
                               make_key<(uint32_t)(RPT - 2 - i)>(e[1], kmask));
    });
    best = max(bq[0], bq[1]);
  }
  __syncthreads();
  if (a.dbg_useq)
    for (int k = t; k < K; k += NT) debug_useq(a, CLS_F32_64, id, k, sm.coef_u[k]);
  eval_and_write_call<true, float, float2>(T, J, val, I, Jb, sm.coef_u, sm.coef_d, sm.tw, sm.red, t,
                                      NT, a.server != 0);
}

// ---------------------------------------------------------------------------
// Paired-bin layout of the F = 64 executor (ROWS = ROWS_PAIRED, 4 warps).
// Thread t = 32 g + p owns the bins (k1, p) and (k1, p + 32) for the 16 rows
// k1 = 16 m + 4 g + j (m, j = 0..3), held as pairs: RX[4m + j] = (Re R(k1, p),
// Re R(k1, p + 32)), RY likewise for Im.  W is a table of 16-byte slots,
// slot (r, d) = (Re W(r, d), Re W(r, d ^ 32), Im W(r, d), Im W(r, d ^ 32)), so
// one 16-byte load gives W(k - u) for both bins of a pair, split into real and
// imaginary pairs: the update and the energy of two bins are six paired FP32
// instructions (fma.rn.f32x2 / mul.rn.f32x2) that round exactly like the
// scalar forms.  Each thread reads its rows in four runs of four; the table
// repeats rows 0..2 as rows 64..66 so a run that wraps stays contiguous.
// ---------------------------------------------------------------------------
constexpr int ROWS_PAIRED = 134;  // 67 rows of 64 float4 slots, counted in float2 rows

template <int NWB, int ROWS, int U>
__device__ __forceinline__ void item_f32_64p(const ExecArgs& a, int id, CtaSmem64<NWB, ROWS>& sm, int t) {
  static_assert(NWB == 4 && ROWS == ROWS_PAIRED, "paired layout: 4 warps, 67 table rows");
  constexpr int NT = 128;
  const ClassArgs& C = a.c[CLS_F32_64];
  float2* zbuf = sm.Wd;  // the FFT buffer is table rows 0..31
  float4* Wt = reinterpret_cast<float4*>(sm.Wd);
  const float rbar = stage_fft64<NT>(a, id, sm, zbuf, t);
  const int2 it = ld_in(C.items + id, a.server != 0);
  const TileDev& T = sm.T;
  const JobDev& J = sm.J;
  const int I = it.y >> 16, Jb = it.y & 0xFFFF;
  const int K = J.K;
  float* val = a.val_f + T.val_off;
  const int p = t & 31, g = t >> 5, lane = p, warp = g;

  // Hermitian split of Z = DFT(w + i w (r - rbar)): W = (Z(k) + conj Z(-k)) / 2
  // into the table, R = rbar W + (Z(k) - conj Z(-k)) / 2i into registers.  Table rows >= 32
  // lie past the FFT buffer and are written at once; rows < 32 wait for every
  // thread's reads.
  float2 RX[16], RY[16];
  float4 wlo[8];
  static_for<0, 16>([&](auto P) {
    constexpr int pi = decltype(P)::value, m = pi >> 2, j = pi & 3;
    const int k1 = 16 * m + 4 * g + j, k1m = (64 - k1) & 63;
    float2 w[2], r[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int col = p + 32 * h, colm = (64 - col) & 63;
      const float2 z = zbuf[swz<64>(k1, col)], zm = zbuf[swz<64>(k1m, colm)];
      w[h] = make_float2(0.5f * (z.x + zm.x), 0.5f * (z.y - zm.y));
      r[h] = make_float2(fmaf(rbar, w[h].x, 0.5f * (z.y + zm.y)), fmaf(rbar, w[h].y, 0.5f * (zm.x - z.x)));
    }
    RX[pi] = make_float2(r[0].x, r[1].x);
    RY[pi] = make_float2(r[0].y, r[1].y);
    const float4 slot = make_float4(w[0].x, w[1].x, w[0].y, w[1].y);
    if constexpr (m >= 2) {
      Wt[k1 * 64 + p] = slot;
      Wt[k1 * 64 + p + 32] = swap_pair(slot);
    } else {
      wlo[pi] = slot;
    }
  });
  __syncthreads();
  static_for<0, 8>([&](auto P) {
    constexpr int pi = decltype(P)::value, m = pi >> 2, j = pi & 3;
    const int k1 = 16 * m + 4 * g + j;
    Wt[k1 * 64 + p] = wlo[pi];
    Wt[k1 * 64 + p + 32] = swap_pair(wlo[pi]);
    if (m == 0 && j < 3 && g == 0) {
      Wt[(k1 + 64) * 64 + p] = wlo[pi];
      Wt[(k1 + 64) * 64 + p + 32] = swap_pair(wlo[pi]);
    }
  });
  __syncthreads();
  const float W0 = Wt[0].x;
  if (!(W0 > 0.f)) {
    if (t == 0) atomicAdd(&C.q->n_empty, 1);
    return;
  }
  const float gs = J.gamma_f / W0;
  // key: energy bits with the low 5 bits replaced by 31 - l, l = 2 pi + h the
  // thread's bin index (increasing with the flat index k1 * 64 + column);
  // equal keys are resolved by the lowest flat index (lane ballot, then warps)
  const uint32_t kmask = opaque(~31u);
  uint32_t bq[2] = {0u, 0u};
  static_for<0, 16>([&](auto P) {
    constexpr int pi = decltype(P)::value;
    float2 e = __fmul2_rn(RX[pi], RX[pi]);
    e = __ffma2_rn(RY[pi], RY[pi], e);
    bq[pi & 1] = max3u(bq[pi & 1], make_key<(uint32_t)(31 - 2 * pi)>(e.x, kmask),
                       make_key<(uint32_t)(30 - 2 * pi)>(e.y, kmask));
  });
  uint32_t best = max(bq[0], bq[1]);
#pragma unroll U  // K-loop unroll factor (autotuned)
  for (int iter = 0; iter < K; ++iter) {
    {
      const uint32_t wbest = __reduce_max_sync(0xffffffffu, best);
      const int l_w = __ffs(__ballot_sync(0xffffffffu, best == wbest)) - 1;
      const int ell = 31 - (int)(wbest & 31u), pw = ell >> 1;
      const int flat_w = (16 * (pw >> 2) + 4 * warp + (pw & 3)) * 64 + l_w + 32 * (ell & 1);
      float2 view[32];  // bin l as (Re, Im): register aliases, no copies
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        view[2 * k] = make_float2(RX[k].x, RY[k].x);
        view[2 * k + 1] = make_float2(RX[k].y, RY[k].y);
      }
      const float2 v = select_reg32(view, ell);  // meaningful in lane l_w only
      st_shared_if(lane == l_w, &sm.xrec[iter & 1][warp],
                   make_float4(__uint_as_float(wbest), __int_as_float(flat_w), v.x, v.y));
    }
    __syncthreads();
    // Equal keys of two warps name the same thread-local bin, so the lower
    // warp holds the lower row and the lower flat index: a two-level tree on
    // the keys alone, keeping the left record on ties.
    const float4 r0 = sm.xrec[iter & 1][0], r1 = sm.xrec[iter & 1][1];
    const float4 r2 = sm.xrec[iter & 1][2], r3 = sm.xrec[iter & 1][3];
    const float4 ra = __float_as_uint(r1.x) > __float_as_uint(r0.x) ? r1 : r0;
    const float4 rc = __float_as_uint(r3.x) > __float_as_uint(r2.x) ? r3 : r2;
    const float4 rb = __float_as_uint(rc.x) > __float_as_uint(ra.x) ? rc : ra;
    const int flat = __float_as_int(rb.y);
    const int u1 = flat >> 6, u2 = flat & 63;
    const float dx = gs * rb.z, dy = gs * rb.w;
    st_shared_if(t == 0, &sm.coef_u[iter], flat);
    st_shared_if(t == 0, &sm.coef_d[iter], make_float2(dx, dy));
    if (iter + 1 == K) break;
    const int d = (p - u2) & 63;
    const float4* wp[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) wp[m] = Wt + ((16 * m + 4 * g - u1) & 63) * 64 + d;
    const float2 ndx2 = make_float2(-dx, -dx), dy2 = make_float2(dy, dy), ndy2 = make_float2(-dy, -dy);
    bq[0] = bq[1] = 0u;
    static_for<0, 16>([&](auto P) {
      constexpr int pi = decltype(P)::value, m = pi >> 2, j = pi & 3;
      const float4 w = wp[m][j * 64];
      const float2 wx = make_float2(w.x, w.y), wy = make_float2(w.z, w.w);
      float2 rx = __ffma2_rn(ndx2, wx, RX[pi]);
      rx = __ffma2_rn(dy2, wy, rx);
      float2 ry = __ffma2_rn(ndx2, wy, RY[pi]);
      ry = __ffma2_rn(ndy2, wx, ry);
      RX[pi] = rx;
      RY[pi] = ry;
      float2 e = __fmul2_rn(rx, rx);
      e = __ffma2_rn(ry, ry, e);
      bq[pi & 1] = max3u(bq[pi & 1], make_key<(uint32_t)(31 - 2 * pi)>(e.x, kmask),
                         make_key<(uint32_t)(30 - 2 * pi)>(e.y, kmask));
    });
    best = max(bq[0], bq[1]);
  }
  __syncthreads();
  if (a.dbg_useq)
    for (int k = t; k < K; k += NT) debug_useq(a, CLS_F32_64, id, k, sm.coef_u[k]);
  eval_and_write_call<true, float, float2>(T, J, val, I, Jb, sm.coef_u, sm.coef_d, sm.tw, sm.red, t,
                                      NT, a.server != 0);
}

template <int NWB, int ROWS, int U>
__device__ __forceinline__ void run_item64(const ExecArgs& a, int id, CtaSmem64<NWB, ROWS>& sm, int t) {
  if constexpr (ROWS == ROWS_PAIRED) item_f32_64p<NWB, ROWS, U>(a, id, sm, t);
  else item_f32_64<NWB, ROWS>(a, id, sm, t);
}

template <int NWB, int ROWS = 128, int U = 1>
__global__ void __launch_bounds__(NWB * 32, NWB == 8 ? 2 : (NWB == 2 ? 4 : (ROWS == 96 ? 4 : 3)))
    k_exec_f32_64(const __grid_constant__ ExecArgs a) {
  constexpr int NT = NWB * 32;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  CtaSmem64<NWB, ROWS>& sm = *reinterpret_cast<CtaSmem64<NWB, ROWS>*>(smem_raw);
  const int t = threadIdx.x;
  if (t < 64) sm.tw[t] = make_float2(c_twf[t].x, -c_twf[t].y);
  __syncthreads();
  const ClassArgs& C = a.c[CLS_F32_64];
  if (a.single_item >= 0) {
    if (blockIdx.x == 0) run_item64<NWB, ROWS, U>(a, a.single_item, sm, t);
    return;
  }
  if (a.level_mode) {
    const int n = min(C.q->n_items, C.cap);
    for (int id = blockIdx.x; id < n; id += gridDim.x)
      if (a.level_of[(size_t)CLS_F32_64 * a.level_stride + id] == a.level) {
        run_item64<NWB, ROWS, U>(a, id, sm, t);
        __syncthreads();
      }
    return;
  }
  for (;;) {
    if (t < 32) {
      const int id = a.server ? server_pop_warp(a, C, CLS_F32_64, t) : queue_pop_warp(C, a.timeout_ns, t);
      if (t == 0) {
        sm.item = id;
        sm.skip = a.server && id >= 0 && !(id & SRV_CMD_BIT) && server_cancelled(a, C, id);
      }
    }
    __syncthreads();
    const int id = sm.item;
    if (id < 0) break;
    if (id & SRV_CMD_BIT) {  // a request joins the running executor
      server_admit<true>(a, C, CLS_F32_64, id & ~SRV_CMD_BIT, t, NT);
      continue;
    }
    if (sm.skip) {  // cancelled: release only (decided once, by thread 0)
      const int2 it = ld_in(C.items + id, a.server != 0);
      copy_desc(&sm.T, a.tiles + it.x, t, NT, a.server != 0);
      __syncthreads();
      copy_desc(&sm.J, a.jobs + sm.T.job, t, NT, a.server != 0);
    } else {
      run_item64<NWB, ROWS, U>(a, id, sm, t);
    }
    __threadfence();
    __syncthreads();
    const int2 it = ld_in(C.items + id, a.server != 0);
    release_successors(a, C, sm.T, sm.J, it.y >> 16, it.y & 0xFFFF, t, NT);
    if (t == 0) {
      atomicAdd(&C.q->n_done, 1);
      if (a.server) server_block_done(a, sm.T.job);
    }
    __syncthreads();
  }
}

// ===========================================================================
// Executor 3: FP64 validation path (F = 32 or 64).  One CTA of 256 threads
// per block, spectrum and weight spectrum both in shared memory, FFT lines in
// shared memory, argmax with the tie rule "lowest flat index among
// |R|^2 >= (1 - tau) max |R|^2" (tau = 1e-9).  Same staging, model and
// write-back code as the FP32 executors.
// ===========================================================================
constexpr int NT64 = 256;
struct alignas(16) CtaSmemD {
  double2 R[64 * 64];
  double2 Wb[64 * 64];
  double2 coef_d[KMAX];
  int32_t coef_u[KMAX];
  double2 tw[64];
  double red[NT64];
  int32_t redi[NT64];
  int item;
};
constexpr size_t SMEMD = sizeof(CtaSmemD);

// In-place radix-2 DIT FFT of one line of n = 32/64 elements at stride `st`.
__device__ void fft_line_d(double2* x, int st, int n, int logn) {
  for (int i = 0; i < n; ++i) {
    int j = 0;
    for (int b = 0; b < logn; ++b) j |= ((i >> b) & 1) << (logn - 1 - b);
    if (i < j) {
      const double2 tmp = x[i * st];
      x[i * st] = x[j * st];
      x[j * st] = tmp;
    }
  }
  for (int s = 0; s < logn; ++s) {
    const int half = 1 << s;
    for (int g = 0; g < n; g += 2 * half)
      for (int k = 0; k < half; ++k) {
        const double2 w = c_twd[k * (32 >> s)];
        const double2 a = x[(g + k) * st], b = x[(g + k + half) * st];
        const double2 tt = make_double2(w.x * b.x - w.y * b.y, w.x * b.y + w.y * b.x);
        x[(g + k) * st] = make_double2(a.x + tt.x, a.y + tt.y);
        x[(g + k + half) * st] = make_double2(a.x - tt.x, a.y - tt.y);
      }
  }
}

__device__ __forceinline__ void item_f64(const ExecArgs& a, int id, CtaSmemD& sm, int t) {
  const ClassArgs& C = a.c[CLS_F64];
  const int2 it = ld_in(C.items + id, a.server != 0);
  const TileDev T = a.tiles[it.x];
  const JobDev J = a.jobs[T.job];
  const int I = it.y >> 16, Jb = it.y & 0xFFFF;
  const int S = J.S, K = J.K, F = J.F, FF = F * F, logF = F == 32 ? 5 : 6;
  double* val = a.val_d + T.val_off;
  if (t == 0) debug_record(a, CLS_F64, id, T, it.x, I, Jb);
  // stage into a plain (unswizzled) F x F buffer
  for (int e = t; e < FF; e += NT64) sm.R[e] = make_double2(0.0, 0.0);
  __syncthreads();
  {
    const int oy = I * J.b - J.B, ox = Jb * J.b - J.B;
    for (int e = t; e < S * S; e += NT64) {
      const int m = e / S, n = e - m * S;
      double wv = 0, zr = 0;
      const int ty = oy + m, tx = ox + n;
      if (ty >= 0 && ty < T.eh && tx >= 0 && tx < T.ew) {
        const size_t gi = (size_t)(T.ey + ty) * J.pitch + (T.ex + tx);
        const double wi = J.wiso_d[e];
        if (__ldg(J.mask + gi) == 0) {
          wv = wi;
          zr = wi * (double)__ldg(J.image + gi);
        } else if (J.order != ORDER_INDEPENDENT) {
          const double v = __ldcg(val + (size_t)ty * T.ew + tx);
          if (!isnan(v)) {
            wv = J.delta * wi;
            zr = wv * v;
          }
        }
      }
      sm.R[m * F + n] = make_double2(wv, zr);
    }
  }
  __syncthreads();
  if (t < F) fft_line_d(sm.R + t * F, 1, F, logF);
  __syncthreads();
  if (t < F) fft_line_d(sm.R + t, F, F, logF);
  __syncthreads();
  // Hermitian split, pairwise in place
  for (int k = t; k < FF; k += NT64) {
    const int k1 = k / F, k2 = k % F;
    const int km = ((F - k1) & (F - 1)) * F + ((F - k2) & (F - 1));
    if (km < k) continue;
    const double2 z = sm.R[k], zm = sm.R[km];
    sm.Wb[k] = make_double2(0.5 * (z.x + zm.x), 0.5 * (z.y - zm.y));
    sm.Wb[km] = make_double2(0.5 * (zm.x + z.x), 0.5 * (zm.y - z.y));
    sm.R[k] = make_double2(0.5 * (z.y + zm.y), 0.5 * (zm.x - z.x));
    sm.R[km] = make_double2(0.5 * (zm.y + z.y), 0.5 * (z.x - zm.x));
  }
  __syncthreads();
  const double W0 = sm.Wb[0].x;
  if (!(W0 > 0.0)) {
    if (t == 0) atomicAdd(&C.q->n_empty, 1);
    return;
  }
  const double gs = J.gamma / W0;
  for (int iter = 0; iter < K; ++iter) {
    double emax = 0;
    for (int k = t; k < FF; k += NT64) emax = fmax(emax, sm.R[k].x * sm.R[k].x + sm.R[k].y * sm.R[k].y);
    sm.red[t] = emax;
    __syncthreads();
    for (int s = NT64 / 2; s > 0; s >>= 1) {
      if (t < s) sm.red[t] = fmax(sm.red[t], sm.red[t + s]);
      __syncthreads();
    }
    const double thr = (1.0 - TAU_F64) * sm.red[0];
    int kmin = FF;
    for (int k = t; k < FF; k += NT64)
      if (sm.R[k].x * sm.R[k].x + sm.R[k].y * sm.R[k].y >= thr) { kmin = k; break; }
    sm.redi[t] = kmin;
    __syncthreads();
    for (int s = NT64 / 2; s > 0; s >>= 1) {
      if (t < s) sm.redi[t] = min(sm.redi[t], sm.redi[t + s]);
      __syncthreads();
    }
    const int u = sm.redi[0];
    const double2 ru = sm.R[u];
    const double dx = gs * ru.x, dy = gs * ru.y;
    __syncthreads();
    if (t == 0) {
      sm.coef_u[iter] = u;
      sm.coef_d[iter] = make_double2(dx, dy);
      debug_useq(a, CLS_F64, id, iter, u);
    }
    const int u1 = u / F, u2 = u % F;
    for (int k = t; k < FF; k += NT64) {
      const int k1 = k / F, k2 = k % F;
      const double2 w = sm.Wb[((k1 - u1) & (F - 1)) * F + ((k2 - u2) & (F - 1))];
      double2 r = sm.R[k];
      r.x -= dx * w.x - dy * w.y;
      r.y -= dx * w.y + dy * w.x;
      sm.R[k] = r;
    }
    __syncthreads();
  }
  eval_and_write_call<true, double, double2>(T, J, val, I, Jb, sm.coef_u, sm.coef_d, sm.tw, sm.red, t,
                                        NT64, a.server != 0);
}

__global__ void __launch_bounds__(NT64) k_exec_f64(const __grid_constant__ ExecArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  CtaSmemD& sm = *reinterpret_cast<CtaSmemD*>(smem_raw);
  const int t = threadIdx.x;
  if (t < 64) sm.tw[t] = make_double2(c_twd[t].x, -c_twd[t].y);
  __syncthreads();
  const ClassArgs& C = a.c[CLS_F64];
  if (a.single_item >= 0) {
    if (blockIdx.x == 0) item_f64(a, a.single_item, sm, t);
    return;
  }
  if (a.level_mode) {
    const int n = min(C.q->n_items, C.cap);
    for (int id = blockIdx.x; id < n; id += gridDim.x)
      if (a.level_of[(size_t)CLS_F64 * a.level_stride + id] == a.level) {
        item_f64(a, id, sm, t);
        __syncthreads();
      }
    return;
  }
  for (;;) {
    if (t < 32) {
      const int id = queue_pop_warp(C, a.timeout_ns, t);
      if (t == 0) sm.item = id;
    }
    __syncthreads();
    const int id = sm.item;
    if (id < 0) break;
    item_f64(a, id, sm, t);
    __threadfence();
    __syncthreads();
    const int2 it = ld_in(C.items + id, a.server != 0);
    const TileDev T = a.tiles[it.x];
    const JobDev J = a.jobs[T.job];
    release_successors(a, C, T, J, it.y >> 16, it.y & 0xFFFF, t, NT64);
    if (t == 0) atomicAdd(&C.q->n_done, 1);
    __syncthreads();
  }
}

// ===========================================================================
// Planner kernels
// ===========================================================================

// out = mask ? 0 : image; out_f32 likewise.  grid.y = job.
__global__ void k_init_out(const JobDev* jobs) {
  const JobDev J = jobs[blockIdx.y];
  const int64_t npx = (int64_t)J.W * J.H;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npx;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int y = (int)(p / J.W), x = (int)(p - (int64_t)y * J.W);
    const size_t gi = (size_t)y * J.pitch + x;
    const uint8_t v = J.mask[gi] ? 0 : J.image[gi];
    J.out[gi] = v;
    if (J.out_f32) J.out_f32[p] = (float)v;
    if (J.out_f64) J.out_f64[p] = (double)v;
  }
}

// One thread per block of a tile's grid: lost if any pixel of the block
// (inside the extended tile) is lost.  grid.y = tile.
__global__ void k_mark(const __grid_constant__ ExecArgs a) {
  const TileDev T = a.tiles[blockIdx.y];
  const JobDev J = a.jobs[T.job];
  const int nb = T.nbx * T.nby;
  const ClassArgs& C = a.c[T.cls];
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nb; k += gridDim.x * blockDim.x) {
    const int I = k / T.nbx, Jb = k - I * T.nbx;
    bool lost = false, core = false;
    const int y0 = I * J.b, x0 = Jb * J.b;
    for (int yy = y0; yy < min(y0 + J.b, T.eh); ++yy)
      for (int xx = x0; xx < min(x0 + J.b, T.ew); ++xx) {
        const int gy = T.ey + yy, gx = T.ex + xx;
        if (J.mask[(size_t)gy * J.pitch + gx]) {
          lost = true;
          if (gx >= T.x && gx < T.x + T.w && gy >= T.y && gy < T.y + T.h) core = true;
        }
      }
    int id = -1;
    if (lost) {
      id = atomicAdd(&C.q->n_items, 1);
      if (id < C.cap) {
        C.items[id] = make_int2(blockIdx.y, (I << 16) | Jb);
        if (core) atomicAdd(&C.q->n_core, 1);
      } else {
        atomicOr(&C.q->error, ERR_BOUNDS);
        id = -1;
      }
    }
    a.map[T.map_off + k] = id;
  }
}

// Pending-predecessor count of every item; items without any are queued.
// Ordered enumeration, pass 1: mark the lost blocks of every tile (map -2,
// or -3 when the block touches the core) and count them per tile.
__device__ __forceinline__ void lost_test(const TileDev& T, const JobDev& J, int I, int Jb, bool& lost, bool& core) {
  lost = false;
  core = false;
  const int y0 = I * J.b, x0 = Jb * J.b;
  for (int yy = y0; yy < min(y0 + J.b, T.eh); ++yy)
    for (int xx = x0; xx < min(x0 + J.b, T.ew); ++xx) {
      const int gy = T.ey + yy, gx = T.ex + xx;
      if (J.mask[(size_t)gy * J.pitch + gx]) {
        lost = true;
        if (gx >= T.x && gx < T.x + T.w && gy >= T.y && gy < T.y + T.h) core = true;
      }
    }
}

__global__ void k_mark_count(const __grid_constant__ ExecArgs a) {
  const TileDev T = a.tiles[blockIdx.y];
  const JobDev J = a.jobs[T.job];
  const int nb = T.nbx * T.nby;
  const ClassArgs& C = a.c[T.cls];
  const int lane = threadIdx.x & 31;
  for (int k0 = blockIdx.x * blockDim.x; k0 < nb; k0 += gridDim.x * blockDim.x) {  // uniform per warp
    const int k = k0 + threadIdx.x;
    bool lost = false, core = false;
    if (k < nb) {
      lost_test(T, J, k / T.nbx, k % T.nbx, lost, core);
      a.map[T.map_off + k] = lost ? (core ? -3 : -2) : -1;
    }
    const unsigned bl = __ballot_sync(0xffffffffu, lost), bc = __ballot_sync(0xffffffffu, core);
    if (lane == 0 && bl) atomicAdd(&a.tile_cnt[blockIdx.y], __popc(bl));
    if (lane == 0 && bc) atomicAdd(&C.q->n_core, __popc(bc));
  }
}

// Pass 2 (one block): per class, the first item id of every tile, tiles in
// order; the class's item count.
__global__ void k_mark_scan(const __grid_constant__ ExecArgs a) {
  __shared__ int wsum[32];
  __shared__ int carry[MAX_CLS];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5, nw = blockDim.x >> 5;
  if (t < MAX_CLS) carry[t] = 0;
  __syncthreads();
  for (int t0 = 0; t0 < a.n_tiles; t0 += blockDim.x) {
    const int i = t0 + t;
    const int cls = i < a.n_tiles ? a.tiles[i].cls : -1;
    const int cnt = i < a.n_tiles ? a.tile_cnt[i] : 0;
    for (int k = 0; k < MAX_CLS; ++k) {
      const int v = cls == k ? cnt : 0;
      int x = v;  // inclusive warp scan
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      if (lane == 31) wsum[w] = x;
      __syncthreads();
      int before = 0;
      for (int q = 0; q < w; ++q) before += wsum[q];
      if (cls == k) a.tile_base[i] = carry[k] + before + x - v;
      __syncthreads();
      if (t == 0) {
        int tot = 0;
        for (int q = 0; q < nw; ++q) tot += wsum[q];
        carry[k] += tot;
      }
      __syncthreads();
    }
  }
  if (t < MAX_CLS) {
    QueueDev* q = a.c[t].q;
    q->n_items = carry[t];
    if (carry[t] > a.c[t].cap) atomicOr(&q->error, ERR_BOUNDS);
  }
}

// Pass 3: ids within each tile's range (a warp's lost blocks consecutive).
__global__ void k_mark_assign(const __grid_constant__ ExecArgs a) {
  const TileDev T = a.tiles[blockIdx.y];
  const int nb = T.nbx * T.nby;
  const ClassArgs& C = a.c[T.cls];
  const int lane = threadIdx.x & 31;
  for (int k0 = blockIdx.x * blockDim.x; k0 < nb; k0 += gridDim.x * blockDim.x) {  // uniform per warp
    const int k = k0 + threadIdx.x;
    const int m = k < nb ? a.map[T.map_off + k] : -1;
    const bool lost = m <= -2;
    const unsigned bl = __ballot_sync(0xffffffffu, lost);
    int base = 0;
    if (lane == 0 && bl) base = atomicAdd(&a.tile_ctr[blockIdx.y], __popc(bl));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (lost) {
      const int id = a.tile_base[blockIdx.y] + base + __popc(bl & ((1u << lane) - 1u));
      if (id < C.cap) {
        C.items[id] = make_int2(blockIdx.y, ((k / T.nbx) << 16) | (k % T.nbx));
        a.map[T.map_off + k] = id;
      } else {
        a.map[T.map_off + k] = -1;
      }
    }
  }
}

__global__ void k_deps(const __grid_constant__ ExecArgs a, int cls) {
  const ClassArgs& C = a.c[cls];
  const int n = min(C.q->n_items, C.cap);
  const int lane = threadIdx.x & 31;
  for (int id0 = blockIdx.x * blockDim.x; id0 < n; id0 += gridDim.x * blockDim.x) {  // uniform per warp
    const int id = id0 + threadIdx.x;
    int cnt = -1;
    if (id < n) {
      const int2 it = ld_in(C.items + id, a.server != 0);
      const TileDev T = a.tiles[it.x];
      const JobDev J = a.jobs[T.job];
      const int I = it.y >> 16, Jb = it.y & 0xFFFF;
      cnt = count_preds(J, T, a.map + T.map_off, I, Jb, false);
      C.cnt[id] = cnt;
      if (a.level_of) a.level_of[(size_t)cls * a.level_stride + id] =
          J.order == ORDER_PHASED ? (I % J.P) * J.P + (Jb % J.P) : 0;
    }
    if (C.window > 0) {
      // fed roots: a warp's roots take consecutive places in id order; the
      // first `window` start, the others wait
      const unsigned br = __ballot_sync(0xffffffffu, cnt == 0);
      int base = 0;
      if (lane == 0 && br) base = atomicAdd(&C.q->n_roots, __popc(br));
      base = __shfl_sync(0xffffffffu, base, 0);
      if (cnt == 0) {
        const int r = base + __popc(br & ((1u << lane) - 1u));
        if (r < C.window) queue_push(C, id);
        else C.roots[r] = id;
      }
    } else if (cnt == 0) {
      queue_push(C, id);
    }
  }
}

__global__ void k_probe(const __grid_constant__ ExecArgs a) {
  const int id = queue_pop_warp(a.c[0], a.timeout_ns, threadIdx.x & 31);
  if (id >= 0 && threadIdx.x == 0) atomicAdd(&a.c[0].q->n_done, 1);
}

// ===========================================================================
// launchers
// ===========================================================================
// Executor variants: one kernel per (class, layout, K-loop unroll).
namespace {
struct Variant {
  int cls, layout, unroll;
  const void* fn;
  int threads;
  size_t smem;
};
const Variant kVariants[] = {
    {CLS_F32_32, 3, 1, (const void*)k_exec_f32_32<WarpSmem32R, 1>, NW32 * 32, SMEM32R},
    {CLS_F32_32, 3, 2, (const void*)k_exec_f32_32<WarpSmem32R, 2>, NW32 * 32, SMEM32R},
    {CLS_F32_32, 2, 1, (const void*)k_exec_f32_32<WarpSmem32P, 1>, NW32 * 32, SMEM32P},
    {CLS_F32_32, 2, 2, (const void*)k_exec_f32_32<WarpSmem32P, 2>, NW32 * 32, SMEM32P},
    {CLS_F32_32, 1, 1, (const void*)k_exec_f32_32<WarpSmem32, 1>, NW32 * 32, SMEM32},
    {CLS_F32_32, 4, 1, (const void*)k_exec_f32_32<WarpSmem32C, 1>, NW32 * 32, SMEM32C},
    {CLS_F32_32, 4, 2, (const void*)k_exec_f32_32<WarpSmem32C, 2>, NW32 * 32, SMEM32C},
    {CLS_F32_64, 6, 1, (const void*)k_exec_f32_64<4, ROWS_PAIRED, 1>, 128, sizeof(CtaSmem64<4, ROWS_PAIRED>)},
    {CLS_F32_64, 6, 2, (const void*)k_exec_f32_64<4, ROWS_PAIRED, 2>, 128, sizeof(CtaSmem64<4, ROWS_PAIRED>)},
    {CLS_F32_64, 5, 1, (const void*)k_exec_f32_64<4, 96>, 128, sizeof(CtaSmem64<4, 96>)},
    {CLS_F32_64, 4, 1, (const void*)k_exec_f32_64<4>, 128, sizeof(CtaSmem64<4>)},
    {CLS_F32_64, 2, 1, (const void*)k_exec_f32_64<2>, 64, sizeof(CtaSmem64<2>)},
    {CLS_F32_64, 8, 1, (const void*)k_exec_f32_64<8>, 256, sizeof(CtaSmem64<8>)},
    {CLS_F64, 0, 1, (const void*)k_exec_f64, NT64, SMEMD},
};

const Variant& variant(int cls, const ExecCfg& c) {
  const int lay = cls == CLS_F32_32 ? c.lay32 : (cls == CLS_F32_64 ? c.lay64 : 0);
  const int un = cls == CLS_F32_32 ? c.unroll32 : (cls == CLS_F32_64 ? c.unroll64 : 1);
  const Variant* fallback = nullptr;
  for (const Variant& v : kVariants) {
    if (v.cls != cls) continue;
    if (!fallback) fallback = &v;  // the first listed is the class default
    if (v.layout == lay && v.unroll == un) return v;
  }
  for (const Variant& v : kVariants)  // an unroll the layout lacks: its unroll-1 form
    if (v.cls == cls && v.layout == lay && v.unroll == 1) return v;
  return *fallback;
}
}  // namespace

bool exec_cfg_valid(int cls, int layout, int unroll) {
  for (const Variant& v : kVariants)
    if (v.cls == cls && v.layout == layout && v.unroll == unroll) return true;
  return false;
}
int exec_threads(int cls, const ExecCfg& c) { return variant(cls, c).threads; }
size_t exec_smem(int cls, const ExecCfg& c) { return variant(cls, c).smem; }
const void* exec_kernel_ptr(int cls, const ExecCfg& c) { return variant(cls, c).fn; }

cudaError_t exec_setup(int device) {
  (void)device;
  for (const Variant& v : kVariants) {
    const cudaError_t e = cudaFuncSetAttribute(v.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)v.smem);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_init_out(const JobDev* jobs_dev, int n_jobs, int max_pixels, cudaStream_t st) {
  if (n_jobs == 0) return cudaSuccess;
  dim3 grid((unsigned)std::min(1024, (max_pixels + 255) / 256 + 1), (unsigned)n_jobs);
  k_init_out<<<grid, 256, 0, st>>>(jobs_dev);
  return cudaGetLastError();
}

cudaError_t launch_mark(const ExecArgs& a, int n_tiles, int max_tile_blocks, cudaStream_t st) {
  if (n_tiles == 0) return cudaSuccess;
  dim3 grid((unsigned)std::min(4096, (max_tile_blocks + 255) / 256 + 1), (unsigned)n_tiles);
  if (!a.tile_cnt) {
    k_mark<<<grid, 256, 0, st>>>(a);
    return cudaGetLastError();
  }
  k_mark_count<<<grid, 256, 0, st>>>(a);
  k_mark_scan<<<1, 1024, 0, st>>>(a);
  k_mark_assign<<<grid, 256, 0, st>>>(a);
  return cudaGetLastError();
}

static int sm_count_of_device() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
    return 132;
  return n;
}

cudaError_t launch_deps(const ExecArgs& a, int cls, int cap, cudaStream_t st) {
  if (cap == 0) return cudaSuccess;
  // with fed roots a grid of one wave keeps the roots close to id order
  const int blocks = a.c[cls].window > 0 ? std::min(sm_count_of_device() * 8, (cap + 255) / 256)
                                         : std::min(8192, (cap + 255) / 256);
  k_deps<<<(unsigned)std::max(1, blocks), 256, 0, st>>>(a, cls);
  return cudaGetLastError();
}

cudaError_t launch_exec(const ExecArgs& a, int cls, int grid, cudaStream_t st, const ExecCfg& c) {
  if (grid <= 0) return cudaSuccess;
  const Variant& v = variant(cls, c);
  void* args[] = {const_cast<ExecArgs*>(&a)};
  return cudaLaunchKernel(v.fn, dim3((unsigned)grid), dim3((unsigned)v.threads), args, v.smem, st);
}

cudaError_t launch_probe(const ExecArgs& a, cudaStream_t st) {
  k_probe<<<1, 32, 0, st>>>(a);
  return cudaGetLastError();
}

// Row re-pitch of `planes` byte planes of W x H (host-buffer path): the host
// copies move whole contiguous planes, this kernel moves rows between the
// packed and the 16-byte-padded layouts.
__global__ void k_repitch(const uint8_t* __restrict__ src, int src_pitch, size_t src_plane,
                          uint8_t* __restrict__ dst, int dst_pitch, size_t dst_plane, int W, int H) {
  const uint8_t* s = src + blockIdx.y * src_plane;
  uint8_t* d = dst + blockIdx.y * dst_plane;
  for (int y = blockIdx.x; y < H; y += gridDim.x) {
    const uint8_t* sr = s + (size_t)y * src_pitch;
    uint8_t* dr = d + (size_t)y * dst_pitch;
    for (int x = threadIdx.x; x < W; x += blockDim.x) dr[x] = sr[x];
  }
}

cudaError_t launch_repitch(const uint8_t* src, int src_pitch, size_t src_plane, uint8_t* dst, int dst_pitch,
                           size_t dst_plane, int W, int H, int planes, cudaStream_t st) {
  if (W <= 0 || H <= 0 || planes <= 0) return cudaSuccess;
  const dim3 grid((unsigned)std::min(H, 2048), (unsigned)planes);
  k_repitch<<<grid, 256, 0, st>>>(src, src_pitch, src_plane, dst, dst_pitch, dst_plane, W, H);
  return cudaGetLastError();
}

}  // namespace fse
