// Serving loop with continuous batching (fse_server_* in fse.h).
//
// One resident executor per served work class (the persistent FP32 kernels in
// server mode) runs for the whole life of the server and drains one work
// queue per class that all resident requests share.  A worker thread
//   - admits queued requests in arrival order as job slots and arena memory
//     free up: it copies the request's inputs and descriptors to the device and
//     posts an "admit" command; the running executor takes the command into
//     its queue, and the group that pops it enumerates the request's lost
//     blocks, sets their dependency counts and pushes the ready ones, so the
//     new request's blocks interleave with those of the requests already on
//     the GPU (no launch, no lane to wait for);
//   - retires requests whose last block has finished (the executor publishes
//     each request's completion to host-mapped memory): outputs copied to the
//     caller's buffers, latency recorded, waiters woken;
//   - advances a heartbeat that bounds every wait of the executor (a stale
//     heartbeat means the host is gone and the kernels exit with an error);
//   - restarts the executor between epochs when the queue's item capacity
//     runs low (the queue counts items for the life of an epoch).
// A request's blocks never read another request's data, and each block's
// arithmetic is that of the batch path, so every result equals the result of
// the same job run alone.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstddef>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/fse.h"
#include "fse_context.h"
#include "fse_internal.h"

namespace {

using Clock = std::chrono::steady_clock;
using fse::MAX_CLS;
using fse::SRV_MAXJ;
using fse::SRV_MAXT;

struct Request {
  uint64_t ticket = 0;
  fse_job_t job;  // the caller's job; image/mask point at the copies below
  std::vector<uint8_t> image, mask;
  int state = FSE_REQ_QUEUED;
  int status = FSE_OK;
  int cls = 0;
  std::atomic<bool> cancel{false};  // set by fse_cancel, read by the worker
  size_t dev_bytes = 0;
  int64_t block_bound = 0;  // blocks of all its extended tiles (>= its lost blocks)
  std::vector<fse_tile_t> tiles;
  Clock::time_point t_submit, t_launch, t_done;
};
using ReqPtr = std::shared_ptr<Request>;

struct Slot {
  ReqPtr req;  // null = free
  int gen = 0;
  size_t off = 0, bytes = 0;  // arena range of the request's buffers
  size_t o_out = 0, o_f32 = 0;
};

// First-fit allocator over an arena range (offsets; 256-byte granules).
class Pool {
 public:
  void reset(size_t begin, size_t end) {
    free_.clear();
    if (end > begin) free_[begin] = end - begin;
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = (bytes + 255) / 256 * 256;
    for (auto it = free_.begin(); it != free_.end(); ++it)
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes, at = it->first + bytes;
        free_.erase(it);
        if (rest) free_[at] = rest;
        return true;
      }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = (bytes + 255) / 256 * 256;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t largest() const {
    size_t m = 0;
    for (auto& kv : free_) m = std::max(m, kv.second);
    return m;
  }

 private:
  std::map<size_t, size_t> free_;
};

inline size_t align256(size_t v) { return (v + 255) / 256 * 256; }

}  // namespace

struct fse_server {
  int device = 0;
  fse::ExecCfg cfg;
  int classes = 3;              // bit k: class k is served (FSE_OPT_SERVER_CLASSES)
  int grid[MAX_CLS] = {0, 0, 0};
  int sm_count = 0;
  int64_t hb_timeout_ns = 0;
  char* arena = nullptr;
  size_t arena_bytes = 0;
  size_t pool_capacity = 0;  // bytes of the request pool
  // arena layout
  fse::ServerDevCtl* dctl = nullptr;
  fse::QueueDev* dq = nullptr;
  fse::JobDev* djobs = nullptr;
  fse::TileDev* dtiles = nullptr;
  float* dwiso = nullptr;  // 64 * 64 per slot
  int2* items[MAX_CLS] = {nullptr, nullptr, nullptr};
  int32_t* cnt[MAX_CLS] = {nullptr, nullptr, nullptr};
  int32_t* slots[MAX_CLS] = {nullptr, nullptr, nullptr};
  int64_t cap = 0;  // queue entries (items and admit commands) per class per epoch
  int64_t consumers[MAX_CLS] = {0, 0, 0};  // queue positions the idle consumers may hold
  Pool pool;
  // host side
  fse::ServerDevCtl* mirror = nullptr;   // pinned: the host-written fields, copied to dctl
  fse::ServerHostCtl* hctl = nullptr;    // host-mapped: written by the device
  fse::ServerHostCtl* hctl_dev = nullptr;
  char* staging = nullptr;  // pinned
  size_t staging_bytes = 0;
  cudaStream_t exec[MAX_CLS] = {nullptr, nullptr, nullptr};
  cudaStream_t copy = nullptr, ctl = nullptr;
  bool running = false;
  int64_t used[MAX_CLS] = {0, 0, 0};  // queue entries reserved this epoch (bounds)
  int cmds[MAX_CLS] = {0, 0, 0};       // admit commands posted this epoch
  int next_gen = 1;
  Slot slot[SRV_MAXJ];
  int max_queue = 64, max_resident = 64;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<ReqPtr> queue;
  std::unordered_map<uint64_t, ReqPtr> table;
  std::deque<double> latencies;
  uint64_t next_ticket = 1;
  int resident = 0;
  bool stop = false;
  std::thread worker;
};

namespace {

// Copies `bytes` of the pinned mirror at `field` to the same place of dctl.
cudaError_t ctl_write(fse_server* s, const void* field, size_t bytes, cudaStream_t st) {
  const size_t off = (const char*)field - (const char*)s->mirror;
  return cudaMemcpyAsync((char*)s->dctl + off, field, bytes, cudaMemcpyHostToDevice, st);
}

fse::ExecArgs exec_args(fse_server* s) {
  fse::ExecArgs a;
  memset(&a, 0, sizeof(a));
  a.jobs = s->djobs;
  a.tiles = s->dtiles;
  a.map = reinterpret_cast<int32_t*>(s->arena);
  a.val_f = reinterpret_cast<float*>(s->arena);
  for (int k = 0; k < MAX_CLS; ++k) {
    a.c[k].items = s->items[k];
    a.c[k].cnt = s->cnt[k];
    a.c[k].slots = s->slots[k];
    a.c[k].q = s->dq + k;
    a.c[k].cap = (int32_t)s->cap;
  }
  a.timeout_ns = s->hb_timeout_ns;
  a.single_item = -1;
  a.server = 1;
  a.srv = s->dctl;
  a.host = s->hctl_dev;
  return a;
}

// Fresh epoch: empty queues, no posted command, executor launched.
int start_executor(fse_server* s) {
  for (int k = 0; k < MAX_CLS; ++k) {
    s->used[k] = 0;
    s->cmds[k] = 0;
  }
  memset(s->mirror, 0, offsetof(fse::ServerDevCtl, cmd));
  cudaError_t e = cudaMemsetAsync(s->dq, 0, sizeof(fse::QueueDev) * MAX_CLS, s->ctl);
  for (int k = 0; k < MAX_CLS && e == cudaSuccess; ++k)
    if (s->slots[k]) e = cudaMemsetAsync(s->slots[k], 0xFF, sizeof(int32_t) * s->cap, s->ctl);
  if (e == cudaSuccess) e = ctl_write(s, s->mirror, offsetof(fse::ServerDevCtl, cmd), s->ctl);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->ctl);
  if (e != cudaSuccess) return fse::cuda_fail(e, "server executor reset");
  const fse::ExecArgs a = exec_args(s);
  for (int k = 0; k < MAX_CLS; ++k)
    if (s->grid[k] > 0) {
      e = fse::launch_exec(a, k, s->grid[k], s->exec[k], s->cfg);
      if (e != cudaSuccess) return fse::cuda_fail(e, "server executor launch");
    }
  s->running = true;
  return FSE_OK;
}

// Stops the executor (its consumers exit once idle) and waits for it.
int stop_executor(fse_server* s) {
  if (!s->running) return FSE_OK;
  s->mirror->stop = 1;
  cudaError_t e = ctl_write(s, &s->mirror->stop, sizeof(int32_t), s->ctl);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->ctl);
  for (int k = 0; k < MAX_CLS && e == cudaSuccess; ++k)
    if (s->exec[k]) e = cudaStreamSynchronize(s->exec[k]);
  s->running = false;
  if (e != cudaSuccess) return fse::cuda_fail(e, "server executor stop");
  return FSE_OK;
}

// Device bytes of a request: inputs, outputs, per tile its block map and
// value plane.
size_t request_bytes(const fse_job_t& j, const std::vector<fse_tile_t>& tl, int64_t* blocks) {
  const size_t px = (size_t)j.W * j.H;
  size_t b = align256(px) * 3 + (j.out_f32 ? align256(px * 4) : 0);
  int64_t nb = 0;
  for (const fse_tile_t& t : tl) {
    const int64_t nbx = (t.ew + j.p.block - 1) / j.p.block, nby = (t.eh + j.p.block - 1) / j.p.block;
    nb += nbx * nby;
    b += align256(sizeof(int32_t) * nbx * nby) + align256(sizeof(float) * (size_t)t.ew * t.eh);
  }
  *blocks = nb;
  return b;
}

// Copies and posts one request; returns false when it must wait (no slot,
// memory or queue capacity now).  Only copy-engine transfers are used: no
// kernel can start while the resident executor holds the SMs.
bool admit(fse_server* s, const ReqPtr& r, size_t* staging_used) {
  const int k = r->cls;
  int si = -1;
  for (int i = 0; i < SRV_MAXJ && i < s->max_resident; ++i)
    if (!s->slot[i].req) {
      si = i;
      break;
    }
  if (si < 0) return false;
  // every queue position taken this epoch: the items and commands pushed, plus
  // one position held by each waiting consumer
  if (s->used[k] + r->block_bound + 1 + s->consumers[k] > s->cap) return false;
  const size_t px = (size_t)r->job.W * r->job.H;
  if (*staging_used + align256(px) * 2 + 65536 > s->staging_bytes && *staging_used > 0) return false;
  size_t off = 0;
  if (!s->pool.alloc(r->dev_bytes, &off)) return false;
  Slot& sl = s->slot[si];
  sl.req = r;
  sl.gen = s->next_gen++;
  sl.off = off;
  sl.bytes = r->dev_bytes;
  s->used[k] += r->block_bound + 1;
  // device layout of the request
  const fse_job_t& j = r->job;
  const fse_params_t& p = j.p;
  size_t o = off;
  auto take = [&](size_t bytes) { const size_t at = o; o += align256(bytes); return at; };
  const size_t o_img = take(px), o_msk = take(px);
  sl.o_out = take(px);
  sl.o_f32 = j.out_f32 ? take(px * 4) : 0;
  fse::JobDev J;
  memset(&J, 0, sizeof(J));
  J.image = (const uint8_t*)(s->arena + o_img);
  J.mask = (const uint8_t*)(s->arena + o_msk);
  J.out = (uint8_t*)(s->arena + sl.o_out);
  J.out_f32 = j.out_f32 ? (float*)(s->arena + sl.o_f32) : nullptr;
  J.W = j.W;
  J.H = j.H;
  J.pitch = j.W;
  J.b = p.block;
  J.B = p.border;
  J.S = p.block + 2 * p.border;
  J.F = p.fft;
  J.K = p.K;
  J.order = p.order;
  J.P = (p.border + p.block - 1) / p.block + 1;
  J.D = (p.border + p.block - 1) / p.block;
  J.cls = k;
  J.rho = p.rho;
  J.delta = p.delta;
  J.gamma = p.gamma;
  J.rho_f = (float)p.rho;
  J.delta_f = (float)p.delta;
  J.gamma_f = (float)p.gamma;
  J.wiso_f = s->dwiso + (size_t)si * 64 * 64;
  // staging: image, mask, weights, job and tiles
  char* st = s->staging + *staging_used;
  size_t so = 0;
  auto stage = [&](const void* src, size_t bytes) {
    char* at = st + so;
    memcpy(at, src, bytes);
    so += align256(bytes);
    return at;
  };
  const char* s_img = stage(r->image.data(), px);
  const char* s_msk = stage(r->mask.data(), px);
  std::vector<float> w((size_t)J.S * J.S);
  const double mc = p.border + (p.block - 1) / 2.0;
  for (int m = 0; m < J.S; ++m)
    for (int q = 0; q < J.S; ++q)
      w[(size_t)m * J.S + q] = (float)std::pow(p.rho, std::sqrt((m - mc) * (m - mc) + (q - mc) * (q - mc)));
  const char* s_w = stage(w.data(), sizeof(float) * w.size());
  const char* s_job = stage(&J, sizeof(J));
  std::vector<fse::TileDev> tiles(r->tiles.size());
  for (size_t t = 0; t < r->tiles.size(); ++t) {
    const fse_tile_t& tl = r->tiles[t];
    fse::TileDev& T = tiles[t];
    memset(&T, 0, sizeof(T));
    T.job = si;
    T.x = tl.x; T.y = tl.y; T.w = tl.w; T.h = tl.h;
    T.ex = tl.ex; T.ey = tl.ey; T.ew = tl.ew; T.eh = tl.eh;
    T.nbx = (T.ew + J.b - 1) / J.b;
    T.nby = (T.eh + J.b - 1) / J.b;
    T.cls = k;
    T.vp = T.ew;
    T.map_off = (int64_t)(take(sizeof(int32_t) * (size_t)T.nbx * T.nby) / sizeof(int32_t));
    const size_t o_val = take(sizeof(float) * (size_t)T.ew * T.eh);
    T.val_off = (int64_t)(o_val / sizeof(float));
  }
  const char* s_tiles = stage(tiles.data(), sizeof(fse::TileDev) * tiles.size());
  *staging_used += so;
  // copies, then the command that publishes them (one stream: in order)
  cudaStream_t cs = s->copy;
  cudaError_t e = cudaMemcpyAsync(s->arena + o_img, s_img, px, cudaMemcpyHostToDevice, cs);
  if (e == cudaSuccess) e = cudaMemcpyAsync(s->arena + o_msk, s_msk, px, cudaMemcpyHostToDevice, cs);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync((void*)J.wiso_f, s_w, sizeof(float) * w.size(), cudaMemcpyHostToDevice, cs);
  if (e == cudaSuccess) e = cudaMemcpyAsync(s->djobs + si, s_job, sizeof(J), cudaMemcpyHostToDevice, cs);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(s->dtiles + (size_t)si * SRV_MAXT, s_tiles, sizeof(fse::TileDev) * tiles.size(),
                        cudaMemcpyHostToDevice, cs);
  // (the value planes are set to pending by the admit itself: a memset would be
  // a kernel, which cannot start while the resident executor holds the SMs)
  const int ci = s->cmds[k]++;
  fse::ServerCmd& cmd = s->mirror->cmd[k][ci % fse::SRV_CMD_RING];
  cmd.job = si;
  cmd.gen = sl.gen;
  cmd.n_tiles = (int)tiles.size();
  cmd.pad_ = 0;
  s->mirror->cmd_tail[k] = ci + 1;  // published once per admission round (post_commands)
  if (e == cudaSuccess) e = ctl_write(s, &cmd, sizeof(cmd), cs);
  r->t_launch = Clock::now();
  if (e != cudaSuccess) {
    r->status = fse::cuda_fail(e, "server admission");
  }
  return true;
}

// Publishes the commands of an admission round: one copy of the posted counts
// after every record's copy on the same stream.  (A copy reads its pinned
// source when it executes, so a count copied per command could already carry
// a later command whose record has not landed yet.)
cudaError_t post_commands(fse_server* s) {
  return ctl_write(s, s->mirror->cmd_tail, sizeof(s->mirror->cmd_tail), s->copy);
}

// Delivers the finished requests of `done` (slot indices): outputs back to
// the callers' buffers through the staging area (in chunks that fit it),
// waiters woken, slots and memory freed.
void retire(fse_server* s, const std::vector<int>& done, int status_all) {
  size_t next = 0;
  while (next < done.size()) {
    std::vector<std::pair<int, char*>> at;
    size_t so = 0;
    cudaError_t e = cudaSuccess;
    for (; next < done.size(); ++next) {
      const int si = done[next];
      const Slot& sl = s->slot[si];
      const fse_job_t& j = sl.req->job;
      const size_t px = (size_t)j.W * j.H;
      const size_t need = align256(px) + (j.out_f32 ? align256(px * 4) : 0);
      char* dst = nullptr;
      if (status_all == FSE_OK) {
        if (so + need > s->staging_bytes && !at.empty()) break;  // the next chunk takes it
        dst = s->staging + so;
        so += need;
        if (e == cudaSuccess) e = cudaMemcpyAsync(dst, s->arena + sl.o_out, px, cudaMemcpyDeviceToHost, s->copy);
        if (e == cudaSuccess && j.out_f32)
          e = cudaMemcpyAsync(dst + align256(px), s->arena + sl.o_f32, px * 4, cudaMemcpyDeviceToHost, s->copy);
      }
      at.emplace_back(si, dst);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->copy);
    const auto now = Clock::now();
    std::vector<ReqPtr> fin;
    for (auto& pr : at) {
      Slot& sl = s->slot[pr.first];
      Request& r = *sl.req;
      const fse_job_t& dst = r.job;
      int status = status_all != FSE_OK ? status_all : (e != cudaSuccess ? FSE_ECUDA : r.status);
      if (status == FSE_OK && r.cancel) status = FSE_ECANCELLED;
      if (status == FSE_OK) {
        const size_t px = (size_t)dst.W * dst.H;
        for (int y = 0; y < dst.H; ++y)
          memcpy(dst.out + (size_t)y * dst.pitch, pr.second + (size_t)y * dst.W, dst.W);
        if (dst.out_f32) memcpy(dst.out_f32, pr.second + align256(px), sizeof(float) * px);
      }
      r.status = status;
      r.t_done = now;
      fin.push_back(sl.req);
      s->pool.release(sl.off, sl.bytes);
      sl.req.reset();
    }
    std::lock_guard<std::mutex> lk(s->mu);
    for (auto& rp : fin) {
      rp->state = rp->status == FSE_OK ? FSE_REQ_DONE : FSE_REQ_FAILED;
      s->latencies.push_back(std::chrono::duration<double>(rp->t_done - rp->t_submit).count());
      if (s->latencies.size() > 1000000) s->latencies.pop_front();
    }
    s->resident -= (int)fin.size();
    s->cv_done.notify_all();
  }
}

void worker_main(fse_server* s) {
  cudaSetDevice(s->device);
  auto last_hb = Clock::now();
  Clock::time_point t_stop{};
  bool stopping = false;
  for (;;) {
    bool progressed = false;
    const auto now = Clock::now();
    if (now - last_hb > std::chrono::milliseconds(2)) {
      s->mirror->heartbeat += 1;
      ctl_write(s, &s->mirror->heartbeat, sizeof(int32_t), s->ctl);
      last_hb = now;
    }
    // a device error fails every resident request and restarts the executor
    const int err = __atomic_load_n(&s->hctl->error, __ATOMIC_ACQUIRE);
    std::vector<int> done;
    if (err) {
      for (int i = 0; i < SRV_MAXJ; ++i)
        if (s->slot[i].req) done.push_back(i);
      stop_executor(s);
      retire(s, done, (err & fse::ERR_TIMEOUT) ? FSE_ETIMEOUT : FSE_ENOMEM);
      __atomic_store_n(&s->hctl->error, 0, __ATOMIC_RELEASE);
      start_executor(s);
      progressed = true;
      done.clear();
    }
    // completions
    for (int i = 0; i < SRV_MAXJ; ++i)
      if (s->slot[i].req && __atomic_load_n(&s->hctl->done_gen[i], __ATOMIC_ACQUIRE) == s->slot[i].gen)
        done.push_back(i);
    if (!done.empty()) {
      retire(s, done, FSE_OK);
      progressed = true;
    }
    // cancellations of resident requests
    for (int i = 0; i < SRV_MAXJ; ++i) {
      Slot& sl = s->slot[i];
      if (sl.req && sl.req->cancel && s->mirror->cancel_gen[i] != sl.gen) {
        s->mirror->cancel_gen[i] = sl.gen;
        ctl_write(s, &s->mirror->cancel_gen[i], sizeof(int32_t), s->ctl);
        progressed = true;
      }
    }
    // admissions, in arrival order
    size_t staging_used = 0;
    int admitted = 0;
    for (;;) {
      ReqPtr r;
      {
        // taken off the queue and marked running under the lock, so that a
        // concurrent fse_cancel sees it either queued or running
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->queue.empty() || s->resident >= s->max_resident) break;
        r = s->queue.front();
        s->queue.pop_front();
        r->state = FSE_REQ_RUNNING;
        ++s->resident;
      }
      bool ok = admit(s, r, &staging_used);
      if (!ok) {
        // a new epoch once the queue capacity is spent and nothing is resident
        bool idle = true;
        for (int i = 0; i < SRV_MAXJ; ++i) idle &= !s->slot[i].req;
        if (idle && s->used[r->cls] > 0 && staging_used == 0) {
          stop_executor(s);
          start_executor(s);
          ok = admit(s, r, &staging_used);
        }
      }
      if (!ok) {  // back to the front of the queue (or out, if cancelled meanwhile)
        std::lock_guard<std::mutex> lk(s->mu);
        --s->resident;
        if (r->cancel) {
          r->state = FSE_REQ_FAILED;
          r->status = FSE_ECANCELLED;
          r->t_done = Clock::now();
          s->cv_done.notify_all();
        } else {
          r->state = FSE_REQ_QUEUED;
          s->queue.push_front(r);
        }
        break;
      }
      ++admitted;
    }
    if (admitted) {
      post_commands(s);
      cudaStreamSynchronize(s->copy);  // the records are out, the staging area is free again
      progressed = true;
    }
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->stop && s->queue.empty() && s->resident == 0) break;
    if (s->stop) {
      // destroy drains the server, within bounds: after 10 s the requests
      // still resident are cancelled, after 20 s the executor is stopped and
      // what remains fails with FSE_ETIMEOUT
      if (!stopping) {
        stopping = true;
        t_stop = now;
      }
      if (now - t_stop > std::chrono::seconds(10))
        for (int i = 0; i < SRV_MAXJ; ++i)
          if (s->slot[i].req) s->slot[i].req->cancel = true;
      if (now - t_stop > std::chrono::seconds(20)) {
        for (auto& r : s->queue) {
          r->state = FSE_REQ_FAILED;
          r->status = FSE_ETIMEOUT;
        }
        s->queue.clear();
        lk.unlock();
        stop_executor(s);
        std::vector<int> rest;
        for (int i = 0; i < SRV_MAXJ; ++i)
          if (s->slot[i].req) rest.push_back(i);
        retire(s, rest, FSE_ETIMEOUT);
        break;
      }
    }
    if (!progressed)
      s->cv_work.wait_for(lk, std::chrono::microseconds(s->resident > 0 ? 20 : 1000));
  }
}

// CTAs per SM of each served class's resident executor: one class alone at
// full occupancy; F = 32 beside F = 64 with the F = 64 class one CTA per SM
// below its occupancy and the F = 32 class filling what remains.
void plan_grid(fse_server* s, const cudaDeviceProp& prop) {
  struct Need { int regs, smem, threads; };
  Need need[MAX_CLS];
  int occ[MAX_CLS] = {0, 0, 0};
  for (int k = 0; k < MAX_CLS; ++k) {
    cudaFuncAttributes fa;
    cudaFuncGetAttributes(&fa, fse::exec_kernel_ptr(k, s->cfg));
    const int thr = fse::exec_threads(k, s->cfg);
    need[k].regs = (thr / 32) * ((fa.numRegs * 32 + 255) / 256 * 256);
    need[k].smem = (int)fse::exec_smem(k, s->cfg) + (int)prop.reservedSharedMemPerBlock;
    need[k].threads = thr;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[k], fse::exec_kernel_ptr(k, s->cfg), thr,
                                                  fse::exec_smem(k, s->cfg));
    occ[k] = std::max(occ[k], 1);
  }
  const bool f32 = s->classes & 1, f64 = s->classes & 2;
  int n32 = f32 ? occ[fse::CLS_F32_32] : 0, n64 = f64 ? occ[fse::CLS_F32_64] : 0;
  if (f32 && f64) {
    auto fits = [&](int a64, int a32) {
      return a64 * need[1].regs + a32 * need[0].regs <= prop.regsPerMultiprocessor &&
             a64 * need[1].smem + a32 * need[0].smem <= (int)prop.sharedMemPerMultiprocessor &&
             a64 * need[1].threads + a32 * need[0].threads <= prop.maxThreadsPerMultiProcessor;
    };
    n64 = std::max(1, occ[1] - 1);
    n32 = 0;
    while (fits(n64, n32 + 1) && n32 + 1 <= occ[0]) ++n32;
    if (n32 == 0) {
      n64 = std::max(1, n64 - 1);
      while (fits(n64, n32 + 1) && n32 + 1 <= occ[0]) ++n32;
    }
    n32 = std::max(n32, 1);
  }
  s->grid[fse::CLS_F32_32] = n32 * s->sm_count;
  s->grid[fse::CLS_F32_64] = n64 * s->sm_count;
  s->grid[fse::CLS_F64] = 0;
  for (int k = 0; k < MAX_CLS; ++k)  // consumers: warps of the F = 32 executor, CTAs of the F = 64 one
    s->consumers[k] = (int64_t)s->grid[k] * (k == fse::CLS_F32_32 ? fse::exec_threads(k, s->cfg) / 32 : 1);
}

void destroy_all(fse_server* s) {
  if (s->running) stop_executor(s);
  for (int k = 0; k < MAX_CLS; ++k)
    if (s->exec[k]) cudaStreamDestroy(s->exec[k]);
  if (s->copy) cudaStreamDestroy(s->copy);
  if (s->ctl) cudaStreamDestroy(s->ctl);
  if (s->mirror) cudaFreeHost(s->mirror);
  if (s->hctl) cudaFreeHost(s->hctl);
  if (s->staging) cudaFreeHost(s->staging);
  if (s->arena) cudaFree(s->arena);
  delete s;
}

}  // namespace

extern "C" {

int fse_server_create(fse_server_t** out, fse_context_t* ctx, const fse_server_cfg_t* cfg) {
  if (!out || !ctx || !cfg) return fse::fail(FSE_EINVAL, "NULL argument");
  *out = nullptr;
  if (cfg->arena_bytes < (64u << 20)) return fse::fail(FSE_EINVAL, "server arena below 64 MiB");
  if (cudaSetDevice(ctx->device) != cudaSuccess) return fse::fail(FSE_ECUDA, "cudaSetDevice");
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return fse::fail(FSE_ECUDA, "cudaMemGetInfo");
  if (cfg->arena_bytes > free_b)
    return fse::fail(FSE_ENOMEM, "server arena %zu > free %zu", cfg->arena_bytes, free_b);
  fse_server* s = new fse_server();
  s->device = ctx->device;
  s->sm_count = ctx->sm_count;
  s->cfg = ctx->cfg;
  s->classes = ctx->server_classes;
  if ((s->classes & 1) && (s->classes & 2)) s->cfg.lay32 = 4;  // beside F = 64: the compact F = 32 form
  if (!fse::exec_cfg_valid(fse::CLS_F32_32, s->cfg.lay32, s->cfg.unroll32)) s->cfg.unroll32 = 1;
  s->hb_timeout_ns = (int64_t)std::max(ctx->timeout_ms, 1000) * 1000000ll;
  s->max_queue = cfg->max_queue > 0 ? cfg->max_queue : 64;
  s->max_resident = std::min(cfg->max_resident > 0 ? cfg->max_resident : 64, SRV_MAXJ);
  s->arena_bytes = cfg->arena_bytes / 256 * 256;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, s->device) != cudaSuccess) {
    delete s;
    return fse::fail(FSE_ECUDA, "cudaGetDeviceProperties");
  }
  if (cudaMalloc(&s->arena, s->arena_bytes) != cudaSuccess) {
    cudaGetLastError();
    delete s;
    return fse::fail(FSE_ENOMEM, "server arena of %zu bytes", cfg->arena_bytes);
  }
  // arena: control, queues, job and tile tables, weights, per served class the
  // queue arrays (a quarter of the arena at most), then the request pool
  size_t o = 0;
  auto take = [&](size_t bytes) { const size_t at = align256(o); o = at + bytes; return at; };
  s->dctl = reinterpret_cast<fse::ServerDevCtl*>(s->arena + take(sizeof(fse::ServerDevCtl)));
  s->dq = reinterpret_cast<fse::QueueDev*>(s->arena + take(sizeof(fse::QueueDev) * MAX_CLS));
  s->djobs = reinterpret_cast<fse::JobDev*>(s->arena + take(sizeof(fse::JobDev) * SRV_MAXJ));
  s->dtiles = reinterpret_cast<fse::TileDev*>(s->arena + take(sizeof(fse::TileDev) * SRV_MAXJ * SRV_MAXT));
  s->dwiso = reinterpret_cast<float*>(s->arena + take(sizeof(float) * 64 * 64 * SRV_MAXJ));
  const int n_cls = ((s->classes & 1) ? 1 : 0) + ((s->classes & 2) ? 1 : 0);
  s->cap = std::min<int64_t>((int64_t)(s->arena_bytes / 4 / 16 / std::max(n_cls, 1)), (int64_t)1 << 28);
  for (int k = 0; k < 2; ++k) {
    if (!((s->classes >> k) & 1)) continue;
    s->items[k] = reinterpret_cast<int2*>(s->arena + take(sizeof(int2) * s->cap));
    s->cnt[k] = reinterpret_cast<int32_t*>(s->arena + take(sizeof(int32_t) * s->cap));
    s->slots[k] = reinterpret_cast<int32_t*>(s->arena + take(sizeof(int32_t) * s->cap));
  }
  s->pool.reset(align256(o), s->arena_bytes);
  s->pool_capacity = s->arena_bytes > align256(o) ? s->arena_bytes - align256(o) : 0;
  s->staging_bytes = (size_t)256 << 20;
  cudaError_t e = cudaMallocHost(&s->mirror, sizeof(fse::ServerDevCtl));
  if (e == cudaSuccess) e = cudaHostAlloc(&s->hctl, sizeof(fse::ServerHostCtl), cudaHostAllocMapped);
  if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&s->hctl_dev, s->hctl, 0);
  if (e == cudaSuccess) e = cudaMallocHost(&s->staging, s->staging_bytes);
  for (int k = 0; k < MAX_CLS && e == cudaSuccess; ++k)
    e = cudaStreamCreateWithFlags(&s->exec[k], cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->copy, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->ctl, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    cudaGetLastError();
    destroy_all(s);
    return fse::fail(FSE_ENOMEM, "server set-up: %s", cudaGetErrorString(e));
  }
  memset(s->mirror, 0, sizeof(fse::ServerDevCtl));
  memset(s->hctl, 0, sizeof(fse::ServerHostCtl));
  for (int i = 0; i < SRV_MAXJ; ++i) s->mirror->cancel_gen[i] = -1;
  e = cudaMemsetAsync(s->dctl, 0, sizeof(fse::ServerDevCtl), s->ctl);
  if (e == cudaSuccess) e = ctl_write(s, s->mirror->cancel_gen, sizeof(s->mirror->cancel_gen), s->ctl);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->ctl);
  if (e != cudaSuccess) {
    destroy_all(s);
    return fse::cuda_fail(e, "server control init");
  }
  plan_grid(s, prop);
  const int rc = start_executor(s);
  if (rc) {
    destroy_all(s);
    return rc;
  }
  s->worker = std::thread(worker_main, s);
  *out = s;
  return FSE_OK;
}

int fse_submit(fse_server_t* s, const fse_job_t* job, uint64_t* ticket) {
  if (!s || !job || !ticket) return fse::fail(FSE_EINVAL, "NULL argument");
  int rc = fse::check_job(*job, 0);
  if (rc) return rc;
  const int cls = job->p.precision == 64 ? fse::CLS_F64 : (job->p.fft == 32 ? fse::CLS_F32_32 : fse::CLS_F32_64);
  if (cls == fse::CLS_F64 || !((s->classes >> cls) & 1))
    return fse::fail(FSE_EINVAL, "the server runs FP32 jobs of the classes FSE_OPT_SERVER_CLASSES names (%d)",
                     s->classes);
  if (job->p.n_tiles > SRV_MAXT) return fse::fail(FSE_EINVAL, "at most %d tiles per request", SRV_MAXT);
  auto r = std::make_shared<Request>();
  r->tiles.resize(job->p.n_tiles);
  int32_t nt = 0;
  rc = fse::plan_tiles_mode(job->p.tiling, job->W, job->H, job->p.n_tiles, job->p.overlap, r->tiles.data(),
                            job->p.n_tiles, &nt);
  if (rc) return rc;
  r->job = *job;
  r->cls = cls;
  r->dev_bytes = request_bytes(*job, r->tiles, &r->block_bound);
  const size_t px = (size_t)job->W * job->H;
  // against the pool's capacity: a request that fits waits in the queue until
  // memory frees up (the free map itself belongs to the worker thread)
  if (r->dev_bytes > s->pool_capacity || r->block_bound + 1 + s->consumers[cls] > s->cap ||
      align256(px) * 2 + 65536 > s->staging_bytes || align256(px) * 5 > s->staging_bytes)
    return fse::fail(FSE_ENOMEM, "request needs %zu device bytes and %lld queue entries; the server has "
                                 "%zu bytes of request memory and %lld entries", r->dev_bytes, (long long)r->block_bound,
                     s->pool_capacity, (long long)s->cap);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return fse::fail(FSE_ECANCELLED, "server shutting down");
    if ((int)s->queue.size() >= s->max_queue) return fse::fail(FSE_EBUSY, "queue full");
  }
  r->image.resize(px);
  r->mask.resize(px);
  for (int y = 0; y < job->H; ++y) {
    memcpy(r->image.data() + (size_t)y * job->W, job->image + (size_t)y * job->pitch, job->W);
    memcpy(r->mask.data() + (size_t)y * job->W, job->mask + (size_t)y * job->pitch, job->W);
  }
  r->job.image = r->image.data();
  r->job.mask = r->mask.data();
  r->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if ((int)s->queue.size() >= s->max_queue) return fse::fail(FSE_EBUSY, "queue full");
    r->ticket = s->next_ticket++;
    s->table[r->ticket] = r;
    s->queue.push_back(r);
    *ticket = r->ticket;
  }
  s->cv_work.notify_one();
  return FSE_OK;
}

int fse_poll(fse_server_t* s, uint64_t ticket, int32_t* state) {
  if (!s || !state) return fse::fail(FSE_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->table.find(ticket);
  if (it == s->table.end()) return fse::fail(FSE_ENOTFOUND, "ticket %llu", (unsigned long long)ticket);
  *state = it->second->state;
  return FSE_OK;
}

int fse_cancel(fse_server_t* s, uint64_t ticket) {
  if (!s) return fse::fail(FSE_EINVAL, "NULL server");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->table.find(ticket);
  if (it == s->table.end()) return fse::fail(FSE_ENOTFOUND, "ticket %llu", (unsigned long long)ticket);
  Request& r = *it->second;
  if (r.state == FSE_REQ_QUEUED) {
    for (auto q = s->queue.begin(); q != s->queue.end(); ++q)
      if ((*q)->ticket == ticket) {
        s->queue.erase(q);
        break;
      }
    r.state = FSE_REQ_FAILED;
    r.status = FSE_ECANCELLED;
    r.t_done = Clock::now();
    s->cv_done.notify_all();
  } else if (r.state == FSE_REQ_RUNNING) {
    r.cancel = true;  // the worker marks its slot; its remaining blocks are skipped
    s->cv_work.notify_one();
  }
  return FSE_OK;
}

int fse_wait(fse_server_t* s, uint64_t ticket, int32_t timeout_ms, fse_stats_t* st) {
  if (!s) return fse::fail(FSE_EINVAL, "NULL server");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->table.find(ticket);
  if (it == s->table.end()) return fse::fail(FSE_ENOTFOUND, "ticket %llu", (unsigned long long)ticket);
  ReqPtr r = it->second;
  auto done = [&] { return r->state == FSE_REQ_DONE || r->state == FSE_REQ_FAILED; };
  if (timeout_ms < 0) {
    s->cv_done.wait(lk, done);
  } else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done)) {
    return fse::fail(FSE_ETIMEOUT, "ticket %llu not done after %d ms", (unsigned long long)ticket, timeout_ms);
  }
  if (st) {
    memset(st, 0, sizeof(*st));
    st->jobs = 1;
    st->pixels = (int64_t)r->job.W * r->job.H;
    st->device_ms = (float)std::chrono::duration<double, std::milli>(r->t_done - r->t_launch).count();
    st->exec_ms = (float)std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
  }
  const int status = r->status;
  if (status == FSE_OK) {
    s->table.erase(ticket);
    return FSE_OK;
  }
  return fse::fail(status, "request %llu failed", (unsigned long long)ticket);
}

int32_t fse_server_latencies(fse_server_t* s, double* out, int32_t cap) {
  if (!s || (!out && cap > 0)) return fse::fail(FSE_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  const int32_t n = (int32_t)std::min<size_t>(cap, s->latencies.size());
  for (int32_t i = 0; i < n; ++i) out[i] = s->latencies[s->latencies.size() - n + i];
  return n;
}

int32_t fse_server_debug_state(fse_server_t* s, int64_t* out, int32_t cap) {
  if (!s || !out || cap < 16 + 8 * SRV_MAXJ) return fse::fail(FSE_EINVAL, "bad arguments");
  cudaSetDevice(s->device);
  fse::QueueDev q[MAX_CLS];
  fse::ServerDevCtl* d = (fse::ServerDevCtl*)malloc(sizeof(fse::ServerDevCtl));
  cudaStream_t st;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  cudaMemcpyAsync(q, s->dq, sizeof(q), cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(d, s->dctl, sizeof(fse::ServerDevCtl), cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  cudaStreamDestroy(st);
  int32_t n = 0;
  for (int k = 0; k < 2; ++k) {
    out[n++] = q[k].n_items;
    out[n++] = q[k].head;
    out[n++] = q[k].tail;
    out[n++] = q[k].n_done;
    out[n++] = d->cmd_tail[k];
    out[n++] = d->cmd_taken[k];
    out[n++] = s->cmds[k];
    out[n++] = s->used[k];
  }
  std::lock_guard<std::mutex> lk(s->mu);
  for (int i = 0; i < SRV_MAXJ; ++i) {
    out[n++] = s->slot[i].req ? (int64_t)s->slot[i].req->ticket : -1;
    out[n++] = s->slot[i].gen;
    out[n++] = d->gen[i];
    out[n++] = d->total[i];
    out[n++] = d->done[i];
    out[n++] = __atomic_load_n(&s->hctl->done_gen[i], __ATOMIC_ACQUIRE);
    out[n++] = d->cancel_gen[i];
    out[n++] = s->slot[i].req ? s->slot[i].req->state : -1;
  }
  free(d);
  return n;
}

void fse_server_destroy(fse_server_t* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  cudaSetDevice(s->device);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    for (auto& kv : s->table)
      if (kv.second->state == FSE_REQ_QUEUED) {
        kv.second->state = FSE_REQ_FAILED;
        kv.second->status = FSE_ECANCELLED;
      }
  }
  s->cv_done.notify_all();
  destroy_all(s);
}

}  // extern "C"
