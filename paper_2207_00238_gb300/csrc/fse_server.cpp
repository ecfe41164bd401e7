// Serving loop with continuous batching (fse_server_* in fse.h).
//
// The server owns one device arena, cut into L lanes.  A lane is a CUDA
// stream, a slice of the arena and a pinned host staging buffer.  A worker
// thread
//   - retires lanes whose batch finished (outputs copied to the callers'
//     buffers, latency recorded, waiters woken), and
//   - admits queued requests into every free lane at once: as many, in arrival
//     order, as fit the lane's device bytes and the resident limit.
// Requests that arrive while other batches run start as soon as a lane frees
// up, and the batches of different lanes run concurrently on the GPU, so the
// persistent kernels of a new batch fill SMs that earlier batches release.
// Every request is extrapolated exactly as it would be alone (the batches only
// share launches, never data).
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/fse.h"
#include "fse_context.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t ticket = 0;
  fse_job_t job;  // the caller's job; image/mask point at the copies below
  std::vector<uint8_t> image, mask;
  int state = FSE_REQ_QUEUED;
  int status = FSE_OK;
  size_t dev_bytes = 0, host_bytes = 0;
  Clock::time_point t_submit, t_launch, t_done;
};
using ReqPtr = std::shared_ptr<Request>;

struct Lane {
  fse::Context* ctx = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  char* pinned = nullptr;
  size_t pinned_bytes = 0;
  std::vector<ReqPtr> reqs;
  std::vector<fse_job_t> staged;  // jobs pointing into `pinned`
  bool busy = false;
};

size_t host_bytes_of(const fse_job_t& j) {
  const size_t px = (size_t)j.W * j.H;
  return ((px * 3 + 255) / 256 + 3) * 256 + (j.out_f32 ? px * 4 + 256 : 0) +
         (j.out_f64 ? px * 8 + 256 : 0);
}

}  // namespace

struct fse_server {
  int device = 0;
  char* arena = nullptr;
  size_t lane_bytes = 0;
  std::vector<Lane> lanes;
  int max_queue = 64, max_resident = 64, max_batch = 16;
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

void finish(fse_server* s, Lane& ln, int status) {
  const auto now = Clock::now();
  for (size_t i = 0; i < ln.reqs.size(); ++i) {
    Request& r = *ln.reqs[i];
    const fse_job_t& st = ln.staged[i];
    const fse_job_t& dst = r.job;
    if (status == FSE_OK) {
      for (int y = 0; y < dst.H; ++y)
        memcpy(dst.out + (size_t)y * dst.pitch, st.out + (size_t)y * st.pitch, dst.W);
      if (dst.out_f32) memcpy(dst.out_f32, st.out_f32, sizeof(float) * dst.W * dst.H);
      if (dst.out_f64) memcpy(dst.out_f64, st.out_f64, sizeof(double) * dst.W * dst.H);
    }
    r.t_done = now;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  for (auto& rp : ln.reqs) {
    rp->state = status == FSE_OK ? FSE_REQ_DONE : FSE_REQ_FAILED;
    rp->status = status;
    s->latencies.push_back(std::chrono::duration<double>(rp->t_done - rp->t_submit).count());
    if (s->latencies.size() > 1000000) s->latencies.pop_front();
  }
  s->resident -= (int)ln.reqs.size();
  ln.reqs.clear();
  ln.staged.clear();
  ln.busy = false;
  s->cv_done.notify_all();
}

// Stages the batch in the lane's pinned buffer and enqueues it on its stream.
int launch(Lane& ln) {
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t r = (off + 255) / 256 * 256; off = r + bytes; return ln.pinned + r; };
  ln.staged.clear();
  for (auto& rp : ln.reqs) {
    Request& r = *rp;
    fse_job_t j = r.job;
    const size_t px = (size_t)j.W * j.H;
    uint8_t* im = (uint8_t*)take(px);
    uint8_t* mk = (uint8_t*)take(px);
    memcpy(im, r.image.data(), px);
    memcpy(mk, r.mask.data(), px);
    j.image = im;
    j.mask = mk;
    j.out = (uint8_t*)take(px);
    j.out_f32 = r.job.out_f32 ? (float*)take(px * 4) : nullptr;
    j.out_f64 = r.job.out_f64 ? (double*)take(px * 8) : nullptr;
    j.pitch = j.W;
    ln.staged.push_back(j);
    r.t_launch = Clock::now();
    r.state = FSE_REQ_RUNNING;
  }
  int rc = fse::enqueue_host(ln.ctx, ln.staged.data(), (int32_t)ln.staged.size(), ln.stream, nullptr);
  if (rc) return rc;
  if (cudaEventRecord(ln.done, ln.stream) != cudaSuccess) return fse::fail(FSE_ECUDA, "event");
  ln.busy = true;
  return FSE_OK;
}

// Device status of the lane's finished batch (bounded-wait timeouts etc.).
int lane_status(Lane& ln) {
  if (!ln.ctx->last_q) return FSE_OK;
  fse::QueueDev q[fse::MAX_CLS];
  if (cudaMemcpy(q, ln.ctx->last_q, sizeof(q), cudaMemcpyDeviceToHost) != cudaSuccess)
    return FSE_ECUDA;
  int err = 0;
  for (int k = 0; k < fse::MAX_CLS; ++k) err |= q[k].error;
  if (err & fse::ERR_TIMEOUT) return FSE_ETIMEOUT;
  if (err) return FSE_ENOMEM;
  return FSE_OK;
}

void worker_main(fse_server* s) {
  cudaSetDevice(s->device);
  for (;;) {
    bool progressed = false;
    // retire finished lanes
    for (Lane& ln : s->lanes) {
      if (!ln.busy) continue;
      const cudaError_t q = cudaEventQuery(ln.done);
      if (q == cudaErrorNotReady) continue;
      finish(s, ln, q == cudaSuccess ? lane_status(ln) : FSE_ECUDA);
      progressed = true;
    }
    // admit queued requests into free lanes
    for (Lane& ln : s->lanes) {
      if (ln.busy) continue;
      {
        std::lock_guard<std::mutex> lk(s->mu);
        size_t dev = 0, host = 0;
        while (!s->queue.empty() && (int)ln.reqs.size() < s->max_batch &&
               s->resident < s->max_resident) {
          const ReqPtr& r = s->queue.front();
          if (dev + r->dev_bytes > s->lane_bytes || host + r->host_bytes > ln.pinned_bytes) break;
          dev += r->dev_bytes;
          host += r->host_bytes;
          ln.reqs.push_back(r);
          s->queue.pop_front();
          ++s->resident;
        }
      }
      if (ln.reqs.empty()) continue;
      const int rc = launch(ln);
      if (rc != FSE_OK) finish(s, ln, rc);
      progressed = true;
    }
    std::unique_lock<std::mutex> lk(s->mu);
    bool any_busy = false;
    for (Lane& ln : s->lanes) any_busy |= ln.busy;
    if (s->stop && s->queue.empty() && !any_busy) break;
    if (!progressed) {
      // woken by a submission; polls the lanes' events every 50 us while busy
      s->cv_work.wait_for(lk, std::chrono::microseconds(any_busy ? 50 : 2000));
    }
  }
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
  if (cfg->arena_bytes > free_b) return fse::fail(FSE_ENOMEM, "server arena %zu > free %zu", cfg->arena_bytes, free_b);
  fse_server* s = new fse_server();
  s->device = ctx->device;
  s->max_queue = cfg->max_queue > 0 ? cfg->max_queue : 64;
  s->max_resident = cfg->max_resident > 0 ? cfg->max_resident : 64;
  s->max_batch = cfg->max_batch > 0 ? cfg->max_batch : 16;
  const int n_lanes = 4;
  if (cudaMalloc(&s->arena, cfg->arena_bytes) != cudaSuccess) {
    cudaGetLastError();
    delete s;
    return fse::fail(FSE_ENOMEM, "server arena of %zu bytes", cfg->arena_bytes);
  }
  s->lane_bytes = cfg->arena_bytes / n_lanes / 256 * 256;
  s->lanes.resize(n_lanes);
  int rc = FSE_OK;
  for (int i = 0; i < n_lanes && rc == FSE_OK; ++i) {
    Lane& ln = s->lanes[i];
    rc = fse::context_create_alias(&ln.ctx, s->device, s->arena + i * s->lane_bytes, s->lane_bytes);
    if (rc) break;
    ln.ctx->exec_mode = ctx->exec_mode;
    ln.ctx->ctas_per_sm = ctx->ctas_per_sm;
    ln.ctx->timeout_ms = ctx->timeout_ms;
    ln.ctx->cfg = ctx->cfg;  // the parent context's executor variants and tuning
    for (int k = 0; k < fse::MAX_CLS; ++k) ln.ctx->tuned_ctas[k] = ctx->tuned_ctas[k];
    ln.ctx->concurrent = ctx->concurrent;
    ln.ctx->class_order = ctx->class_order;
    fse::update_occupancy(ln.ctx);
    ln.pinned_bytes = std::min<size_t>(s->lane_bytes / 2, (size_t)1 << 30);
    if (cudaStreamCreateWithFlags(&ln.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&ln.done, cudaEventDisableTiming) != cudaSuccess ||
        cudaMallocHost(&ln.pinned, ln.pinned_bytes) != cudaSuccess) {
      cudaGetLastError();
      rc = fse::fail(FSE_ENOMEM, "lane %d setup", i);
    }
  }
  if (rc) {
    fse_server_destroy(s);
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
  int32_t nt = 0;
  std::vector<fse_tile_t> tl(job->p.n_tiles);
  rc = fse::plan_tiles_mode(job->p.tiling, job->W, job->H, job->p.n_tiles, job->p.overlap, tl.data(),
                            job->p.n_tiles, &nt);
  if (rc) return rc;
  auto r = std::make_shared<Request>();
  r->job = *job;
  r->dev_bytes = fse::job_device_bytes(*job);
  r->host_bytes = host_bytes_of(*job);
  if (r->dev_bytes > s->lane_bytes || r->host_bytes > s->lanes[0].pinned_bytes)
    return fse::fail(FSE_ENOMEM, "request needs %zu device bytes, a lane has %zu", r->dev_bytes,
                     s->lane_bytes);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return fse::fail(FSE_ECANCELLED, "server shutting down");
    if ((int)s->queue.size() >= s->max_queue) return fse::fail(FSE_EBUSY, "queue full");
  }
  const size_t px = (size_t)job->W * job->H;
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
  for (Lane& ln : s->lanes) {
    if (ln.stream) cudaStreamSynchronize(ln.stream);
    if (ln.ctx) fse::context_destroy(ln.ctx);
    if (ln.stream) cudaStreamDestroy(ln.stream);
    if (ln.done) cudaEventDestroy(ln.done);
    if (ln.pinned) cudaFreeHost(ln.pinned);
  }
  if (s->arena) cudaFree(s->arena);
  delete s;
}

}  // extern "C"
