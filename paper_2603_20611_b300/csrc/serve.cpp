// serve.cpp -- request loop of the slice projection library: resident Gaussian
// sets, a queue of slice / stack / voxelize requests, admission by free device
// memory, and continuous batching onto several workers, each with its own
// context (workspace) and CUDA stream, so requests that arrive while others run
// are admitted as soon as a worker and memory are free and their kernels overlap
// on the device.
//
// Batching: a worker that takes a slice or stack request also takes every other
// pending request for the same set, axis, image size and sigma_z (up to
// max_batch_slices planes) and renders all their planes in one call into its
// staging stack, then copies each request's planes to that request's output.
// Every (plane, tile) list and every tile's summation order depend only on the
// set and the plane, so a request's result is bitwise the same alone and in a
// batch.  Pending voxelize requests for the same set and grid ask for the same
// volume: a worker takes them together, voxelizes once and copies the volume to
// each of their outputs.
//
// A request carries its own copy of the set's descriptor (pointers, count,
// scale modifier), taken under the lock when it is submitted, so a worker never
// reads the server's set table, which a concurrent load may grow.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "gp_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t ticket;
  gp_request r;
  gp_set set{};          // the set's descriptor as registered (a copy)
  std::vector<float> z;  // copy of the plane positions
  gp::View view{};       // slice orientation (the request's view, or its axis's)
  Clock::time_point submitted;
  int64_t est_bytes;
};

struct Worker {
  gp_ctx* ctx = nullptr;
  cudaStream_t stream = nullptr;
  float* staging = nullptr;  // batched slice stack
  size_t staging_floats = 0;
  std::thread th;
};

}  // namespace

struct gp_server {
  gp_ctx* owner = nullptr;
  int device = 0;
  gp_serve_cfg cfg{};
  std::vector<gp_set> sets;
  std::vector<void*> owned;  // device memory of sets decoded by the server
  std::vector<Worker> workers;
  std::mutex mu;
  std::condition_variable cv_work;   // workers wait for requests
  std::condition_variable cv_done;   // pollers wait for results
  std::deque<Request> pending;
  std::map<uint64_t, gp_result> done;
  uint64_t next_ticket = 1;
  int64_t inflight_bytes = 0;
  bool stop = false;
  gp_serve_stats stats{};
};

namespace {

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

// Device bytes a request may add while it runs (workspace and staging), a
// conservative estimate used for admission.
int64_t estimate_bytes(const gp_set& g, const gp_request& r) {
  if (r.kind == GP_REQ_VOXELIZE) {
    // the voxelizer bins the grid's Z planes of 16 x 16 tiles: records + tile
    // ranges + pair buffers (20 B per pair; a Gaussian of std 1.5 voxels
    // reaches ~16 planes and ~2 tiles on each)
    const int64_t tiles = (int64_t)((r.X + 15) / 16) * ((r.Y + 15) / 16) * r.Z;
    return g.n * 64 + tiles * 8 + g.n * 32 * 20;
  }
  const int64_t px = (int64_t)r.S * r.H * r.W;
  return px * 4 + g.n * 64 + g.n * 24 * 20;  // staging + records + pair buffers
}

bool same_batch(const Request& qa, const Request& qb) {
  const gp_request &a = qa.r, &b = qb.r;
  if (a.kind == GP_REQ_VOXELIZE || b.kind == GP_REQ_VOXELIZE)
    return a.kind == b.kind && a.set_id == b.set_id && a.X == b.X && a.Y == b.Y && a.Z == b.Z;
  return (a.kind == GP_REQ_SLICE || a.kind == GP_REQ_STACK) && (b.kind == GP_REQ_SLICE || b.kind == GP_REQ_STACK) &&
         a.set_id == b.set_id && gp::same_view(qa.view, qb.view) && a.H == b.H && a.W == b.W &&
         a.sigma_z == b.sigma_z;
}

int64_t free_device_bytes(int device) {
  size_t f = 0, t = 0;
  cudaSetDevice(device);
  if (cudaMemGetInfo(&f, &t) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return (int64_t)f;
}

// Result of a request that leaves the queue without running (deadline passed,
// cancelled).  Caller holds s->mu.
void drop_locked(gp_server* s, const Request& q, gp_status st, Clock::time_point now) {
  gp_result res{};
  res.status = st;
  res.latency_ms = ms_between(q.submitted, now);
  res.queue_ms = res.latency_ms;
  res.batch_size = 0;
  s->done[q.ticket] = res;
  s->stats.completed += 1;
  s->stats.failed += 1;
  if (st == GP_ERR_TIMEOUT) s->stats.expired += 1;
  if (st == GP_ERR_CANCELLED) s->stats.cancelled += 1;
  s->cv_done.notify_all();
}

// Drops the queued requests whose deadline has passed.  Caller holds s->mu.
void expire_locked(gp_server* s) {
  const Clock::time_point now = Clock::now();
  for (auto it = s->pending.begin(); it != s->pending.end();) {
    if (it->r.timeout_ms > 0.0 && ms_between(it->submitted, now) > it->r.timeout_ms) {
      drop_locked(s, *it, GP_ERR_TIMEOUT, now);
      it = s->pending.erase(it);
    } else {
      ++it;
    }
  }
}

void finish(gp_server* s, const std::vector<Request>& reqs, gp_status st, Clock::time_point started) {
  const Clock::time_point now = Clock::now();
  std::lock_guard<std::mutex> lk(s->mu);
  for (const Request& q : reqs) {
    gp_result res;
    res.status = st;
    res.latency_ms = ms_between(q.submitted, now);
    res.queue_ms = ms_between(q.submitted, started);
    res.batch_size = (int)reqs.size();
    s->done[q.ticket] = res;
    s->inflight_bytes -= q.est_bytes;
    s->stats.inflight_requests -= 1;
    s->stats.completed += 1;
    if (st != GP_OK) s->stats.failed += 1;
  }
  s->stats.batches += 1;
  s->cv_done.notify_all();
  s->cv_work.notify_all();
}

gp_status run_slices(gp_server* s, Worker& w, std::vector<Request>& batch) {
  const gp_request& r0 = batch[0].r;
  int S = 0;
  for (const Request& q : batch) S += q.r.S;
  std::vector<float> z;
  z.reserve(S);
  for (const Request& q : batch) z.insert(z.end(), q.z.begin(), q.z.end());
  const size_t need = (size_t)S * r0.H * r0.W;
  float* dst = batch.size() == 1 ? r0.out : nullptr;
  if (!dst) {
    if (need > w.staging_floats) {
      if (w.staging) cudaFree(w.staging);
      w.staging = nullptr;
      w.staging_floats = 0;
      if (cudaMalloc(&w.staging, need * 4) != cudaSuccess) {
        cudaGetLastError();
        return GP_ERR_OOM;
      }
      w.staging_floats = need;
    }
    dst = w.staging;
  }
  gp_view v;
  memcpy(v.R, batch[0].view.R, sizeof(v.R));
  memcpy(v.t, batch[0].view.t, sizeof(v.t));
  gp_status st = gp_render_slices_view(w.ctx, &batch[0].set, &v, z.data(), S, r0.H, r0.W, r0.sigma_z, dst,
                                       w.stream);
  if (st != GP_OK) return st;
  if (batch.size() > 1) {
    size_t off = 0;
    for (const Request& q : batch) {
      const size_t n = (size_t)q.r.S * q.r.H * q.r.W;
      if (cudaMemcpyAsync(q.r.out, dst + off, n * 4, cudaMemcpyDeviceToDevice, w.stream) != cudaSuccess) {
        cudaGetLastError();
        return GP_ERR_CUDA;
      }
      off += n;
    }
  }
  if (cudaStreamSynchronize(w.stream) != cudaSuccess) {
    cudaGetLastError();
    return GP_ERR_CUDA;
  }
  return GP_OK;
}

// Voxelize requests of one set and grid: one volume, copied to every output.
gp_status run_voxelize(Worker& w, std::vector<Request>& batch) {
  const gp_request& r0 = batch[0].r;
  gp_status st = gp_voxelize(w.ctx, &batch[0].set, r0.X, r0.Y, r0.Z, r0.out, w.stream);
  if (st != GP_OK) return st;
  const size_t bytes = (size_t)r0.X * r0.Y * r0.Z * 4;
  for (size_t i = 1; i < batch.size(); ++i)
    if (cudaMemcpyAsync(batch[i].r.out, r0.out, bytes, cudaMemcpyDeviceToDevice, w.stream) != cudaSuccess) {
      cudaGetLastError();
      return GP_ERR_CUDA;
    }
  if (cudaStreamSynchronize(w.stream) != cudaSuccess) {
    cudaGetLastError();
    return GP_ERR_CUDA;
  }
  return GP_OK;
}

void worker_loop(gp_server* s, int wi) {
  Worker& w = s->workers[wi];
  cudaSetDevice(s->device);
  for (;;) {
    std::vector<Request> batch;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      int64_t budget = 0;
      for (;;) {
        if (s->stop) return;
        expire_locked(s);
        if (!s->pending.empty()) {
          // admission: the oldest request first; it runs if its estimate fits in
          // the memory budget (always, when nothing else is in flight)
          const Request& head = s->pending.front();
          budget = s->cfg.hbm_budget_bytes > 0
                       ? s->cfg.hbm_budget_bytes
                       : free_device_bytes(s->device) - s->cfg.hbm_reserve_bytes + s->inflight_bytes;
          if (s->inflight_bytes == 0 || s->inflight_bytes + head.est_bytes <= budget) break;
          s->stats.admission_waits += 1;
        }
        s->cv_work.wait_for(lk, std::chrono::milliseconds(5));
      }
      batch.push_back(std::move(s->pending.front()));
      s->pending.pop_front();
      s->inflight_bytes += batch[0].est_bytes;
      if (batch[0].r.kind != GP_REQ_VOXELIZE) {
        int planes = batch[0].r.S;
        for (auto it = s->pending.begin(); it != s->pending.end();) {
          if (same_batch(batch[0], *it) && planes + it->r.S <= s->cfg.max_batch_slices &&
              s->inflight_bytes + it->est_bytes <= budget) {
            planes += it->r.S;
            s->inflight_bytes += it->est_bytes;
            batch.push_back(std::move(*it));
            it = s->pending.erase(it);
          } else {
            ++it;
          }
        }
      } else {
        // the same volume again: no workspace beyond the first request's, but
        // like a slice it joins only while the memory in flight is in budget
        for (auto it = s->pending.begin(); it != s->pending.end();) {
          if ((int)batch.size() < s->cfg.max_batch_slices && same_batch(batch[0], *it) &&
              s->inflight_bytes <= budget) {
            it->est_bytes = 0;
            batch.push_back(std::move(*it));
            it = s->pending.erase(it);
          } else {
            ++it;
          }
        }
      }
      s->stats.inflight_requests += (int64_t)batch.size();
      s->stats.max_inflight_requests = std::max(s->stats.max_inflight_requests, s->stats.inflight_requests);
    }
    const Clock::time_point started = Clock::now();
    gp::NvtxRange range(batch[0].r.kind == GP_REQ_VOXELIZE ? "gp:serve_voxelize" : "gp:serve_slices");
    gp_status st;
    if (batch[0].r.kind == GP_REQ_VOXELIZE) {
      st = run_voxelize(w, batch);
    } else {
      st = run_slices(s, w, batch);
    }
    finish(s, batch, st, started);
  }
}

gp_status check_request(gp_server* s, const gp_request* r) {
  if (!r) return GP_ERR_ARG;
  if (r->set_id < 0 || r->set_id >= (int)s->sets.size()) return GP_ERR_ARG;
  if (!r->out || !(r->timeout_ms >= 0.0)) return GP_ERR_ARG;
  if (r->kind == GP_REQ_VOXELIZE) {
    if (r->X <= 0 || r->Y <= 0 || r->Z <= 0) return GP_ERR_ARG;
    return GP_OK;
  }
  if (r->kind != GP_REQ_SLICE && r->kind != GP_REQ_STACK) return GP_ERR_ARG;
  if (r->S <= 0 || !r->z || r->H <= 0 || r->W <= 0 || !(r->sigma_z > 0.0f)) return GP_ERR_ARG;
  gp::View v;
  if (r->view ? !gp::check_view(r->view, &v) : !gp::axis_view(r->axis, &v)) return GP_ERR_ARG;
  if (r->kind == GP_REQ_SLICE && r->S != 1) return GP_ERR_ARG;
  if (r->S > s->cfg.max_batch_slices) return GP_ERR_ARG;
  return GP_OK;
}

}  // namespace

extern "C" {

gp_status gp_serve_open(gp_ctx* ctx, const gp_serve_cfg* cfg, gp_server** out) {
  if (!ctx || !out) return GP_ERR_ARG;
  *out = nullptr;
  gp_server* s = new (std::nothrow) gp_server();
  if (!s) return GP_ERR_OOM;
  s->owner = ctx;
  s->device = ctx->impl.device;
  gp_serve_cfg c{};
  c.workers = 4;
  c.max_batch_slices = 64;
  c.hbm_budget_bytes = 0;
  c.hbm_reserve_bytes = (int64_t)4 << 30;
  if (cfg) {
    c = *cfg;
    if (c.workers <= 0 || c.workers > 64 || c.max_batch_slices <= 0 || c.hbm_budget_bytes < 0 ||
        c.hbm_reserve_bytes < 0) {
      delete s;
      return GP_ERR_ARG;
    }
  }
  s->cfg = c;
  s->workers.resize(c.workers);
  gp_config wc = ctx->impl.cfg;
  for (int i = 0; i < c.workers; ++i) {
    Worker& w = s->workers[i];
    gp_status st = gp_create(&w.ctx, s->device, &wc);
    if (st == GP_OK && cudaStreamCreateWithFlags(&w.stream, cudaStreamNonBlocking) != cudaSuccess) st = GP_ERR_CUDA;
    if (st != GP_OK) {
      for (int j = 0; j <= i; ++j) {
        if (s->workers[j].stream) cudaStreamDestroy(s->workers[j].stream);
        if (s->workers[j].ctx) gp_destroy(s->workers[j].ctx);
      }
      delete s;
      return st;
    }
  }
  for (int i = 0; i < c.workers; ++i) s->workers[i].th = std::thread(worker_loop, s, i);
  *out = s;
  return GP_OK;
}

gp_status gp_serve_load_set(gp_server* s, const gp_set* set, int* set_id) {
  if (!s || !set || !set_id) return GP_ERR_ARG;
  if (set->n < 0 || (set->n > 0 && (!set->mu || !set->scale || !set->quat || !set->alpha))) return GP_ERR_ARG;
  if (set->n > 0 && ((uintptr_t)set->quat & 15u)) return GP_ERR_ARG;
  if (!(set->scale_mod > 0.0f)) return GP_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  s->sets.push_back(*set);
  *set_id = (int)s->sets.size() - 1;
  return GP_OK;
}

gp_status gp_serve_load_encoded(gp_server* s, const gp_codec_header* header, const uint16_t* streams,
                                float scale_mod, int* set_id) {
  if (!s || !header || !set_id || header->n < 0 || !(scale_mod > 0.0f)) return GP_ERR_ARG;
  const int64_t n = header->n;
  gp_set set{};
  set.n = n;
  set.scale_mod = scale_mod;
  void* mem = nullptr;
  if (n > 0) {
    if (cudaSetDevice(s->device) != cudaSuccess || cudaMalloc(&mem, (size_t)n * 11 * 4) != cudaSuccess) {
      cudaGetLastError();
      return GP_ERR_OOM;
    }
    float* base = (float*)mem;  // quat first: 16-byte aligned
    set.quat = base;
    set.mu = base + 4 * n;
    set.scale = base + 7 * n;
    set.alpha = base + 10 * n;
    gp_status st = gp_decode(s->owner, header, streams, (float*)set.mu, (float*)set.scale, (float*)set.quat,
                             (float*)set.alpha, nullptr);
    if (st == GP_OK && cudaStreamSynchronize(nullptr) != cudaSuccess) st = GP_ERR_CUDA;
    if (st != GP_OK) {
      cudaFree(mem);
      return st;
    }
  }
  std::lock_guard<std::mutex> lk(s->mu);
  s->sets.push_back(set);
  if (mem) s->owned.push_back(mem);
  *set_id = (int)s->sets.size() - 1;
  return GP_OK;
}

gp_status gp_serve_submit(gp_server* s, const gp_request* r, uint64_t* ticket) {
  if (!s || !ticket) return GP_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  gp_status st = check_request(s, r);
  if (st != GP_OK) return st;
  Request q;
  q.ticket = s->next_ticket++;
  q.r = *r;
  if (r->kind != GP_REQ_VOXELIZE) {
    q.z.assign(r->z, r->z + r->S);
    if (r->view)
      gp::check_view(r->view, &q.view);
    else
      gp::axis_view(r->axis, &q.view);
  }
  q.r.view = nullptr;  // the caller's view need not outlive the submit
  q.set = s->sets[r->set_id];
  q.submitted = Clock::now();
  q.est_bytes = estimate_bytes(q.set, *r);
  *ticket = q.ticket;
  s->pending.push_back(std::move(q));
  s->stats.submitted += 1;
  s->cv_work.notify_one();
  return GP_OK;
}

gp_status gp_serve_poll(gp_server* s, uint64_t ticket, int timeout_ms, gp_result* out) {
  if (!s || !out || ticket == 0) return GP_ERR_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  if (ticket >= s->next_ticket) return GP_ERR_ARG;
  const auto deadline = Clock::now() + std::chrono::milliseconds(std::max(timeout_ms, 0));
  for (;;) {
    expire_locked(s);
    auto it = s->done.find(ticket);
    if (it != s->done.end()) {
      *out = it->second;
      s->done.erase(it);
      return GP_OK;
    }
    if (timeout_ms <= 0 || Clock::now() >= deadline) return GP_PENDING;
    // wake at least every 5 ms, so that a queued request's deadline is seen
    s->cv_done.wait_until(lk, std::min(deadline, Clock::now() + std::chrono::milliseconds(5)));
  }
}

gp_status gp_serve_cancel(gp_server* s, uint64_t ticket) {
  if (!s || ticket == 0) return GP_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  if (ticket >= s->next_ticket) return GP_ERR_ARG;
  for (auto it = s->pending.begin(); it != s->pending.end(); ++it) {
    if (it->ticket == ticket) {
      drop_locked(s, *it, GP_ERR_CANCELLED, Clock::now());
      s->pending.erase(it);
      return GP_OK;
    }
  }
  return GP_ERR_STATE;
}

gp_status gp_serve_stats_get(gp_server* s, gp_serve_stats* out) {
  if (!s || !out) return GP_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  expire_locked(s);
  *out = s->stats;
  out->pending = (int64_t)s->pending.size();
  out->inflight_bytes = s->inflight_bytes;
  return GP_OK;
}

gp_status gp_serve_close(gp_server* s) {
  if (!s) return GP_ERR_ARG;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->cv_work.notify_all();
  }
  for (Worker& w : s->workers)
    if (w.th.joinable()) w.th.join();
  cudaSetDevice(s->device);
  for (Worker& w : s->workers) {
    if (w.stream) {
      cudaStreamSynchronize(w.stream);
      cudaStreamDestroy(w.stream);
    }
    if (w.staging) cudaFree(w.staging);
    if (w.ctx) gp_destroy(w.ctx);
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    for (const Request& q : s->pending) {
      gp_result res{};
      res.status = GP_ERR_STATE;
      s->done[q.ticket] = res;
    }
    s->pending.clear();
  }
  for (void* m : s->owned) cudaFree(m);
  delete s;
  return GP_OK;
}

}  // extern "C"
