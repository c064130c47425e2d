// Serving loop: continuous batching of plan re-optimisation requests on one
// GPU.  Requests of uneven sizes are admitted while earlier ones run, as long
// as their device footprint fits under a memory cap and an active slot is
// free; every admitted plan keeps its matrices and iteration state resident
// on its own stream, and the iterations of all active plans are enqueued in
// rounds so that their kernels overlap on the device.  Every tile shape of a
// plan depends on that plan alone, so a result is bit-identical whether the
// plan runs alone or among others.
//
// Threads: a loader thread admits queued requests (FIFO) and loads them
// (upload, validation, CSC copy, schedules); a scheduler thread keeps each
// active plan's stream fed with rounds of iterations and finishes plans
// whose iterations are done (final FP64 pass, outputs to the caller's host
// buffers).  The public calls only touch the request table under a mutex.
#include "fredopt.h"
#include "fredopt_internal.cuh"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

namespace {

using Clock = std::chrono::steady_clock;

enum Status { QUEUED = 0, LOADING = 1, RUNNING = 2, DONE = 3 };

struct Req {
  int64_t id = 0;
  fredopt_request r{};
  std::vector<fredopt_constraint> con;
  std::vector<fredopt_objective_term> obj;
  int status = QUEUED;  // or a negative error code
  int64_t footprint = 0;
  double t_submit = 0, t_admit = 0, t_start = 0, t_done = 0;
  fredopt_t h = nullptr;
  int enqueued = 0;            // iterations enqueued so far
  cudaEvent_t round_done = nullptr;
  bool round_pending = false;
  fredopt_report rep{};
  cudaStream_t stream = nullptr;  // the plan's stream, created with `prio`
  int prio = 0;
};

}  // namespace

struct fredopt_server {
  int device = 0;
  int64_t mem_cap = 0;
  int max_active = 1;
  int round_iters = 10;
  Clock::time_point t0;

  std::mutex mu;
  std::condition_variable cv;      // wakes the loader / waiters
  std::condition_variable cv_sched;
  std::map<int64_t, std::shared_ptr<Req>> table;
  std::deque<int64_t> queue;       // waiting for admission (FIFO)
  std::vector<std::shared_ptr<Req>> active;
  int64_t mem_used = 0;
  int n_loading = 0;
  int prio_least = 0, prio_greatest = 0;  // CUDA stream priority range (greatest is numerically lowest)
  int64_t next_id = 1;
  bool stop = false;
  std::thread loader, scheduler;

  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace {

// Destroy a plan's handle and then its stream.
void release(Req& q) {
  if (q.h) fredopt_destroy(q.h);
  q.h = nullptr;
  if (q.stream) cudaStreamDestroy(q.stream);
  q.stream = nullptr;
}

void set_error(fredopt_server* s, const std::shared_ptr<Req>& q, int code) {
  std::lock_guard<std::mutex> lk(s->mu);
  q->status = code;
  q->t_done = s->now();
  s->mem_used -= q->footprint;
  s->cv.notify_all();
}

void loader_main(fredopt_server* s) {
  cudaSetDevice(s->device);
  while (true) {
    std::shared_ptr<Req> q;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv.wait(lk, [&] {
        if (s->stop) return true;
        if (s->queue.empty()) return false;
        const auto& f = s->table[s->queue.front()];
        const int busy = (int)s->active.size() + s->n_loading;
        return busy < s->max_active && s->mem_used + f->footprint <= s->mem_cap;
      });
      if (s->stop) return;
      q = s->table[s->queue.front()];
      s->queue.pop_front();
      s->mem_used += q->footprint;
      s->n_loading += 1;
      q->status = LOADING;
      q->t_admit = s->now();
      // Stream priority.  Admitted with no backlog (latency matters): the
      // level below the youngest plan in flight, so the block scheduler
      // serves older plans first and younger ones fill the SMs they leave
      // idle.  Admitted while requests still wait (throughput matters): the
      // lowest level, shared, so the plans interleave freely.
      int lvl = s->prio_greatest;
      for (const auto& kv : s->table) {
        const Req& o = *kv.second;
        if (&o != q.get() && (o.status == LOADING || o.status == RUNNING) && o.stream)
          lvl = std::max(lvl, o.prio + 1);
      }
      q->prio = s->queue.empty() ? std::min(lvl, s->prio_least) : s->prio_least;
    }
    const fredopt_request& r = q->r;
    fredopt_t h = nullptr;
    int rc = cudaStreamCreateWithPriority(&q->stream, cudaStreamNonBlocking, q->prio) == cudaSuccess
                 ? FREDOPT_OK
                 : FREDOPT_ERR_CUDA;
    if (rc == FREDOPT_OK) rc = fredopt_create(&h, s->device, q->stream);
    if (rc == FREDOPT_OK)
      rc = fredopt_load_influence(h, r.n_vox, r.n_spots, r.nnz, r.row_ptr, r.col, r.D_val, r.L_val,
                                  r.voxel_mask, r.format | (s->max_active > 1 ? FREDOPT_SHARED : 0u), 0);
    if (rc == FREDOPT_OK) rc = fredopt_set_constraints(h, (int)q->con.size(), q->con.data());
    if (rc == FREDOPT_OK) rc = fredopt_set_objective(h, (int)q->obj.size(), q->obj.data());
    if (rc == FREDOPT_OK) rc = fredopt_begin(h, r.w0, r.alpha, r.relaxation, &r.params, 0);
    if (rc == FREDOPT_OK && cudaEventCreateWithFlags(&q->round_done, cudaEventDisableTiming) != cudaSuccess)
      rc = FREDOPT_ERR_CUDA;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->n_loading -= 1;
    }
    if (rc != FREDOPT_OK) {
      q->h = h;
      release(*q);
      set_error(s, q, rc);
      continue;
    }
    {
      std::lock_guard<std::mutex> lk(s->mu);
      q->h = h;
      q->status = RUNNING;
      q->t_start = s->now();
      s->active.push_back(q);
    }
    s->cv_sched.notify_all();
  }
}

// Finish a plan whose iterations have all run: final pass and outputs.
void finish(fredopt_server* s, const std::shared_ptr<Req>& q) {
  const fredopt_request& r = q->r;
  fredopt_report rep{};
  int rc = fredopt_end(q->h, r.w_out, r.dose_out, r.letd_out, &rep, 0);
  cudaEventDestroy(q->round_done);
  release(*q);
  std::lock_guard<std::mutex> lk(s->mu);
  q->rep = rep;
  q->status = rc == FREDOPT_OK ? DONE : rc;
  q->t_done = s->now();
  s->mem_used -= q->footprint;
  s->active.erase(std::remove(s->active.begin(), s->active.end(), q), s->active.end());
  s->cv.notify_all();
}

void scheduler_main(fredopt_server* s) {
  cudaSetDevice(s->device);
  while (true) {
    std::vector<std::shared_ptr<Req>> act;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_sched.wait_for(lk, std::chrono::microseconds(200), [&] { return s->stop || !s->active.empty(); });
      if (s->stop && s->active.empty()) return;
      act = s->active;
    }
    bool progressed = false;
    for (auto& q : act) {
      if (q->round_pending) {
        const cudaError_t e = cudaEventQuery(q->round_done);
        if (e == cudaErrorNotReady) continue;
        q->round_pending = false;
      }
      if (q->enqueued < q->r.iters) {
        const int n = std::min(s->round_iters, q->r.iters - q->enqueued);
        int rc = fredopt_iterate(q->h, n);
        if (rc == FREDOPT_OK && cudaEventRecord(q->round_done, fo::handle_stream(q->h)) != cudaSuccess)
          rc = FREDOPT_ERR_CUDA;
        if (rc != FREDOPT_OK) {
          cudaEventDestroy(q->round_done);
          release(*q);
          {
            std::lock_guard<std::mutex> lk(s->mu);
            s->active.erase(std::remove(s->active.begin(), s->active.end(), q), s->active.end());
          }
          set_error(s, q, rc);
          continue;
        }
        q->enqueued += n;
        q->round_pending = true;
        progressed = true;
      } else {
        finish(s, q);
        progressed = true;
      }
    }
    if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

void fill_info(const Req& q, fredopt_ticket_info* info) {
  if (!info) return;
  std::memset(info, 0, sizeof(*info));
  info->status = q.status;
  info->t_submit = q.t_submit;
  info->t_admit = q.t_admit;
  info->t_start = q.t_start;
  info->t_done = q.t_done;
  info->footprint_bytes = q.footprint;
  info->report = q.rep;
}

}  // namespace

extern "C" {

int64_t fredopt_footprint_bytes(int64_t n_vox, int32_t n_spots, int64_t nnz, int format) {
  if (n_vox < 0 || n_spots < 1 || nnz < 0) return -1;
  const int fmt = format & 0xff;
  const int64_t vb = fmt == FREDOPT_FP32 ? 4 : 2;
  const int64_t na = ((nnz + 255) & ~255LL) + fo::kPadElems;
  // peaks of the load: FP32 upload + gathered copy; the CSC fill's CSR + CSC
  // + one scratch record per entry (16 bytes with FP32 values, 8 with 16-bit);
  // while the 16-bit index copies are made, CSR + CSC (int32 indices) + both
  // 16-bit copies
  const int64_t rec = vb == 4 ? 16 : 8;
  const int64_t load_peak =
      std::max(std::max(2 * na * 12, na * (2 * (4 + 2 * vb) + 4)), na * (2 * (4 + 2 * vb) + rec));
  // resident: CSR with 16-bit columns and CSC with int32 and based 16-bit
  // rows (as much as two int32 copies), the 16-bit copies' FP32 staging, the
  // block headers of the based rows, and their overflow table for wide blocks
  // (one per column boundary plus one in 16 blocks; a plan whose rows are
  // sparser than that can exceed the estimate, and its load then fails with
  // FREDOPT_ERR_OOM without disturbing the plans in flight)
  const int64_t headers = na / 128 * 4;
  const int64_t overflow = ((int64_t)n_spots + na / 128 / 16) * 128 * 4;
  const int64_t resident = na * (4 + 2 * vb) * 2 + (fmt ? na * 8 : 0) + headers + overflow;
  const int64_t per_row = n_vox * (8 + 8 + 4 + 24 + 4 * 8 + 16 + 8 + 16 + 8 + (fmt ? 8 : 0));
  const int64_t per_spot = (int64_t)n_spots * (4 * 4 + 8 + 4) + (int64_t)2 * 152 * n_spots * 4;
  const int64_t tables = na / 256 * 16 + ((int64_t)16 << 20);
  return std::max(load_peak, resident) + per_row + per_spot + tables;
}

int fredopt_server_create(fredopt_server_t* out, int device, int64_t mem_cap_bytes, int max_active,
                          int round_iters) {
  if (!out || mem_cap_bytes <= 0 || max_active < 1 || round_iters < 1) return FREDOPT_ERR_INVALID_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return FREDOPT_ERR_INVALID_ARG;
  }
  fredopt_server* s = new fredopt_server();
  s->device = device;
  s->mem_cap = mem_cap_bytes;
  s->max_active = max_active;
  s->round_iters = round_iters;
  s->t0 = Clock::now();
  {
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(device);
    if (cudaDeviceGetStreamPriorityRange(&s->prio_least, &s->prio_greatest) != cudaSuccess) {
      cudaGetLastError();
      s->prio_least = s->prio_greatest = 0;
    }
    cudaSetDevice(cur);
  }
  s->loader = std::thread(loader_main, s);
  s->scheduler = std::thread(scheduler_main, s);
  *out = s;
  return FREDOPT_OK;
}

int fredopt_server_submit(fredopt_server_t s, const fredopt_request* r, int64_t* ticket) {
  if (!s || !r || !ticket) return FREDOPT_ERR_INVALID_ARG;
  if (r->iters < 0 || !r->w0 || !r->row_ptr || !r->voxel_mask || r->n_constraints < 0 ||
      r->n_objective < 0 || (r->n_constraints > 0 && !r->constraints) || (r->n_objective > 0 && !r->objective))
    return FREDOPT_ERR_INVALID_ARG;
  const int64_t fp = fredopt_footprint_bytes(r->n_vox, r->n_spots, r->nnz, r->format);
  if (fp < 0) return FREDOPT_ERR_SHAPE;
  auto q = std::make_shared<Req>();
  q->r = *r;
  q->con.assign(r->constraints, r->constraints + r->n_constraints);
  q->obj.assign(r->objective, r->objective + r->n_objective);
  q->footprint = fp;
  std::lock_guard<std::mutex> lk(s->mu);
  if (fp > s->mem_cap) return FREDOPT_ERR_OOM;  // could never be admitted
  q->id = s->next_id++;
  q->t_submit = s->now();
  s->table[q->id] = q;
  s->queue.push_back(q->id);
  *ticket = q->id;
  s->cv.notify_all();
  return FREDOPT_OK;
}

int fredopt_server_poll(fredopt_server_t s, int64_t ticket, fredopt_ticket_info* info) {
  if (!s) return FREDOPT_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->table.find(ticket);
  if (it == s->table.end()) return FREDOPT_ERR_INVALID_ARG;
  fill_info(*it->second, info);
  return FREDOPT_OK;
}

int fredopt_server_wait(fredopt_server_t s, int64_t ticket, double timeout_s, fredopt_ticket_info* info) {
  if (!s) return FREDOPT_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->table.find(ticket);
  if (it == s->table.end()) return FREDOPT_ERR_INVALID_ARG;
  auto q = it->second;
  const bool ok = s->cv.wait_for(lk, std::chrono::duration<double>(timeout_s),
                                 [&] { return q->status == DONE || q->status < 0; });
  fill_info(*q, info);
  return ok ? FREDOPT_OK : FREDOPT_ERR_TIMEOUT;
}

int fredopt_server_drain(fredopt_server_t s, double timeout_s) {
  if (!s) return FREDOPT_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  const bool ok = s->cv.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] {
    for (auto& kv : s->table)
      if (kv.second->status >= 0 && kv.second->status != DONE) return false;
    return true;
  });
  return ok ? FREDOPT_OK : FREDOPT_ERR_TIMEOUT;
}

int fredopt_server_stats(fredopt_server_t s, int64_t* mem_used, int* n_active, int* n_queued) {
  if (!s) return FREDOPT_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  if (mem_used) *mem_used = s->mem_used;
  if (n_active) *n_active = (int)s->active.size() + s->n_loading;
  if (n_queued) *n_queued = (int)s->queue.size();
  return FREDOPT_OK;
}

int fredopt_server_destroy(fredopt_server_t s) {
  if (!s) return FREDOPT_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->queue.clear();
  }
  s->cv.notify_all();
  s->cv_sched.notify_all();
  s->loader.join();
  // the scheduler finishes the plans that are already active
  s->scheduler.join();
  delete s;
  return FREDOPT_OK;
}

}  // extern "C"
