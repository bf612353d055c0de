// server.cu -- luda_server: continuous batching of compaction jobs on one GPU.
//
// Slots: each slot is a host thread with its own non-blocking CUDA stream. A slot takes
// the oldest queued job, runs it through the ordinary single-job pipeline, and takes the
// next one as soon as it is done, so jobs that arrive while others run start as soon as a
// slot frees up and their kernels overlap with the running jobs' on the device.
//
// Memory: the pipeline calls the slot's admission gate after its sizing pass with the
// job's peak device bytes. The gate admits jobs first come, first served while the sum of
// admitted bytes stays within the budget; a job bigger than the budget is admitted alone.
// A job releases its bytes when it completes (its new tables then belong to the caller).
// Waiting jobs hold only their sizing buffers and running jobs never wait, so the gate
// cannot deadlock.
#include <cuda_runtime.h>

#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.cuh"
#include "luda.h"

using namespace luda;

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

enum class TState { kQueued, kRunning, kDone };

struct Ticket {
  uint64_t id = 0;
  luda_job job{};
  std::vector<luda_input> inputs;
  std::vector<uint8_t> range_lo, range_hi;  // copies of the job's range keys
  TState state = TState::kQueued;
  luda_status rc = LUDA_OK;
  luda_outputs out{};
  luda_job_stats stats{};
  bool host = false;  // inputs and outputs in host memory
  char detail[512] = {0};
  Clock::time_point t_submit, t_start, t_gate, t_admit, t_done;
};

}  // namespace

struct luda_server {
  luda_server_config cfg{};
  luda_tuning tuning{};               // copy of cfg.opts.tuning (cfg.opts.tuning points here)
  int device = 0;
  std::vector<cudaStream_t> streams;
  std::vector<std::thread> slots;

  std::mutex mu;
  std::condition_variable cv_queue;   // a job was queued, or stopping
  std::condition_variable cv_done;    // a job completed
  std::condition_variable cv_budget;  // budget released or the admission queue moved
  std::deque<Ticket*> queue;
  std::unordered_map<uint64_t, std::unique_ptr<Ticket>> tickets;
  std::deque<uint64_t> completed;     // not yet returned by luda_server_next
  std::deque<uint64_t> gate_fifo;     // jobs waiting for admission, in arrival order
  uint64_t next_id = 1;
  uint64_t used = 0;
  uint32_t running = 0;               // admitted jobs
  bool stopping = false;
  std::mutex copy_mu[2];              // host jobs: inputs in / tables out, one job at a time each
  luda_server_stats st{};
};

namespace {

struct SlotGate final : AdmitGate {
  luda_server* s;
  Ticket* t;
  SlotGate(luda_server* srv, Ticket* tk) : s(srv), t(tk) {}
  bool admit(uint64_t bytes) override {
    std::unique_lock<std::mutex> lk(s->mu);
    t->t_gate = Clock::now();
    s->gate_fifo.push_back(t->id);
    s->cv_budget.wait(lk, [&] {
      return s->gate_fifo.front() == t->id && (s->used + bytes <= s->cfg.hbm_budget || s->running == 0);
    });
    s->gate_fifo.pop_front();
    s->used += bytes;
    s->running += 1;
    if (s->used > s->st.budget_peak) s->st.budget_peak = s->used;
    if (s->running > s->st.running_peak) s->st.running_peak = s->running;
    t->stats.reserved_bytes = bytes;
    t->stats.running_at_admit = s->running;
    t->t_admit = Clock::now();
    s->cv_budget.notify_all();  // the next waiting job may fit as well
    return true;
  }
  void copy_begin(int dir) override { s->copy_mu[dir].lock(); }
  void copy_end(int dir) override { s->copy_mu[dir].unlock(); }
};

void slot_main(luda_server* s, uint32_t slot) {
  cudaSetDevice(s->device);
  luda::warm_thread();  // best effort: a job sets up whatever is still missing itself
  for (;;) {
    Ticket* t = nullptr;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_queue.wait(lk, [&] { return !s->queue.empty() || s->stopping; });
      if (s->queue.empty()) return;  // stopping and drained
      t = s->queue.front();
      s->queue.pop_front();
      t->state = TState::kRunning;
      t->t_start = Clock::now();
    }
    luda_options o = s->cfg.opts;
    o.stream = s->streams[slot];
    o.bottommost = t->job.bottommost;
    SlotGate gate(s, t);
    const luda_status rc = t->host ? compact_job_host(t->job, &o, &t->out, &gate)
                                   : compact_job_device(t->job, &o, &t->out, &gate);
    if (rc) snprintf(t->detail, sizeof t->detail, "%s", luda_last_error_detail());
    const Clock::time_point now = Clock::now();
    std::lock_guard<std::mutex> lk(s->mu);
    if (t->stats.reserved_bytes) {
      s->used -= t->stats.reserved_bytes;
      s->running -= 1;
    } else {
      t->t_gate = t->t_admit = now;  // failed before admission
    }
    t->rc = rc;
    t->state = TState::kDone;
    t->t_done = now;
    t->stats.slot = slot;
    t->stats.queue_ms = ms_between(t->t_submit, t->t_start);
    t->stats.admit_wait_ms = ms_between(t->t_gate, t->t_admit);
    t->stats.run_ms = ms_between(t->t_start, now);
    t->stats.latency_ms = ms_between(t->t_submit, now);
    s->st.completed += 1;
    if (rc) s->st.failed += 1;
    s->completed.push_back(t->id);
    s->cv_budget.notify_all();
    s->cv_done.notify_all();
  }
}

template <class Pred>
bool wait_for(std::condition_variable& cv, std::unique_lock<std::mutex>& lk, int64_t timeout_ms, Pred pred) {
  if (timeout_ms < 0) {
    cv.wait(lk, pred);
    return true;
  }
  return cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred);
}

}  // namespace

extern "C" {

luda_status luda_server_create(const luda_server_config* cfg, luda_server** server) {
  luda::set_error_detail("");
  if (!cfg || !server) return LUDA_ERR_INVALID_ARG;
  *server = nullptr;
  if (cfg->n_slots < 1 || cfg->n_slots > 64 || cfg->hbm_budget == 0) {
    luda::set_error_detail("n_slots must be 1..64 and hbm_budget > 0");
    return LUDA_ERR_INVALID_ARG;
  }
  auto s = std::make_unique<luda_server>();
  s->cfg = *cfg;
  if (cfg->opts.tuning) {
    if (!luda::tuning_valid(cfg->opts.tuning)) return LUDA_ERR_INVALID_ARG;
    s->tuning = *cfg->opts.tuning;
    s->cfg.opts.tuning = &s->tuning;
  }
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    luda::set_error_detail("no usable CUDA device");
    return LUDA_ERR_CUDA;
  }
  for (uint32_t i = 0; i < cfg->n_slots; ++i) {
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      for (cudaStream_t x : s->streams) cudaStreamDestroy(x);
      luda::set_error_detail("cudaStreamCreateWithFlags failed");
      return LUDA_ERR_CUDA;
    }
    s->streams.push_back(st);
  }
  if (cfg->prewarm_bytes && !cfg->opts.dev_alloc) {
    void* p = nullptr;
    if (cudaMallocAsync(&p, cfg->prewarm_bytes, s->streams[0]) == cudaSuccess) cudaFreeAsync(p, s->streams[0]);
    cudaStreamSynchronize(s->streams[0]);
    cudaGetLastError();  // a prewarm that does not fit is not an error
  }
  for (uint32_t i = 0; i < cfg->n_slots; ++i) s->slots.emplace_back(slot_main, s.get(), i);
  *server = s.release();
  return LUDA_OK;
}

static luda_status submit(luda_server* s, const luda_job* job, uint64_t* ticket, bool host) {
  if (!s || !job || !ticket || (!job->inputs && job->n_inputs)) return LUDA_ERR_INVALID_ARG;
  auto t = std::make_unique<Ticket>();
  t->host = host;
  t->inputs.assign(job->inputs, job->inputs + job->n_inputs);
  t->job = *job;
  t->job.inputs = t->inputs.data();
  if (job->range_lo) {
    t->range_lo.assign(job->range_lo, job->range_lo + job->range_lo_len);
    t->range_lo.push_back(0);  // never empty, so data() is a valid pointer
    t->job.range_lo = t->range_lo.data();
  }
  if (job->range_hi) {
    t->range_hi.assign(job->range_hi, job->range_hi + job->range_hi_len);
    t->range_hi.push_back(0);
    t->job.range_hi = t->range_hi.data();
  }
  for (const luda_input& in : t->inputs) t->stats.input_bytes += in.size;
  t->t_submit = Clock::now();
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stopping) return LUDA_ERR_INVALID_ARG;
  t->id = s->next_id++;
  *ticket = t->id;
  s->queue.push_back(t.get());
  s->tickets.emplace(t->id, std::move(t));
  s->st.submitted += 1;
  s->cv_queue.notify_one();
  return LUDA_OK;
}

luda_status luda_server_submit(luda_server* s, const luda_job* job, uint64_t* ticket) {
  return submit(s, job, ticket, false);
}

luda_status luda_server_submit_host(luda_server* s, const luda_job* job, uint64_t* ticket) {
  return submit(s, job, ticket, true);
}

luda_status luda_server_next(luda_server* s, int64_t timeout_ms, uint64_t* ticket) {
  if (!s || !ticket) return LUDA_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  if (!wait_for(s->cv_done, lk, timeout_ms, [&] { return !s->completed.empty(); })) return LUDA_ERR_TIMEOUT;
  *ticket = s->completed.front();
  s->completed.pop_front();
  return LUDA_OK;
}

luda_status luda_server_wait(luda_server* s, uint64_t ticket, int64_t timeout_ms, luda_outputs* out,
                             luda_job_stats* stats) {
  if (!s || !out) return LUDA_ERR_INVALID_ARG;
  std::unique_ptr<Ticket> t;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) {
      luda::set_error_detail("unknown or already collected ticket");
      return LUDA_ERR_INVALID_ARG;
    }
    Ticket* raw = it->second.get();
    if (!wait_for(s->cv_done, lk, timeout_ms, [&] { return raw->state == TState::kDone; })) return LUDA_ERR_TIMEOUT;
    t = std::move(s->tickets[ticket]);
    s->tickets.erase(ticket);
    for (auto c = s->completed.begin(); c != s->completed.end(); ++c)
      if (*c == ticket) {
        s->completed.erase(c);
        break;
      }
  }
  *out = t->out;
  if (stats) *stats = t->stats;
  luda::set_error_detail(t->detail);
  return t->rc;
}

luda_status luda_server_stats_get(luda_server* s, luda_server_stats* stats) {
  if (!s || !stats) return LUDA_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  *stats = s->st;
  return LUDA_OK;
}

void luda_server_destroy(luda_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stopping = true;
    s->cv_queue.notify_all();
  }
  for (std::thread& th : s->slots) th.join();
  for (auto& kv : s->tickets) luda_outputs_free(&kv.second->out);
  for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
  delete s;
}

}  // extern "C"
