// pdmcf_serve.cu — asynchronous solves with continuous batching
// (mcf_submit / mcf_poll / mcf_wait / mcf_cancel / mcf_serving_config).
//
// A scheduler thread owns one BatchEngine per device. Between chunks of batched PDHG
// iterations it admits queued requests whose device footprint fits the HBM budget and a
// free slot (first come, first served; a request that does not fit yet waits, later small
// ones may pass it), and retires requests whose stop rule fired. Requests that arrive while
// others are on the GPU therefore join the running batch at the next chunk boundary, and
// their work shares every launch with the resident ones. A problem keeps its iterate
// (F, Y, omega) resident after a solve, so a request with warm_start = 1 re-solves from it
// (Sec. 3.1, warm start). Requests the batched kernels do not serve (FP64 or BF16 storage,
// a forced launch shape) run one at a time on a helper thread.
//
// A problem has at most one outstanding ticket: from mcf_submit until the ticket is
// collected (the poll or wait that reports its final status, or mcf_cancel of a finished
// ticket). A finished ticket's T, F and Y are read from the problem's device state when it is
// collected, so no other solve may touch that state in between; the same rule means the
// scheduler never holds the problem lock of one ticket while trying to take it for another.
#include <stdint.h>

#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "pdmcf_batch_engine.h"
#include "pdmcf_internal.h"

namespace pdmcf {

namespace {

constexpr int kChunk = 10;   // batched iterations between scheduling decisions

struct Ticket {
  mcf_ticket id = 0;
  mcf_problem* p = nullptr;
  mcf_options opts{};
  int status = MCF_PENDING;
  bool started = false;
  bool cancelled = false;
  bool solo = false;
  int64_t bytes = 0;
  int slot = -1;
  mcf_result res{};
  std::chrono::steady_clock::time_point t_submit, t_start;
};

bool batchable(const mcf_problem* p, const mcf_options& o) {
  return o.precision == MCF_FP32 && o.shape < 0 && batch_admit_shape(p) >= 0;
}

class Server {
 public:
  ~Server() { shutdown(false); }

  int submit(mcf_problem* p, const mcf_options* o, mcf_ticket* out) {
    const bool batch = batchable(p, *o);
    const int64_t bytes = device_bytes(p, batch ? MCF_FP32 : o->precision) +
                          (batch ? BatchEngine::extra_bytes(p) : 0);
    std::lock_guard<std::mutex> g(mu_);
    if (bytes > budget_) {
      set_error("request footprint exceeds the serving HBM budget");
      return MCF_ERR_OOM_BUDGET;
    }
    if ((int)queue_.size() + (int)solo_queue_.size() >= max_queue_) {
      set_error("submission queue is full");
      return MCF_ERR_BUSY;
    }
    int idle = 0;
    if (!p->busy.compare_exchange_strong(idle, 1)) {
      set_error("the problem has an outstanding ticket: collect it with mcf_poll or mcf_wait, "
                "or discard it with mcf_cancel, before submitting another");
      return MCF_ERR_BUSY;
    }
    auto t = std::make_shared<Ticket>();
    t->id = next_id_++;
    t->p = p;
    t->opts = *o;
    t->opts.check_log = nullptr;   // the caller's string need not outlive the call
    t->bytes = bytes;
    t->solo = !batch;
    t->t_submit = std::chrono::steady_clock::now();
    tickets_[t->id] = t;
    if (t->solo) {
      solo_queue_.push_back(t);
      if (!solo_.joinable()) solo_ = std::thread([this] { solo_loop(); });
      cv_solo_.notify_one();
    } else {
      queue_.push_back(t);
      if (!sched_.joinable()) sched_ = std::thread([this] { schedule_loop(); });
      cv_work_.notify_one();
    }
    *out = t->id;
    return MCF_OK;
  }

  int poll(mcf_ticket id, int* status, mcf_result* res, int64_t timeout_ms, bool block) {
    std::unique_lock<std::mutex> g(mu_);
    auto it = tickets_.find(id);
    if (it == tickets_.end()) {
      set_error("unknown ticket");
      return MCF_ERR_INVALID;
    }
    std::shared_ptr<Ticket> t = it->second;
    if (block) {
      auto pred = [&] { return t->status != MCF_PENDING; };
      if (timeout_ms < 0) cv_done_.wait(g, pred);
      else if (!cv_done_.wait_for(g, std::chrono::milliseconds(timeout_ms), pred)) {
        if (status) *status = MCF_PENDING;
        set_error("timed out");
        return MCF_ERR_TIMEOUT;
      }
    }
    if (status) *status = t->status;
    if (t->status == MCF_PENDING) return MCF_PENDING;
    tickets_.erase(id);
    g.unlock();
    int rc = MCF_OK;
    if (res) {
      double *T = res->T, *F = res->F, *Y = res->Y;
      *res = t->res;
      res->T = T;
      res->F = F;
      res->Y = Y;
      res->status = t->status;
      if ((T || F || Y) && (t->status == MCF_OK || t->status == MCF_ERR_NOT_CONVERGED)) {
        std::lock_guard<std::mutex> pg(t->p->lock);
        rc = device_copy_outputs(t->p, res);
      }
    }
    t->p->busy.store(0);   // collected: the problem takes new work again
    return rc;
  }

  int cancel(mcf_ticket id) {
    std::lock_guard<std::mutex> g(mu_);
    auto it = tickets_.find(id);
    if (it == tickets_.end()) {
      set_error("unknown ticket");
      return MCF_ERR_INVALID;
    }
    std::shared_ptr<Ticket> t = it->second;
    if (t->status != MCF_PENDING) {   // finished and not collected: discard the result
      tickets_.erase(it);
      t->p->busy.store(0);
      return MCF_OK;
    }
    t->cancelled = true;
    if (!t->started) {
      auto& q = t->solo ? solo_queue_ : queue_;
      for (auto qi = q.begin(); qi != q.end(); ++qi)
        if ((*qi)->id == id) { q.erase(qi); break; }
      finish_unstarted(t);
    }
    // a started batched ticket leaves its slot at the next chunk boundary (schedule_loop);
    // a started one-at-a-time ticket runs to its stop rule and then reports the cancellation
    return MCF_OK;
  }

  int config(int64_t budget, int max_resident) {
    if (budget <= 0 || max_resident < 0) {
      set_error("budget must be > 0 and max_resident >= 0");
      return MCF_ERR_INVALID;
    }
    std::lock_guard<std::mutex> g(mu_);
    budget_ = budget;
    max_resident_ = max_resident;
    cv_work_.notify_all();
    cv_solo_.notify_all();
    return MCF_OK;
  }

  // Stop both threads. Every ticket not finished yet ends with MCF_ERR_CANCELLED: queued
  // ones at once, running batched ones after the chunk in progress (their slots are
  // released, leaving the problem's iterate where the chunk ended, when release_state),
  // a running one-at-a-time solve when it returns. A later mcf_submit starts the threads
  // again. At process exit (release_state false) no CUDA call is made: the engines are
  // left to the driver's teardown.
  void shutdown(bool release_state) {
    {
      std::lock_guard<std::mutex> g(mu_);
      stop_ = true;
      release_state_ = release_state;
    }
    cv_work_.notify_all();
    cv_solo_.notify_all();
    if (sched_.joinable()) sched_.join();
    if (solo_.joinable()) solo_.join();
    std::lock_guard<std::mutex> g(mu_);
    if (release_state) {
      engines_.clear();
    } else {
      for (auto& kv : engines_) (void)kv.second.release();
      engines_.clear();
    }
    stop_ = false;
  }

 private:
  BatchEngine* engine_for(int device) {
    auto it = engines_.find(device);
    if (it != engines_.end()) return it->second.get();
    auto e = std::make_unique<BatchEngine>(device, kMaxSlots);
    if (e->init() != MCF_OK) return nullptr;
    BatchEngine* raw = e.get();
    engines_[device] = std::move(e);
    return raw;
  }

  // Admit queued requests that fit (called with mu_ held; unlocks around GPU work).
  void admit(std::unique_lock<std::mutex>& g) {
    for (auto qi = queue_.begin(); qi != queue_.end();) {
      std::shared_ptr<Ticket> t = *qi;
      if (resident_ >= max_resident_) break;
      if (in_use_ + t->bytes > budget_) { ++qi; continue; }
      BatchEngine* eng = engine_for(t->opts.device);
      if (!eng) {   // no usable device: the request cannot run
        qi = queue_.erase(qi);
        finish_unstarted(t, MCF_ERR_CUDA);
        continue;
      }
      if (eng->free_slots() == 0) { ++qi; continue; }
      if (!t->p->lock.try_lock()) { ++qi; continue; }   // a synchronous call holds it
      qi = queue_.erase(qi);
      t->started = true;
      t->t_start = std::chrono::steady_clock::now();
      in_use_ += t->bytes;
      ++resident_;
      g.unlock();
      int slot = -1;
      const int nchunks = ((t->p->n + 7) / 8 * 8) / 4;
      const int cls = batch_class_for(t->opts.device, nchunks, t->opts.autotune != 0);
      const int rc = eng->add(t->p, t->opts, t.get(), &slot, cls);
      g.lock();
      if (rc != MCF_OK) {
        t->p->lock.unlock();
        finish(t, rc);
      } else {
        t->slot = slot;
        running_[t.get()] = t;
      }
      qi = queue_.begin();   // the queue may have changed while unlocked
    }
  }

  void finish(const std::shared_ptr<Ticket>& t, int rc) {   // mu_ held
    in_use_ -= t->bytes;
    --resident_;
    t->status = t->cancelled ? MCF_ERR_CANCELLED : rc;
    t->res.status = t->status;
    t->res.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t->t_submit).count();
    cv_done_.notify_all();
  }

  void finish_unstarted(const std::shared_ptr<Ticket>& t, int rc = MCF_ERR_CANCELLED) {
    // mu_ held; the ticket was never admitted
    t->status = rc;
    t->res.status = rc;
    t->res.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t->t_submit).count();
    cv_done_.notify_all();
  }

  // Release the engine slots of these running tickets (no lock held: the engines belong to
  // the scheduler thread), then, with mu_ held, unlock their problems and finish them.
  void retire(std::unique_lock<std::mutex>& g, std::vector<std::shared_ptr<Ticket>>& ts, int rc,
              bool release) {
    for (auto& t : ts) running_.erase(t.get());
    g.unlock();
    if (release)
      for (auto& t : ts) {
        auto it = engines_.find(t->opts.device);
        if (it != engines_.end() && t->slot >= 0) it->second->release(t->slot);
      }
    g.lock();
    for (auto& t : ts) {
      t->p->lock.unlock();
      finish(t, rc);
    }
    ts.clear();
  }

  void schedule_loop() {
    std::unique_lock<std::mutex> g(mu_);
    for (;;) {
      if (stop_) {   // shutdown: cancel what runs and what waits
        std::vector<std::shared_ptr<Ticket>> all;
        for (auto& kv : running_) {
          kv.second->cancelled = true;
          all.push_back(kv.second);
        }
        retire(g, all, MCF_ERR_CANCELLED, release_state_);
        for (auto& t : queue_) finish_unstarted(t);
        queue_.clear();
        return;
      }
      admit(g);
      if (running_.empty()) {
        const bool paused = max_resident_ == 0;
        if (queue_.empty() || paused)
          cv_work_.wait(g, [&] { return stop_ || (!queue_.empty() && max_resident_ > 0); });
        else   // queued work whose problem a synchronous call still holds
          cv_work_.wait_for(g, std::chrono::milliseconds(2));
        continue;
      }
      // running tickets cancelled since the last chunk leave their slots now
      std::vector<std::shared_ptr<Ticket>> gone;
      for (auto& kv : running_)
        if (kv.second->cancelled) gone.push_back(kv.second);
      if (!gone.empty()) {
        retire(g, gone, MCF_ERR_CANCELLED, true);
        continue;
      }
      g.unlock();
      std::vector<std::pair<Ticket*, mcf_result>> done;
      int err = MCF_OK;
      for (auto& kv : engines_) {
        BatchEngine* eng = kv.second.get();
        if (eng->active_count() == 0) continue;
        const int rc = eng->step(kChunk);
        if (rc != MCF_OK) err = rc;
        for (int s : eng->take_finished()) {
          Ticket* tk = static_cast<Ticket*>(eng->slot(s).tag);
          eng->release(s);
          mcf_result r = eng->slot(s).res;
          r.status = eng->slot(s).status;
          done.emplace_back(tk, r);
        }
      }
      g.lock();
      for (auto& dn : done) {
        auto it = running_.find(dn.first);
        if (it == running_.end()) continue;
        std::shared_ptr<Ticket> t = it->second;
        running_.erase(it);
        t->res = dn.second;
        t->p->lock.unlock();
        finish(t, dn.second.status);
      }
      if (err != MCF_OK) {   // a device error ends every running request
        std::vector<std::shared_ptr<Ticket>> all;
        for (auto& kv : running_) all.push_back(kv.second);
        retire(g, all, err, true);
        // rebuild the engines on the next admission rather than reuse a failed one
        g.unlock();
        engines_.clear();
        g.lock();
      }
    }
  }

  void solo_loop() {
    std::unique_lock<std::mutex> g(mu_);
    for (;;) {
      cv_solo_.wait(g, [&] { return stop_ || (!solo_queue_.empty() && max_resident_ > 0); });
      if (stop_) {
        for (auto& t : solo_queue_) finish_unstarted(t);
        solo_queue_.clear();
        return;
      }
      std::shared_ptr<Ticket> t = solo_queue_.front();
      solo_queue_.pop_front();
      t->started = true;
      in_use_ += t->bytes;
      ++resident_;
      g.unlock();
      mcf_result r{};
      int rc;
      {
        std::lock_guard<std::mutex> pg(t->p->lock);
        rc = device_solve(t->p, &t->opts, &r);
      }
      g.lock();
      t->res = r;
      finish(t, rc);
    }
  }

  static constexpr int kMaxSlots = 256;
  std::mutex mu_;
  std::condition_variable cv_work_, cv_done_, cv_solo_;
  std::deque<std::shared_ptr<Ticket>> queue_, solo_queue_;
  std::unordered_map<mcf_ticket, std::shared_ptr<Ticket>> tickets_;
  std::map<Ticket*, std::shared_ptr<Ticket>> running_;
  std::map<int, std::unique_ptr<BatchEngine>> engines_;
  std::thread sched_, solo_;
  mcf_ticket next_id_ = 1;
  int64_t budget_ = (int64_t)120 * 1000 * 1000 * 1000;
  int64_t in_use_ = 0;
  int max_resident_ = kMaxSlots;
  int resident_ = 0;
  int max_queue_ = 1 << 16;
  bool stop_ = false;
  bool release_state_ = true;
};

Server& server() {
  static Server s;
  return s;
}

}  // namespace
}  // namespace pdmcf

using namespace pdmcf;

extern "C" {

int mcf_submit(mcf_problem* p, const mcf_options* opts, mcf_ticket* ticket) {
  if (!p || !ticket) {
    set_error("problem or ticket is NULL");
    return MCF_ERR_INVALID;
  }
  int rc = validate_options(opts);
  if (rc != MCF_OK) return rc;
  return server().submit(p, opts, ticket);
}

int mcf_poll(mcf_ticket ticket, int* status, mcf_result* res) {
  return server().poll(ticket, status, res, 0, false);
}

int mcf_wait(mcf_ticket ticket, int64_t timeout_ms, int* status, mcf_result* res) {
  return server().poll(ticket, status, res, timeout_ms, true);
}

int mcf_cancel(mcf_ticket ticket) { return server().cancel(ticket); }

int mcf_serving_config(int64_t hbm_budget_bytes, int max_resident) {
  return server().config(hbm_budget_bytes, max_resident);
}

int mcf_serving_shutdown(void) {
  server().shutdown(true);
  return MCF_OK;
}

}  // extern "C"
