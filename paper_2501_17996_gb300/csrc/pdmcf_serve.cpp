// pdmcf_serve.cpp — asynchronous solves (mcf_submit / mcf_poll / mcf_wait / mcf_cancel).
//
// Requests wait in a FIFO until their device footprint fits the HBM budget and a resident
// slot is free; admitted requests run concurrently, each on its problem's own CUDA stream,
// so the work of requests that arrive while others are running overlaps on the device.
// A problem keeps its iterate (F, Y, omega) resident after a solve, so a later request
// with warm_start = 1 re-solves from it (Sec. 3.1, warm start).
#include <stdint.h>

#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "pdmcf_internal.h"

namespace pdmcf {

int validate_options(const mcf_options* o);

namespace {

struct Ticket {
  mcf_ticket id = 0;
  mcf_problem* p = nullptr;
  mcf_options opts{};
  int status = MCF_PENDING;
  bool started = false;
  bool cancelled = false;
  int64_t bytes = 0;
  mcf_result res{};
};

class Server {
 public:
  ~Server() {
    {
      std::lock_guard<std::mutex> g(mu_);
      stop_ = true;
    }
    cv_work_.notify_all();
    for (auto& t : workers_)
      if (t.joinable()) t.join();
  }

  int submit(mcf_problem* p, const mcf_options* o, mcf_ticket* out) {
    const int64_t bytes = device_bytes(p, o->precision);
    std::lock_guard<std::mutex> g(mu_);
    if (bytes > budget_) {
      set_error("request footprint exceeds the serving HBM budget");
      return MCF_ERR_OOM_BUDGET;
    }
    if ((int)queue_.size() >= max_queue_) {
      set_error("submission queue is full");
      return MCF_ERR_BUSY;
    }
    auto t = std::make_shared<Ticket>();
    t->id = next_id_++;
    t->p = p;
    t->opts = *o;
    t->bytes = bytes;
    p->busy.fetch_add(1);
    tickets_[t->id] = t;
    queue_.push_back(t);
    ensure_workers();
    *out = t->id;
    cv_work_.notify_one();
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
    if (res) {
      double *T = res->T, *F = res->F, *Y = res->Y;
      *res = t->res;
      res->T = T;
      res->F = F;
      res->Y = Y;
      res->status = t->status;
      if ((T || F || Y) && (t->status == MCF_OK || t->status == MCF_ERR_NOT_CONVERGED)) {
        std::lock_guard<std::mutex> pg(t->p->lock);
        int rc = device_copy_outputs(t->p, res);
        if (rc != MCF_OK) return rc;
      }
    }
    return MCF_OK;
  }

  int cancel(mcf_ticket id) {
    std::lock_guard<std::mutex> g(mu_);
    auto it = tickets_.find(id);
    if (it == tickets_.end()) {
      set_error("unknown ticket");
      return MCF_ERR_INVALID;
    }
    std::shared_ptr<Ticket> t = it->second;
    if (t->status != MCF_PENDING) return MCF_OK;
    t->cancelled = true;
    if (!t->started) {
      for (auto q = queue_.begin(); q != queue_.end(); ++q)
        if ((*q)->id == id) { queue_.erase(q); break; }
      t->status = MCF_ERR_CANCELLED;
      t->p->busy.fetch_sub(1);
      cv_done_.notify_all();
    }
    return MCF_OK;
  }

  int config(int64_t budget, int max_resident) {
    if (budget <= 0 || max_resident <= 0) {
      set_error("budget and max_resident must be > 0");
      return MCF_ERR_INVALID;
    }
    std::lock_guard<std::mutex> g(mu_);
    budget_ = budget;
    max_resident_ = max_resident;
    cv_work_.notify_all();
    return MCF_OK;
  }

 private:
  void ensure_workers() {
    const int want = kWorkers;
    while ((int)workers_.size() < want) workers_.emplace_back([this] { work(); });
  }

  bool admissible() const {
    if (queue_.empty()) return false;
    const auto& t = queue_.front();
    return resident_ < max_resident_ && in_use_ + t->bytes <= budget_;
  }

  void work() {
    for (;;) {
      std::shared_ptr<Ticket> t;
      {
        std::unique_lock<std::mutex> g(mu_);
        cv_work_.wait(g, [&] { return stop_ || admissible(); });
        if (stop_) return;
        t = queue_.front();
        queue_.pop_front();
        t->started = true;
        in_use_ += t->bytes;
        ++resident_;
      }
      mcf_result r{};
      int rc;
      {
        std::lock_guard<std::mutex> pg(t->p->lock);
        const auto t0 = std::chrono::steady_clock::now();
        rc = device_solve(t->p, &t->opts, &r);
        r.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      }
      {
        std::lock_guard<std::mutex> g(mu_);
        in_use_ -= t->bytes;
        --resident_;
        t->res = r;
        t->status = t->cancelled ? MCF_ERR_CANCELLED : rc;
        t->p->busy.fetch_sub(1);
      }
      cv_done_.notify_all();
      cv_work_.notify_all();
    }
  }

  static constexpr int kWorkers = 16;
  std::mutex mu_;
  std::condition_variable cv_work_, cv_done_;
  std::deque<std::shared_ptr<Ticket>> queue_;
  std::unordered_map<mcf_ticket, std::shared_ptr<Ticket>> tickets_;
  std::vector<std::thread> workers_;
  mcf_ticket next_id_ = 1;
  int64_t budget_ = (int64_t)120 * 1000 * 1000 * 1000;
  int64_t in_use_ = 0;
  int max_resident_ = 256;
  int resident_ = 0;
  int max_queue_ = 1 << 16;
  bool stop_ = false;
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

}  // extern "C"
