// Request server: a long-lived thread that admits queued decode requests
// into a context as slots and HBM free up (continuous batching), and the
// replay of an arrival schedule built on it.
//
// Producers on any thread enqueue requests (jxl_recon_server_enqueue) and
// wait for them (jxl_recon_server_wait).  The server thread scans the queue
// in arrival order and submits each request the context accepts.  A request
// refused for want of HBM under the cap is passed over by smaller ones
// behind it, until it has waited longer than the age bound: from then on
// nothing behind it is admitted before it.  Admitted requests run on their
// slots' streams and overlap on the device; the context runs a request on a
// stream whose priority rises with its image size, so large requests (the
// tail of the latency) take the SMs they need and small ones fill the rest.
// Optionally the largest requests run alone: one of them is admitted only
// onto an idle device (the requests behind it wait too, so the device
// drains), and nothing is admitted beside it.
// Latency = completion - enqueue (queueing included).
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "../../include/jxl_recon.h"
#include "internal.h"

using Clock = std::chrono::steady_clock;

// Images from this size up run alone in the replay of jxl_recon_serve: they
// set the tail latency, and requests beside them slow them down at every
// kernel boundary (measured: p99 at 30-50% load 1.2-1.4x that of one image
// at a time otherwise).
constexpr double kServeExclusiveMpx = 8.0;

struct jxl_recon_server {
  jxl_recon_ctx* ctx = nullptr;
  double age_bound_s = 0.005;
  bool bypass = true;
  uint64_t exclusive_px = 0;       // requests at least this large run alone (0: none)
  std::thread th;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  struct Pending {
    jxl_recon_request r;
    uint64_t id;
    Clock::time_point arrival;
  };
  struct Flight {
    uint64_t ticket, id;
    Clock::time_point arrival;
    bool exclusive;
  };
  struct Result {
    jxlr_status st;
    double latency_ms;
  };
  std::deque<Pending> pending;                     // guarded by mu
  std::unordered_map<uint64_t, Result> results;    // guarded by mu
  std::unordered_set<uint64_t> open;               // enqueued, not yet waited for (mu)
  uint64_t next_id = 1;                            // guarded by mu
  bool stopping = false;                           // guarded by mu
  // statistics (guarded by mu)
  uint64_t busy = 0, bypassed = 0, completed = 0;
  uint32_t max_in_flight = 0;
  Clock::time_point first_arrival, last_done;
  bool any = false;

  void loop();
};

void jxl_recon_server::loop() {
  std::vector<Flight> flight;          // this thread only
  std::vector<Pending> snap;
  std::vector<uint64_t> admitted;
  for (;;) {
    bool progressed = false;
    {
      std::unique_lock<std::mutex> lock(mu);
      if (stopping && pending.empty() && flight.empty()) break;
      snap.assign(pending.begin(), pending.end());
    }
    // ---- admission, in arrival order ----
    admitted.clear();
    const auto now = Clock::now();
    bool passed = false;   // a refused request is ahead of the ones tried now
    bool alone = false;    // a request that runs alone is in flight
    for (const Flight& f : flight) alone = alone || f.exclusive;
    for (size_t i = 0; i < snap.size() && !alone; ++i) {
      if (jxlr::ctx_idle_slots(ctx) == 0) break;
      const jxl_recon_request& r = snap[i].r;
      const bool excl = exclusive_px && r.coeffs &&
                        uint64_t(r.coeffs->xsize) * r.coeffs->ysize >= exclusive_px;
      uint64_t t = 0;
      // a request that runs alone waits for the device to drain
      const jxlr_status st = excl && !flight.empty()
                                 ? JXLR_EBUSY
                                 : jxl_recon_submit(ctx, r.coeffs, r.varblock_map, r.quant_field,
                                                    r.cfl_map, r.filter_params, r.out, &t);
      if (st == JXLR_EBUSY) {
        {
          std::lock_guard<std::mutex> lock(mu);
          ++busy;
        }
        if (excl) break;   // nothing passes a request waiting to run alone
        // a refused request that has waited past the age bound is passed by none
        const double age = std::chrono::duration<double>(now - snap[i].arrival).count();
        if (!bypass || age > age_bound_s) break;
        passed = true;
        continue;
      }
      admitted.push_back(snap[i].id);
      progressed = true;
      if (st != JXLR_OK) {   // rejected outright: report it as the request's result
        std::lock_guard<std::mutex> lock(mu);
        results[snap[i].id] = {st, 0.0};
        ++completed;
        cv_done.notify_all();
        continue;
      }
      if (passed) {
        std::lock_guard<std::mutex> lock(mu);
        ++bypassed;
      }
      flight.push_back({t, snap[i].id, snap[i].arrival, excl});
      alone = excl;
    }
    if (!admitted.empty()) {
      std::lock_guard<std::mutex> lock(mu);
      for (uint64_t id : admitted)
        for (auto it = pending.begin(); it != pending.end(); ++it)
          if (it->id == id) {
            pending.erase(it);
            break;
          }
      max_in_flight = std::max<uint32_t>(max_in_flight, static_cast<uint32_t>(flight.size()));
    }
    // ---- completions ----
    for (size_t k = 0; k < flight.size();) {
      const jxlr_status st = jxl_recon_poll(ctx, flight[k].ticket, 0, nullptr);
      if (st == JXLR_EAGAIN) {
        ++k;
        continue;
      }
      const auto done = Clock::now();
      {
        std::lock_guard<std::mutex> lock(mu);
        results[flight[k].id] = {
            st, std::chrono::duration<double, std::milli>(done - flight[k].arrival).count()};
        ++completed;
        last_done = done;
      }
      cv_done.notify_all();
      flight[k] = flight.back();
      flight.pop_back();
      progressed = true;
    }
    if (!progressed) {
      if (flight.empty()) {
        // nothing on the device: sleep until a request arrives (or shortly,
        // when refused requests wait for the cap)
        std::unique_lock<std::mutex> lock(mu);
        if (!stopping)
          cv_work.wait_for(lock, std::chrono::microseconds(pending.empty() ? 500 : 20));
      } else {
        std::this_thread::yield();   // completions are polled
      }
    }
  }
}

extern "C" {

jxlr_status jxl_recon_server_start(jxl_recon_ctx* ctx, const jxl_recon_server_config* cfg,
                                   jxl_recon_server** out) {
  if (!ctx || !out) {
    jxlr::set_last_error("server_start: null argument");
    return JXLR_EINVAL;
  }
  auto* s = new jxl_recon_server();
  s->ctx = ctx;
  if (cfg) {
    s->bypass = cfg->bypass != 0;
    if (cfg->age_bound_ms >= 0) s->age_bound_s = cfg->age_bound_ms * 1e-3;
    if (cfg->exclusive_mpx > 0) s->exclusive_px = static_cast<uint64_t>(cfg->exclusive_mpx * 1e6);
  }
  s->th = std::thread([s] { s->loop(); });
  *out = s;
  return JXLR_OK;
}

jxlr_status jxl_recon_server_enqueue(jxl_recon_server* s, const jxl_recon_request* r,
                                     uint64_t* id) {
  if (!s || !r || !id) {
    jxlr::set_last_error("server_enqueue: null argument");
    return JXLR_EINVAL;
  }
  {
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->stopping) {
      jxlr::set_last_error("server_enqueue: server is stopping");
      return JXLR_EINVAL;
    }
    const auto now = Clock::now();
    if (!s->any) {
      s->first_arrival = now;
      s->any = true;
    }
    *id = s->next_id++;
    s->open.insert(*id);
    s->pending.push_back({*r, *id, now});
  }
  s->cv_work.notify_one();
  return JXLR_OK;
}

jxlr_status jxl_recon_server_wait(jxl_recon_server* s, uint64_t id, int64_t timeout_us,
                                  double* latency_ms) {
  if (!s) {
    jxlr::set_last_error("server_wait: null server");
    return JXLR_EINVAL;
  }
  std::unique_lock<std::mutex> lock(s->mu);
  if (!s->open.count(id)) {
    jxlr::set_last_error("server_wait: unknown request, or already waited for");
    return JXLR_EINVAL;
  }
  auto ready = [&] { return s->results.count(id) != 0; };
  if (timeout_us < 0) {
    s->cv_done.wait(lock, ready);
  } else if (!s->cv_done.wait_for(lock, std::chrono::microseconds(timeout_us), ready)) {
    return timeout_us == 0 ? JXLR_EAGAIN : JXLR_ETIMEDOUT;
  }
  const auto res = s->results[id];
  s->results.erase(id);
  s->open.erase(id);
  if (latency_ms) *latency_ms = res.latency_ms;
  if (res.st != JXLR_OK) jxlr::set_last_error("server: request failed");
  return res.st;
}

jxlr_status jxl_recon_server_stop(jxl_recon_server* s, jxl_recon_serve_stats* stats) {
  if (!s) return JXLR_OK;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stopping = true;
  }
  s->cv_work.notify_all();
  s->th.join();
  if (stats) {
    stats->makespan_s =
        s->any ? std::chrono::duration<double>(s->last_done - s->first_arrival).count() : 0.0;
    stats->busy_refusals = s->busy;
    stats->completed = s->completed;
    stats->max_in_flight = s->max_in_flight;
    stats->bypassed = s->bypassed;
  }
  delete s;
  return JXLR_OK;
}

jxlr_status jxl_recon_serve(jxl_recon_ctx* ctx, const jxl_recon_request* reqs, size_t n,
                            const double* arrival_s, double* latency_ms,
                            jxl_recon_serve_stats* stats) {
  if (!ctx || (!reqs && n) || (!arrival_s && n) || (!latency_ms && n)) {
    jxlr::set_last_error("serve: null argument");
    return JXLR_EINVAL;
  }
  for (size_t i = 1; i < n; ++i)
    if (arrival_s[i] < arrival_s[i - 1]) {
      jxlr::set_last_error("serve: arrival times must be non-decreasing");
      return JXLR_EINVAL;
    }
  jxl_recon_server* s = nullptr;
  jxl_recon_server_config cfg = {5.0, 1, kServeExclusiveMpx};
  jxlr_status st = jxl_recon_server_start(ctx, &cfg, &s);
  if (st != JXLR_OK) return st;
  // this thread feeds the arrivals on schedule
  std::vector<uint64_t> ids(n);
  const auto t0 = Clock::now();
  for (size_t i = 0; i < n; ++i) {
    for (;;) {
      const double wait =
          arrival_s[i] - std::chrono::duration<double>(Clock::now() - t0).count();
      if (wait <= 0) break;
      if (wait > 200e-6)
        std::this_thread::sleep_for(std::chrono::duration<double>(wait - 100e-6));
      else
        std::this_thread::yield();
    }
    jxl_recon_server_enqueue(s, &reqs[i], &ids[i]);
  }
  jxlr_status failure = JXLR_OK;
  for (size_t i = 0; i < n; ++i) {
    const jxlr_status r = jxl_recon_server_wait(s, ids[i], -1, &latency_ms[i]);
    if (r != JXLR_OK && failure == JXLR_OK) failure = r;
  }
  jxl_recon_serve_stats ss;
  jxl_recon_server_stop(s, &ss);
  if (stats) *stats = ss;
  return failure;
}

}  // extern "C"
