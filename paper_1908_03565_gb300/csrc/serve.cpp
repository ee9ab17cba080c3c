// Native request loop: replays an arrival schedule through submit/poll.
//
// Requests are admitted in arrival order as soon as the context accepts
// them (a free slot and room under the HBM cap); a refused request waits at
// the head of the queue until a running one completes.  Admitted requests
// run on their slots' streams and overlap on the device with the ones in
// flight (continuous batching); with one slot the loop is the plain
// one-request-at-a-time path.  Latency = completion - arrival, so it
// includes the time a request waited for admission.
#include <chrono>
#include <thread>
#include <vector>

#include "../../include/jxl_recon.h"
#include "internal.h"

extern "C" jxlr_status jxl_recon_serve(jxl_recon_ctx* ctx, const jxl_recon_request* reqs,
                                       size_t n, const double* arrival_s, double* latency_ms,
                                       jxl_recon_serve_stats* stats) {
  using Clock = std::chrono::steady_clock;
  if (!ctx || (!reqs && n) || (!arrival_s && n) || (!latency_ms && n)) {
    jxlr::set_last_error("serve: null argument");
    return JXLR_EINVAL;
  }
  for (size_t i = 1; i < n; ++i)
    if (arrival_s[i] < arrival_s[i - 1]) {
      jxlr::set_last_error("serve: arrival times must be non-decreasing");
      return JXLR_EINVAL;
    }
  struct Flight {
    uint64_t ticket;
    size_t index;
  };
  std::vector<Flight> flight;
  const auto t0 = Clock::now();
  auto now_s = [&] { return std::chrono::duration<double>(Clock::now() - t0).count(); };
  size_t next = 0, done = 0;
  uint64_t busy = 0;
  double max_in_flight = 0;
  jxlr_status failure = JXLR_OK;
  while (done < n) {
    bool progressed = false;
    // admit every arrived request the context accepts, in order
    while (failure == JXLR_OK && next < n && arrival_s[next] <= now_s()) {
      const jxl_recon_request& r = reqs[next];
      uint64_t t = 0;
      jxlr_status st = jxl_recon_submit(ctx, r.coeffs, r.varblock_map, r.quant_field, r.cfl_map,
                                        r.filter_params, r.out, &t);
      if (st == JXLR_EBUSY) {
        ++busy;
        break;
      }
      if (st != JXLR_OK) {
        failure = st;
        break;
      }
      flight.push_back({t, next});
      if (flight.size() > max_in_flight) max_in_flight = static_cast<double>(flight.size());
      ++next;
      progressed = true;
    }
    // retire finished requests
    for (size_t k = 0; k < flight.size();) {
      double lat = 0;
      jxlr_status st = jxl_recon_poll(ctx, flight[k].ticket, 0, &lat);
      if (st == JXLR_EAGAIN) {
        ++k;
        continue;
      }
      const size_t i = flight[k].index;
      latency_ms[i] = (now_s() - arrival_s[i]) * 1e3;
      if (st != JXLR_OK && failure == JXLR_OK) failure = st;
      flight[k] = flight.back();
      flight.pop_back();
      ++done;
      progressed = true;
    }
    if (failure != JXLR_OK && flight.empty()) break;
    if (!progressed) {
      // nothing to do: wait for the next arrival or completion
      const double wait = next < n && flight.empty() ? arrival_s[next] - now_s() : 0.0;
      if (wait > 200e-6)
        std::this_thread::sleep_for(std::chrono::duration<double>(wait - 100e-6));
      else
        std::this_thread::yield();
    }
  }
  if (stats) {
    stats->makespan_s = now_s() - (n ? arrival_s[0] : 0.0);
    stats->busy_refusals = busy;
    stats->completed = done;
    stats->max_in_flight = static_cast<uint32_t>(max_in_flight);
  }
  return failure;
}
