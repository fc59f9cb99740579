// fp_replay.cpp -- trace replay for measurements (include/fpparse_bench.h):
// requests submitted at their arrival times from a native thread, so that
// the client keeps to the schedule, through the request server or through
// the plain per-request entry point.
#include <atomic>
#include <chrono>
#include <thread>
#include <vector>

#include "../../include/fpparse.h"
#include "../../include/fpparse_bench.h"

namespace {

int64_t steady_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

// Spin until the steady clock reaches t (a sleep would wake too late).
void wait_until(int64_t t) {
  while (steady_ns() < t) {
  }
}

bool valid_trace(const fp_replay_body_t* bodies, uint32_t n_bodies, const uint32_t* order,
                 const int64_t* arrival_ns, size_t n, const int64_t* out_ns) {
  if (!bodies || !order || !arrival_ns || !out_ns || n_bodies == 0) return false;
  for (size_t i = 0; i < n; i++) {
    if (order[i] >= n_bodies) return false;
    if (i && arrival_ns[i] < arrival_ns[i - 1]) return false;
  }
  return true;
}

}  // namespace

extern "C" fp_err_t fp_replay_server(fp_server* server, const fp_replay_body_t* bodies,
                                     uint32_t n_bodies, const uint32_t* order,
                                     const int64_t* arrival_ns, size_t n, int64_t lead_ns,
                                     int64_t* out_ns) {
  if (!server || !valid_trace(bodies, n_bodies, order, arrival_ns, n, out_ns) || lead_ns < 0)
    return FP_ERR_ARG;
  std::vector<uint64_t> ids(n, 0);
  std::atomic<size_t> submitted{0};
  std::atomic<bool> ended{false};  // the submitter will submit no more
  std::atomic<int> first_err{FP_OK};
  const int64_t t0 = steady_ns() + lead_ns;
  // the waiter: requests in submission order, each as soon as it is submitted
  std::thread waiter([&]() {
    for (size_t i = 0; i < n; i++) {
      while (submitted.load(std::memory_order_acquire) <= i) {
        if (ended.load(std::memory_order_acquire) &&
            submitted.load(std::memory_order_acquire) <= i)
          return;
        std::this_thread::yield();
      }
      fp_request_info_t info;
      const fp_err_t e = fp_server_wait(server, ids[i], -1, &info);
      out_ns[4 * i + 2] = info.launch_ns;
      out_ns[4 * i + 3] = info.done_ns;
      int expect = FP_OK;
      if (e != FP_OK) first_err.compare_exchange_strong(expect, (int)e);
    }
  });
  for (size_t i = 0; i < n; i++) {
    const fp_replay_body_t& b = bodies[order[i]];
    const int64_t ta = t0 + arrival_ns[i];
    wait_until(ta);
    uint64_t id = 0;
    const int64_t ts = steady_ns();
    const fp_err_t e =
        fp_server_submit(server, b.host_text, b.len, b.host_f64, b.host_status, b.out_cap, &id);
    out_ns[4 * i] = ta;
    out_ns[4 * i + 1] = ts;
    if (e != FP_OK) {  // stop the trace here; the waiter ends after request i - 1
      int expect = FP_OK;
      first_err.compare_exchange_strong(expect, (int)e);
      ended.store(true, std::memory_order_release);
      waiter.join();
      return (fp_err_t)first_err.load();
    }
    ids[i] = id;
    submitted.store(i + 1, std::memory_order_release);
  }
  ended.store(true, std::memory_order_release);
  waiter.join();
  return (fp_err_t)first_err.load();
}

extern "C" fp_err_t fp_replay_plain(const fp_replay_body_t* bodies, uint32_t n_bodies,
                                    const uint32_t* order, const int64_t* arrival_ns, size_t n,
                                    int64_t lead_ns, char delim, struct CUstream_st* stream,
                                    int64_t* out_ns) {
  if (!valid_trace(bodies, n_bodies, order, arrival_ns, n, out_ns) || lead_ns < 0)
    return FP_ERR_ARG;
  const int64_t t0 = steady_ns() + lead_ns;
  for (size_t i = 0; i < n; i++) {
    const fp_replay_body_t& b = bodies[order[i]];
    const int64_t ta = t0 + arrival_ns[i];
    wait_until(ta);
    uint64_t count = 0;
    const fp_err_t e =
        fp_parse_f64_host(b.host_text, b.len, delim, b.host_f64, b.host_status, &count, stream);
    out_ns[2 * i] = ta;
    out_ns[2 * i + 1] = steady_ns();
    if (e != FP_OK) return e;
  }
  return FP_OK;
}
