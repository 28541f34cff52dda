// Serving loop: replays a trace of timed requests for several functions on one
// GPU with continuous batching.
//
// Requests arrive at their trace times.  A function is prepared (its read-only
// data staged, Sec. 5.1) when its first request arrives; while it stages, its
// requests queue.  Admission is by device memory: a prepare that does not fit the
// pool budget evicts idle resident functions (least recently used first) and
// otherwise waits.  Each function owns `lanes` streams, each with its own
// workspace slot; whenever lanes are idle and requests are queued, the queue is
// split evenly over the idle lanes and each lane's share (up to the batch limits)
// is fused into one launch chain -- so requests that arrive while others run are
// batched as soon as a lane frees up, and the lanes of one function and of
// different functions overlap on the device.  A resident
// function with nothing queued or in flight keeps its data for `linger_s`
// (the first stage of the paper's multi-stage exit, Sec. 6.3) and is then
// released.  With sm_partition each function's lanes are streams of its own SM
// partition (a green context holding SMs / n_fns SMs), so that one function's
// batches never occupy another's SMs.
#include <stdio.h>

#include <algorithm>
#include <chrono>
#include <deque>
#include <memory>
#include <thread>
#include <vector>

#include "../../include/sage.h"
#include "kernels.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Lane {
  cudaStream_t s = nullptr;
  cudaEvent_t ev = nullptr;
  bool busy = false;
  std::vector<int> reqs;
};

struct FnState {
  sage_fn_desc desc{};
  sage_fn h = nullptr;
  bool ready = false;
  bool failed = false;
  double ready_at = -1;
  double last_active = 0;
  std::deque<int> queue;
  std::vector<Lane> lanes;
  int inflight = 0;
};

double pct(std::vector<double> v, double q) {
  if (v.empty()) return 0;
  std::sort(v.begin(), v.end());
  const size_t i = std::min(v.size() - 1, static_cast<size_t>(q * (v.size() - 1) + 0.5));
  return v[i];
}

}  // namespace

extern "C" sage_status sage_serve(sage_pool pool, const sage_fn_desc* fns, int n_fns, const sage_request* reqs,
                                  int n, const sage_serve_config* cfg_in, sage_request_result* results,
                                  sage_serve_stats* stats) {
  if (!pool || !fns || n_fns < 1 || n < 0 || (n > 0 && (!reqs || !results)))
    return sage::set_last_error("bad serve arguments"), SAGE_ERR_INVALID;
  sage_serve_config cfg{};
  if (cfg_in) cfg = *cfg_in;
  const int max_inv = cfg.max_batch_invocations > 0 ? std::min(cfg.max_batch_invocations, 256) : 256;
  const int64_t max_rows = cfg.max_batch_rows > 0 ? cfg.max_batch_rows : 65536;
  const int lanes = cfg.lanes_per_fn > 0 ? cfg.lanes_per_fn : 2;
  const double timeout_s = cfg.timeout_s > 0 ? cfg.timeout_s : 600.0;
  for (int i = 0; i < n; ++i) {
    if (reqs[i].fn < 0 || reqs[i].fn >= n_fns || reqs[i].inv.batch < 0)
      return sage::set_last_error("request with a bad function index or batch"), SAGE_ERR_INVALID;
    if (!sage::host_csr_valid(reqs[i].inv, fns[reqs[i].fn].num_tables))
      return sage::set_last_error("request whose offsets do not start at 0, decrease or do not end at num_indices"),
             SAGE_ERR_INVALID;
    results[i] = sage_request_result{-1.0, -1.0, -1.0, 0, 0, SAGE_PENDING};
  }
  std::unique_ptr<sage::Partition> part;
  if (cfg.sm_partition) {
    int dev = 0;
    cudaGetDevice(&dev);
    sage::Partition* p = nullptr;
    const sage_status ps = sage::Partition::create(dev, n_fns, 0, &p);
    if (ps != SAGE_OK) return ps;
    part.reset(p);
  }
  std::vector<FnState> F(n_fns);
  // every exit destroys the lanes' events and streams (partition streams belong to the partition)
  struct LaneGuard {
    std::vector<FnState>& F;
    bool own_streams;
    ~LaneGuard() {
      for (auto& S : F)
        for (auto& L : S.lanes) {
          if (L.ev) cudaEventDestroy(L.ev);
          if (L.s && own_streams) cudaStreamDestroy(L.s);
          L.ev = nullptr;
          L.s = nullptr;
        }
    }
  } guard{F, !cfg.sm_partition};
  for (int f = 0; f < n_fns; ++f) {
    F[f].desc = fns[f];
    F[f].desc.workspace_slots = std::max(lanes, fns[f].workspace_slots);
    F[f].lanes.resize(lanes);
    for (auto& L : F[f].lanes) {
      if (part) {
        const sage_status ps = part->stream(f, &L.s);  // owned (and destroyed) by the partition
        if (ps != SAGE_OK) return ps;
      } else if (cudaStreamCreateWithFlags(&L.s, cudaStreamNonBlocking) != cudaSuccess) {
        return sage::set_last_error("stream creation failed"), SAGE_ERR_CUDA;
      }
      if (cudaEventCreateWithFlags(&L.ev, cudaEventDisableTiming) != cudaSuccess)
        return sage::set_last_error("event creation failed"), SAGE_ERR_CUDA;
    }
  }
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return reqs[a].arrival_s < reqs[b].arrival_s; });

  sage_serve_stats st{};
  const auto t0 = Clock::now();
  auto now_s = [&] { return std::chrono::duration<double>(Clock::now() - t0).count(); };
  size_t next = 0;
  int done = 0, inflight_total = 0;
  sage_status result = SAGE_OK;
  std::vector<sage_host_invocation> hb;
  hb.reserve(256);

  while (done < n) {
    double t = now_s();
    if (t > timeout_s) {
      result = SAGE_ERR_TIMEOUT;
      sage::set_last_error("serving did not finish within its timeout");
      break;
    }
    bool progressed = false;
    // 1. arrivals
    while (next < order.size() && reqs[order[next]].arrival_s <= t) {
      const int id = order[next++];
      F[reqs[id].fn].queue.push_back(id);
      results[id].cold = F[reqs[id].fn].ready ? 0 : 1;
      progressed = true;
    }
    // 2. admission: prepare functions with demand
    for (int f = 0; f < n_fns; ++f) {
      FnState& S = F[f];
      if (S.h || S.failed || S.queue.empty()) continue;
      sage_fn h = nullptr;
      sage_status ps = sage_prepare(pool, &S.desc, &h);
      while (ps == SAGE_ERR_NOMEM) {
        // evict the least recently used idle resident function, then retry
        int victim = -1;
        for (int g = 0; g < n_fns; ++g) {
          if (g == f || !F[g].h || !F[g].ready || F[g].inflight || !F[g].queue.empty()) continue;
          if (victim < 0 || F[g].last_active < F[victim].last_active) victim = g;
        }
        if (victim < 0) break;
        if (sage_release(F[victim].h) != SAGE_OK) result = SAGE_ERR_CUDA;
        F[victim].h = nullptr;
        F[victim].ready = false;
        st.evictions++;
        ps = sage_prepare(pool, &S.desc, &h);
      }
      if (ps == SAGE_OK) {
        S.h = h;
        S.ready = false;
        S.last_active = t;
        st.prepares++;
        progressed = true;
      } else if (ps != SAGE_ERR_NOMEM) {
        S.failed = true;
        for (int id : S.queue) {
          results[id].status = ps;
          ++done;
        }
        S.queue.clear();
        result = ps;
      }
    }
    // 3. launches on idle lanes of ready functions
    for (int f = 0; f < n_fns; ++f) {
      FnState& S = F[f];
      if (!S.h || S.queue.empty()) continue;
      if (!S.ready) {
        sage_status q = sage_fn_query(S.h);
        if (q == SAGE_PENDING) continue;
        if (q != SAGE_OK) {
          S.failed = true;
          for (int id : S.queue) {
            results[id].status = q;
            ++done;
          }
          S.queue.clear();
          result = q;
          continue;
        }
        S.ready = true;
        S.ready_at = now_s();
      }
      // the queue is split evenly over the idle lanes (each then runs its share as one
      // fused batch), so that queued requests run side by side instead of all in one
      // lane's batch while the other lanes idle
      int idle = 0;
      for (const Lane& L : S.lanes) idle += L.busy ? 0 : 1;
      for (int li = 0; li < lanes && !S.queue.empty(); ++li) {
        Lane& L = S.lanes[li];
        if (L.busy) continue;
        const int share = static_cast<int>((S.queue.size() + idle - 1) / idle);
        --idle;
        hb.clear();
        L.reqs.clear();
        int64_t rows = 0;
        while (!S.queue.empty() && static_cast<int>(hb.size()) < std::min(max_inv, share)) {
          const int id = S.queue.front();
          if (!hb.empty() && rows + reqs[id].inv.batch > max_rows) break;
          S.queue.pop_front();
          hb.push_back(reqs[id].inv);
          L.reqs.push_back(id);
          rows += reqs[id].inv.batch;
        }
        const double tl = now_s();
        sage_status ls = sage::host_batch_async(S.h, hb.data(), static_cast<int>(hb.size()), L.s, li);
        if (ls == SAGE_OK && cudaEventRecord(L.ev, L.s) != cudaSuccess) ls = SAGE_ERR_CUDA;
        if (ls != SAGE_OK) {
          for (int id : L.reqs) {
            results[id].status = ls;
            ++done;
          }
          L.reqs.clear();
          result = ls;
          continue;
        }
        for (int id : L.reqs) {
          results[id].queue_ms = (tl - reqs[id].arrival_s) * 1e3;
          results[id].batch_invocations = static_cast<int>(L.reqs.size());
        }
        L.busy = true;
        S.inflight++;
        inflight_total++;
        st.batches++;
        st.max_inflight_batches = std::max<int64_t>(st.max_inflight_batches, inflight_total);
        progressed = true;
      }
    }
    // 4. completions
    for (int f = 0; f < n_fns; ++f) {
      for (auto& L : F[f].lanes) {
        if (!L.busy) continue;
        cudaError_t q = cudaEventQuery(L.ev);
        if (q == cudaErrorNotReady) continue;
        const double tc = now_s();
        for (int id : L.reqs) {
          results[id].latency_ms = (tc - reqs[id].arrival_s) * 1e3;
          results[id].service_ms = (tc - reqs[id].arrival_s) * 1e3 - results[id].queue_ms;
          results[id].status = q == cudaSuccess ? SAGE_OK : SAGE_ERR_CUDA;
          ++done;
        }
        if (q != cudaSuccess) result = SAGE_ERR_CUDA;
        L.reqs.clear();
        L.busy = false;
        F[f].inflight--;
        inflight_total--;
        F[f].last_active = tc;
        progressed = true;
      }
    }
    // 5. linger: release idle functions whose linger time ran out
    if (cfg.linger_s >= 0) {
      for (auto& S : F) {
        if (S.h && S.ready && !S.inflight && S.queue.empty() && t - S.last_active > cfg.linger_s) {
          if (sage_release(S.h) != SAGE_OK) result = SAGE_ERR_CUDA;
          S.h = nullptr;
          S.ready = false;
          st.evictions++;
        }
      }
    }
    if (!progressed) {
      // nothing to do now.  With batches in flight, poll: a serving thread that sleeps
      // between requests comes back slower on hosts whose idle cores clock down.  With
      // requests queued only behind a function's staging, yield the core to the staging
      // producers (short sleeps).  Idle: sleep until 1 ms before the next arrival, then poll.
      bool queued = false;
      for (const FnState& S : F) queued = queued || !S.queue.empty();
      const double gap = next < order.size() ? reqs[order[next]].arrival_s - now_s() : 1e9;
      if (inflight_total == 0 && queued)
        std::this_thread::sleep_for(std::chrono::microseconds(20));
      else if (inflight_total == 0 && gap > 2e-3)
        std::this_thread::sleep_for(std::chrono::duration<double>(gap - 1e-3));
    }
  }
  // drain and release
  for (auto& S : F) {
    for (auto& L : S.lanes) {
      if (L.busy) cudaEventSynchronize(L.ev);
    }
    if (S.h && sage_release(S.h) != SAGE_OK && result == SAGE_OK) result = SAGE_ERR_CUDA;
  }
  st.wall_s = now_s();
  std::vector<double> all, cold, warm;
  for (int i = 0; i < n; ++i) {
    if (results[i].status != SAGE_OK) continue;
    st.completed++;
    all.push_back(results[i].latency_ms);
    (results[i].cold ? cold : warm).push_back(results[i].latency_ms);
  }
  st.cold_requests = static_cast<int64_t>(cold.size());
  st.p50_ms = pct(all, 0.50);
  st.p99_ms = pct(all, 0.99);
  st.warm_p50_ms = pct(warm, 0.50);
  st.warm_p99_ms = pct(warm, 0.99);
  st.cold_p50_ms = pct(cold, 0.50);
  st.cold_p99_ms = pct(cold, 0.99);
  double sum = 0;
  for (double v : all) sum += v;
  st.mean_ms = all.empty() ? 0 : sum / all.size();
  st.invocations_per_s = st.wall_s > 0 ? st.completed / st.wall_s : 0;
  if (stats) *stats = st;
  return result;
}
