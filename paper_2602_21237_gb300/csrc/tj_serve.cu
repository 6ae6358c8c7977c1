// Serving loop (no counterpart in the paper, whose P99 framing of Sec. 5.2 /
// Sec. 6 it measures): continuous batching of join and sort requests under a
// device-memory budget.
//
// Requests wait in one queue in arrival order.  A request is admitted as soon
// as a worker is free and its footprint (the library scratch its call may
// hold plus its output buffer) fits in what the budget has left; it then runs
// on its worker's own CUDA stream, so admitted requests overlap on the
// device.  When the oldest request does not fit yet, a later one that does
// may go first, but no request is passed more than kMaxBypass times (then the
// queue waits for it), so none starves.  When a request completes, its
// reservation is released and the next one is admitted immediately --
// requests that arrive while others run join the mix as slots and memory
// free up.  Latency = completion - arrival.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "tj_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

// times a queued request may be passed by later ones that fit the budget
constexpr int kMaxBypass = 8;
// requests of the queue's front looked at for one that fits
constexpr size_t kScan = 64;
// latencies kept for the percentiles (a uniform sample beyond this many)
constexpr size_t kLatCap = 1 << 20;

struct Pending {
  int64_t ticket;
  tj_request req;
  size_t footprint;
  Clock::time_point arrival;
  int bypassed;
};

}  // namespace

struct tj_server {
  size_t budget = 0;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv;  // queue / completion changes
  std::deque<Pending> queue;
  std::unordered_map<int64_t, tj_result> done;  // completed, not yet waited on
  std::unordered_set<int64_t> open;             // submitted, not yet waited on
  std::vector<double> lat_ms;                   // this stats window's latencies (sampled)
  int64_t lat_seen = 0;                         // latencies the window has seen
  uint64_t lat_rng = 0x9E3779B97F4A7C15ull;
  int64_t bypasses = 0;
  size_t reserved = 0;
  size_t peak_reserved = 0;
  int inflight = 0;
  int peak_inflight = 0;
  int64_t next = 0;
  int64_t tuples = 0;
  bool stop = false;
  Clock::time_point first_arrival{}, last_done{};
  bool any = false;
  std::vector<std::thread> workers;
};

namespace {

size_t rows_bytes(tj_dtype dt) { return dt == TJ_I32 ? 4 : 8; }

// What the library may hold for the call (single-pass sort buffers, look-back,
// join state) plus the output buffer the request pins.
size_t footprint_of(const tj_request& r) {
  const size_t w = rows_bytes((tj_dtype)r.dt);
  if (r.op == TJ_OP_SORT) return (size_t)r.n_r * (2 * w + 2) + (2u << 20);
  const size_t rows = (size_t)(r.n_r + r.n_s);
  return rows * (4 * w + 2) + (size_t)r.out_capacity * 2 * w + (2u << 20);
}

// The queued request to admit now (index into the queue), or -1: the first
// one of the front kScan that fits what the budget has left, unless a request
// before it has been passed kMaxBypass times already.
long pick(const tj_server* S) {
  const size_t n = std::min(S->queue.size(), kScan);
  for (size_t i = 0; i < n; ++i) {
    const Pending& q = S->queue[i];
    if (S->reserved + q.footprint <= S->budget) return (long)i;
    if (q.bypassed >= kMaxBypass) return -1;  // it goes next: wait for room
  }
  return -1;
}

void worker_main(tj_server* S) {
  cudaSetDevice(S->device);
  cudaStream_t st = nullptr;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  while (true) {
    Pending p;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv.wait(lk, [&] { return S->stop || pick(S) >= 0; });
      if (S->stop && S->queue.empty()) break;
      const long i = pick(S);
      if (i < 0) continue;
      for (long j = 0; j < i; ++j) S->queue[(size_t)j].bypassed += 1;
      S->bypasses += i;
      p = S->queue[(size_t)i];
      S->queue.erase(S->queue.begin() + i);
      S->reserved += p.footprint;
      S->peak_reserved = std::max(S->peak_reserved, S->reserved);
      S->inflight += 1;
      S->peak_inflight = std::max(S->peak_inflight, S->inflight);
    }
    tj_result res = {};
    const tj_request& r = p.req;
    const size_t w = rows_bytes((tj_dtype)r.dt);
    if (r.op == TJ_OP_SORT) {
      res.status = tj_sort((tj_dtype)r.dt, r.keys_r, r.ids_r, r.n_r, st);
    } else {
      // the call's working set stays inside the reservation minus its output
      const size_t lib = p.footprint - (size_t)r.out_capacity * 2 * w;
      void* out = r.out_pairs;
      if (!out && r.out_capacity > 0 &&
          cudaMallocAsync(&out, (size_t)r.out_capacity * 2 * w, st) != cudaSuccess) {
        out = nullptr;
        res.status = TJ_ERR_CUDA;
      }
      if (res.status == TJ_OK)
        res.status = tj_join_inner((tj_dtype)r.dt, r.keys_r, r.ids_r, r.n_r, r.keys_s, r.ids_s,
                                   r.n_s, lib, out, r.out_capacity, &res.out_count, st);
      if (!r.out_pairs && out) {  // a server-owned output is counted, then released
        cudaFreeAsync(out, st);
        cudaStreamSynchronize(st);
      }
    }
    const Clock::time_point t1 = Clock::now();
    res.latency_ms = std::chrono::duration<double, std::milli>(t1 - p.arrival).count();
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->reserved -= p.footprint;
      S->inflight -= 1;
      S->done[p.ticket] = res;
      // reservoir sample of the window's latencies (all of them up to kLatCap)
      S->lat_seen += 1;
      if (S->lat_ms.size() < kLatCap) {
        S->lat_ms.push_back(res.latency_ms);
      } else {
        S->lat_rng = S->lat_rng * 6364136223846793005ull + 1442695040888963407ull;
        const uint64_t k = (S->lat_rng >> 11) % (uint64_t)S->lat_seen;
        if (k < kLatCap) S->lat_ms[(size_t)k] = res.latency_ms;
      }
      S->tuples += r.op == TJ_OP_SORT ? r.n_r : r.n_r + r.n_s;
      if (t1 > S->last_done) S->last_done = t1;
    }
    S->cv.notify_all();
  }
  cudaStreamDestroy(st);
}

// q-quantile of sorted v (linear between neighbours)
double pct(const std::vector<double>& v, double q) {
  if (v.empty()) return 0.0;
  const double pos = q * (double)(v.size() - 1);
  const size_t i = (size_t)pos;
  const double f = pos - (double)i;
  return i + 1 < v.size() ? v[i] * (1 - f) + v[i + 1] * f : v[i];
}

}  // namespace

extern "C" {

tj_status tj_server_create(size_t mem_budget_bytes, int workers, tj_server** out) {
  if (!out || workers < 1 || workers > 64 || mem_budget_bytes == 0) return TJ_ERR_INVALID;
  tj_server* S = new tj_server();
  S->budget = mem_budget_bytes;
  if (cudaGetDevice(&S->device) != cudaSuccess) {
    delete S;
    return TJ_ERR_CUDA;
  }
  for (int i = 0; i < workers; ++i) S->workers.emplace_back(worker_main, S);
  *out = S;
  return TJ_OK;
}

tj_status tj_server_submit(tj_server* S, const tj_request* r, int64_t* ticket) {
  if (!S || !r || !ticket) return TJ_ERR_INVALID;
  if (r->op != TJ_OP_JOIN && r->op != TJ_OP_SORT) return TJ_ERR_INVALID;
  Pending p;
  p.req = *r;
  p.footprint = footprint_of(*r);
  p.arrival = Clock::now();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    p.ticket = S->next++;
    *ticket = p.ticket;
    if (!S->any) {
      S->first_arrival = p.arrival;
      S->any = true;
    }
    S->open.insert(p.ticket);
    if (p.footprint > S->budget) {  // can never be admitted
      tj_result res = {};
      res.status = TJ_ERR_BUDGET;
      S->done[p.ticket] = res;
      S->cv.notify_all();
      return TJ_OK;
    }
    p.bypassed = 0;
    S->queue.push_back(p);
  }
  S->cv.notify_all();
  return TJ_OK;
}

tj_status tj_server_wait(tj_server* S, int64_t ticket, tj_result* res) {
  if (!S || !res) return TJ_ERR_INVALID;
  std::unique_lock<std::mutex> lk(S->mu);
  if (S->open.count(ticket) == 0) return TJ_ERR_INVALID;  // unknown, or waited on already
  S->cv.wait(lk, [&] { return S->done.count(ticket) > 0; });
  auto it = S->done.find(ticket);
  *res = it->second;
  S->done.erase(it);  // each result is collected once: the server keeps no history
  S->open.erase(ticket);
  return TJ_OK;
}

tj_status tj_server_replay(tj_server* S, const tj_request* reqs, const double* arrival_s,
                           int64_t n, int64_t* tickets) {
  if (!S || (n > 0 && (!reqs || !arrival_s || !tickets))) return TJ_ERR_INVALID;
  const Clock::time_point t0 = Clock::now();
  for (int64_t i = 0; i < n; ++i) {
    const auto due = t0 + std::chrono::duration_cast<Clock::duration>(
                              std::chrono::duration<double>(arrival_s[i]));
    std::this_thread::sleep_until(due);
    tj_status st = tj_server_submit(S, &reqs[i], &tickets[i]);
    if (st != TJ_OK) return st;
  }
  return TJ_OK;
}

tj_status tj_server_drain(tj_server* S) {
  if (!S) return TJ_ERR_INVALID;
  std::unique_lock<std::mutex> lk(S->mu);
  S->cv.wait(lk, [&] { return S->queue.empty() && S->inflight == 0; });
  return TJ_OK;
}

tj_status tj_server_report(tj_server* S, tj_server_stats* out) {
  if (!S || !out) return TJ_ERR_INVALID;
  tj_server_stats r = {};
  std::vector<double> lat;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    lat = S->lat_ms;  // sorted outside the lock
    r.completed = S->lat_seen;
    r.tuples = S->tuples;
    r.makespan_s = S->any ? std::chrono::duration<double>(S->last_done - S->first_arrival).count()
                          : 0.0;
    r.peak_reserved = (int64_t)S->peak_reserved;
    r.peak_inflight = S->peak_inflight;
    r.bypasses = S->bypasses;
  }
  std::sort(lat.begin(), lat.end());
  r.p50_ms = pct(lat, 0.50);
  r.p99_ms = pct(lat, 0.99);
  r.max_ms = lat.empty() ? 0.0 : lat.back();
  double sum = 0;
  for (double x : lat) sum += x;
  r.mean_ms = lat.empty() ? 0.0 : sum / (double)lat.size();
  *out = r;
  return TJ_OK;
}

tj_status tj_server_reset_stats(tj_server* S) {
  if (!S) return TJ_ERR_INVALID;
  std::lock_guard<std::mutex> lk(S->mu);
  S->lat_ms.clear();
  S->lat_seen = 0;
  S->bypasses = 0;
  S->tuples = 0;
  S->any = false;
  S->peak_reserved = S->reserved;
  S->peak_inflight = S->inflight;
  return TJ_OK;
}

void tj_server_destroy(tj_server* S) {
  if (!S) return;
  tj_server_drain(S);
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv.notify_all();
  for (auto& t : S->workers) t.join();
  delete S;
}

}  // extern "C"
