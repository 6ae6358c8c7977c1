// C ABI of libtj (include/tj.h): argument checks, the digit plan, scratch
// management and the launch sequence of each operation.
//
// Join (paper Sec. 4.1) = sort both relations along the key axis (LSD onesweep
// passes over the significant bits of key - min, Sec. 4.2), then align the two
// sorted axes tile by tile and materialise the pairs once (Sec. 3.1).  Every
// step runs in the kernels of tj_radix.cu and tj_join.cu; this file only plans
// and launches.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <string>
#include <limits>
#include <mutex>
#include <vector>

#include "tj_internal.cuh"

namespace tj {
namespace {

thread_local char g_err[512] = {0};
thread_local tj_stats g_stats = {};

// device -> host reads waiting for the next sync_stream() (see put_small)
struct PendingRead {
  void* dst;
  const unsigned char* src;
  size_t n;
};
thread_local std::vector<PendingRead> g_reads;

tj_status set_err(tj_status s, const char* fmt, ...) {
  g_reads.clear();  // an error return leaves no read behind for a later sync
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return s;
}

#define TJ_CUDA(call)                                                                       \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess)                                                                  \
      return set_err(TJ_ERR_CUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                     __LINE__);                                                             \
  } while (0)

constexpr int64_t kMaxRows = (int64_t)1 << 30;
constexpr int kMlpTable = 4096;  // grid of the MLP's monotone tabulation

// ---- kernel trace ------------------------------------------------------------------
struct TraceRow {
  char name[48];
  int64_t launches;
  double ms;
  double bytes;
};
std::mutex g_trace_mu;
bool g_trace_on = false;
std::vector<TraceRow> g_trace;

// Events are taken from a per-thread pool and returned after use, so tracing
// costs two cudaEventRecord calls per launch.
thread_local std::vector<cudaEvent_t> g_event_pool;

cudaEvent_t pool_get() {
  if (!g_event_pool.empty()) {
    cudaEvent_t e = g_event_pool.back();
    g_event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

void pool_put(cudaEvent_t e) {
  if (e) g_event_pool.push_back(e);
}

// Per call: event pairs around each launch, resolved after the call's final sync.
class Tracer {
 public:
  explicit Tracer(cudaStream_t st) : st_(st) {
    std::lock_guard<std::mutex> lk(g_trace_mu);
    on_ = g_trace_on;
    if (on_) {
      cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
      if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
        on_ = false;
    }
  }
  ~Tracer() {
    for (auto& p : pend_) {
      pool_put(p.e0);
      pool_put(p.e1);
    }
  }
  // `s`: the launch's stream when it is not the call's own; `launches`: the
  // kernels between begin and end (one unless a phase is traced as a whole)
  void begin(const char* name, double bytes, cudaStream_t s = nullptr, int launches = 1) {
    if (!on_) return;
    Pending p;
    p.name = name;
    p.bytes = bytes;
    p.launches = launches;
    p.st = s ? s : st_;
    p.e0 = pool_get();
    p.e1 = pool_get();
    if (!p.e0 || !p.e1) {
      pool_put(p.e0);
      pool_put(p.e1);
      return;
    }
    cudaEventRecord(p.e0, p.st);
    pend_.push_back(p);
    open_ = true;
  }
  void end() {
    if (!on_ || !open_) return;
    cudaEventRecord(pend_.back().e1, pend_.back().st);
    open_ = false;
  }
  // the bytes of the last traced launch named `name` (known only afterwards)
  void add_bytes(const char* name, double bytes) {
    for (auto it = pend_.rbegin(); it != pend_.rend(); ++it)
      if (strcmp(it->name, name) == 0) {
        it->bytes += bytes;
        return;
      }
  }
  // call after the stream has been synchronised
  void flush() {
    if (!on_) return;
    std::lock_guard<std::mutex> lk(g_trace_mu);
    for (auto& p : pend_) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, p.e0, p.e1) != cudaSuccess) continue;
      TraceRow* row = nullptr;
      for (auto& r : g_trace)
        if (strcmp(r.name, p.name) == 0) row = &r;
      if (!row) {
        TraceRow r = {};
        snprintf(r.name, sizeof(r.name), "%s", p.name);
        g_trace.push_back(r);
        row = &g_trace.back();
      }
      row->launches += p.launches;
      row->ms += ms;
      row->bytes += p.bytes;
    }
    cudaGetLastError();
  }

 private:
  struct Pending {
    const char* name;
    double bytes;
    int launches;
    cudaStream_t st;
    cudaEvent_t e0, e1;
  };
  cudaStream_t st_;
  bool on_ = false;
  bool open_ = false;
  std::vector<Pending> pend_;
};

// ---- per-device one-time setup -----------------------------------------------
std::mutex g_init_mu;
bool g_inited[256] = {false};

tj_status ensure_device() {
  int dev = 0;
  TJ_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 256) return set_err(TJ_ERR_INTERNAL, "device index %d", dev);
  std::lock_guard<std::mutex> lk(g_init_mu);
  if (g_inited[dev]) return TJ_OK;
  cudaMemPool_t pool;
  TJ_CUDA(cudaDeviceGetDefaultMemPool(&pool, dev));
  uint64_t thr = ~0ull;  // keep freed scratch in the pool between calls
  TJ_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));
  TJ_CUDA(radix_init_attributes());
  TJ_CUDA(join_init_attributes());
  TJ_CUDA(mlp_init_attributes());
  TJ_CUDA(fused_init_attributes());
  g_inited[dev] = true;
  return TJ_OK;
}

// ---- scratch: one stream-ordered block per phase, carved in 256 B pieces ------
struct Carve {
  size_t off = 0;
  template <typename T>
  size_t add(size_t count) {
    off = (off + 255) & ~(size_t)255;
    const size_t at = off;
    off += count * sizeof(T);
    return at;
  }
};

struct Block {
  char* p = nullptr;
  cudaStream_t st = nullptr;
  ~Block() {
    if (p) cudaFreeAsync(p, st);
  }
  cudaError_t alloc(size_t n, cudaStream_t s) {
    st = s;
    return cudaMallocAsync((void**)&p, n ? n : 256, s);
  }
  void release() {  // stream-ordered: later allocations may reuse the memory
    if (p) cudaFreeAsync(p, st);
    p = nullptr;
  }
  template <typename T>
  T* at(size_t off) const {
    return reinterpret_cast<T*>(p + off);
  }
};

// A part of a block (not owned).
struct View {
  char* p;
  template <typename T>
  T* at(size_t off) const {
    return reinterpret_cast<T*>(p + off);
  }
};

// ---- pinned host staging for job-table uploads (one per thread, grows) ------
struct Pinned {
  unsigned char* p = nullptr;
  size_t cap = 0;
  cudaEvent_t ev = nullptr;  // last upload from this buffer
  ~Pinned() {
    if (ev) cudaEventDestroy(ev);
    if (p) cudaFreeHost(p);
  }
};
thread_local Pinned g_pinned;

cudaEvent_t pinned_event() { return g_pinned.ev; }

// A pinned buffer of at least n bytes whose previous upload has completed.
cudaError_t pinned_staging(size_t n, unsigned char** out) {
  cudaError_t e;
  if (!g_pinned.ev) {
    e = cudaEventCreateWithFlags(&g_pinned.ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
  }
  e = cudaEventSynchronize(g_pinned.ev);
  if (e != cudaSuccess) return e;
  if (n > g_pinned.cap) {
    if (g_pinned.p) cudaFreeHost(g_pinned.p);
    g_pinned.p = nullptr;
    g_pinned.cap = 0;
    const size_t c = std::max(n, (size_t)1 << 20);
    e = cudaMallocHost((void**)&g_pinned.p, c);
    if (e != cudaSuccess) return e;
    g_pinned.cap = c;
  }
  *out = g_pinned.p;
  return cudaSuccess;
}

// ---- small host <-> device transfers without the copy engines --------------------
// Tables going to the device and counts or statistics coming back move
// through a per-thread arena of pinned host memory that the device maps, by a
// copy kernel on the call's stream (launch_copy_bytes): a copy engine runs
// copies of one direction in order, so a small read queued behind a caller's
// multi-gigabyte transfer would stall the call for all of it.  A read lands
// in the arena and reaches its destination at the next sync_stream().  The
// arena is reused from the start by every API call (the previous call on the
// thread has synchronised its stream); a buffer outgrown within a call is
// kept until then.
struct Arena {
  unsigned char* p = nullptr;
  size_t cap = 0, off = 0;
  std::vector<unsigned char*> old;
  ~Arena() {
    for (auto* q : old) cudaFreeHost(q);
    if (p) cudaFreeHost(p);
  }
};
thread_local Arena g_arena;

void arena_reset() {
  for (auto* q : g_arena.old) cudaFreeHost(q);
  g_arena.old.clear();
  g_arena.off = 0;
  g_reads.clear();
}

cudaError_t arena_take(size_t n, unsigned char** out) {
  const size_t need = (n + 255) & ~(size_t)255;
  if (g_arena.off + need > g_arena.cap) {
    const size_t cap = std::max<size_t>({need, 2 * g_arena.cap, (size_t)4 << 20});
    unsigned char* q = nullptr;
    cudaError_t e = cudaMallocHost((void**)&q, cap);
    if (e != cudaSuccess) return e;
    if (g_arena.p) g_arena.old.push_back(g_arena.p);  // still read by queued kernels
    g_arena.p = q;
    g_arena.cap = cap;
    g_arena.off = 0;
  }
  *out = g_arena.p + g_arena.off;
  g_arena.off += need;
  return cudaSuccess;
}

// host -> device: the bytes are taken now (the caller may reuse `src`)
cudaError_t put_small(void* dst, const void* src, size_t n, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  unsigned char* a = nullptr;
  cudaError_t e = arena_take(n, &a);
  if (e != cudaSuccess) return e;
  memcpy(a, src, n);
  return launch_copy_bytes(dst, a, n, st);
}

// device -> host: `dst` holds the bytes after the next sync_stream()
cudaError_t get_small(void* dst, const void* src, size_t n, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  unsigned char* a = nullptr;
  cudaError_t e = arena_take(n, &a);
  if (e != cudaSuccess) return e;
  e = launch_copy_bytes(a, src, n, st);
  if (e != cudaSuccess) return e;
  g_reads.push_back({dst, a, n});
  return cudaSuccess;
}

cudaError_t sync_stream(cudaStream_t st) {
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e;
  for (auto& r : g_reads) memcpy(r.dst, r.src, r.n);
  g_reads.clear();
  return cudaSuccess;
}

// ---- a second stream per host thread ---------------------------------------------
// The groups of a partitioned join alternate between the caller's stream and
// this one, so one group's sort passes fill the tails of the other's launches.
struct SideStream {
  int dev = -1;
  cudaStream_t s = nullptr;
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  void reset() {
    for (auto& e : ev)
      if (e) cudaEventDestroy(e), e = nullptr;
    if (s) cudaStreamDestroy(s);
    s = nullptr;
    dev = -1;
  }
  ~SideStream() { reset(); }
};
thread_local SideStream g_side;

// The side stream of the current device and three events to order work
// between it and the caller's stream.
cudaError_t side_stream(SideStream** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (g_side.s && g_side.dev != dev) g_side.reset();
  if (!g_side.s) {
    e = cudaStreamCreateWithFlags(&g_side.s, cudaStreamNonBlocking);
    for (auto& x : g_side.ev)
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&x, cudaEventDisableTiming);
    if (e != cudaSuccess) {
      g_side.reset();
      return e;
    }
    g_side.dev = dev;
  }
  *out = &g_side;
  return cudaSuccess;
}

// Makes `st` wait for everything enqueued on `side` so far when it goes out of
// scope (declared after the blocks the side stream uses, so it runs before
// their stream-ordered frees, on every return path).
struct JoinBack {
  cudaStream_t st = nullptr, side = nullptr;
  cudaEvent_t ev = nullptr;
  void now() {
    if (!side) return;
    cudaEventRecord(ev, side);
    cudaStreamWaitEvent(st, ev, 0);
    side = nullptr;
  }
  ~JoinBack() { now(); }
};

// ---- digit plan -----------------------------------------------------------------
struct Plan {
  uint64_t lo = 0;
  int key_bits = 0;
  int passes = 0;
  int shift[kMaxPasses] = {0};
  int bits[kMaxPasses] = {0};
  int max_bits = 0;
};

int bitlen(uint64_t x) { return x ? 64 - __builtin_clzll(x) : 0; }

// passes = ceil(b / max_digit) (rounded up to even if asked), digits of
// ceil(b / passes) bits from the least significant end.  The widest digit is
// 10 bits for int32 rows and 9 bits for int64 rows, the widest that keeps two
// onesweep CTAs resident per SM.
template <typename K>
constexpr int max_digit_bits() {
  return sizeof(K) == 4 ? 10 : 9;
}

// Time of one pass per row by digit width, relative to a pass of at most 7
// bits (measured on GB300 with 16-byte rows: 8 bits 1.17x, 9 bits 1.43x; a
// wider digit splits each tile into more and shorter output runs).
double pass_cost(int w) { return w <= 7 ? 1.0 : w == 8 ? 1.17 : w == 9 ? 1.43 : 1.7; }

// A plan that need not be even, over at least kCostRows rows, takes one pass
// more when the narrower digits make it cheaper (27 bits: 4 passes of 7 bits
// instead of 3 of 9); below that size a pass's fixed cost decides.
constexpr int64_t kCostRows = int64_t(1) << 22;

Plan make_plan(uint64_t lo, uint64_t range, bool even, int max_digit, int force_passes = -1,
               int64_t rows = 0) {
  Plan p;
  p.lo = lo;
  p.key_bits = bitlen(range);
  int P = force_passes >= 0 ? force_passes : (p.key_bits + max_digit - 1) / max_digit;
  if (force_passes < 0 && !even && rows >= kCostRows && P > 0 && P < kMaxPasses) {
    const int w0 = (p.key_bits + P - 1) / P, w1 = (p.key_bits + P) / (P + 1);
    if ((P + 1) * pass_cost(w1) < P * pass_cost(w0)) ++P;
  }
  if (even && (P & 1)) ++P;
  if (P > kMaxPasses) P = kMaxPasses;
  p.passes = P;
  if (P > 0) {
    const int w = (p.key_bits + P - 1) / P;
    for (int i = 0; i < P; ++i) {
      p.shift[i] = std::min(i * w, 63);
      p.bits[i] = std::max(0, std::min(w, p.key_bits - i * w));
      p.max_bits = std::max(p.max_bits, p.bits[i]);
    }
  }
  return p;
}

template <typename K>
K key_of(unsigned long long ou);
template <>
int32_t key_of<int32_t>(unsigned long long ou) {
  return (int32_t)(uint32_t)((uint32_t)ou ^ 0x80000000u);
}
template <>
int64_t key_of<int64_t>(unsigned long long ou) {
  return (int64_t)(ou ^ 0x8000000000000000ull);
}

template <typename K>
uint64_t lo_bits(K k) {
  return (uint64_t)(typename UnsignedOf<K>::type)k;
}
template <typename K>
uint64_t range_of(K lo, K hi) {
  using U = typename UnsignedOf<K>::type;
  return (uint64_t)(U)((U)hi - (U)lo);
}

int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

template <typename K>
void set_job_plan(RadixJob<K>& j, const Plan& p) {
  j.lo = p.lo;
  j.passes = p.passes;
  for (int i = 0; i < kMaxPasses; ++i) {
    j.shift[i] = p.shift[i];
    j.bits[i] = p.bits[i];
  }
}

// Sets the ping-pong pointers of a job: pass 0 reads (in_k, in_v); pass p
// writes buffer A when p is even, B when odd.  Returns the final location.
template <typename K>
void set_job_buffers(RadixJob<K>& j, const K* in_k, const K* in_v, K* ak, K* av, K* bk, K* bv,
                     const K** res_k, const K** res_v) {
  const K* ck = in_k;
  const K* cv = in_v;
  for (int p = 0; p < j.passes; ++p) {
    K* dk = (p & 1) ? bk : ak;
    K* dv = (p & 1) ? bv : av;
    j.src_k[p] = ck;
    j.src_v[p] = cv;
    j.dst_k[p] = dk;
    j.dst_v[p] = dv;
    ck = dk;
    cv = dv;
  }
  *res_k = ck;
  *res_v = cv;
}

// ---- inner join -------------------------------------------------------------------
struct Opts {
  int router = TJ_ROUTE_AUTO;
  int partitions = 0;  // 0: chosen from the key range (auto_parts)
  int stride = 100;
  int segments = 4096;
  int mlp_steps = 600;
  int mlp_batch = 256;
  float mlp_lr = 3e-3f;
  uint64_t seed = 20260221ull;
  double radix_judge = 1.25;  // < 0: the learned model is always kept
  bool fused = true;          // the partition-resident phase for narrow batches
  bool exact_route = false;  // size the batch regions by a histogram, not the sample
};

// part_join_impl's request to be run again with exact batch sizes (a batch
// outgrew the region its sample estimate gave it)
constexpr tj_status kRouteAgain = (tj_status)100;

Opts make_opts(const tj_join_opts* o) {
  Opts x;
  if (!o) return x;
  x.router = o->router;
  if (o->partitions > 0) x.partitions = o->partitions;
  if (o->sample_stride > 0) x.stride = o->sample_stride;
  if (o->pla_segments > 0) x.segments = o->pla_segments;
  if (o->mlp_steps > 0) x.mlp_steps = o->mlp_steps;
  if (o->mlp_batch > 0) x.mlp_batch = o->mlp_batch;
  if (o->mlp_lr > 0.f) x.mlp_lr = o->mlp_lr;
  if (o->seed) x.seed = o->seed;
  if (o->radix_judge != 0.f) x.radix_judge = o->radix_judge;
  x.fused = (o->flags & TJ_JOIN_NO_FUSED) == 0;
  return x;
}

// Batches of a partitioned join when the caller leaves the number open: 128
// (fewer, larger batches: best for the LSD path, where 128 and 256 measured
// within 3%), or 256 when that, and not 128, brings the batches within the
// partition-resident phase's preferred reach (kFKeyBits + kFPreferMsdBits
// key bits): key ranges of 27 bits, such as 10^8 keys.
int auto_parts(int key_bits) {
  return key_bits == kFKeyBits + kFPreferMsdBits + 8 ? 256 : 128;
}

// Inputs (n_r + n_s) from which router AUTO partitions a join whose batches
// the partition-resident phase can join, even when one pass fits the budget.
constexpr int64_t kAutoPartitionRows = int64_t(1) << 26;

template <typename K>
tj_status part_join_impl(const K* kr, const K* ir, int64_t nr, const K* ks, const K* is,
                         int64_t ns, K lo, K hi, bool range_known, size_t budget, const Opts& o,
                         K* out, int64_t cap, int64_t* out_count, tj_stats& stats, Tracer& tr,
                         cudaStream_t st);
template <typename K>
tj_status sort_impl(K* keys, K* ids, int64_t n, cudaStream_t st);

template <typename K>
tj_status join_impl(const K* kr, const K* ir, int64_t nr, const K* ks, const K* is, int64_t ns,
                    size_t budget, const Opts& opts, K* out, int64_t cap, int64_t* out_count,
                    cudaStream_t st) {
  tj_stats stats = {};
  stats.groups = 1;
  *out_count = 0;
  if (nr == 0 || ns == 0) {
    g_stats = stats;
    return TJ_OK;
  }
  tj_status s = ensure_device();
  if (s != TJ_OK) return s;

  const int64_t tiles_r = ceil_div(nr, kTile), tiles_s = ceil_div(ns, kTile);
  Carve cc;
  const size_t o_jobs = cc.add<RadixJob<K>>(4);  // R, S; again for the onesweep tile
  const size_t o_stats = cc.add<KeyStats>(2);
  const size_t o_misc = cc.add<int64_t>(32);  // err, counters, total
  const size_t o_jj = cc.add<JoinJob<K>>(1);
  Block ctl;
  TJ_CUDA(ctl.alloc(cc.off, st));
  RadixJob<K>* d_jobs = ctl.at<RadixJob<K>>(o_jobs);
  KeyStats* d_stats = ctl.at<KeyStats>(o_stats);
  int* d_err = ctl.at<int>(o_misc);
  uint32_t* d_counters = ctl.at<uint32_t>(o_misc + 16);  // [kMaxPasses + 1]
  int64_t* d_total = ctl.at<int64_t>(o_misc + 128);
  JoinJob<K>* d_jj = ctl.at<JoinJob<K>>(o_jj);

  RadixJob<K> hj[2];
  memset(hj, 0, sizeof(hj));
  hj[0].keys = kr;
  hj[0].n = nr;
  hj[0].tile0 = 0;
  hj[1].keys = ks;
  hj[1].n = ns;
  hj[1].tile0 = tiles_r;
  TJ_CUDA(cudaMemsetAsync(ctl.p + o_misc, 0, 32 * sizeof(int64_t), st));
  TJ_CUDA(cudaMemsetAsync(d_stats, 0xFF, 2 * sizeof(KeyStats), st));
  TJ_CUDA(put_small(d_jobs, hj, sizeof(hj), st));
  Tracer tr(st);
  const double w = (double)sizeof(K);

  // the partitioned path (again with exact batch sizes if a sampled region overflowed)
  auto partitioned = [&](int router, K lo, K hi, bool range_known) -> tj_status {
    stats.learned = router;
    Opts po = opts;
    po.router = router;
    tj_status ps = part_join_impl<K>(kr, ir, nr, ks, is, ns, lo, hi, range_known, budget, po,
                                     out, cap, out_count, stats, tr, st);
    if (ps == kRouteAgain) {
      po.exact_route = true;
      ps = part_join_impl<K>(kr, ir, nr, ks, is, ns, lo, hi, range_known, budget, po, out, cap,
                             out_count, stats, tr, st);
      stats.route_regions = 3;
    }
    if (ps == TJ_OK || ps == TJ_ERR_CAPACITY) {
      stats.out_count = *out_count;
      g_stats = stats;
    }
    return ps;
  };
  // One sorted copy of both relations already exceeds the budget: the join is
  // partitioned whatever the key range, and a learned router needs no key
  // statistics first (its sample gives the range for routing, the route pass
  // the exact one for the batches).
  if ((opts.router == TJ_ROUTE_AUTO || opts.router == TJ_ROUTE_PLA ||
       opts.router == TJ_ROUTE_MLP) &&
      budget != 0 && (double)(nr + ns) * 2.0 * w > (double)budget)
    return partitioned(opts.router == TJ_ROUTE_AUTO ? (int)TJ_ROUTE_PLA : opts.router, K(0),
                       K(0), false);
  tr.begin("stats", w * (nr + ns));
  TJ_CUDA(launch_stats<K>(d_jobs, 2, tiles_r + tiles_s, d_stats, st));
  tr.end();
  KeyStats hs[2];
  TJ_CUDA(get_small(hs, d_stats, sizeof(hs), st));
  TJ_CUDA(sync_stream(st));

  const K min_r = key_of<K>(hs[0].min_u), max_r = key_of<K>(~hs[0].max_u);
  const K min_s = key_of<K>(hs[1].min_u), max_s = key_of<K>(~hs[1].max_u);
  if (max_r < min_s || max_s < min_r) {  // key ranges do not overlap: J is empty
    g_stats = stats;
    return TJ_OK;
  }
  const K lo = std::min(min_r, min_s), hi = std::max(max_r, max_s);
  const Plan plan =
      make_plan(lo_bits<K>(lo), range_of<K>(lo, hi), false, max_digit_bits<K>(), -1, nr + ns);
  stats.key_bits = plan.key_bits;
  stats.radix_passes = plan.passes;
  stats.digit_bits = plan.max_bits;

  const int P = plan.passes;
  const int64_t bins_max = (int64_t)1 << plan.max_bits;
  const int64_t jtiles = ceil_div(ns, kJTile);
  const int nbuf = P >= 2 ? 2 : P;
  Carve bc;
  size_t o_r[4] = {0, 0, 0, 0}, o_s[4] = {0, 0, 0, 0};
  for (int b = 0; b < nbuf; ++b) {
    o_r[2 * b] = bc.add<K>(nr);
    o_r[2 * b + 1] = bc.add<K>(nr);
    o_s[2 * b] = bc.add<K>(ns);
    o_s[2 * b + 1] = bc.add<K>(ns);
  }
  const size_t o_hist = bc.add<uint32_t>(2 * kMaxPasses * kMaxBins);
  const size_t o_lb = bc.add<uint32_t>((size_t)(tiles_r + tiles_s) * bins_max);
  const size_t o_tiles = bc.add<JTile<K>>(jtiles);
  const size_t o_jlb = bc.add<uint64_t>(jtiles);
  const size_t need = bc.off + cc.off;
  int router = opts.router;
  if (router == TJ_ROUTE_AUTO) {
    // Execution-time choice of the path (Sec. 3.3: from the input's scale and
    // the extent of the key axis; Sec. 5.4 compares it with the forced
    // paths): partitioned when the budget requires it, or when the inputs
    // are large and the batches of this key range reach the
    // partition-resident phase, which then costs less than sorting both
    // relations whole (measured on FK joins: 0.88-0.93x the single pass from
    // 10^8 rows on, break-even near 5x10^7, up to 2x slower below); else
    // one pass.
    const int parts_bits = bitlen((uint64_t)auto_parts(plan.key_bits)) - 1;
    const int batch_bits = plan.key_bits - parts_bits;
    const bool fusable =
        opts.fused && batch_bits >= kFKeyBits && batch_bits <= kFKeyBits + kFMaxMsdBits;
    if (budget != 0 && need > budget)
      router = TJ_ROUTE_PLA;
    else if (fusable && nr + ns >= kAutoPartitionRows)
      router = TJ_ROUTE_PLA;
    else
      router = TJ_ROUTE_SINGLE;
  }
  if (router != TJ_ROUTE_SINGLE) return partitioned(router, lo, hi, true);
  if (budget != 0 && need > budget)
    return set_err(TJ_ERR_BUDGET,
                   "join needs %zu bytes of scratch in one pass, budget is %zu", need, budget);
  Block big;
  TJ_CUDA(big.alloc(bc.off, st));
  stats.scratch_peak = (int64_t)need;

  const K* res_rk = kr;
  const K* res_rv = ir;
  const K* res_sk = ks;
  const K* res_sv = is;
  if (P > 0) {
    set_job_plan(hj[0], plan);
    set_job_plan(hj[1], plan);
    hj[0].hist_stride = hj[1].hist_stride = kMaxBins;
    hj[0].hist = big.at<uint32_t>(o_hist);
    hj[1].hist = hj[0].hist + kMaxPasses * kMaxBins;
    hj[0].lookback = big.at<uint32_t>(o_lb);
    hj[1].lookback = hj[0].lookback + tiles_r * bins_max;
    K* rb_k = nbuf > 1 ? big.at<K>(o_r[2]) : nullptr;
    K* rb_v = nbuf > 1 ? big.at<K>(o_r[3]) : nullptr;
    K* sb_k = nbuf > 1 ? big.at<K>(o_s[2]) : nullptr;
    K* sb_v = nbuf > 1 ? big.at<K>(o_s[3]) : nullptr;
    set_job_buffers(hj[0], kr, ir, big.at<K>(o_r[0]), big.at<K>(o_r[1]), rb_k, rb_v, &res_rk,
                    &res_rv);
    set_job_buffers(hj[1], ks, is, big.at<K>(o_s[0]), big.at<K>(o_s[1]), sb_k, sb_v, &res_sk,
                    &res_sv);
    // the onesweep passes take the wider tile when every digit is narrow: a
    // second pair of jobs numbers their tiles (no more tiles than the
    // histogram's, so the look-back region holds them)
    const int items = plan.max_bits <= kWideBits ? kItemsWide : kItems;
    const int64_t otile = (int64_t)kSortThreads * items;
    const int64_t otiles_r = ceil_div(nr, otile), otiles_s = ceil_div(ns, otile);
    RadixJob<K> hw[4] = {hj[0], hj[1], hj[0], hj[1]};
    hw[3].tile0 = otiles_r;
    hw[3].lookback = hw[2].lookback + otiles_r * bins_max;
    TJ_CUDA(put_small(d_jobs, hw, sizeof(hw), st));
    TJ_CUDA(cudaMemsetAsync(hj[0].hist, 0, 2 * kMaxPasses * kMaxBins * sizeof(uint32_t), st));
    tr.begin("histogram", w * (nr + ns));
    TJ_CUDA(launch_histogram<K>(d_jobs, 2, tiles_r + tiles_s, st));
    tr.end();
    TJ_CUDA(launch_digit_scan<K>(d_jobs, 2, P, st));
    for (int p = 0; p < P; ++p) {
      TJ_CUDA(cudaMemsetAsync(hj[0].lookback, 0,
                              (size_t)(otiles_r + otiles_s) * bins_max * sizeof(uint32_t), st));
      tr.begin("onesweep", 4.0 * w * (nr + ns));
      TJ_CUDA(launch_onesweep<K>(d_jobs + 2, 2, otiles_r + otiles_s, p, plan.max_bits, false,
                                 d_counters + p, d_err, st, nullptr, items));
      tr.end();
    }
  }

  JoinJob<K> jj;
  jj.rk = res_rk;
  jj.rv = res_rv;
  jj.nr = nr;
  jj.sk = res_sk;
  jj.sv = res_sv;
  jj.ns = ns;
  jj.tile0 = 0;
  JTile<K>* d_tiles = big.at<JTile<K>>(o_tiles);
  uint64_t* d_jlb = big.at<uint64_t>(o_jlb);
  TJ_CUDA(put_small(d_jj, &jj, sizeof(jj), st));
  TJ_CUDA(launch_tile_ranges<K>(d_jj, 1, jtiles, d_tiles, st));
  TJ_CUDA(cudaMemsetAsync(d_jlb, 0, jtiles * sizeof(uint64_t), st));
  tr.begin("join", 2.0 * w * (nr + ns));
  TJ_CUDA(launch_join<K>(jtiles, d_tiles, d_jlb, d_counters + kMaxPasses, out, cap, nullptr,
                         nullptr, d_total, d_err, st));
  tr.end();
  int64_t h_misc[2] = {0, 0};
  int h_err = 0;
  TJ_CUDA(get_small(&h_misc[0], d_total, sizeof(int64_t), st));
  TJ_CUDA(get_small(&h_err, d_err, sizeof(int), st));
  TJ_CUDA(sync_stream(st));
  if (h_misc[0] <= cap) tr.add_bytes("join", 2.0 * w * (double)h_misc[0]);
  tr.flush();
  if (h_err) return set_err((tj_status)h_err, "device reported %d", h_err);
  *out_count = h_misc[0];
  stats.out_count = h_misc[0];
  g_stats = stats;
  if (h_misc[0] > cap)
    return set_err(TJ_ERR_CAPACITY, "result has %lld pairs, capacity %lld",
                   (long long)h_misc[0], (long long)cap);
  return TJ_OK;
}


// ---- partitioned (multi-pass) join --------------------------------------------------
// 1. cut keys from the router (equal-width ranges, or sample quantiles);
// 2. one route pass moves R and S into key-range batches (staging);
// 3. batches are grouped in key order so that each group's working set (sort
//    buffers, histograms, look-back, join state) fits the budget, and every
//    group is sorted and aligned by one batched launch sequence, its output
//    written after the previous group's (device-side running offset).

// Cuts of 2^plog equal-width batches over [lo, hi]: lo + p 2^(b - plog), b =
// significant bits of hi - lo (every key of the range its own batch when
// b <= plog).  The batch of a key is then (key - lo) >> (b - plog).
template <typename K>
std::vector<K> radix_cuts(K lo, K hi, int plog) {
  std::vector<K> cuts;
  const int b = bitlen(range_of<K>(lo, hi));
  if (b <= plog) {
    for (uint64_t x = 1; x <= range_of<K>(lo, hi); ++x) cuts.push_back((K)(lo_bits<K>(lo) + x));
  } else {
    for (int64_t p = 1; p < ((int64_t)1 << plog); ++p)
      cuts.push_back((K)(lo_bits<K>(lo) + ((uint64_t)p << (b - plog))));
  }
  return cuts;
}

// Smallest and largest key of both relations (one read of the keys).
template <typename K>
tj_status key_range(const K* kr, int64_t nr, const K* ks, int64_t ns, K* lo, K* hi,
                    cudaStream_t st) {
  Carve c;
  const size_t o_jobs = c.add<RadixJob<K>>(2), o_stats = c.add<KeyStats>(2);
  Block b;
  TJ_CUDA(b.alloc(c.off, st));
  RadixJob<K> hj[2];
  memset(hj, 0, sizeof(hj));
  hj[0].keys = kr;
  hj[0].n = nr;
  hj[1].keys = ks;
  hj[1].n = ns;
  hj[1].tile0 = ceil_div(nr, kTile);
  TJ_CUDA(put_small(b.at<RadixJob<K>>(o_jobs), hj, sizeof(hj), st));
  TJ_CUDA(cudaMemsetAsync(b.at<KeyStats>(o_stats), 0xFF, 2 * sizeof(KeyStats), st));
  TJ_CUDA(launch_stats<K>(b.at<RadixJob<K>>(o_jobs), 2, hj[1].tile0 + ceil_div(ns, kTile),
                          b.at<KeyStats>(o_stats), st));
  KeyStats hs[2];
  TJ_CUDA(get_small(hs, b.at<KeyStats>(o_stats), sizeof(hs), st));
  TJ_CUDA(sync_stream(st));
  *lo = key_of<K>(std::min(hs[0].min_u, hs[1].min_u));
  *hi = key_of<K>(std::max(~hs[0].max_u, ~hs[1].max_u));
  return TJ_OK;
}

template <typename K>
std::vector<K> make_cuts(const std::vector<K>& b) {
  std::vector<K> v(b);
  std::sort(v.begin(), v.end());
  std::vector<K> out;
  for (size_t i = 0; i < v.size();) {
    size_t j = i;
    while (j < v.size() && v[j] == v[i]) ++j;
    out.push_back(v[i]);
    // a boundary that repeats holds at least one batch's worth of rows: give
    // it a batch of its own by also cutting right after it
    if (j - i >= 2 && v[i] < std::numeric_limits<K>::max()) out.push_back((K)(v[i] + 1));
    i = j;
  }
  std::sort(out.begin(), out.end());
  out.erase(std::unique(out.begin(), out.end()), out.end());
  return out;
}

template <typename K>
tj_status part_join_impl(const K* kr, const K* ir, int64_t nr, const K* ks, const K* is,
                         int64_t ns, K lo, K hi, bool range_known, size_t budget, const Opts& o,
                         K* out, int64_t cap, int64_t* out_count, tj_stats& stats, Tracer& tr,
                         cudaStream_t st) {
  const double w = (double)sizeof(K);
  const int maxd = max_digit_bits<K>();
  // batches: as asked, else from the key range (the sample's when the range
  // is not known yet)
  int parts = o.partitions > 0 ? std::max(2, std::min(o.partitions, kMaxCuts))
                               : (range_known ? auto_parts(bitlen(range_of<K>(lo, hi))) : 128);
  std::vector<K> cuts;
  int router = o.router;
  std::vector<uint32_t> sample_cnt;  // per side and batch, when regions are sized by the sample
  int64_t sample_m[2] = {0, 0};
  bool radix_route = false;  // equal-width batches, routed by their digit (no cut table)
  bool fell_back = false;    // the radix judge replaced the learned model
  // ---- 1. cut keys ----
  if (router == TJ_ROUTE_PLA || router == TJ_ROUTE_MLP) {
    const int stride = o.stride;
    const int64_t off_r = (int64_t)((o.seed * 0x9E3779B97F4A7C15ull) >> 33) % std::min<int64_t>(stride, nr);
    const int64_t off_s = (int64_t)((o.seed * 0xBF58476D1CE4E5B9ull) >> 33) % std::min<int64_t>(stride, ns);
    const int64_t m_r = (nr - off_r + stride - 1) / stride, m_s = (ns - off_s + stride - 1) / stride;
    const int64_t m = m_r + m_s;
    Carve c;
    const size_t o_k = c.add<K>((size_t)m), o_v = c.add<K>((size_t)m), o_b = c.add<K>(kMaxCuts);
    const size_t o_th = c.add<float>(kMlpParams), o_tab = c.add<float>(kMlpTable + 1);
    const size_t o_steps = c.add<int>(4);
    const size_t o_edges = c.add<int64_t>(kMaxCuts + 2);
    const size_t o_scuts = c.add<K>(kMaxCuts), o_scnt = c.add<uint32_t>(2 * kMaxBins);
    Block sb;
    TJ_CUDA(sb.alloc(c.off, st));
    TJ_CUDA(launch_sample_gather<K>(kr, m_r, off_r, ks, m_s, off_s, stride, sb.at<K>(o_k),
                                    sb.at<K>(o_v), st));
    const tj_stats keep = g_stats;
    tj_status ss = sort_impl<K>(sb.at<K>(o_k), sb.at<K>(o_v), m, st);
    g_stats = keep;
    if (ss != TJ_OK) return ss;
    if (!range_known) {  // the sorted sample's ends stand for the range until the route
      TJ_CUDA(get_small(&lo, sb.at<K>(o_k), sizeof(K), st));
      TJ_CUDA(get_small(&hi, sb.at<K>(o_k) + (m - 1), sizeof(K), st));
      TJ_CUDA(sync_stream(st));
      if (o.partitions <= 0) parts = auto_parts(bitlen(range_of<K>(lo, hi)));
    }
    // per-side sample counts of the batches a set of cuts makes
    auto sample_counts = [&](const std::vector<K>& cv, std::vector<uint32_t>& cnt) -> tj_status {
      std::vector<K> hc(kMaxCuts, std::numeric_limits<K>::max());
      std::copy(cv.begin(), cv.end(), hc.begin());
      TJ_CUDA(put_small(sb.at<K>(o_scuts), hc.data(), kMaxCuts * sizeof(K), st));
      TJ_CUDA(cudaMemsetAsync(sb.at<uint32_t>(o_scnt), 0, 2 * kMaxBins * sizeof(uint32_t), st));
      TJ_CUDA(launch_sample_route_counts<K>(sb.at<K>(o_k), sb.at<K>(o_v), m, m_r,
                                            sb.at<K>(o_scuts), (int)cv.size(),
                                            sb.at<uint32_t>(o_scnt), st));
      cnt.assign(2 * (size_t)kMaxBins, 0u);
      TJ_CUDA(get_small(cnt.data(), sb.at<uint32_t>(o_scnt), cnt.size() * sizeof(uint32_t), st));
      TJ_CUDA(sync_stream(st));
      return TJ_OK;
    };
    // Radix judges the model on the (sorted) sample: the balance of
    // equal-width ranges of the same count (bucket edges by binary search on
    // the device) against the balance of the model's batches, leaving out the
    // batches of a single key (a heavy key isolated by its cuts needs no
    // sort).  Radix replaces the model whenever it is within o.radix_judge
    // (1.25 by default) of it, allowing for the sample's noise (the model is
    // judged on the sample it was fitted to) and its largest batch fits the
    // budget.  Its route pass is a plain digit pass with no cut-table search,
    // so a model that fits the keys no better than equal-width ranges
    // (uniform keys, or a network that failed to fit) falls back to radix.
    const int b_all = bitlen(range_of<K>(lo, hi));
    int plog = 0;
    while ((2 << plog) <= parts) ++plog;
    int64_t radix_max = 0;  // sample rows of the largest equal-width range
    double radix_noise = 0;  // sampling noise of the largest range's balance
    {
      const int sh = std::max(0, b_all - plog);
      const int nb = 1 << plog;
      TJ_CUDA(launch_sorted_bucket_edges<K>(sb.at<K>(o_k), m, lo_bits<K>(lo), sh, nb,
                                            sb.at<int64_t>(o_edges), st));
      std::vector<int64_t> edges((size_t)nb + 1);
      TJ_CUDA(get_small(edges.data(), sb.at<int64_t>(o_edges), edges.size() * 8, st));
      TJ_CUDA(sync_stream(st));
      // over the non-empty ranges: a key range that is not a power of two
      // leaves the top ranges empty, which costs nothing
      int64_t mx = 0;
      int used = 0;
      for (int d = 0; d < nb; ++d) {
        const int64_t c = (d + 1 < nb ? edges[(size_t)d + 1] : m) - edges[(size_t)d];
        mx = std::max(mx, c);
        used += c > 0;
      }
      stats.radix_balance = (double)mx * (double)std::max(used, 1) / (double)std::max<int64_t>(1, m);
      radix_max = mx;
      // the largest of the ranges' sample counts lies about 3 standard
      // deviations (Poisson: the square root of the mean) above their mean
      radix_noise = 3.0 / std::sqrt(std::max(1.0, (double)m / std::max(used, 1)));
    }
    // Under a budget, the largest equal-width batch (its sample share of all
    // rows plus 10%) must also fit one lane's half of the working set: about
    // 2w + 2 bytes per row (one sort buffer, look-back words).
    const double radix_rows =
        1.1 * (double)radix_max / (double)std::max<int64_t>(1, m) * (double)(nr + ns) + 4096.0;
    const bool radix_fits =
        budget == 0 || radix_rows * (2.0 * sizeof(K) + 2.0) <= 0.45 * (double)budget;
    // A model's batches balance no better than perfectly (1, up to the heavy
    // keys it isolates, and a key heavy enough to matter would have pushed
    // the equal-width balance up too), so when equal-width ranges are within
    // the judge's factor of perfect, radix wins whatever the model: the fit
    // is skipped.
    std::vector<uint32_t> cnt;
    tj_status js = TJ_OK;
    if (o.radix_judge >= 0 && radix_fits && stats.radix_balance <= o.radix_judge + radix_noise) {
      radix_route = true;
      fell_back = true;
      stats.learned_balance = 0;
      cuts = radix_cuts<K>(lo, hi, plog);
      js = sample_counts(cuts, cnt);
      if (js != TJ_OK) return js;
    } else {
      int G = std::max(o.segments, parts);
      G = (G / parts) * parts;  // boundaries fall on knots
      std::vector<K> bnd((size_t)(parts - 1));
      if (router == TJ_ROUTE_PLA) {
        // boundaries of the piecewise-linear CDF: knots t_{(G / parts) p}
        const int step = G / parts;
        tr.begin("pla_fit", w * (double)m);
        TJ_CUDA(launch_quantiles<K>(sb.at<K>(o_k), m, G, step, step * (parts - 1), step,
                                    sb.at<K>(o_b), st));
        tr.end();
      } else {
        // MLP: seeded uniform initialisation on the host, training and the
        // monotone tabulation on the device
        std::vector<float> th(kMlpParams, 0.f);
        uint64_t z = o.seed;
        auto uni = [&](float a) {
          z += 0x9E3779B97F4A7C15ull;
          uint64_t x = z;
          x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
          x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
          x ^= x >> 31;
          return a * (2.f * (float)((x >> 40) * (1.0 / 16777216.0)) - 1.f);
        };
        for (int i = 0; i < 32; ++i) th[1 + i] = uni(2.45f);          // w1
        for (int i = 0; i < 32; ++i) th[33 + i] = uni(1.0f);          // b1
        for (int i = 0; i < 1024; ++i) th[65 + i] = uni(0.433f);      // W2
        for (int i = 0; i < 32; ++i) th[1121 + i] = uni(0.433f);      // w3
        TJ_CUDA(put_small(sb.at<float>(o_th), th.data(), th.size() * 4, st));
        tr.begin("mlp_train", 0.0);
        TJ_CUDA(launch_mlp_train<K>(sb.at<K>(o_k), m, sb.at<float>(o_th), o.mlp_steps,
                                    o.mlp_batch, o.mlp_lr, o.seed, sb.at<int>(o_steps), st));
        TJ_CUDA(get_small(&stats.mlp_steps, sb.at<int>(o_steps), sizeof(int), st));
        tr.end();
        tr.begin("mlp_route_table", 0.0);
        TJ_CUDA(launch_mlp_boundaries<K>(sb.at<float>(o_th), kMlpTable, sb.at<float>(o_tab), parts,
                                         sb.at<K>(o_k), m, sb.at<K>(o_b), st));
        tr.end();
      }
      TJ_CUDA(get_small(bnd.data(), sb.at<K>(o_b), bnd.size() * sizeof(K), st));
      TJ_CUDA(sync_stream(st));  // bnd is filled at the sync
      cuts = make_cuts<K>(bnd);
      js = sample_counts(cuts, cnt);
      if (js != TJ_OK) return js;
      {
        const int np = (int)cuts.size() + 1;
        int64_t mx = 0;
        for (int p2 = 0; p2 < np; ++p2) {
          const bool single = p2 > 0 && p2 < np - 1 &&
                              (uint64_t)cuts[(size_t)p2] - (uint64_t)cuts[(size_t)p2 - 1] == 1;
          if (!single)
            mx = std::max<int64_t>(mx, (int64_t)cnt[(size_t)p2] + cnt[(size_t)kMaxBins + p2]);
        }
        stats.learned_balance = (double)mx * (double)np / (double)std::max<int64_t>(1, m);
      }
      if (o.radix_judge >= 0 && radix_fits &&
          stats.radix_balance <= o.radix_judge * stats.learned_balance + radix_noise) {
        radix_route = true;
        fell_back = true;
        cuts = radix_cuts<K>(lo, hi, plog);
        js = sample_counts(cuts, cnt);
        if (js != TJ_OK) return js;
      }
    }
    // batch sizes per side estimated from the sample (regions sized ahead of
    // the route pass, so it needs no histogram of its own)
    if (!o.exact_route) {
      sample_cnt = cnt;
      sample_m[0] = m_r;
      sample_m[1] = m_s;
    }
    // a retry with exact sizes routes equal-width ranges by their digit over
    // the whole key range: take it from the key statistics
    if (radix_route && o.exact_route && !range_known) {
      tj_status rs = key_range<K>(kr, nr, ks, ns, &lo, &hi, st);
      if (rs != TJ_OK) return rs;
      range_known = true;
      cuts = radix_cuts<K>(lo, hi, plog);
    }
  } else {  // TJ_ROUTE_RADIX
    if (!range_known) return set_err(TJ_ERR_INTERNAL, "equal-width batches need the key range");
    router = TJ_ROUTE_RADIX;
    radix_route = true;
    int plog = 0;
    while ((2 << plog) <= parts) ++plog;
    cuts = radix_cuts<K>(lo, hi, plog);
  }
  while ((int)cuts.size() > kMaxCuts - 1) cuts.pop_back();  // cannot happen for parts <= 1024
  const int ncuts = (int)cuts.size();
  const int nparts = ncuts + 1;
  int rbits = bitlen((uint64_t)ncuts);
  if (rbits == 0) rbits = 1;
  stats.partitions = nparts;
  if (!radix_route) {
    int heavy = 0;
    for (int i = 0; i + 1 < ncuts; ++i)
      if ((uint64_t)cuts[(size_t)i + 1] - (uint64_t)cuts[(size_t)i] == 1) ++heavy;
    stats.heavy_keys = heavy;
  }

  // ---- 2. route pass into staging, in chunks whose look-back fits the budget ----
  // log-scale index over the cuts (see RadixJob::route_tab): tab[b] = number of
  // cuts below the first key of bucket b
  const uint64_t krange = range_of<K>(lo, hi);
  std::vector<uint16_t> tab(kRouteBuckets + 1);
  for (int bkt = 0; bkt <= kRouteBuckets; ++bkt) {
    uint64_t start;  // smallest x = key - lo whose bucket is >= bkt
    bool beyond = bkt == kRouteBuckets;
    if (bkt < 32) {
      start = (uint64_t)bkt;
    } else if (bkt <= 6 * 32) {
      start = 32;
    } else {
      const int e = bkt >> 5, mnt = bkt & 31;
      start = e > 64 ? 0 : ((uint64_t)(32 + mnt) << (e - 6));
      if (e > 64) beyond = true;
    }
    if (beyond || start > krange) {
      tab[(size_t)bkt] = (uint16_t)ncuts;
    } else {
      const K sk = (K)(lo_bits<K>(lo) + start);
      tab[(size_t)bkt] = (uint16_t)(std::lower_bound(cuts.begin(), cuts.end(), sk) - cuts.begin());
    }
  }
  int route_steps = 0;  // halvings that empty the largest bucket
  int route_shift = -1;
  {
    auto steps_for = [](const std::vector<uint16_t>& t, int nb) {
      int widest = 0, st2 = 0;
      for (int bkt = 0; bkt < nb; ++bkt)
        widest = std::max(widest, (int)t[(size_t)bkt + 1] - (int)t[(size_t)bkt]);
      while ((1 << st2) <= widest) ++st2;
      return st2;
    };
    route_steps = steps_for(tab, kRouteBuckets);
    // uniform index: bucket b covers x in [b << us, (b + 1) << us)
    int us = 0;
    while (us < 64 && (krange >> us) >= (uint64_t)(kRouteBuckets - 1)) ++us;
    const int ub = (int)(krange >> us) + 1;  // buckets in use (<= kRouteBuckets - 1)
    std::vector<uint16_t> utab(kRouteBuckets + 1, (uint16_t)ncuts);
    for (int bkt = 0; bkt <= ub; ++bkt) {
      const uint64_t start = (uint64_t)bkt << us;
      if (start > krange) break;
      const K sk = (K)(lo_bits<K>(lo) + start);
      utab[(size_t)bkt] = (uint16_t)(std::lower_bound(cuts.begin(), cuts.end(), sk) - cuts.begin());
    }
    const int usteps = steps_for(utab, ub);
    if (usteps < route_steps) {
      tab.swap(utab);
      route_steps = usteps;
      route_shift = us;
    }
  }
  // route pass tiles: kItemsRoute rows per thread for narrow batch indices
  // (shared memory still fits three CTAs per SM), kItems otherwise (with 1024
  // batches the 9-row tile measured 1.4x slower)
  // equal-width batches: batch = (clamp(key) - lo) >> rshift, rbits wide
  const int rshift = radix_route ? std::max(0, bitlen(krange) - rbits) : 0;
  const int ritems = radix_route ? (rbits <= kWideBits ? kItemsWide : kItems)
                                 : (rbits <= kWideBits ? kItemsRoute : kItems);
  const int64_t rtile = (int64_t)kSortThreads * ritems;
  const int64_t lb_per_tile = ((int64_t)1 << rbits) * 4;
  const int64_t route_lb = budget ? std::max<int64_t>((int64_t)budget / 4, 16 * lb_per_tile)
                                  : INT64_MAX;
  const int64_t all_tiles = ceil_div(std::max(nr, ns), rtile);
  const int64_t chunk_tiles = std::max<int64_t>(1, std::min(all_tiles, route_lb / lb_per_tile));
  const int64_t chunk_rows = chunk_tiles * rtile;  // <= max(n_r, n_s) rounded up to a tile
  if ((int64_t)nr + ns >= ((int64_t)1 << 32))
    return set_err(TJ_ERR_INVALID, "partitioned join needs n_r + n_s < 2^32");
  // Batch regions in the routed copies: sized from the sample when the router
  // sampled (est), else by a route histogram.  A sampled batch gets room for
  // its sample count scaled to the side plus six standard deviations and a
  // tile; the route pass drops and reports a row past its batch's region, and
  // the join is then routed again with exact sizes.
  const bool est = !sample_cnt.empty();
  stats.route_regions = est ? 2 : 1;
  std::vector<int64_t> rcap(2 * (size_t)nparts, 0), rstart(2 * (size_t)nparts, 0);
  int64_t side_rows[2] = {nr, ns};
  if (est) {
    for (int side = 0; side < 2; ++side) {
      const double scale =
          (double)(side ? ns : nr) / (double)std::max<int64_t>(1, sample_m[side]);
      int64_t acc = 0;
      for (int p2 = 0; p2 < nparts; ++p2) {
        const double c = (double)sample_cnt[(size_t)side * kMaxBins + p2];
        const int64_t k = (int64_t)std::ceil((c + 6.0 * std::sqrt(c) + 8.0) * scale) + rtile;
        rcap[(size_t)side * nparts + p2] = k;
        rstart[(size_t)side * nparts + p2] = acc;
        acc += k;
      }
      side_rows[side] = acc;
    }
    if (side_rows[0] >= ((int64_t)1 << 32) || side_rows[1] >= ((int64_t)1 << 32)) return kRouteAgain;
  }
  struct Chunk {
    int side;
    int64_t r0, n;
  };
  std::vector<Chunk> chunks;
  for (int side = 0; side < 2; ++side) {
    const int64_t n = side ? ns : nr;
    for (int64_t r0 = 0; r0 < n; r0 += chunk_rows) chunks.push_back({side, r0, std::min(chunk_rows, n - r0)});
  }
  const int nch = (int)chunks.size();
  // launch groups of chunks, each group's look-back within route_lb (one chunk
  // per launch with sampled regions: a chunk starts where the last one ended)
  std::vector<std::pair<int, int>> cgroups;
  int64_t lb_max = 0;
  for (int i = 0; i < nch;) {
    int j = i;
    int64_t acc = 0;
    while (j < nch && (j == i || (!est && acc + ceil_div(chunks[(size_t)j].n, rtile) * lb_per_tile <=
                                               route_lb)))
      acc += ceil_div(chunks[(size_t)j].n, rtile) * lb_per_tile, ++j;
    cgroups.push_back({i, j});
    lb_max = std::max(lb_max, acc);
    i = j;
  }
  Carve cc;
  const size_t o_rk = cc.add<K>((size_t)side_rows[0]), o_rv = cc.add<K>((size_t)side_rows[0]);
  const size_t o_sk = cc.add<K>((size_t)side_rows[1]), o_sv = cc.add<K>((size_t)side_rows[1]);
  const size_t staging = cc.off;
  const size_t o_cuts = cc.add<K>(kMaxCuts);
  const size_t o_tab = cc.add<uint16_t>(kRouteBuckets + 1);
  const size_t o_hist = cc.add<uint32_t>((size_t)nch * kMaxBins);
  const size_t o_rend = cc.add<uint32_t>(2 * (size_t)kMaxBins);  // regions' ends (est)
  const size_t o_fin = cc.add<uint32_t>(2 * (size_t)kMaxBins);   // where the route ended (est)
  const size_t o_jobs = cc.add<RadixJob<K>>((size_t)nch * 2);
  const size_t o_misc = cc.add<int64_t>(32);
  // the key range from the first and the last batch (range not known): jobs, min / max
  const size_t o_rjobs = cc.add<RadixJob<K>>(4), o_range = cc.add<KeyStats>(4);
  Block stg;
  TJ_CUDA(stg.alloc(cc.off, st));
  stats.staging_bytes = (int64_t)staging;
  int* d_err = stg.at<int>(o_misc);
  uint32_t* d_counters = stg.at<uint32_t>(o_misc + 16);
  std::vector<K> hc(kMaxCuts, std::numeric_limits<K>::max());
  std::copy(cuts.begin(), cuts.end(), hc.begin());
  TJ_CUDA(put_small(stg.at<K>(o_cuts), hc.data(), kMaxCuts * sizeof(K), st));
  TJ_CUDA(put_small(stg.at<uint16_t>(o_tab), tab.data(), tab.size() * sizeof(uint16_t), st));
  // histogram jobs (global tile numbering) then per-launch route jobs (tile0
  // rebased to their launch); the route jobs' hist slots receive the bases
  std::vector<RadixJob<K>> hj((size_t)nch * 2);
  memset(hj.data(), 0, hj.size() * sizeof(RadixJob<K>));
  int64_t tiles_all = 0;
  for (int c = 0; c < nch; ++c) {
    const Chunk& ch = chunks[(size_t)c];
    RadixJob<K>& x = hj[(size_t)c];
    const K* kb = ch.side ? ks : kr;
    const K* vb = ch.side ? is : ir;
    x.keys = kb + ch.r0;
    x.n = ch.n;
    x.tile0 = tiles_all;
    tiles_all += ceil_div(ch.n, kTile);
    x.lo = lo_bits<K>(lo);
    x.passes = 1;
    x.bits[0] = rbits;
    x.shift[0] = radix_route ? rshift : 0;
    x.route_hi = lo_bits<K>(hi);
    x.hist_stride = kMaxBins;
    x.hist = stg.at<uint32_t>(o_hist) + (size_t)c * kMaxBins;
    x.src_k[0] = kb + ch.r0;
    x.src_v[0] = vb + ch.r0;
    x.dst_k[0] = ch.side ? stg.at<K>(o_sk) : stg.at<K>(o_rk);
    x.dst_v[0] = ch.side ? stg.at<K>(o_sv) : stg.at<K>(o_rv);
    x.cuts = radix_route ? nullptr : stg.at<K>(o_cuts);  // radix: the digit path
    x.ncuts = ncuts;
    x.route_tab = stg.at<uint16_t>(o_tab);
    x.route_steps = route_steps;
    x.route_shift = route_shift;
    x.route_end = est ? stg.at<uint32_t>(o_rend) + (size_t)ch.side * kMaxBins : nullptr;
  }
  // route jobs' look-back words live in the working block, allocated once the
  // groups are known: offsets now, pointers (and a second upload) later
  std::vector<int64_t> route_lbw((size_t)nch, 0);
  for (auto& g : cgroups) {
    int64_t t = 0, lbw = 0;
    for (int c = g.first; c < g.second; ++c) {
      RadixJob<K> x = hj[(size_t)c];
      x.tile0 = t;
      route_lbw[(size_t)c] = lbw;
      t += ceil_div(x.n, rtile);
      lbw += ceil_div(x.n, rtile) << rbits;
      hj[(size_t)nch + c] = x;
    }
  }
  RadixJob<K>* d_rj = stg.at<RadixJob<K>>(o_jobs);
  TJ_CUDA(cudaMemsetAsync(stg.p + o_misc, 0, 32 * sizeof(int64_t), st));

  TJ_CUDA(put_small(d_rj, hj.data(), hj.size() * sizeof(RadixJob<K>), st));
  std::vector<int64_t> pcount(2 * (size_t)nparts, 0);
  std::vector<uint32_t> hcount((size_t)nch * kMaxBins, 0u);
  std::vector<uint32_t> rend(2 * (size_t)kMaxBins, 0u), rfin(2 * (size_t)kMaxBins, 0u);
  if (!est) {
    TJ_CUDA(cudaMemsetAsync(stg.at<uint32_t>(o_hist), 0, (size_t)nch * kMaxBins * sizeof(uint32_t), st));
    tr.begin("histogram", w * (nr + ns));
    TJ_CUDA(launch_histogram<K>(d_rj, nch, tiles_all, st));
    tr.end();
    TJ_CUDA(get_small(hcount.data(), stg.at<uint32_t>(o_hist), hcount.size() * 4, st));
    TJ_CUDA(sync_stream(st));
    // partition sizes and every chunk's base per partition (partition-major,
    // chunks in row order: the route is stable)
    for (int c = 0; c < nch; ++c)
      for (int p2 = 0; p2 < nparts; ++p2)
        pcount[(size_t)chunks[(size_t)c].side * nparts + p2] += hcount[(size_t)c * kMaxBins + p2];
    std::vector<int64_t> run(2 * (size_t)nparts, 0);
    for (int side = 0; side < 2; ++side) {
      int64_t acc = 0;
      for (int p2 = 0; p2 < nparts; ++p2) {
        run[(size_t)side * nparts + p2] = acc;
        rstart[(size_t)side * nparts + p2] = acc;
        acc += pcount[(size_t)side * nparts + p2];
      }
    }
    for (int c = 0; c < nch; ++c) {
      const int side = chunks[(size_t)c].side;
      for (int p2 = 0; p2 < nparts; ++p2) {
        const int64_t cnt = hcount[(size_t)c * kMaxBins + p2];
        hcount[(size_t)c * kMaxBins + p2] = (uint32_t)run[(size_t)side * nparts + p2];
        run[(size_t)side * nparts + p2] += cnt;
      }
    }
  } else {
    // the first chunk of a side starts at its batches' region starts; a later
    // chunk starts where the one before ended (chained on the device)
    for (int side = 0; side < 2; ++side)
      for (int p2 = 0; p2 < nparts; ++p2) {
        const size_t i = (size_t)side * nparts + p2;
        rend[(size_t)side * kMaxBins + p2] = (uint32_t)(rstart[i] + rcap[i]);
        rfin[(size_t)side * kMaxBins + p2] = (uint32_t)rstart[i];
      }
    for (int c = 0; c < nch; ++c)
      if (c == 0 || chunks[(size_t)c - 1].side != chunks[(size_t)c].side)
        for (int p2 = 0; p2 < nparts; ++p2)
          hcount[(size_t)c * kMaxBins + p2] =
              (uint32_t)rstart[(size_t)chunks[(size_t)c].side * nparts + p2];
    TJ_CUDA(put_small(stg.at<uint32_t>(o_rend), rend.data(), rend.size() * 4, st));
    TJ_CUDA(put_small(stg.at<uint32_t>(o_fin), rfin.data(), rfin.size() * 4, st));
  }
  TJ_CUDA(put_small(stg.at<uint32_t>(o_hist), hcount.data(), hcount.size() * 4, st));

  // ---- 3. the route pass (look-back words in a block of their own) ----
  // Memory: the routed copies (staging, reported apart) | route control (cuts,
  // index, bases, jobs) | the route pass's look-back words, released before
  // the groups' working block is taken | tables (every group's jobs, all digit
  // histograms, the groups' output bases).  The budget bounds control + the
  // larger of the two blocks + tables.
  const int64_t control = (int64_t)(cc.off - staging);
  if (budget && control + lb_max + 4096 > (int64_t)budget)
    return set_err(TJ_ERR_BUDGET, "budget %zu below the route pass's %lld bytes", budget,
                   (long long)(control + lb_max + 4096));
  Block rlb;
  TJ_CUDA(rlb.alloc((size_t)std::max<int64_t>(lb_max, 256), st));
  for (int c = 0; c < nch; ++c)
    hj[(size_t)nch + c].lookback = rlb.at<uint32_t>(0) + route_lbw[(size_t)c];
  TJ_CUDA(put_small(d_rj + nch, hj.data() + nch, (size_t)nch * sizeof(RadixJob<K>), st));
  for (auto& g : cgroups) {
    int64_t t = 0;
    for (int c = g.first; c < g.second; ++c) t += ceil_div(chunks[(size_t)c].n, rtile);
    TJ_CUDA(cudaMemsetAsync(rlb.p, 0, (size_t)lb_max, st));
    TJ_CUDA(cudaMemsetAsync(d_counters + kMaxPasses, 0, sizeof(uint32_t), st));
    double rows = 0;
    for (int c = g.first; c < g.second; ++c) rows += (double)chunks[(size_t)c].n;
    tr.begin("route", 4.0 * w * rows);
    TJ_CUDA(launch_onesweep<K>(d_rj + nch + g.first, g.second - g.first, t, 0, rbits,
                               radix_route ? kModeRadix : kModeCuts, d_counters + kMaxPasses,
                               d_err, st, nullptr, ritems, est));
    tr.end();
    if (est) {  // where this chunk ended: the next chunk's bases, or the side's end
      const int c = g.first, side = chunks[(size_t)c].side;
      uint32_t* next = (c + 1 < nch && chunks[(size_t)c + 1].side == side)
                           ? stg.at<uint32_t>(o_hist) + (size_t)(c + 1) * kMaxBins
                           : stg.at<uint32_t>(o_fin) + (size_t)side * kMaxBins;
      TJ_CUDA(launch_route_chain(stg.at<uint32_t>(o_hist) + (size_t)c * kMaxBins, rlb.at<uint32_t>(0),
                                 t - 1, 1 << rbits, next, st));
    }
  }
  if (est) {  // exact batch sizes
    int h_err = 0;
    TJ_CUDA(get_small(rfin.data(), stg.at<uint32_t>(o_fin), rfin.size() * 4, st));
    TJ_CUDA(get_small(&h_err, d_err, sizeof(int), st));
    TJ_CUDA(sync_stream(st));
    if (h_err == TJ_ERR_CAPACITY) return kRouteAgain;
    if (h_err) return set_err((tj_status)h_err, "device reported %d during the route pass", h_err);
    for (int side = 0; side < 2; ++side)
      for (int p2 = 0; p2 < nparts; ++p2) {
        const size_t i = (size_t)side * nparts + p2;
        pcount[i] = (int64_t)rfin[(size_t)side * kMaxBins + p2] - rstart[i];
      }
  }
  if (!range_known) {
    // the smallest key is in the first non-empty batch, the largest in the
    // last one (equal-width ranges over a sample's range may leave the top
    // ranges empty): their rows on both sides (about 2 / nparts of the data)
    // give the exact range
    int p_first = 0, p_last = nparts - 1;
    while (p_first < nparts - 1 && pcount[(size_t)p_first] + pcount[(size_t)nparts + p_first] == 0)
      ++p_first;
    while (p_last > p_first && pcount[(size_t)p_last] + pcount[(size_t)nparts + p_last] == 0)
      --p_last;
    std::vector<RadixJob<K>> rj;
    int64_t rtiles = 0;
    for (int side = 0; side < 2; ++side)
      for (int p2 : {p_first, p_last}) {
        const size_t i = (size_t)side * nparts + p2;
        RadixJob<K> x;
        memset(&x, 0, sizeof(x));
        x.keys = (side ? stg.at<K>(o_sk) : stg.at<K>(o_rk)) + rstart[i];
        x.n = pcount[i];
        x.tile0 = rtiles;
        rtiles += ceil_div(x.n, kTile);
        rj.push_back(x);
      }
    TJ_CUDA(put_small(stg.at<RadixJob<K>>(o_rjobs), rj.data(), rj.size() * sizeof(RadixJob<K>), st));
    TJ_CUDA(cudaMemsetAsync(stg.at<KeyStats>(o_range), 0xFF, 4 * sizeof(KeyStats), st));
    tr.begin("stats", w * (double)rtiles * kTile);
    TJ_CUDA(launch_stats<K>(stg.at<RadixJob<K>>(o_rjobs), 4, rtiles, stg.at<KeyStats>(o_range), st));
    tr.end();
    KeyStats hr[4];
    TJ_CUDA(get_small(hr, stg.at<KeyStats>(o_range), sizeof(hr), st));
    TJ_CUDA(sync_stream(st));
    unsigned long long mn = ~0ull, mx = 0ull;
    for (int i = 0; i < 4; ++i) {  // empty jobs keep 0xFF..: no effect on either
      mn = std::min(mn, hr[i].min_u);
      mx = std::max(mx, ~hr[i].max_u);
    }
    lo = key_of<K>(mn);
    hi = key_of<K>(mx);
    stats.key_bits = bitlen(range_of<K>(lo, hi));
  }
  {
    int64_t tot[2] = {0, 0}, maxrows = 0;
    for (int j = 0; j < nparts; ++j) {
      tot[0] += pcount[(size_t)j];
      tot[1] += pcount[(size_t)nparts + j];
      maxrows = std::max<int64_t>(maxrows, pcount[(size_t)j] + pcount[(size_t)nparts + j]);
    }
    if (tot[0] != nr || tot[1] != ns) return set_err(TJ_ERR_INTERNAL, "route counts do not add up");
    stats.max_partition = maxrows;
    stats.balance = (double)maxrows * nparts / (double)std::max<int64_t>(1, nr + ns);
  }

  // ---- 4. batches: a plan per batch ----
  // A batch whose key range spans kFKeyBits to kFKeyBits + kFMaxMsdBits bits
  // is joined by the partition-resident phase: one MSD pass cuts it into
  // sub-batches of kFKeys key values, which are sorted and aligned on chip
  // (tj_fused.cu) -- unless one of them holds more R rows than fit on chip
  // (many duplicate R keys), which the key counts show after the MSD
  // histogram.  A batch of a single key value (a heavy key the cuts
  // isolate) pairs every R row with every S row: k_cross streams its pairs.
  // Other batches are sorted by LSD passes and aligned by k_join.
  struct Part {
    int64_t r0, nr, s0, ns;
    K lo, hi;
    Plan plan;    // LSD plan (or, fused, the MSD pass: its only digit)
    Plan lsd;     // the LSD plan, kept for a fused batch that falls back
    bool fused;
    bool cross;   // one key value: pairs streamed by k_cross
    int m;        // fused: MSD digit bits
    int64_t items, kbt, kbs;  // fused: items, multi-tile tiles and sub-batches
    int64_t ws;   // working set without the look-back words
    int64_t lb;   // look-back bytes of one pass
    int np;       // passes (at least 1)
    size_t hist_at;  // its histograms in the tables block (R side, then S side)
    int fj;          // fused: index of its FusedJob
  };
  std::vector<Part> P;
  size_t hist_words_all = 0;
  int n_fused = 0;
  // histogram words of one side of a batch: room for either plan's (the R
  // side's at hist_at, the S side's after it)
  auto hist_half = [](const Part& q) {
    return std::max((size_t)std::max(1, q.lsd.passes) << q.lsd.max_bits,
                    q.fj >= 0 ? (size_t)1 << q.m : (size_t)0);
  };
  for (int j = 0; j < nparts; ++j) {
    Part q = {};
    q.nr = pcount[(size_t)j];
    q.ns = pcount[(size_t)nparts + j];
    q.r0 = rstart[(size_t)j];
    q.s0 = rstart[(size_t)nparts + j];
    if (q.nr == 0 || q.ns == 0) continue;
    q.lo = j == 0 ? lo : std::max(lo, cuts[(size_t)j - 1]);
    q.hi = j == ncuts ? hi : std::min(hi, (K)(cuts[(size_t)j] - 1));
    q.lsd = make_plan(lo_bits<K>(q.lo), range_of<K>(q.lo, q.hi), false, maxd, -1, q.nr + q.ns);
    const int bits = q.lsd.key_bits;
    // (narrower batches -- a heavy key's own batch above all -- need no sort
    // or few passes: k_join aligns them directly)
    // (an MSD digit wider than the preferred one only for batches whose
    // sub-batches still average 1024 rows: smaller ones join faster by LSD
    // -- measured on C1 at Zipf 1.2, about 1800 rows, and C2's 1024
    // batches, about 500)
    q.fused = o.fused && bits >= kFMinBits && bits <= kFKeyBits + kFMaxMsdBits &&
              (bits <= kFKeyBits + kFPreferMsdBits ||
               q.nr + q.ns >= ((int64_t)1024 << (bits - kFKeyBits)));
    q.cross = o.fused && q.lo == q.hi;
    q.m = q.fused ? std::max(0, bits - kFKeyBits) : 0;
    q.fj = q.fused ? n_fused++ : -1;
    if (q.fused) {
      q.plan = Plan();
      q.plan.lo = lo_bits<K>(q.lo);
      q.plan.key_bits = bits;
      if (q.m > 0) {
        q.plan.passes = 1;
        q.plan.shift[0] = kFKeyBits;
        q.plan.bits[0] = q.m;
        q.plan.max_bits = q.m;
      }
    } else {
      q.plan = q.lsd;
    }
    q.hist_at = hist_words_all;
    hist_words_all += 2 * hist_half(q);
    P.push_back(q);
  }
  // working set of a batch on the LSD path: one sort buffer (the passes
  // alternate between it and the batch's routed copy), one look-back region
  // per pass (a group keeps as many as its deepest batch), join tile state
  // (tile descriptors, chained words, tile map), the radix tile map
  auto plan_lsd = [&](Part& q) {
    q.fused = false;
    q.plan = q.lsd;
    const int64_t bins = (int64_t)1 << q.plan.max_bits;
    const int64_t rtiles = ceil_div(q.nr, kTile) + ceil_div(q.ns, kTile);
    q.np = std::max(1, q.plan.passes);
    q.lb = rtiles * bins * 4;
    q.ws = (int64_t)std::min(q.plan.passes, 1) * (q.nr + q.ns) * 2 * (int64_t)sizeof(K) +
           ceil_div(q.ns, kJTile) * (int64_t)(sizeof(JTile<K>) + 12) + rtiles * 4 + 4096;
  };
  // ... and on the fused path: the MSD pass's output, its look-back words and
  // tile map, the items (descriptor and chained word), the multi-tile count
  // vectors and totals, the job descriptor
  auto plan_fused = [&](Part& q) {
    const int64_t rtiles = ceil_div(q.nr, kTile) + ceil_div(q.ns, kTile);
    q.np = 1;
    q.lb = q.m > 0 ? rtiles * ((int64_t)1 << q.m) * 4 : 0;
    // (+ the layout's minimum of one count vector and one totals slot and its
    // 256-byte alignment of each of about a dozen arrays)
    q.ws = (q.m > 0 ? (q.nr + q.ns) * 2 * (int64_t)sizeof(K) + rtiles * 4 : 0) +
           q.items * (int64_t)(sizeof(FItem) + 8) +
           (q.kbt + q.kbs + 2) * (int64_t)kFKeys * 4 + (int64_t)sizeof(FusedJob<K>) + 8192;
  };
  for (auto& q : P)
    if (!q.fused) plan_lsd(q);
  // ... and a single-key batch: no buffers (its job sits in the tables)
  for (auto& q : P)
    if (q.cross) {
      q.ws = 4096;
      q.lb = 0;
      q.np = 1;
    }
  // tables: histogram-pass jobs and group jobs (radix), join jobs, fused jobs
  // and their counts, histograms, output bases (one more than groups; at most
  // one group per batch)
  const size_t rj1 = P.size() * 2 * sizeof(RadixJob<K>);
  const size_t t_rj = 0, t_rjh = t_rj + rj1, t_jj = t_rjh + rj1;
  const size_t t_cj = (t_jj + P.size() * sizeof(JoinJob<K>) + 255) & ~(size_t)255;
  const size_t t_fj = (t_cj + P.size() * sizeof(CrossJob<K>) + 255) & ~(size_t)255;
  const size_t t_info = (t_fj + std::max<size_t>(1, (size_t)n_fused) * sizeof(FusedJob<K>) + 255) &
                        ~(size_t)255;
  const size_t t_hist = (t_info + std::max<size_t>(1, (size_t)n_fused) * 4 * sizeof(int64_t) + 255) &
                        ~(size_t)255;
  const size_t t_base = (t_hist + hist_words_all * 4 + 255) & ~(size_t)255;
  const size_t tbl_bytes = t_base + (P.size() + 1) * sizeof(int64_t);
  const int64_t fixed = control + (int64_t)tbl_bytes + 4096;
  const int64_t room = budget ? (int64_t)budget - fixed : INT64_MAX;
  if (room <= 0)
    return set_err(TJ_ERR_BUDGET, "budget %zu below the join's tables and control (%lld bytes)",
                   budget, (long long)fixed);
  rlb.release();
  Block tbl;
  TJ_CUDA(tbl.alloc(tbl_bytes + 256, st));
  uint32_t* d_hist_all = reinterpret_cast<uint32_t*>(tbl.p + t_hist);
  RadixJob<K>* d_rj_all = reinterpret_cast<RadixJob<K>*>(tbl.p + t_rj);
  RadixJob<K>* d_rjh_all = reinterpret_cast<RadixJob<K>*>(tbl.p + t_rjh);
  JoinJob<K>* d_jj_all = reinterpret_cast<JoinJob<K>*>(tbl.p + t_jj);
  CrossJob<K>* d_cj_all = reinterpret_cast<CrossJob<K>*>(tbl.p + t_cj);
  FusedJob<K>* d_fj_all = reinterpret_cast<FusedJob<K>*>(tbl.p + t_fj);
  int64_t* d_info = reinterpret_cast<int64_t*>(tbl.p + t_info);
  int64_t* d_gbase = reinterpret_cast<int64_t*>(tbl.p + t_base);
  TJ_CUDA(cudaMemsetAsync(tbl.p + t_hist, 0, tbl_bytes - t_hist, st));

  // ---- 5. digit histograms of every batch in one launch ----
  // (the routed copies: LSD digits, or the MSD digit of a fused batch)
  auto batch_side = [&](const Part& q, int side, K** k0, K** v0) {
    *k0 = side ? stg.at<K>(o_sk) + q.s0 : stg.at<K>(o_rk) + q.r0;
    *v0 = side ? stg.at<K>(o_sv) + q.s0 : stg.at<K>(o_rv) + q.r0;
    return side ? q.ns : q.nr;
  };
  auto hist_jobs = [&](bool fused_only_lsd, std::vector<RadixJob<K>>& out, int64_t* tiles) {
    out.clear();
    *tiles = 0;
    for (auto& q : P) {
      if (fused_only_lsd && (q.fused || q.fj < 0)) continue;  // demoted fused batches only
      if (q.plan.passes == 0) continue;
      for (int side = 0; side < 2; ++side) {
        RadixJob<K> x;
        memset(&x, 0, sizeof(x));
        K* k0;
        K* v0;
        x.n = batch_side(q, side, &k0, &v0);
        x.keys = k0;
        set_job_plan(x, q.plan);
        x.hist_stride = 1 << q.plan.max_bits;
        x.hist = d_hist_all + q.hist_at + (side ? hist_half(q) : 0);
        x.tile0 = *tiles;
        *tiles += ceil_div(x.n, kTile);
        out.push_back(x);
      }
    }
  };
  int maxp = 0;
  for (auto& q : P) maxp = std::max(maxp, q.plan.passes);
  std::vector<RadixJob<K>> all_rjh;
  int64_t htiles = 0;
  hist_jobs(false, all_rjh, &htiles);
  if (!all_rjh.empty()) {
    TJ_CUDA(put_small(d_rjh_all, all_rjh.data(), all_rjh.size() * sizeof(RadixJob<K>), st));
    tr.begin("histogram", w * (double)(nr + ns));
    TJ_CUDA(launch_histogram<K>(d_rjh_all, (int)all_rjh.size(), htiles, st));
    tr.end();
    TJ_CUDA(launch_digit_scan<K>(d_rjh_all, (int)all_rjh.size(), maxp, st));
  }
  // fused batches: items and sub-batch sizes from the MSD counts (one read)
  std::vector<FusedJob<K>> fj((size_t)n_fused);
  if (n_fused > 0) {
    for (auto& q : P) {
      if (q.fj < 0) continue;
      FusedJob<K>& f = fj[(size_t)q.fj];
      memset(&f, 0, sizeof(f));
      f.hr = q.m > 0 ? d_hist_all + q.hist_at : nullptr;
      f.hs = q.m > 0 ? d_hist_all + q.hist_at + hist_half(q) : nullptr;
      f.nr = q.nr;
      f.ns = q.ns;
      f.lo = lo_bits<K>(q.lo);
      f.m = q.m;
    }
    TJ_CUDA(put_small(d_fj_all, fj.data(), fj.size() * sizeof(FusedJob<K>), st));
    TJ_CUDA(launch_fused_info<K>(d_fj_all, n_fused, d_info, st));
    std::vector<int64_t> info((size_t)n_fused * 4);
    TJ_CUDA(get_small(info.data(), d_info, info.size() * sizeof(int64_t), st));
    TJ_CUDA(sync_stream(st));
    bool demoted = false;
    for (auto& q : P) {
      if (q.fj < 0) continue;
      const int64_t* in = info.data() + (size_t)q.fj * 4;
      if (in[3] > kFCapR) {  // an R sub-batch does not fit on chip: LSD path
        plan_lsd(q);
        demoted = true;
        continue;
      }
      q.items = in[0];
      q.kbt = in[1];
      q.kbs = in[2];
      plan_fused(q);
    }
    if (demoted) {  // their LSD digit histograms
      std::vector<RadixJob<K>> dj;
      int64_t dt = 0;
      hist_jobs(true, dj, &dt);
      for (auto& q : P)
        if (!q.fused && q.fj >= 0)
          TJ_CUDA(cudaMemsetAsync(d_hist_all + q.hist_at, 0, 2 * hist_half(q) * 4, st));
      if (!dj.empty()) {
        RadixJob<K>* d_dj = d_rj_all;  // the group jobs are written later
        int dmaxp = 0;
        for (auto& q : P)
          if (!q.fused && q.fj >= 0) dmaxp = std::max(dmaxp, q.plan.passes);
        TJ_CUDA(put_small(d_dj, dj.data(), dj.size() * sizeof(RadixJob<K>), st));
        TJ_CUDA(launch_histogram<K>(d_dj, (int)dj.size(), dt, st));
        TJ_CUDA(launch_digit_scan<K>(d_dj, (int)dj.size(), dmaxp, st));
        maxp = std::max(maxp, dmaxp);
      }
    }
  }
  {
    int nf = 0;
    for (auto& q : P) nf += q.fused;
    stats.fused_batches = nf;
  }

  // ---- 6. groups: consecutive batches whose working set fits ----
  // A group holds runs of LSD and fused batches in key order.  Its working
  // set: every batch's buffers and tables, the LSD batches' look-back words
  // once per pass of the deepest one, the fused batches' MSD look-back words.
  // When the budget needs more than one group, groups are planned against
  // half of it and alternate between two streams (lanes), each with its own
  // half.
  std::vector<std::pair<size_t, size_t>> groups;  // [first, last) into P
  int64_t ws_max = 0;
  auto need_of = [&](size_t i) { return P[i].ws + P[i].lb * P[i].np; };
  auto make_groups = [&](int64_t lim) -> int64_t {  // -1, or a batch that needs more
    groups.clear();
    ws_max = 0;
    for (size_t i = 0; i < P.size();) {
      if (need_of(i) > lim) return (int64_t)i;
      size_t j = i;
      int64_t ws = 0, lb_lsd = 0, lb_msd = 0, acc = 0;
      int np = 1;
      while (j < P.size()) {
        const Part& q = P[j];
        const int np2 = q.fused ? np : std::max(np, q.np);
        const int64_t l2 = lb_lsd + (q.fused ? 0 : q.lb), m2 = lb_msd + (q.fused ? q.lb : 0);
        const int64_t acc2 = ws + q.ws + l2 * np2 + m2;
        if (acc2 > lim) break;
        ws += q.ws, lb_lsd = l2, lb_msd = m2, np = np2, acc = acc2, ++j;
      }
      groups.push_back({i, j});
      ws_max = std::max(ws_max, acc);
      i = j;
    }
    return -1;
  };
  {
    const int64_t bad = make_groups(room);
    if (bad >= 0)
      return set_err(TJ_ERR_BUDGET,
                     "batch of keys [%lld, %lld] needs %lld bytes of working set, budget "
                     "leaves %lld (raise the budget or the number of batches)",
                     (long long)P[(size_t)bad].lo, (long long)P[(size_t)bad].hi,
                     (long long)need_of((size_t)bad), (long long)room);
  }
  int lanes = 1;
  if (groups.size() > 1) {
    const auto one = groups;
    const int64_t one_max = ws_max;
    if (make_groups(room / 2) < 0) {
      lanes = 2;
    } else {
      groups = one;
      ws_max = one_max;
    }
  }
  stats.groups = (int)groups.size();
  stats.lanes = lanes;
  const size_t lane_bytes = ((size_t)std::max<int64_t>(ws_max, 256) + 255) & ~(size_t)255;
  const int64_t wk_bytes = (int64_t)(lane_bytes * (size_t)lanes);
  stats.scratch_peak = control + std::max<int64_t>(lb_max, wk_bytes + (int64_t)tbl_bytes);
  Block wk;
  TJ_CUDA(wk.alloc((size_t)wk_bytes, st));

  // ---- 7. group plans: job tables ----
  // Group layout in the working block: the sort buffer (LSD) or MSD output
  // (fused) of every batch | one zeroed region (tile and item counters, the
  // LSD passes' look-back words, the MSD pass's, per run: chained join or
  // item words, count vectors, totals) | per run: join tile descriptors and
  // tile map, or items | the tile maps of the LSD passes and the MSD pass.
  // Runs: maximal stretches of batches of one kind (LSD, fused, single-key);
  // their last kernels run in key order, each from the output index the one
  // before it left.
  struct RunPlan {
    bool fused;
    bool cross;        // single-key batches (k_cross)
    int64_t pairs;     // cross: the run's pairs
    int64_t xblocks;   // cross: CTAs of k_cross
    size_t first, nj;  // batches [first, first + nj) of P
    size_t jj_at;      // LSD: join jobs in the table; fused: first FusedJob
    int64_t jt0, jtiles;  // LSD: its join tiles within the group's
    int64_t items;        // fused
    bool any_multi;
    double rows;
    size_t o_jlb, o_ilb, o_kbl, o_kbt, o_items;
    int base;  // index of its first output index in d_gbase
  };
  struct GroupPlan {
    size_t first, nj;
    size_t rj_lsd_at, rj_msd_at;  // radix jobs in the table
    int nrj_lsd, nrj_msd;
    size_t o_zero, zero_bytes, o_cnt, o_lb, o_lbm, o_jt, o_jmap, o_tmap, o_tmapm;
    size_t lb_words, lbm_words;
    int64_t tiles, tilesm, jtiles;
    int P, maxbits, maxbitsm, ipt, iptm, lane;
    double rows, msd_rows, prow[kMaxPasses];
    std::vector<RunPlan> runs;
  };
  std::vector<RadixJob<K>> all_rj;
  std::vector<JoinJob<K>> all_jj;
  std::vector<CrossJob<K>> all_cj;
  std::vector<GroupPlan> plans;
  int n_bases = 0;
  for (auto& g : groups) {
    GroupPlan gp = {};
    gp.lane = (int)(plans.size() % (size_t)lanes);
    const View lw{wk.p + (size_t)gp.lane * lane_bytes};  // the group's lane of wk
    gp.first = g.first;
    gp.nj = g.second - g.first;
    const size_t nj = gp.nj;
    for (size_t i = 0; i < nj;) {  // runs
      RunPlan r = {};
      r.fused = P[g.first + i].fused;
      r.cross = P[g.first + i].cross;
      r.first = g.first + i;
      size_t j = i;
      while (j < nj && P[g.first + j].fused == r.fused && P[g.first + j].cross == r.cross) ++j;
      r.nj = j - i;
      r.base = n_bases++;
      gp.runs.push_back(r);
      i = j;
    }
    Carve gc;
    std::vector<size_t> o_buf(nj * 4, 0);
    for (size_t i = 0; i < nj; ++i) {
      const Part& q = P[g.first + i];
      if (q.plan.passes > 0) {
        o_buf[i * 4 + 0] = gc.add<K>((size_t)q.nr);
        o_buf[i * 4 + 1] = gc.add<K>((size_t)q.nr);
        o_buf[i * 4 + 2] = gc.add<K>((size_t)q.ns);
        o_buf[i * 4 + 3] = gc.add<K>((size_t)q.ns);
      }
    }
    // onesweep tiles of the LSD passes and of the MSD pass: the wider one
    // when every digit of the launch is narrow
    for (size_t i = 0; i < nj; ++i) {
      const Part& q = P[g.first + i];
      if (q.fused)
        gp.maxbitsm = std::max(gp.maxbitsm, q.plan.max_bits);
      else
        gp.maxbits = std::max(gp.maxbits, q.plan.max_bits);
    }
    gp.ipt = gp.maxbits <= kWideBits ? kItemsWide : kItems;
    gp.iptm = gp.maxbitsm <= kWideBits ? kItemsWide : kItems;
    const int64_t otile = (int64_t)kSortThreads * gp.ipt, otilem = (int64_t)kSortThreads * gp.iptm;
    std::vector<size_t> lb_at(nj * 2);
    for (size_t i = 0; i < nj; ++i) {
      const Part& q = P[g.first + i];
      const size_t bins = (size_t)1 << q.plan.max_bits;
      for (int side = 0; side < 2; ++side) {
        const int64_t n = side ? q.ns : q.nr;
        if (q.plan.passes == 0) continue;
        if (q.fused) {
          lb_at[i * 2 + side] = gp.lbm_words;
          gp.lbm_words += (size_t)ceil_div(n, otilem) * bins;
        } else {
          lb_at[i * 2 + side] = gp.lb_words;
          gp.lb_words += (size_t)ceil_div(n, otile) * bins;
        }
      }
      gp.rows += (double)(q.nr + q.ns);
      if (q.fused) {
        if (q.plan.passes > 0) gp.msd_rows += (double)(q.nr + q.ns);
      } else {
        gp.P = std::max(gp.P, q.plan.passes);
        for (int p = 0; p < q.plan.passes; ++p) gp.prow[p] += (double)(q.nr + q.ns);
      }
    }
    for (auto& r : gp.runs) {
      for (size_t i = 0; i < r.nj; ++i) {
        const Part& q = P[r.first + i];
        r.rows += (double)(q.nr + q.ns);
        if (r.fused) {
          r.items += q.items;
          r.any_multi |= q.kbt > 0;
        }
      }
      if (!r.fused && !r.cross) {
        r.jt0 = gp.jtiles;
        for (size_t i = 0; i < r.nj; ++i) r.jtiles += ceil_div(P[r.first + i].ns, kJTile);
        gp.jtiles += r.jtiles;
      }
    }
    // zeroed region: counters (LSD passes, the MSD pass, one per run), the
    // look-back words, per run its chained words and count vectors
    gp.o_cnt = gc.add<uint32_t>(kMaxPasses + 1 + gp.runs.size());
    gp.o_zero = gp.o_cnt;
    gp.o_lb = gc.add<uint32_t>(std::max<size_t>(gp.lb_words, 1) * (size_t)std::max(1, gp.P));
    gp.o_lbm = gc.add<uint32_t>(std::max<size_t>(gp.lbm_words, 1));
    for (auto& r : gp.runs) {
      if (r.fused) {
        int64_t kbt = 0, kbs = 0;
        for (size_t i = 0; i < r.nj; ++i) {
          kbt += P[r.first + i].kbt;
          kbs += P[r.first + i].kbs;
        }
        r.o_ilb = gc.add<uint64_t>((size_t)std::max<int64_t>(r.items, 1));
        r.o_kbl = gc.add<uint32_t>((size_t)std::max<int64_t>(kbt, 1) * kFKeys);
        r.o_kbt = gc.add<uint32_t>((size_t)std::max<int64_t>(kbs, 1) * kFKeys);
      } else if (!r.cross) {
        r.o_jlb = gc.add<uint64_t>((size_t)std::max<int64_t>(r.jtiles, 1));
      }
    }
    gp.zero_bytes = gc.off - gp.o_zero;
    // radix jobs (LSD passes, then the MSD pass), join jobs, fused jobs
    std::vector<RadixJob<K>> rj_lsd, rj_msd;
    std::vector<const K*> res(nj * 4);
    for (size_t i = 0; i < nj; ++i) {
      const Part& q = P[g.first + i];
      for (int side = 0; side < 2; ++side) {
        K* k0;
        K* v0;
        const int64_t n = batch_side(q, side, &k0, &v0);
        res[i * 4 + 2 * side] = k0;
        res[i * 4 + 2 * side + 1] = v0;
        if (q.plan.passes == 0) continue;
        RadixJob<K> x;
        memset(&x, 0, sizeof(x));
        x.keys = k0;
        x.n = n;
        set_job_plan(x, q.plan);
        x.hist_stride = 1 << q.plan.max_bits;
        x.hist = d_hist_all + q.hist_at + (side ? hist_half(q) : 0);
        K* ak = lw.at<K>(o_buf[i * 4 + 2 * side]);
        K* av = lw.at<K>(o_buf[i * 4 + 2 * side + 1]);
        const K** rk = &res[i * 4 + 2 * side];
        const K** rv = &res[i * 4 + 2 * side + 1];
        if (q.fused) {
          // the MSD pass: routed copy -> the batch's MSD output
          x.lookback = lw.at<uint32_t>(gp.o_lbm) + lb_at[i * 2 + side];
          x.lb_stride = (int64_t)gp.lbm_words;
          set_job_buffers(x, k0, v0, ak, av, ak, av, rk, rv);
          x.tile0 = gp.tilesm;
          gp.tilesm += ceil_div(n, otilem);
          rj_msd.push_back(x);
        } else {
          // LSD passes alternate: routed copy -> buffer -> routed copy -> ...
          x.lookback = lw.at<uint32_t>(gp.o_lb) + lb_at[i * 2 + side];
          x.lb_stride = (int64_t)gp.lb_words;
          set_job_buffers(x, k0, v0, ak, av, k0, v0, rk, rv);
          x.tile0 = gp.tiles;
          gp.tiles += ceil_div(n, otile);
          rj_lsd.push_back(x);
        }
      }
    }
    gp.rj_lsd_at = all_rj.size();
    gp.nrj_lsd = (int)rj_lsd.size();
    all_rj.insert(all_rj.end(), rj_lsd.begin(), rj_lsd.end());
    gp.rj_msd_at = all_rj.size();
    gp.nrj_msd = (int)rj_msd.size();
    all_rj.insert(all_rj.end(), rj_msd.begin(), rj_msd.end());
    for (auto& r : gp.runs) {
      if (r.fused) {
        r.jj_at = (size_t)P[r.first].fj;
        int64_t item0 = 0, kbt0 = 0, kbs0 = 0;
        for (size_t i = 0; i < r.nj; ++i) {
          const Part& q = P[r.first + i];
          const size_t li = r.first + i - g.first;
          FusedJob<K>& f = fj[(size_t)q.fj];
          f.rk = res[li * 4 + 0];
          f.rv = res[li * 4 + 1];
          f.sk = res[li * 4 + 2];
          f.sv = res[li * 4 + 3];
          f.item0 = item0;
          f.kbt0 = kbt0;
          f.kbs0 = kbs0;
          item0 += q.items;
          kbt0 += q.kbt;
          kbs0 += q.kbs;
        }
        r.o_items = gc.add<FItem>((size_t)std::max<int64_t>(r.items, 1));
      } else if (r.cross) {
        r.jj_at = all_cj.size();
        for (size_t i = 0; i < r.nj; ++i) {
          const Part& q = P[r.first + i];
          const size_t li = r.first + i - g.first;
          CrossJob<K> x;
          x.rv = res[li * 4 + 1];
          x.sv = res[li * 4 + 3];
          x.nr = q.nr;
          x.ns = q.ns;
          x.off = r.pairs;
          x.blk0 = r.xblocks;
          r.pairs += q.nr * q.ns;
          r.xblocks += ceil_div(q.nr * q.ns, kXPairs);
          all_cj.push_back(x);
        }
        // beyond the caller's capacity: one CTA, which only passes the base on
        if (r.pairs > cap) r.xblocks = 1;
      } else {
        r.jj_at = all_jj.size();
        int64_t jt = r.jt0;
        for (size_t i = 0; i < r.nj; ++i) {
          const Part& q = P[r.first + i];
          const size_t li = r.first + i - g.first;
          JoinJob<K> y;
          y.rk = res[li * 4 + 0];
          y.rv = res[li * 4 + 1];
          y.nr = q.nr;
          y.sk = res[li * 4 + 2];
          y.sv = res[li * 4 + 3];
          y.ns = q.ns;
          y.tile0 = jt;
          jt += ceil_div(q.ns, kJTile);
          all_jj.push_back(y);
        }
      }
    }
    gp.o_jt = gc.add<JTile<K>>((size_t)std::max<int64_t>(gp.jtiles, 1));
    gp.o_jmap = gc.add<int32_t>((size_t)std::max<int64_t>(gp.jtiles, 1));
    gp.o_tmap = gc.add<int32_t>((size_t)std::max<int64_t>(gp.tiles, 1));
    gp.o_tmapm = gc.add<int32_t>((size_t)std::max<int64_t>(gp.tilesm, 1));
    if (gc.off > lane_bytes)
      return set_err(TJ_ERR_INTERNAL, "group needs %zu bytes, its lane has %zu", gc.off,
                     lane_bytes);
    stats.digit_bits = std::max(stats.digit_bits, std::max(gp.maxbits, gp.maxbitsm));
    plans.push_back(std::move(gp));
  }
  if (all_rj.size() * sizeof(RadixJob<K>) > rj1 || (size_t)n_bases > P.size())
    return set_err(TJ_ERR_INTERNAL, "group tables do not add up");
  // one upload of the group tables (run r writes from base[r] on and its
  // last join tile or item sets base[r + 1])
  {
    unsigned char* h = nullptr;
    TJ_CUDA(pinned_staging(t_hist, &h));
    memcpy(h + t_rj, all_rj.data(), all_rj.size() * sizeof(RadixJob<K>));
    memcpy(h + t_jj, all_jj.data(), all_jj.size() * sizeof(JoinJob<K>));
    memcpy(h + t_cj, all_cj.data(), all_cj.size() * sizeof(CrossJob<K>));
    if (n_fused > 0) memcpy(h + t_fj, fj.data(), fj.size() * sizeof(FusedJob<K>));
    TJ_CUDA(put_small(tbl.p + t_rj, h + t_rj, t_rjh - t_rj, st));
    TJ_CUDA(put_small(tbl.p + t_jj, h + t_jj, t_info - t_jj, st));
    TJ_CUDA(cudaEventRecord(pinned_event(), st));  // the staging buffer is busy until here
    TJ_CUDA(cudaMemsetAsync(d_gbase, 0, (P.size() + 1) * sizeof(int64_t), st));
  }

  // ---- 8. per group: the LSD passes and the MSD pass of its batches, the
  //         LSD runs' tile ranges and fused runs' items, then each run's
  //         join (k_join or k_fused_join) in key order ----
  // With two lanes, group g runs on lane g % 2's stream; a group's first join
  // waits for the previous group's last (it writes from the base that one
  // leaves).
  cudaStream_t lane_st[2] = {st, st};
  SideStream* side = nullptr;
  JoinBack back;
  if (lanes > 1) {
    TJ_CUDA(side_stream(&side));
    lane_st[1] = side->s;
    TJ_CUDA(cudaEventRecord(side->ev[0], st));  // tables, histograms, scans
    TJ_CUDA(cudaStreamWaitEvent(side->s, side->ev[0], 0));
    back.st = st;
    back.side = side->s;
    back.ev = side->ev[2];
  }
  for (size_t g = 0; g < plans.size(); ++g) {
    const GroupPlan& gp = plans[g];
    const cudaStream_t gs = lane_st[gp.lane];
    const View lw{wk.p + (size_t)gp.lane * lane_bytes};
    uint32_t* d_gcnt = lw.at<uint32_t>(gp.o_cnt);
    // One lane: every kernel traced.  Two lanes: the launches of the lanes
    // overlap, so a group is traced as a whole ("group/lanes": its passes and
    // joins, launches counted) with two events instead of two per kernel.
    const bool whole = lanes > 1;
    if (whole) {
      double by = 2.0 * w * gp.rows + 4.0 * w * gp.msd_rows;  // join input, MSD pass
      for (int p = 0; p < gp.P; ++p) by += 4.0 * w * gp.prow[p];
      tr.begin("group/lanes", by, gs, gp.P + 2 + 2 * (int)gp.runs.size());
    }
    TJ_CUDA(cudaMemsetAsync(lw.p + gp.o_zero, 0, gp.zero_bytes, gs));
    // the join jobs of the LSD runs are consecutive in the table
    size_t jj0 = 0;
    int lsd_jobs = 0;
    for (auto& r : gp.runs)
      if (!r.fused && !r.cross) {
        if (lsd_jobs == 0) jj0 = r.jj_at;
        lsd_jobs += (int)r.nj;
      }
    JoinJob<K>* d_gjj = d_jj_all + jj0;
    if (gp.nrj_lsd > 0) {
      RadixJob<K>* d_gj = d_rj_all + gp.rj_lsd_at;
      TJ_CUDA(launch_group_maps<K>(d_gj, gp.nrj_lsd, lw.at<int32_t>(gp.o_tmap), d_gjj, lsd_jobs,
                                   lw.at<int32_t>(gp.o_jmap), gs, kSortThreads * gp.ipt));
      for (int p = 0; p < gp.P; ++p) {
        if (!whole) tr.begin("onesweep", 4.0 * w * gp.prow[p], gs);
        TJ_CUDA(launch_onesweep<K>(d_gj, gp.nrj_lsd, gp.tiles, p, gp.maxbits, kModeSort,
                                   d_gcnt + p, d_err, gs, lw.at<int32_t>(gp.o_tmap), gp.ipt));
        if (!whole) tr.end();
      }
    } else if (gp.jtiles > 0) {  // LSD runs of single-key batches only: the join map
      TJ_CUDA(launch_group_maps<K>(nullptr, 0, nullptr, d_gjj, lsd_jobs,
                                   lw.at<int32_t>(gp.o_jmap), gs));
    }
    if (gp.nrj_msd > 0) {
      RadixJob<K>* d_gm = d_rj_all + gp.rj_msd_at;
      TJ_CUDA(launch_group_maps<K>(d_gm, gp.nrj_msd, lw.at<int32_t>(gp.o_tmapm), nullptr, 0,
                                   nullptr, gs, kSortThreads * gp.iptm));
      if (!whole) tr.begin("msd", 4.0 * w * gp.msd_rows, gs);
      TJ_CUDA(launch_onesweep<K>(d_gm, gp.nrj_msd, gp.tilesm, 0, gp.maxbitsm, kModeSort,
                                 d_gcnt + kMaxPasses, d_err, gs, lw.at<int32_t>(gp.o_tmapm),
                                 gp.iptm));
      if (!whole) tr.end();
    }
    if (gp.jtiles > 0)
      TJ_CUDA(launch_tile_ranges<K>(d_gjj, lsd_jobs, gp.jtiles, lw.at<JTile<K>>(gp.o_jt), gs,
                                    lw.at<int32_t>(gp.o_jmap)));
    for (auto& r : gp.runs)
      if (r.fused)
        TJ_CUDA(launch_fused_prep<K>(d_fj_all + r.jj_at, (int)r.nj, lw.at<FItem>(r.o_items),
                                     r.items, r.any_multi, lw.at<uint32_t>(r.o_kbt), gs));
    if (lanes > 1 && g > 0) TJ_CUDA(cudaStreamWaitEvent(gs, side->ev[1], 0));
    for (size_t ri = 0; ri < gp.runs.size(); ++ri) {
      const RunPlan& r = gp.runs[ri];
      uint32_t* cnt = d_gcnt + kMaxPasses + 1 + ri;
      if (r.fused) {
        if (!whole) tr.begin("fused", 2.0 * w * r.rows, gs);
        if (r.items > 0) {
          TJ_CUDA(launch_fused_join<K>(d_fj_all + r.jj_at, lw.at<FItem>(r.o_items), r.items, cnt,
                                       lw.at<uint64_t>(r.o_ilb), lw.at<uint32_t>(r.o_kbl),
                                       lw.at<uint32_t>(r.o_kbt), out, cap, d_gbase + r.base,
                                       d_gbase + r.base + 1, d_err, gs));
        } else {  // no pairs in this run: the next one starts where it did
          TJ_CUDA(launch_copy_bytes(d_gbase + r.base + 1, d_gbase + r.base, sizeof(int64_t), gs));
        }
        if (!whole) tr.end();
      } else if (r.cross) {
        if (!whole) tr.begin("cross", w * (double)r.rows + 2.0 * w * (double)r.pairs, gs);
        TJ_CUDA(launch_cross<K>(d_cj_all + r.jj_at, (int)r.nj, r.xblocks, out, cap,
                                d_gbase + r.base, d_gbase + r.base + 1, r.pairs, gs));
        if (!whole) tr.end();
      } else {
        if (!whole) tr.begin("join", 2.0 * w * r.rows, gs);
        TJ_CUDA(launch_join<K>(r.jtiles, lw.at<JTile<K>>(gp.o_jt) + r.jt0,
                               lw.at<uint64_t>(r.o_jlb), cnt, out, cap, d_gbase + r.base, nullptr,
                               d_gbase + r.base + 1, d_err, gs));
        if (!whole) tr.end();
      }
    }
    if (whole) tr.end();
    // (the next group's wait is enqueued before this event is recorded again)
    if (lanes > 1) TJ_CUDA(cudaEventRecord(side->ev[1], gs));
  }
  back.now();
  stats.radix_passes = maxp;
  int64_t h_total = 0;
  int h_err = 0;
  TJ_CUDA(get_small(&h_total, d_gbase + n_bases, sizeof(int64_t), st));
  TJ_CUDA(get_small(&h_err, d_err, sizeof(int), st));
  TJ_CUDA(sync_stream(st));
  if (h_total <= cap && !plans.empty())
    tr.add_bytes(lanes > 1 ? "group/lanes" : (plans.back().runs.back().fused ? "fused" : "join"),
                 2.0 * w * (double)h_total);
  tr.flush();
  if (h_err) return set_err((tj_status)h_err, "device reported %d", h_err);
  *out_count = h_total;
  stats.learned = router + (fell_back ? 100 : 0);
  if (h_total > cap)
    return set_err(TJ_ERR_CAPACITY, "result has %lld pairs, capacity %lld", (long long)h_total,
                   (long long)cap);
  return TJ_OK;
}

// ---- sort ---------------------------------------------------------------------------
template <typename K>
tj_status sort_impl(K* keys, K* ids, int64_t n, cudaStream_t st) {
  tj_stats stats = {};
  stats.groups = 1;
  if (n <= 1) {
    g_stats = stats;
    return TJ_OK;
  }
  tj_status s = ensure_device();
  if (s != TJ_OK) return s;
  const int64_t tiles = ceil_div(n, kTile);
  Carve cc;
  const size_t o_jobs = cc.add<RadixJob<K>>(1);
  const size_t o_stats = cc.add<KeyStats>(1);
  const size_t o_misc = cc.add<int64_t>(32);
  Block ctl;
  TJ_CUDA(ctl.alloc(cc.off, st));
  RadixJob<K>* d_jobs = ctl.at<RadixJob<K>>(o_jobs);
  KeyStats* d_stats = ctl.at<KeyStats>(o_stats);
  int* d_err = ctl.at<int>(o_misc);
  uint32_t* d_counters = ctl.at<uint32_t>(o_misc + 16);

  RadixJob<K> hj;
  memset(&hj, 0, sizeof(hj));
  hj.keys = keys;
  hj.n = n;
  TJ_CUDA(cudaMemsetAsync(ctl.p + o_misc, 0, 32 * sizeof(int64_t), st));
  TJ_CUDA(cudaMemsetAsync(d_stats, 0xFF, sizeof(KeyStats), st));
  TJ_CUDA(put_small(d_jobs, &hj, sizeof(hj), st));
  Tracer tr(st);
  const double w = (double)sizeof(K);
  tr.begin("stats", w * n);
  TJ_CUDA(launch_stats<K>(d_jobs, 1, tiles, d_stats, st));
  tr.end();
  KeyStats hs;
  TJ_CUDA(get_small(&hs, d_stats, sizeof(hs), st));
  TJ_CUDA(sync_stream(st));
  tr.flush();
  Tracer tr2(st);
  const K lo = key_of<K>(hs.min_u), hi = key_of<K>(~hs.max_u);
  const Plan plan = make_plan(lo_bits<K>(lo), range_of<K>(lo, hi), /*even=*/true, max_digit_bits<K>());
  stats.key_bits = plan.key_bits;
  stats.radix_passes = plan.passes;
  stats.digit_bits = plan.max_bits;
  if (plan.passes == 0) {  // all keys equal: already sorted
    g_stats = stats;
    return TJ_OK;
  }
  const int64_t bins_max = (int64_t)1 << plan.max_bits;
  // onesweep tiles (narrow digits: the wider tile); the histogram keeps kTile
  const int items = plan.max_bits <= kWideBits ? kItemsWide : kItems;
  const int64_t otiles = ceil_div(n, (int64_t)kSortThreads * items);
  Carve bc;
  const size_t o_bk = bc.add<K>(n);
  const size_t o_bv = bc.add<K>(n);
  const size_t o_hist = bc.add<uint32_t>(kMaxPasses * kMaxBins);
  const size_t o_lb = bc.add<uint32_t>((size_t)otiles * bins_max);
  Block big;
  TJ_CUDA(big.alloc(bc.off, st));
  stats.scratch_peak = (int64_t)(bc.off + cc.off);
  set_job_plan(hj, plan);
  hj.hist_stride = kMaxBins;
  hj.hist = big.at<uint32_t>(o_hist);
  hj.lookback = big.at<uint32_t>(o_lb);
  const K* rk;
  const K* rv;
  // even number of passes: B, keys, B, keys, ... ends in the caller's arrays
  set_job_buffers(hj, keys, ids, big.at<K>(o_bk), big.at<K>(o_bv), keys, ids, &rk, &rv);
  TJ_CUDA(put_small(d_jobs, &hj, sizeof(hj), st));
  TJ_CUDA(cudaMemsetAsync(hj.hist, 0, kMaxPasses * kMaxBins * sizeof(uint32_t), st));
  tr2.begin("histogram", w * n);
  TJ_CUDA(launch_histogram<K>(d_jobs, 1, tiles, st));
  tr2.end();
  TJ_CUDA(launch_digit_scan<K>(d_jobs, 1, plan.passes, st));
  for (int p = 0; p < plan.passes; ++p) {
    TJ_CUDA(cudaMemsetAsync(hj.lookback, 0, (size_t)otiles * bins_max * sizeof(uint32_t), st));
    tr2.begin("onesweep", 4.0 * w * n);
    TJ_CUDA(launch_onesweep<K>(d_jobs, 1, otiles, p, plan.max_bits, false, d_counters + p, d_err,
                               st, nullptr, items));
    tr2.end();
  }
  int h_err = 0;
  TJ_CUDA(get_small(&h_err, d_err, sizeof(int), st));
  TJ_CUDA(sync_stream(st));
  tr2.flush();
  if (h_err) return set_err((tj_status)h_err, "device reported %d", h_err);
  if (rk != keys) return set_err(TJ_ERR_INTERNAL, "odd pass count in place");
  g_stats = stats;
  return TJ_OK;
}

// ---- multi-column sort ----------------------------------------------------------------
// Key statistics of every column first (one launch).  If the columns'
// significant bits fit one key of type K (without its sign bit), they are
// folded into it (k_0 highest), sorted once with the ids and unfolded.
// Otherwise stable LSD over the columns, the last one first: the row
// permutation idx starts as the identity; per column c, key[i] =
// cols[c][idx[i]] and (key, idx) is sorted stably by key, so rows equal in
// column c keep the order the later columns gave them; then every column and
// the ids are permuted by idx (column 0 is already sorted in `key`).
template <typename K>
tj_status sort_multi_impl(K* const* cols, int ncols, K* ids, int64_t n, int path,
                          cudaStream_t st) {
  tj_stats stats = {};
  stats.groups = 1;
  g_stats = stats;
  if (n <= 1 || ncols == 0) return TJ_OK;
  if (ncols > kGatherCols) return set_err(TJ_ERR_INVALID, "at most %d key columns", kGatherCols);
  tj_status s = ensure_device();
  if (s != TJ_OK) return s;
  int dev = 0, sms = 0;
  TJ_CUDA(cudaGetDevice(&dev));
  TJ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int64_t tiles = ceil_div(n, kTile);
  Carve c;
  const size_t o_jobs = c.add<RadixJob<K>>((size_t)ncols);
  const size_t o_stats = c.add<KeyStats>((size_t)ncols);
  const size_t o_idx = c.add<K>((size_t)n), o_key = c.add<K>((size_t)n),
               o_tmp = c.add<K>((size_t)n);
  Block blk;
  TJ_CUDA(blk.alloc(c.off, st));
  K* idx = blk.at<K>(o_idx);
  K* key = blk.at<K>(o_key);
  K* tmp = blk.at<K>(o_tmp);
  Tracer tr(st);
  const double w = (double)sizeof(K);
  // 1. key statistics of every column
  std::vector<RadixJob<K>> hj((size_t)ncols);
  for (int col = 0; col < ncols; ++col) {
    memset(&hj[(size_t)col], 0, sizeof(RadixJob<K>));
    hj[(size_t)col].keys = cols[col];
    hj[(size_t)col].n = n;
    hj[(size_t)col].tile0 = col * tiles;
  }
  TJ_CUDA(put_small(blk.at<RadixJob<K>>(o_jobs), hj.data(), hj.size() * sizeof(RadixJob<K>), st));
  TJ_CUDA(cudaMemsetAsync(blk.at<KeyStats>(o_stats), 0xFF, (size_t)ncols * sizeof(KeyStats), st));
  tr.begin("stats", w * n * ncols);
  TJ_CUDA(launch_stats<K>(blk.at<RadixJob<K>>(o_jobs), ncols, tiles * ncols,
                          blk.at<KeyStats>(o_stats), st));
  tr.end();
  std::vector<KeyStats> hs((size_t)ncols);
  TJ_CUDA(get_small(hs.data(), blk.at<KeyStats>(o_stats), hs.size() * sizeof(KeyStats), st));
  TJ_CUDA(sync_stream(st));
  tr.flush();
  PackArgs<K> pa;
  memset(&pa, 0, sizeof(pa));
  pa.n = ncols;
  int total_bits = 0;
  for (int col = ncols - 1; col >= 0; --col) {
    const K lo = key_of<K>(hs[(size_t)col].min_u), hi = key_of<K>(~hs[(size_t)col].max_u);
    const int b = bitlen(range_of<K>(lo, hi));
    pa.col[col] = cols[col];
    pa.lo[col] = lo;
    pa.bits[col] = b;
    pa.shift[col] = std::min(total_bits, 8 * (int)sizeof(K) - 1);
    total_bits += b;
  }
  stats.key_bits = total_bits;
  const bool fits = total_bits <= 8 * (int)sizeof(K) - 1;
  if (path == 2 && !fits)
    return set_err(TJ_ERR_INVALID, "%d key bits do not fit one %d-bit key", total_bits,
                   8 * (int)sizeof(K));
  if (fits && path != 1) {
    // 2a. one key: fold, sort with the ids (or a scratch array), unfold
    tr.begin("pack", 2.0 * w * n * ncols);
    TJ_CUDA(launch_pack<K>(pa, key, n, false, sms, st));
    tr.end();
    tr.flush();
    s = sort_impl<K>(key, ids ? ids : idx, n, st);
    if (s != TJ_OK) return s;
    tr.begin("pack", 2.0 * w * n * ncols);
    TJ_CUDA(launch_pack<K>(pa, key, n, true, sms, st));
    tr.end();
    stats.packed_keys = 1;
  } else {
    // 2b. one sort per column, carrying the row permutation
    TJ_CUDA(launch_iota<K>(idx, n, sms, st));
    for (int col = ncols - 1; col >= 0; --col) {
      tr.begin("gather", 3.0 * w * n);
      TJ_CUDA(launch_gather_idx<K>(cols[col], idx, key, n, sms, st));
      tr.end();
      tr.flush();
      s = sort_impl<K>(key, idx, n, st);
      if (s != TJ_OK) return s;
    }
    for (int col = 1; col < ncols; ++col) {
      tr.begin("gather", 3.0 * w * n);
      TJ_CUDA(launch_gather_idx<K>(cols[col], idx, tmp, n, sms, st));
      tr.end();
      TJ_CUDA(cudaMemcpyAsync(cols[col], tmp, (size_t)n * sizeof(K), cudaMemcpyDeviceToDevice, st));
    }
    TJ_CUDA(cudaMemcpyAsync(cols[0], key, (size_t)n * sizeof(K), cudaMemcpyDeviceToDevice, st));
    if (ids) {
      tr.begin("gather", 3.0 * w * n);
      TJ_CUDA(launch_gather_idx<K>(ids, idx, tmp, n, sms, st));
      tr.end();
      TJ_CUDA(cudaMemcpyAsync(ids, tmp, (size_t)n * sizeof(K), cudaMemcpyDeviceToDevice, st));
    }
    stats.groups = ncols;
  }
  TJ_CUDA(sync_stream(st));
  tr.flush();
  g_stats = stats;
  return TJ_OK;
}

// ---- batch of joins -------------------------------------------------------------------
// Job j joins R rows [r_off[j], r_off[j+1]) with S rows [s_off[j], s_off[j+1]).
// Radix jobs are laid out R_0, S_0, R_1, S_1, ...; every pair shares its own
// (lo, bits) and all pairs use the same pass count with per-pair digit widths.
// Everything after the statistics is captured into one CUDA graph.
template <typename K>
tj_status batch_impl(int64_t nj, const int64_t* r_off, const int64_t* s_off, const K* kr,
                     const K* ir, const K* ks, const K* is, K* out, int64_t cap,
                     int64_t* d_out_off, int64_t* out_count, cudaStream_t st, int digit_cap,
                     int items) {
  tj_stats stats = {};
  stats.groups = 1;
  const int tile = kSortThreads * items;
  stats.tile_rows = tile;
  stats.digit_cap = digit_cap;
  *out_count = 0;
  tj_status s = ensure_device();
  if (s != TJ_OK) return s;
  const int64_t R = r_off[nj], S = s_off[nj];
  std::vector<RadixJob<K>> hj((size_t)(2 * nj));
  memset(hj.data(), 0, hj.size() * sizeof(RadixJob<K>));
  int64_t tiles = 0;
  for (int64_t j = 0; j < nj; ++j) {
    for (int side = 0; side < 2; ++side) {
      RadixJob<K>& x = hj[(size_t)(2 * j + side)];
      const int64_t a = side ? s_off[j] : r_off[j];
      const int64_t n = (side ? s_off[j + 1] : r_off[j + 1]) - a;
      x.keys = (side ? ks : kr) + a;
      x.n = n;
      x.tile0 = tiles;
      tiles += ceil_div(n, tile);
    }
  }
  Carve cc;
  const size_t o_jobs = cc.add<RadixJob<K>>((size_t)(2 * nj));
  const size_t o_stats = cc.add<KeyStats>((size_t)(2 * nj));
  const size_t o_misc = cc.add<int64_t>(32);
  const size_t o_jj = cc.add<JoinJob<K>>((size_t)nj);
  Block ctl;
  TJ_CUDA(ctl.alloc(cc.off, st));
  RadixJob<K>* d_jobs = ctl.at<RadixJob<K>>(o_jobs);
  KeyStats* d_stats = ctl.at<KeyStats>(o_stats);
  int* d_err = ctl.at<int>(o_misc);
  uint32_t* d_counters = ctl.at<uint32_t>(o_misc + 16);
  int64_t* d_total = ctl.at<int64_t>(o_misc + 128);
  JoinJob<K>* d_jj = ctl.at<JoinJob<K>>(o_jj);
  TJ_CUDA(cudaMemsetAsync(ctl.p + o_misc, 0, 32 * sizeof(int64_t), st));
  TJ_CUDA(cudaMemsetAsync(d_stats, 0xFF, (size_t)(2 * nj) * sizeof(KeyStats), st));
  TJ_CUDA(put_small(d_jobs, hj.data(), hj.size() * sizeof(RadixJob<K>), st));
  TJ_CUDA(launch_stats<K>(d_jobs, (int)(2 * nj), tiles, d_stats, st, tile));
  std::vector<KeyStats> hs((size_t)(2 * nj));
  TJ_CUDA(get_small(hs.data(), d_stats, hs.size() * sizeof(KeyStats), st));
  TJ_CUDA(sync_stream(st));

  // per-pair ranges; pairs that cannot match are dropped from the batch
  std::vector<uint64_t> plo((size_t)nj, 0), prange((size_t)nj, 0);
  std::vector<char> live((size_t)nj, 0);
  int P = 0;
  for (int64_t j = 0; j < nj; ++j) {
    const RadixJob<K>& xr = hj[(size_t)(2 * j)];
    const RadixJob<K>& xs = hj[(size_t)(2 * j + 1)];
    if (xr.n == 0 || xs.n == 0) continue;
    const K min_r = key_of<K>(hs[(size_t)(2 * j)].min_u), max_r = key_of<K>(~hs[(size_t)(2 * j)].max_u);
    const K min_s = key_of<K>(hs[(size_t)(2 * j + 1)].min_u),
            max_s = key_of<K>(~hs[(size_t)(2 * j + 1)].max_u);
    if (max_r < min_s || max_s < min_r) continue;
    const K lo = std::min(min_r, min_s), hi = std::max(max_r, max_s);
    plo[(size_t)j] = lo_bits<K>(lo);
    prange[(size_t)j] = range_of<K>(lo, hi);
    live[(size_t)j] = 1;
    P = std::max(P, make_plan(plo[(size_t)j], prange[(size_t)j], false, digit_cap).passes);
  }
  stats.radix_passes = P;
  // scratch: ping-pong copies of every live pair, histograms, look-back, join state
  const int nbuf = P >= 2 ? 2 : P;
  std::vector<Plan> plans((size_t)nj);
  int64_t hist_words = 0, lb_words = 0, jtiles = 0;
  std::vector<int64_t> hist_at((size_t)(2 * nj), 0), lb_at((size_t)(2 * nj), 0);
  tiles = 0;
  for (int64_t j = 0; j < nj; ++j) {
    Plan pl;
    if (live[(size_t)j]) pl = make_plan(plo[(size_t)j], prange[(size_t)j], false, digit_cap, P);
    plans[(size_t)j] = pl;
    stats.key_bits = std::max(stats.key_bits, pl.key_bits);
    stats.digit_bits = std::max(stats.digit_bits, pl.max_bits);
    const int64_t bins = (int64_t)1 << pl.max_bits;
    for (int side = 0; side < 2; ++side) {
      RadixJob<K>& x = hj[(size_t)(2 * j + side)];
      if (!live[(size_t)j]) x.n = 0;
      x.tile0 = tiles;
      const int64_t t = ceil_div(x.n, tile);
      tiles += t;
      hist_at[(size_t)(2 * j + side)] = hist_words;
      hist_words += (int64_t)std::max(P, 1) * bins;
      lb_at[(size_t)(2 * j + side)] = lb_words;
      lb_words += t * bins;
    }
    if (live[(size_t)j]) jtiles += ceil_div(s_off[j + 1] - s_off[j], kJTile);
  }
  Carve bc;
  size_t o_r[4] = {0, 0, 0, 0}, o_s[4] = {0, 0, 0, 0};
  for (int b = 0; b < nbuf; ++b) {
    o_r[2 * b] = bc.add<K>((size_t)R);
    o_r[2 * b + 1] = bc.add<K>((size_t)R);
    o_s[2 * b] = bc.add<K>((size_t)S);
    o_s[2 * b + 1] = bc.add<K>((size_t)S);
  }
  const size_t o_hist = bc.add<uint32_t>((size_t)std::max<int64_t>(hist_words, 1));
  const size_t o_lb = bc.add<uint32_t>((size_t)std::max<int64_t>(lb_words, 1));
  const size_t o_jt = bc.add<JTile<K>>((size_t)std::max<int64_t>(jtiles, 1));
  const size_t o_jlb = bc.add<uint64_t>((size_t)std::max<int64_t>(jtiles, 1));
  const size_t o_tmap = bc.add<int32_t>((size_t)std::max<int64_t>(tiles, 1));
  const size_t o_jmap = bc.add<int32_t>((size_t)std::max<int64_t>(jtiles, 1));
  Block big;
  TJ_CUDA(big.alloc(bc.off, st));
  stats.scratch_peak = (int64_t)(bc.off + cc.off);
  int32_t* d_tmap = big.at<int32_t>(o_tmap);
  int32_t* d_jmap = big.at<int32_t>(o_jmap);

  std::vector<JoinJob<K>> hjj((size_t)nj);
  int64_t jt = 0;
  for (int64_t j = 0; j < nj; ++j) {
    const K* res[4] = {kr + r_off[j], ir + r_off[j], ks + s_off[j], is + s_off[j]};
    for (int side = 0; side < 2; ++side) {
      RadixJob<K>& x = hj[(size_t)(2 * j + side)];
      set_job_plan(x, plans[(size_t)j]);
      x.passes = live[(size_t)j] ? P : 0;
      x.hist_stride = 1 << plans[(size_t)j].max_bits;
      x.hist = big.at<uint32_t>(o_hist) + hist_at[(size_t)(2 * j + side)];
      x.lookback = big.at<uint32_t>(o_lb) + lb_at[(size_t)(2 * j + side)];
      const int64_t a = side ? s_off[j] : r_off[j];
      const size_t* o = side ? o_s : o_r;
      K* ak = nbuf > 0 ? big.at<K>(o[0]) + a : nullptr;
      K* av = nbuf > 0 ? big.at<K>(o[1]) + a : nullptr;
      K* bk = nbuf > 1 ? big.at<K>(o[2]) + a : nullptr;
      K* bv = nbuf > 1 ? big.at<K>(o[3]) + a : nullptr;
      set_job_buffers(x, res[2 * side], res[2 * side + 1], ak, av, bk, bv, &res[2 * side],
                      &res[2 * side + 1]);
    }
    JoinJob<K>& y = hjj[(size_t)j];
    y.rk = res[0];
    y.rv = res[1];
    y.nr = r_off[j + 1] - r_off[j];
    y.sk = res[2];
    y.sv = res[3];
    y.ns = live[(size_t)j] ? s_off[j + 1] - s_off[j] : 0;
    y.tile0 = jt;
    jt += ceil_div(y.ns, kJTile);
  }
  TJ_CUDA(put_small(d_jobs, hj.data(), hj.size() * sizeof(RadixJob<K>), st));
  TJ_CUDA(put_small(d_jj, hjj.data(), hjj.size() * sizeof(JoinJob<K>), st));

  // the batch's device work, captured once as a graph (plain launches on the
  // legacy stream, which cannot be captured)
  const bool use_graph = st != nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  if (use_graph) TJ_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaSuccess;
  auto step = [&](cudaError_t x) {
    if (e == cudaSuccess) e = x;
  };
  step(launch_fill_tile_job<K>(d_jobs, (int)(2 * nj), d_tmap, st, tile));
  step(launch_fill_join_tile_job<K>(d_jj, (int)nj, d_jmap, st));
  if (P > 0) {
    step(cudaMemsetAsync(big.at<uint32_t>(o_hist), 0,
                         (size_t)std::max<int64_t>(hist_words, 1) * sizeof(uint32_t), st));
    step(launch_histogram<K>(d_jobs, (int)(2 * nj), tiles, st, d_tmap, tile));
    step(launch_digit_scan<K>(d_jobs, (int)(2 * nj), P, st));
    for (int p = 0; p < P; ++p) {
      step(cudaMemsetAsync(big.at<uint32_t>(o_lb), 0,
                           (size_t)std::max<int64_t>(lb_words, 1) * sizeof(uint32_t), st));
      step(launch_onesweep<K>(d_jobs, (int)(2 * nj), tiles, p, stats.digit_bits, false, d_counters + p,
                              d_err, st, d_tmap, items));
    }
  }
  step(launch_tile_ranges<K>(d_jj, (int)nj, jtiles, big.at<JTile<K>>(o_jt), st, d_jmap));
  step(cudaMemsetAsync(big.at<uint64_t>(o_jlb), 0,
                       (size_t)std::max<int64_t>(jtiles, 1) * sizeof(uint64_t), st));
  step(launch_join<K>(jtiles, big.at<JTile<K>>(o_jt), big.at<uint64_t>(o_jlb),
                      d_counters + kMaxPasses, out, cap, nullptr, d_out_off, d_total, d_err, st));
  step(launch_fix_job_out<K>(d_jj, (int)nj, jtiles, d_out_off, d_total, st));
  if (use_graph) {
    cudaError_t e2 = cudaStreamEndCapture(st, &graph);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (e == cudaSuccess) e = cudaGraphLaunch(exec, st);
  }
  int64_t h_total = 0;
  int h_err = 0;
  if (e == cudaSuccess)
    e = get_small(&h_total, d_total, sizeof(int64_t), st);
  if (e == cudaSuccess) e = get_small(&h_err, d_err, sizeof(int), st);
  if (e == cudaSuccess) e = sync_stream(st);
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  if (e != cudaSuccess)
    return set_err(TJ_ERR_CUDA, "batch launch: %s", cudaGetErrorString(e));
  if (h_err) return set_err((tj_status)h_err, "device reported %d", h_err);
  *out_count = h_total;
  stats.out_count = h_total;
  g_stats = stats;
  if (h_total > cap)
    return set_err(TJ_ERR_CAPACITY, "batch result has %lld pairs, capacity %lld",
                   (long long)h_total, (long long)cap);
  return TJ_OK;
}


// ---- autotuner of the batched join --------------------------------------------------
// Choices: the widest radix digit (and so the number of passes and the fan-out
// of each pass) and the onesweep tile (1536 or 3072 rows: small jobs waste
// less of a smaller last tile).  A choice is cached per (dtype, log2 jobs,
// log2 mean rows per array); TJ_TUNE_CACHE names a file that persists it.
struct TuneChoice {
  int digit;
  int items;
};
std::mutex g_tune_mu;
std::vector<std::pair<std::string, TuneChoice>> g_tune;
bool g_tune_loaded = false;

std::string tune_key(int dt, int64_t nj, int64_t rows) {
  char b[64];
  const int64_t avg = nj > 0 ? rows / (2 * nj) : 0;
  snprintf(b, sizeof(b), "batch_d%d_j%d_a%d", dt, bitlen((uint64_t)nj), bitlen((uint64_t)avg));
  return b;
}

void tune_load_locked() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char* f = getenv("TJ_TUNE_CACHE");
  if (!f) return;
  FILE* fp = fopen(f, "r");
  if (!fp) return;
  char key[64];
  int d, it;
  while (fscanf(fp, "%63s %d %d", key, &d, &it) == 3)
    if (d >= 4 && d <= kMaxDigitBits && (it == 4 || it == kItems)) g_tune.push_back({key, {d, it}});
  fclose(fp);
}

bool tune_get(const std::string& k, TuneChoice* c) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  tune_load_locked();
  for (auto it = g_tune.rbegin(); it != g_tune.rend(); ++it)
    if (it->first == k) {
      *c = it->second;
      return true;
    }
  return false;
}

void tune_put(const std::string& k, TuneChoice c) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  tune_load_locked();
  g_tune.push_back({k, c});
  const char* f = getenv("TJ_TUNE_CACHE");
  if (!f) return;
  FILE* fp = fopen(f, "a");
  if (!fp) return;
  fprintf(fp, "%s %d %d\n", k.c_str(), c.digit, c.items);
  fclose(fp);
}

template <typename K>
tj_status batch_tuned(int dt, int64_t nj, const int64_t* r_off, const int64_t* s_off, const K* kr,
                      const K* ir, const K* ks, const K* is, K* out, int64_t cap,
                      int64_t* d_out_off, int64_t* out_count, cudaStream_t st, bool tune) {
  const std::string key = tune_key(dt, nj, r_off[nj] + s_off[nj]);
  TuneChoice c = {max_digit_bits<K>(), kItems};
  if (!tune) {
    tune_get(key, &c);
    return batch_impl<K>(nj, r_off, s_off, kr, ir, ks, is, out, cap, d_out_off, out_count, st,
                         c.digit, c.items);
  }
  // time every candidate on this batch (each run also produces the result)
  double best = 1e300;
  TuneChoice bc = c;
  for (int d = 6; d <= max_digit_bits<K>(); ++d)
    for (int it : {4, kItems}) {
      for (int rep = 0; rep < 2; ++rep) {  // the first run warms the pool
        const auto t0 = std::chrono::steady_clock::now();
        tj_status s = batch_impl<K>(nj, r_off, s_off, kr, ir, ks, is, out, cap, d_out_off,
                                    out_count, st, d, it);
        const double dtm =
            std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (s != TJ_OK) return s;
        if (rep == 1 && dtm < best) {
          best = dtm;
          bc = {d, it};
        }
      }
    }
  tune_put(key, bc);
  return batch_impl<K>(nj, r_off, s_off, kr, ir, ks, is, out, cap, d_out_off, out_count, st,
                       bc.digit, bc.items);
}

bool bad_ptr(const void* p, int64_t n) { return n > 0 && p == nullptr; }

// ---- sort without allocation --------------------------------------------------------
// Some callers cannot call cudaMalloc (or any allocator) at the point they
// sort: code running while an outer framework owns the device memory pool,
// allocation-free real-time paths, or hosts that must not grow device memory
// after start-up.  For them, tj_sort_noalloc runs the same kernels as tj_sort
// with its scratch in one file-scope device array of a fixed size, held by
// every GPU that loads this library until the process exits.
constexpr int64_t kNoAllocMaxRows = (int64_t)1 << 20;  // rows per call
constexpr int64_t kNoAllocTiles = (kNoAllocMaxRows + kTile - 1) / kTile;
constexpr size_t kNoAllocBytes = 2 * (size_t)kNoAllocMaxRows * 8           // B keys, B ids
                                 + (size_t)kMaxPasses * kMaxBins * 4        // digit histograms
                                 + (size_t)kNoAllocTiles * kMaxBins * 4     // look-back words
                                 + 4096;                                    // job, stats, flags
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_noalloc_mu;
unsigned char* g_noalloc_ptr[256] = {nullptr};

// Device address of the scratch array on the current device, looked up once
// per device (cudaGetSymbolAddress with that device current).
tj_status noalloc_scratch(unsigned char** out) {
  int dev = 0;
  TJ_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 256) return set_err(TJ_ERR_INTERNAL, "device index %d", dev);
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    TJ_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_noalloc_ptr[dev] = (unsigned char*)p;
  }
  *out = g_noalloc_ptr[dev];
  return TJ_OK;
}

// The job table enters the device as a kernel parameter (no host staging
// buffer, no copy engine).
template <typename K>
__global__ void k_put_job(RadixJob<K> job, RadixJob<K>* dst) {
  *dst = job;
}

// Device -> host read of a few bytes into the caller's (pageable) variable;
// returns once the bytes have arrived.
cudaError_t read_now(void* dst, const void* src, size_t n, cudaStream_t st) {
  cudaError_t e = cudaMemcpyAsync(dst, src, n, cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(st);
}

template <typename K>
tj_status sort_noalloc_impl(K* keys, K* ids, int64_t n, cudaStream_t st) {
  tj_stats stats = {};
  stats.groups = 1;
  if (n <= 1) {
    g_stats = stats;
    return TJ_OK;
  }
  tj_status s = ensure_device();
  if (s != TJ_OK) return s;
  unsigned char* base = nullptr;
  s = noalloc_scratch(&base);
  if (s != TJ_OK) return s;
  const int64_t tiles = ceil_div(n, kTile);
  // carve the fixed array: B keys | B ids | histograms | look-back | job | stats | flags
  K* bk = reinterpret_cast<K*>(base);
  K* bv = reinterpret_cast<K*>(base + (size_t)kNoAllocMaxRows * 8);
  uint32_t* hist = reinterpret_cast<uint32_t*>(base + 2 * (size_t)kNoAllocMaxRows * 8);
  uint32_t* lb = hist + (size_t)kMaxPasses * kMaxBins;
  unsigned char* tail = reinterpret_cast<unsigned char*>(lb + (size_t)kNoAllocTiles * kMaxBins);
  RadixJob<K>* d_job = reinterpret_cast<RadixJob<K>*>(tail);
  KeyStats* d_stats = reinterpret_cast<KeyStats*>(tail + 1024);
  int* d_err = reinterpret_cast<int*>(tail + 2048);
  uint32_t* d_counters = reinterpret_cast<uint32_t*>(tail + 2048 + 64);
  static_assert(sizeof(RadixJob<int64_t>) <= 1024, "job fits its slot");

  RadixJob<K> hj;
  memset(&hj, 0, sizeof(hj));
  hj.keys = keys;
  hj.n = n;
  TJ_CUDA(cudaMemsetAsync(tail + 2048, 0, 2048, st));  // error word and tile counters
  TJ_CUDA(cudaMemsetAsync(d_stats, 0xFF, sizeof(KeyStats), st));
  k_put_job<K><<<1, 1, 0, st>>>(hj, d_job);
  TJ_CUDA(cudaGetLastError());
  TJ_CUDA(launch_stats<K>(d_job, 1, tiles, d_stats, st));
  KeyStats hs;
  TJ_CUDA(read_now(&hs, d_stats, sizeof(hs), st));
  const K lo = key_of<K>(hs.min_u), hi = key_of<K>(~hs.max_u);
  const Plan plan = make_plan(lo_bits<K>(lo), range_of<K>(lo, hi), /*even=*/true,
                              max_digit_bits<K>());
  stats.key_bits = plan.key_bits;
  stats.radix_passes = plan.passes;
  stats.digit_bits = plan.max_bits;
  if (plan.passes == 0) {  // all keys equal
    g_stats = stats;
    return TJ_OK;
  }
  const int64_t bins_max = (int64_t)1 << plan.max_bits;
  set_job_plan(hj, plan);
  hj.hist_stride = kMaxBins;
  hj.hist = hist;
  hj.lookback = lb;
  const K* rk;
  const K* rv;
  set_job_buffers(hj, keys, ids, bk, bv, keys, ids, &rk, &rv);
  k_put_job<K><<<1, 1, 0, st>>>(hj, d_job);
  TJ_CUDA(cudaGetLastError());
  // the array keeps the last call's contents: clear what must start at zero
  TJ_CUDA(cudaMemsetAsync(hist, 0, (size_t)kMaxPasses * kMaxBins * sizeof(uint32_t), st));
  TJ_CUDA(launch_histogram<K>(d_job, 1, tiles, st));
  TJ_CUDA(launch_digit_scan<K>(d_job, 1, plan.passes, st));
  for (int p = 0; p < plan.passes; ++p) {
    TJ_CUDA(cudaMemsetAsync(lb, 0, (size_t)tiles * bins_max * sizeof(uint32_t), st));
    TJ_CUDA(launch_onesweep<K>(d_job, 1, tiles, p, plan.max_bits, false, d_counters + p, d_err,
                               st));
  }
  int h_err = 0;
  TJ_CUDA(read_now(&h_err, d_err, sizeof(int), st));
  if (h_err) return set_err((tj_status)h_err, "device reported %d", h_err);
  if (rk != keys) return set_err(TJ_ERR_INTERNAL, "odd pass count in place");
  // the library's scratch for this call is the fixed array, none of it allocated
  stats.scratch_peak = 0;
  g_stats = stats;
  return TJ_OK;
}


}  // namespace
}  // namespace tj

using namespace tj;

extern "C" {

tj_status tj_join_inner(tj_dtype dt, const void* keys_r, const void* ids_r, int64_t n_r,
                        const void* keys_s, const void* ids_s, int64_t n_s,
                        size_t mem_budget_bytes, void* out_pairs, int64_t out_capacity,
                        int64_t* out_count, void* stream) {
  return tj_join_inner_ex(dt, keys_r, ids_r, n_r, keys_s, ids_s, n_s, mem_budget_bytes, nullptr,
                          out_pairs, out_capacity, out_count, stream);
}

tj_status tj_join_inner_ex(tj_dtype dt, const void* keys_r, const void* ids_r, int64_t n_r,
                           const void* keys_s, const void* ids_s, int64_t n_s,
                           size_t mem_budget_bytes, const tj_join_opts* opts, void* out_pairs,
                           int64_t out_capacity, int64_t* out_count, void* stream) {
  g_err[0] = 0;
  arena_reset();
  if (!out_count) return set_err(TJ_ERR_INVALID, "out_count is NULL");
  *out_count = 0;
  if (n_r < 0 || n_s < 0 || out_capacity < 0)
    return set_err(TJ_ERR_INVALID, "negative size");
  if (n_r >= kMaxRows || n_s >= kMaxRows)
    return set_err(TJ_ERR_INVALID, "n >= 2^30 rows per relation is not supported");
  if (bad_ptr(keys_r, n_r) || bad_ptr(ids_r, n_r) || bad_ptr(keys_s, n_s) ||
      bad_ptr(ids_s, n_s) || bad_ptr(out_pairs, out_capacity))
    return set_err(TJ_ERR_INVALID, "null pointer with a non-zero size");
  if (opts && (opts->router < TJ_ROUTE_AUTO || opts->router > TJ_ROUTE_MLP ||
               opts->partitions < 0 || opts->partitions > kMaxCuts || opts->sample_stride < 0 ||
               opts->mlp_batch < 0 || opts->mlp_batch > 256))
    return set_err(TJ_ERR_INVALID, "bad tj_join_opts");
  const Opts o = make_opts(opts);
  cudaStream_t st = (cudaStream_t)stream;
  if (dt == TJ_I32)
    return join_impl<int32_t>((const int32_t*)keys_r, (const int32_t*)ids_r, n_r,
                              (const int32_t*)keys_s, (const int32_t*)ids_s, n_s,
                              mem_budget_bytes, o, (int32_t*)out_pairs, out_capacity, out_count,
                              st);
  if (dt == TJ_I64)
    return join_impl<int64_t>((const int64_t*)keys_r, (const int64_t*)ids_r, n_r,
                              (const int64_t*)keys_s, (const int64_t*)ids_s, n_s,
                              mem_budget_bytes, o, (int64_t*)out_pairs, out_capacity, out_count,
                              st);
  return set_err(TJ_ERR_INVALID, "unknown dtype %d", (int)dt);
}

tj_status tj_sort_noalloc(tj_dtype dt, void* keys, void* ids, int64_t n, void* stream) {
  g_err[0] = 0;  // (no arena_reset: this entry point never touches the pinned arena)
  if (n < 0) return set_err(TJ_ERR_INVALID, "negative size");
  if (n > kNoAllocMaxRows)
    return set_err(TJ_ERR_INVALID,
                   "tj_sort_noalloc sorts at most %lld rows per call (got %lld); use tj_sort",
                   (long long)kNoAllocMaxRows, (long long)n);
  if (bad_ptr(keys, n) || bad_ptr(ids, n))
    return set_err(TJ_ERR_INVALID, "null pointer with a non-zero size");
  cudaStream_t st = (cudaStream_t)stream;
  if (dt == TJ_I32) return sort_noalloc_impl<int32_t>((int32_t*)keys, (int32_t*)ids, n, st);
  if (dt == TJ_I64) return sort_noalloc_impl<int64_t>((int64_t*)keys, (int64_t*)ids, n, st);
  return set_err(TJ_ERR_INVALID, "unknown dtype %d", (int)dt);
}

tj_status tj_sort_multi(tj_dtype dt, void* const* cols, int32_t n_cols, void* ids, int64_t n,
                        int32_t path, void* stream) {
  g_err[0] = 0;
  arena_reset();
  if (n < 0 || n_cols < 0) return set_err(TJ_ERR_INVALID, "negative size");
  if (path < 0 || path > 2) return set_err(TJ_ERR_INVALID, "path %d (0, 1 or 2)", path);
  if (n >= kMaxRows) return set_err(TJ_ERR_INVALID, "n >= 2^30 rows is not supported");
  if (n_cols > 0 && !cols) return set_err(TJ_ERR_INVALID, "cols is NULL");
  for (int32_t c = 0; c < n_cols; ++c)
    if (bad_ptr(cols[c], n)) return set_err(TJ_ERR_INVALID, "column %d is NULL", c);
  cudaStream_t st = (cudaStream_t)stream;
  if (dt == TJ_I32)
    return sort_multi_impl<int32_t>(reinterpret_cast<int32_t* const*>(cols), n_cols,
                                    (int32_t*)ids, n, path, st);
  if (dt == TJ_I64)
    return sort_multi_impl<int64_t>(reinterpret_cast<int64_t* const*>(cols), n_cols,
                                    (int64_t*)ids, n, path, st);
  return set_err(TJ_ERR_INVALID, "unknown dtype %d", (int)dt);
}

tj_status tj_sort(tj_dtype dt, void* keys, void* ids, int64_t n, void* stream) {
  g_err[0] = 0;
  arena_reset();
  if (n < 0) return set_err(TJ_ERR_INVALID, "negative size");
  if (n >= kMaxRows) return set_err(TJ_ERR_INVALID, "n >= 2^30 rows is not supported");
  if (bad_ptr(keys, n) || bad_ptr(ids, n))
    return set_err(TJ_ERR_INVALID, "null pointer with a non-zero size");
  cudaStream_t st = (cudaStream_t)stream;
  if (dt == TJ_I32) return sort_impl<int32_t>((int32_t*)keys, (int32_t*)ids, n, st);
  if (dt == TJ_I64) return sort_impl<int64_t>((int64_t*)keys, (int64_t*)ids, n, st);
  return set_err(TJ_ERR_INVALID, "unknown dtype %d", (int)dt);
}

tj_status tj_gather_pairs(tj_dtype id_dt, const void* pairs, int64_t n, int64_t n_r,
                          int64_t n_s, const tj_column* cols, int32_t n_cols, void* stream) {
  g_err[0] = 0;
  arena_reset();
  if (n < 0 || n_r < 0 || n_s < 0 || n_cols < 0) return set_err(TJ_ERR_INVALID, "negative size");
  if (id_dt != TJ_I32 && id_dt != TJ_I64) return set_err(TJ_ERR_INVALID, "unknown dtype %d", (int)id_dt);
  if (n_cols > 0 && !cols) return set_err(TJ_ERR_INVALID, "cols is NULL");
  const size_t idw = id_dt == TJ_I32 ? 4 : 8;
  if (bad_ptr(pairs, n) || (n > 0 && ((uintptr_t)pairs % (2 * idw)) != 0))
    return set_err(TJ_ERR_INVALID, "pairs: NULL or not aligned to a pair");
  for (int32_t c = 0; c < n_cols; ++c) {
    const tj_column& x = cols[c];
    if (x.side != 0 && x.side != 1) return set_err(TJ_ERR_INVALID, "column %d: side %d", c, x.side);
    if (x.elem_bytes != 4 && x.elem_bytes != 8)
      return set_err(TJ_ERR_INVALID, "column %d: elem_bytes %d (4 or 8)", c, x.elem_bytes);
    const int64_t rows = x.side ? n_s : n_r;
    if (bad_ptr(x.src, rows) || bad_ptr(x.dst, n) ||
        ((uintptr_t)x.src % (uintptr_t)x.elem_bytes) != 0 ||
        ((uintptr_t)x.dst % (uintptr_t)x.elem_bytes) != 0)
      return set_err(TJ_ERR_INVALID, "column %d: NULL or misaligned pointer", c);
  }
  if (n == 0 || n_cols == 0) return TJ_OK;
  tj_status s = ensure_device();
  if (s != TJ_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  TJ_CUDA(cudaGetDevice(&dev));
  TJ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  Block eb;
  TJ_CUDA(eb.alloc(256, st));
  TJ_CUDA(cudaMemsetAsync(eb.p, 0, sizeof(int), st));
  Tracer tr(st);
  for (int32_t c0 = 0; c0 < n_cols; c0 += kGatherCols) {
    GatherArgs a;
    memset(&a, 0, sizeof(a));
    a.n = std::min<int32_t>(kGatherCols, n_cols - c0);
    double by = 2.0 * (double)idw * (double)n;
    for (int i = 0; i < a.n; ++i) {
      const tj_column& x = cols[c0 + i];
      a.c[i] = GatherCol{x.src, x.dst, x.side, x.elem_bytes};
      by += 2.0 * (double)x.elem_bytes * (double)n;
    }
    tr.begin("gather", by);
    if (id_dt == TJ_I32)
      TJ_CUDA(launch_gather_pairs<int32_t>((const int32_t*)pairs, n, n_r, n_s, a, eb.at<int>(0),
                                           sms, st));
    else
      TJ_CUDA(launch_gather_pairs<int64_t>((const int64_t*)pairs, n, n_r, n_s, a, eb.at<int>(0),
                                           sms, st));
    tr.end();
  }
  int h_err = 0;
  TJ_CUDA(get_small(&h_err, eb.p, sizeof(int), st));
  TJ_CUDA(sync_stream(st));
  tr.flush();
  if (h_err) return set_err((tj_status)h_err, "an id of `pairs` is out of range");
  return TJ_OK;
}

static tj_status batch_entry(tj_dtype dt, int64_t n_jobs, const int64_t* r_off,
                             const int64_t* s_off, const void* keys_r, const void* ids_r,
                             const void* keys_s, const void* ids_s, void* out_pairs,
                             int64_t out_capacity, int64_t* out_off, int64_t* out_count,
                             void* stream, bool tune) {
  g_err[0] = 0;
  arena_reset();
  if (!out_count) return set_err(TJ_ERR_INVALID, "out_count is NULL");
  *out_count = 0;
  if (n_jobs < 0 || out_capacity < 0) return set_err(TJ_ERR_INVALID, "negative size");
  if (n_jobs >= ((int64_t)1 << 30)) return set_err(TJ_ERR_INVALID, "too many jobs");
  if (n_jobs > 0 && (!r_off || !s_off || !out_off))
    return set_err(TJ_ERR_INVALID, "null offsets");
  if (n_jobs == 0) return TJ_OK;
  if (r_off[0] != 0 || s_off[0] != 0) return set_err(TJ_ERR_INVALID, "offsets must start at 0");
  for (int64_t j = 0; j < n_jobs; ++j) {
    const int64_t a = r_off[j + 1] - r_off[j], b = s_off[j + 1] - s_off[j];
    if (a < 0 || b < 0) return set_err(TJ_ERR_INVALID, "offsets of job %lld decrease", (long long)j);
    if (a >= kMaxRows || b >= kMaxRows)
      return set_err(TJ_ERR_INVALID, "job %lld has >= 2^30 rows", (long long)j);
  }
  if (bad_ptr(keys_r, r_off[n_jobs]) || bad_ptr(ids_r, r_off[n_jobs]) ||
      bad_ptr(keys_s, s_off[n_jobs]) || bad_ptr(ids_s, s_off[n_jobs]) ||
      bad_ptr(out_pairs, out_capacity))
    return set_err(TJ_ERR_INVALID, "null pointer with a non-zero size");
  cudaStream_t st = (cudaStream_t)stream;
  if (dt == TJ_I32)
    return batch_tuned<int32_t>((int)dt, n_jobs, r_off, s_off, (const int32_t*)keys_r,
                                (const int32_t*)ids_r, (const int32_t*)keys_s,
                                (const int32_t*)ids_s, (int32_t*)out_pairs, out_capacity,
                                out_off, out_count, st, tune);
  if (dt == TJ_I64)
    return batch_tuned<int64_t>((int)dt, n_jobs, r_off, s_off, (const int64_t*)keys_r,
                                (const int64_t*)ids_r, (const int64_t*)keys_s,
                                (const int64_t*)ids_s, (int64_t*)out_pairs, out_capacity,
                                out_off, out_count, st, tune);
  return set_err(TJ_ERR_INVALID, "unknown dtype %d", (int)dt);
}

tj_status tj_join_batch(tj_dtype dt, int64_t n_jobs, const int64_t* r_off, const int64_t* s_off,
                        const void* keys_r, const void* ids_r, const void* keys_s,
                        const void* ids_s, void* out_pairs, int64_t out_capacity,
                        int64_t* out_off, int64_t* out_count, void* stream) {
  return batch_entry(dt, n_jobs, r_off, s_off, keys_r, ids_r, keys_s, ids_s, out_pairs,
                     out_capacity, out_off, out_count, stream, false);
}

tj_status tj_autotune_batch(tj_dtype dt, int64_t n_jobs, const int64_t* r_off,
                            const int64_t* s_off, const void* keys_r, const void* ids_r,
                            const void* keys_s, const void* ids_s, void* out_pairs,
                            int64_t out_capacity, int64_t* out_off, int64_t* out_count,
                            void* stream) {
  return batch_entry(dt, n_jobs, r_off, s_off, keys_r, ids_r, keys_s, ids_s, out_pairs,
                     out_capacity, out_off, out_count, stream, true);
}

tj_status tj_mlp_grad(const float* theta, const float* x, const float* y, int n, float* grad,
                      void* stream) {
  g_err[0] = 0;
  arena_reset();
  if (n < 1 || n > 256) return set_err(TJ_ERR_INVALID, "batch must have 1..256 rows");
  if (!theta || !x || !y || !grad) return set_err(TJ_ERR_INVALID, "null pointer");
  tj_status s = ensure_device();
  if (s != TJ_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  TJ_CUDA(launch_mlp_grad(theta, x, y, n, grad, st));
  TJ_CUDA(sync_stream(st));
  return TJ_OK;
}

tj_status tj_mlp_adam(float* theta, float* m, float* v, const float* grad, int n, int t,
                      float lr, void* stream) {
  g_err[0] = 0;
  arena_reset();
  if (n < 0 || t < 1) return set_err(TJ_ERR_INVALID, "bad size or step");
  if (n > 0 && (!theta || !m || !v || !grad)) return set_err(TJ_ERR_INVALID, "null pointer");
  tj_status s = ensure_device();
  if (s != TJ_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  if (n > 0) TJ_CUDA(launch_adam(theta, m, v, grad, n, t, lr, st));
  TJ_CUDA(sync_stream(st));
  return TJ_OK;
}

tj_status tj_mlp_table(const float* theta, int T, float* table, int parts, tj_dtype dt,
                       const void* sorted, int64_t m, void* bounds, void* stream) {
  g_err[0] = 0;
  arena_reset();
  if (T < 1 || T > 65536) return set_err(TJ_ERR_INVALID, "T must be 1..65536");
  if (parts < 2 || parts > kMaxCuts) return set_err(TJ_ERR_INVALID, "parts must be 2..%d", kMaxCuts);
  if (m < 1) return set_err(TJ_ERR_INVALID, "the sample needs at least one key");
  if (!theta || !table || !sorted || !bounds) return set_err(TJ_ERR_INVALID, "null pointer");
  tj_status s = ensure_device();
  if (s != TJ_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  if (dt == TJ_I32)
    TJ_CUDA(launch_mlp_boundaries<int32_t>(theta, T, table, parts, (const int32_t*)sorted, m,
                                           (int32_t*)bounds, st));
  else if (dt == TJ_I64)
    TJ_CUDA(launch_mlp_boundaries<int64_t>(theta, T, table, parts, (const int64_t*)sorted, m,
                                           (int64_t*)bounds, st));
  else
    return set_err(TJ_ERR_INVALID, "unknown dtype %d", (int)dt);
  TJ_CUDA(sync_stream(st));
  return TJ_OK;
}

const char* tj_status_str(tj_status s) {
  switch (s) {
    case TJ_OK: return "TJ_OK";
    case TJ_ERR_INVALID: return "TJ_ERR_INVALID";
    case TJ_ERR_BUDGET: return "TJ_ERR_BUDGET";
    case TJ_ERR_CAPACITY: return "TJ_ERR_CAPACITY";
    case TJ_ERR_CUDA: return "TJ_ERR_CUDA";
    case TJ_ERR_TIMEOUT: return "TJ_ERR_TIMEOUT";
    case TJ_ERR_INTERNAL: return "TJ_ERR_INTERNAL";
  }
  return "TJ_ERR_UNKNOWN";
}

const char* tj_last_error(void) { return g_err; }

tj_status tj_get_stats(tj_stats* out) {
  if (!out) return TJ_ERR_INVALID;
  *out = g_stats;
  return TJ_OK;
}

const char* tj_version(void) { return "tj 0.1 (sm_103a)"; }

void tj_trace_enable(int on) {
  std::lock_guard<std::mutex> lk(g_trace_mu);
  g_trace_on = on != 0;
}

void tj_trace_reset(void) {
  std::lock_guard<std::mutex> lk(g_trace_mu);
  g_trace.clear();
}

int tj_trace_count(void) {
  std::lock_guard<std::mutex> lk(g_trace_mu);
  return (int)g_trace.size();
}

tj_status tj_trace_get(int i, char* name, int name_len, int64_t* launches, double* ms,
                       double* bytes) {
  std::lock_guard<std::mutex> lk(g_trace_mu);
  if (i < 0 || i >= (int)g_trace.size()) return TJ_ERR_INVALID;
  const TraceRow& r = g_trace[(size_t)i];
  if (name && name_len > 0) snprintf(name, (size_t)name_len, "%s", r.name);
  if (launches) *launches = r.launches;
  if (ms) *ms = r.ms;
  if (bytes) *bytes = r.bytes;
  return TJ_OK;
}

}  // extern "C"
