// Internal declarations shared by the CUDA translation units of libtj.
//
// Layout of a relation: two device arrays (SoA), keys[n] and ids[n], of the
// same integer width.  Sorting moves both; joins read both and write (r_id,
// s_id) pairs once at the end (late materialisation, paper Sec. 3.1).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/tj.h"

namespace tj {

// ---- launch geometry -------------------------------------------------------
constexpr int kThreads = 256;               // threads per CTA of most kernels (8 warps)
constexpr int kWarps = kThreads / 32;
#ifndef TJ_SORT_THREADS  // 12 warps: three CTAs fit an SM (registers and shared memory)
#define TJ_SORT_THREADS 384
#endif
#ifndef TJ_SORT_MINB
#define TJ_SORT_MINB 3
#endif
#ifndef TJ_SORT_ITEMS
#define TJ_SORT_ITEMS 8
#endif
constexpr int kSortThreads = TJ_SORT_THREADS;  // threads per onesweep CTA
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kItems = TJ_SORT_ITEMS;          // rows per thread in a sort tile
constexpr int kTile = kSortThreads * kItems;   // rows per onesweep tile (3072)
// Rows per thread of sorts whose digits have at most kWideBits bits: 10, a
// 3840-row tile (its shared memory still lets three CTAs share an SM; about
// 8% faster than 8 rows per thread for 7-bit digits, measured).
constexpr int kItemsWide = 10;
constexpr int kWideBits = 7;
constexpr int kTileWide = kSortThreads * kItemsWide;
// rows per thread of a route pass with at most kWideBits of batch index (its
// batch-index tables and per-slot digits take shared memory of their own)
#ifndef TJ_ROUTE_ITEMS
#define TJ_ROUTE_ITEMS 9
#endif
constexpr int kItemsRoute = TJ_ROUTE_ITEMS;
constexpr int kTileRoute = kSortThreads * kItemsRoute;
constexpr int kMaxDigitBits = 10;           // widest radix digit
constexpr int kMaxBins = 1 << kMaxDigitBits;
constexpr int kMaxPasses = 8;               // 64-bit keys at 8 bits per pass
#ifndef TJ_JTILE
#define TJ_JTILE 4096
#endif
constexpr int kJTile = TJ_JTILE;            // S rows per join tile (a power of two)
constexpr int kRCap = kJTile / 2;           // R rows a join tile keeps on chip at once
constexpr int kMaxChunks = 4;               // R chunks a join tile aligns on chip
constexpr int kHTSlots = kJTile;            // on-chip hash table slots (load <= 0.5)
static_assert((kJTile & (kJTile - 1)) == 0 && kJTile >= 1024, "join tile: a power of two");

// ---- decoupled look-back words (30-bit counts) ----------------------------
constexpr uint32_t kFlagAgg = 1u << 30;
constexpr uint32_t kFlagInc = 2u << 30;
constexpr uint32_t kValMask = (1u << 30) - 1u;
// 64-bit words for output offsets (62-bit counts)
constexpr uint64_t kFlagAgg64 = 1ull << 62;
constexpr uint64_t kFlagInc64 = 2ull << 62;
constexpr uint64_t kValMask64 = (1ull << 62) - 1ull;
// bounded waits: iterations of a spin before the device reports TJ_ERR_TIMEOUT
constexpr int kSpinLimit = 1 << 22;
// key-range partitions of one route pass: cuts <= 1023 -> digits of <= 10 bits
constexpr int kMaxCuts = 1024;
constexpr int kRouteBuckets = 65 * 32;  // b(x) < 32 * 65
// predecessors a onesweep digit reads per look-back round trip: the first
// window is issued before the tile's slots are recorded, later ones after.
// Every word read is a separate L2 sector (one predecessor tile each), so wide
// windows cost more in load traffic than they save in round trips; 4 and 8
// measured fastest on GB300 (windows of 16 or 32 were 3-10% slower).
#ifndef TJ_LB_FIRST
#define TJ_LB_FIRST 4
#endif
#ifndef TJ_LB_WIDE
#define TJ_LB_WIDE 8
#endif
constexpr int kLookWindow = TJ_LB_FIRST;
constexpr int kLookWide = TJ_LB_WIDE;

template <typename K> struct UnsignedOf;
template <> struct UnsignedOf<int32_t> { using type = uint32_t; };
template <> struct UnsignedOf<int64_t> { using type = uint64_t; };

// ---- per-array radix job ---------------------------------------------------
// One array being sorted by (key - lo) over `passes` LSD digits.  Pass p reads
// src_k/src_v[p] and writes dst_k/dst_v[p] (ping-pong buffers).
template <typename K>
struct RadixJob {
  const K* keys;        // keys for statistics and the digit histogram
  int64_t n;            // rows
  int64_t tile0;        // first global tile index (kTile rows per tile)
  uint64_t lo;          // subtracted (bit pattern of the key type, wraps)
  int32_t passes;
  int32_t shift[kMaxPasses];
  int32_t bits[kMaxPasses];
  int32_t hist_stride;  // words between passes in `hist`
  uint32_t* hist;       // [passes][hist_stride]: counts, then exclusive bases
  uint32_t* lookback;   // [tiles][1 << bits[p]] words of the current pass
  int64_t lb_stride;    // words between the look-back regions of consecutive
                        // passes (0: one region, cleared before every pass)
  const K* src_k[kMaxPasses];
  const K* src_v[kMaxPasses];
  K* dst_k[kMaxPasses];
  K* dst_v[kMaxPasses];
  // Route digit (pass 0 only, when cuts != nullptr): the digit of a key is the
  // number of cut keys <= key, i.e. the index of its key-range partition.
  const K* cuts;        // sorted cut keys, padded to kMaxCuts with the key type's max
  int32_t ncuts;        // real cuts (<= kMaxCuts - 1); partitions = ncuts + 1
  // Log-scale index over the cuts: with x = key - lo, bucket b(x) = x for
  // x < 32, else 32 * bitlen(x) + the 5 bits below x's leading one; bucket b
  // holds cuts [route_tab[b], route_tab[b + 1]).  Fine-grained at every
  // magnitude, so clustered keys still find their cut in a few steps;
  // route_steps = ceil(log2(largest bucket + 1)) halvings always suffice, so
  // every lane runs the same number of them.
  // When the cuts are spread evenly enough, the index is uniform instead:
  // route_shift >= 0 and bucket b(x) = x >> route_shift (at most
  // kRouteBuckets buckets over the key range); the host keeps whichever index
  // needs fewer halvings.
  const uint16_t* route_tab;  // kRouteBuckets + 1 entries
  int32_t route_steps;
  int32_t route_shift;  // -1: log-scale index
  // Batch regions sized in advance (optional): rows of batch d go below
  // route_end[d]; a row that would not is dropped and the pass reports
  // TJ_ERR_CAPACITY, after which the caller routes again with exact sizes.
  const uint32_t* route_end;
  // Equal-width batches (route passes in kModeRadix): the batch of a key is
  // (clamp(key, lo, route_hi) - lo) >> shift[0]; keys outside the range (a
  // range read off a sample) take the first or the last batch.
  uint64_t route_hi;
};

// Kinds of onesweep pass: a sort digit of key - lo, a route by the cut table
// (batch = number of cuts <= key), a route by equal-width ranges.
constexpr int kModeSort = 0;
constexpr int kModeCuts = 1;
constexpr int kModeRadix = 2;

// Per-array min/max, stored as order-preserving unsigned (key ^ sign bit).
struct KeyStats {
  unsigned long long min_u;
  unsigned long long max_u;
};

// ---- join job ---------------------------------------------------------------
// One join of key-sorted R and key-sorted S.
template <typename K>
struct JoinJob {
  const K* rk;          // sorted R keys
  const K* rv;          // R ids in the same order
  int64_t nr;
  const K* sk;          // sorted S keys
  const K* sv;
  int64_t ns;
  int64_t tile0;        // first global join tile (kJTile S rows per tile)
};

// A batch of one key value (a heavy key the cuts isolate): every R row pairs
// with every S row, so its pairs need neither sort nor table.  Pair p of the
// batch, p = i * nr + j, is (R id j, S id i) at out[base + off + p]: key,
// then S position, then R position.
template <typename K>
struct CrossJob {
  const K* rv;     // R ids of the batch (routed, so in input order)
  const K* sv;     // S ids
  int64_t nr, ns;
  int64_t off;     // first pair relative to its run's base
  int64_t blk0;    // first CTA (kXPairs pairs per CTA)
};
constexpr int kXPairs = 4096;  // pairs per CTA of k_cross
constexpr int kXThreads = 256;

// One join tile as k_tile_ranges leaves it for k_join (one 64-byte load): its
// S rows and the R rows whose keys lie between its first and last key.
template <typename K>
struct alignas(16) JTile {
  const K* sk;   // the tile's first S row (keys, ids)
  const K* sv;
  const K* rk;   // the first R row of its range (keys, ids)
  const K* rv;
  int64_t lt;    // tile index within its job
  int64_t nrr;   // R rows in the range
  int32_t nv;    // S rows of the tile
  int32_t j;     // its job
  int64_t pad;
};
static_assert(sizeof(JTile<int64_t>) == 64 && sizeof(JTile<int32_t>) == 64, "64-byte tiles");

template <typename K> struct PairOf;
template <> struct PairOf<int32_t> { using type = int2; };
template <> struct PairOf<int64_t> { using type = longlong2; };

// ---- partition-resident join (tj_fused.cu) ------------------------------------
// A batch of the partitioned join, cut by one MSD pass into 2^m sub-batches of
// kFKeys consecutive key values; one item = one tile (<= kFCapS S rows) of a
// sub-batch, joined on chip.
constexpr int kFKeyBits = 10;               // key offsets within a sub-batch
#ifndef TJ_FUSED_MIN_BITS
#define TJ_FUSED_MIN_BITS 10
#endif
// narrowest batch key range the resident phase takes (below kFKeyBits: the
// whole batch is one sub-batch, no MSD pass)
constexpr int kFMinBits = TJ_FUSED_MIN_BITS;
constexpr int kFKeys = 1 << kFKeyBits;
constexpr int kFThreads = 512;              // threads of a fused CTA
constexpr int kFCapS = 4608;                // S rows of one item (9 per thread)
constexpr int kFCapR = 2048;                // R rows of a sub-batch (on chip)
#ifndef TJ_FUSED_MAX_MSD
#define TJ_FUSED_MAX_MSD 10
#endif
constexpr int kFMaxMsdBits = TJ_FUSED_MAX_MSD;  // widest MSD digit of the resident phase
constexpr int kFPreferMsdBits = 9;  // widest MSD digit the batch count aims at (a 10-bit pass costs 1.45x a 9-bit one)

template <typename K>
struct FusedJob {
  const K* rk;          // R rows of the batch, sub-batches back to back (MSD order)
  const K* rv;
  const K* sk;          // S rows likewise
  const K* sv;
  const uint32_t* hr;   // first R row of each sub-batch (2^m), nullptr when m == 0
  const uint32_t* hs;   // first S row of each sub-batch
  int64_t nr, ns;
  uint64_t lo;          // the batch's first key (bits of K); sub-batch d starts at lo + d 2^10
  int32_t m;            // MSD digit bits (0: the batch is one sub-batch)
  int32_t pad;
  int64_t item0;        // first item of the batch in its group's item list
  int64_t kbt0;         // first count-vector slot of its multi-tile sub-batches' tiles
  int64_t kbs0;         // first totals slot of its multi-tile sub-batches
};

// One item, resolved by k_fused_items so that a join CTA starts from one
// 64-byte load: where its rows are, how many, and its sub-batch's first key.
struct alignas(16) FItem {
  uint64_t rk, rv;  // the sub-batch's first R row (keys, ids: const K*)
  uint64_t sk, sv;  // the tile's first S row
  uint64_t sublo;   // the sub-batch's first key value (unsigned bits of K)
  int32_t nr;       // R rows of the sub-batch (<= kFCapR)
  int32_t ns;       // S rows of the tile (<= kFCapS)
  int32_t job;      // FusedJob of the group
  uint32_t dt;      // sub-batch (low 11 bits) | tile << 11
  int32_t kbt;      // count-vector slot of the tile (-1: the sub-batch is one tile)
  int32_t kbs;      // totals slot of the sub-batch (-1: one tile)
};
static_assert(sizeof(FItem) == 64, "an item is one 64-byte load");

cudaError_t fused_init_attributes();
// info[4 j + 0..3]: items, multi-tile tiles, multi-tile sub-batches, largest
// R sub-batch with pairs
template <typename K>
cudaError_t launch_fused_info(const FusedJob<K>* d_jobs, int nj, int64_t* d_info,
                              cudaStream_t st);
// the group's item list and (any_multi) the totals of its multi-tile
// sub-batches (d_kb_tot zeroed beforehand)
template <typename K>
cudaError_t launch_fused_prep(const FusedJob<K>* d_jobs, int nj, FItem* d_items, int64_t n_items,
                              bool any_multi, uint32_t* d_kb_tot, cudaStream_t st);
// the joins of the group's items (item and count-vector look-back zeroed);
// pairs from *d_out_base on, *d_total = the end of the group's pairs
template <typename K>
cudaError_t launch_fused_join(const FusedJob<K>* d_jobs, const FItem* d_items, int64_t n_items,
                              uint32_t* d_item_counter, uint64_t* d_item_lb, uint32_t* d_kb_lb,
                              const uint32_t* d_kb_tot, K* out, int64_t capacity,
                              const int64_t* d_out_base, int64_t* d_total, int* d_err,
                              cudaStream_t st);

// ---- late materialisation (tj_gather.cu) ------------------------------------
constexpr int kGatherCols = 16;  // columns per gather launch
struct GatherCol {
  const void* src;  // column of R (side 0) or S (side 1)
  void* dst;        // one element per pair
  int32_t side;
  int32_t bytes;    // 4 or 8
};
struct GatherArgs {
  GatherCol c[kGatherCols];
  int32_t n;
};
template <typename I>
cudaError_t launch_gather_pairs(const I* pairs, int64_t n, int64_t n_r, int64_t n_s,
                                const GatherArgs& a, int* d_err, int sms, cudaStream_t st);
// dst[i] = src[idx[i]] (idx a permutation of [0, n)); out[i] = i
template <typename K>
cudaError_t launch_gather_idx(const K* src, const K* idx, K* dst, int64_t n, int sms,
                              cudaStream_t st);
template <typename K>
cudaError_t launch_iota(K* out, int64_t n, int sms, cudaStream_t st);
// dst[0, n) = src[0, n) by a kernel (one side may be pinned, mapped host memory)
cudaError_t launch_copy_bytes(void* dst, const void* src, size_t n, cudaStream_t st);
// key columns folded into one key (pack) and back (unpack)
template <typename K>
struct PackArgs {
  K* col[kGatherCols];
  K lo[kGatherCols];
  int32_t shift[kGatherCols];
  int32_t bits[kGatherCols];
  int32_t n;
};
template <typename K>
cudaError_t launch_pack(const PackArgs<K>& a, K* packed, int64_t n, bool unpack, int sms,
                        cudaStream_t st);

// ---- launchers (tj_radix.cu) -----------------------------------------------
cudaError_t radix_init_attributes();
// Tiles of the radix kernels have `tile` rows (kTile, or kSortThreads * items
// of a smaller onesweep tile); jobs' tile0 counts tiles of that size.
template <typename K>
cudaError_t launch_stats(const RadixJob<K>* d_jobs, int num_jobs, int64_t total_tiles,
                         KeyStats* d_stats, cudaStream_t st, int tile = kTile);
template <typename K>
cudaError_t launch_histogram(const RadixJob<K>* d_jobs, int num_jobs, int64_t total_tiles,
                             cudaStream_t st, const int32_t* d_tile_job = nullptr,
                             int tile = kTile);
// d_map[t] = index of the job that owns tile t (jobs' tile0 / n in tile or kJTile rows)
template <typename K>
cudaError_t launch_fill_tile_job(const RadixJob<K>* d_jobs, int num_jobs, int32_t* d_map,
                                 cudaStream_t st, int tile = kTile);
template <typename K>
cudaError_t launch_fill_join_tile_job(const JoinJob<K>* d_jobs, int num_jobs, int32_t* d_map,
                                      cudaStream_t st);
template <typename K>
cudaError_t launch_digit_scan(const RadixJob<K>* d_jobs, int num_jobs, int passes,
                              cudaStream_t st);
template <typename K>
cudaError_t launch_onesweep(const RadixJob<K>* d_jobs, int num_jobs, int64_t total_tiles,
                            int pass, int max_bits, int mode, uint32_t* d_tile_counter,
                            int* d_err, cudaStream_t st, const int32_t* d_tile_job = nullptr,
                            int items = kItems, bool guard = false);

// ---- launchers (tj_join.cu) -------------------------------------------------
cudaError_t join_init_attributes();
template <typename K>
cudaError_t launch_tile_ranges(const JoinJob<K>* d_jobs, int num_jobs, int64_t total_tiles,
                               JTile<K>* d_tiles, cudaStream_t st,
                               const int32_t* d_tile_job = nullptr);
template <typename K>
cudaError_t launch_join(int64_t total_tiles, const JTile<K>* d_tiles, uint64_t* d_lookback,
                        uint32_t* d_tile_counter, K* out, int64_t capacity,
                        const int64_t* d_out_base, int64_t* d_job_out, int64_t* d_total,
                        int* d_err, cudaStream_t st);
// k_cross over a run of single-key batches: reads the run's base, writes
// base + run_pairs for the next run (CTA 0), and writes a batch's pairs only
// if all of them fit `capacity`.
template <typename K>
cudaError_t launch_cross(const CrossJob<K>* d_jobs, int num_jobs, int64_t blocks, K* out,
                         int64_t capacity, const int64_t* d_base, int64_t* d_next,
                         int64_t run_pairs, cudaStream_t st);
// tile -> job maps of a group's radix jobs (tile of kTile rows) and join jobs
template <typename K>
cudaError_t launch_group_maps(const RadixJob<K>* d_rjobs, int nr, int32_t* d_rmap,
                              const JoinJob<K>* d_jjobs, int nj, int32_t* d_jmap,
                              cudaStream_t st, int tile = kTile);

// ---- launchers (tj_learned.cu) ----------------------------------------------
template <typename K>
cudaError_t launch_sample_gather(const K* a, int64_t ma, int64_t off_a, const K* b, int64_t mb,
                                 int64_t off_b, int stride, K* out_k, K* out_v, cudaStream_t st);
template <typename K>
cudaError_t launch_quantiles(const K* sorted, int64_t m, int G, int first, int last, int step,
                             K* out, cudaStream_t st);
template <typename K>
cudaError_t launch_sorted_bucket_edges(const K* sorted, int64_t m, uint64_t lo, int shift, int nb,
                                       int64_t* edges, cudaStream_t st);
// counts[side * kMaxBins + p] += sample rows of the side (index < m_r: R) in batch p
template <typename K>
cudaError_t launch_sample_route_counts(const K* keys, const K* idx, int64_t m, int64_t m_r,
                                       const K* cuts, int ncuts, uint32_t* counts,
                                       cudaStream_t st);
// next[d] = base[d] + the inclusive count of digit d over a route launch's
// tiles (the last tile's look-back word), d < bins
cudaError_t launch_route_chain(const uint32_t* base, const uint32_t* lookback, int64_t last_tile,
                               int bins, uint32_t* next, cudaStream_t st);
template <typename K>
cudaError_t launch_fix_job_out(const JoinJob<K>* d_jobs, int num_jobs, int64_t total_tiles,
                               int64_t* d_job_out, const int64_t* d_total, cudaStream_t st);

// ---- launchers (tj_mlp.cu) ---------------------------------------------------
constexpr int kMlpParams = 1153;
cudaError_t mlp_init_attributes();
template <typename K>
cudaError_t launch_mlp_train(const K* sorted, int64_t m, float* theta, int steps, int batch,
                             float lr, uint64_t seed, int* steps_run, cudaStream_t st);
cudaError_t launch_mlp_grad(const float* theta, const float* x, const float* y, int n,
                            float* grad, cudaStream_t st);
cudaError_t launch_adam(float* theta, float* m, float* v, const float* g, int n, int t, float lr,
                        cudaStream_t st);
template <typename K>
cudaError_t launch_mlp_boundaries(const float* theta, int T, float* table, int parts,
                                  const K* sorted, int64_t m, K* out, cudaStream_t st);

}  // namespace tj
