/*
 * tj.h -- C ABI of the GB300 (sm_103a) tensor-path join and sort library
 * (libtj.so, built from paper_2602_21237_gb300/csrc).
 *
 * The operations follow arXiv 2602.21237:
 *   - tj_join_inner: the inner equi-join of two relations aligned on their
 *     common key axis (Sec. 4.1; Sec. 3.2 "join = alignment on the common
 *     axis"), with the result ordered by that key, key and row-id columns kept
 *     as separate device arrays until the single final materialisation of
 *     (r_id, s_id) pairs (Sec. 3.1, late materialisation).  The device memory
 *     budget plays the role of the paper's work_mem (Sec. 6, M): under it the
 *     join runs in several partitioned passes and never spills to the host.
 *   - tj_sort: ORDER BY one key, a stable relocation of rows along the key
 *     axis (Sec. 4.2).
 *
 * Conventions for every entry point:
 *   - Keys and ids are two's-complement signed integers of one width, given by
 *     tj_dtype (int32 or int64); every key value is legal (no reserved value).
 *   - Array arguments are caller-owned DEVICE pointers on the current CUDA
 *     device; sizes are element counts.  Inputs marked const are never written.
 *     Arrays need the natural alignment of their element type.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  All device
 *     work is ordered on it.  The library allocates its own scratch
 *     stream-ordered from the device's default memory pool and frees it before
 *     returning; nothing the caller owns is freed.
 *   - Errors are returned, never printed or thrown.  tj_last_error() gives a
 *     one-line detail for the calling thread's last failed call.
 *   - Relations are limited to n < 2^30 rows per array per call (the decoupled
 *     look-back words hold 30-bit counts); larger n returns TJ_ERR_INVALID.
 */
#ifndef TJ_H
#define TJ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TJ_OK = 0,
  TJ_ERR_INVALID = 1,  /* bad argument: null pointer with n > 0, n too large, bad dtype */
  TJ_ERR_BUDGET = 2,   /* mem_budget_bytes below the minimum working set of the plan */
  TJ_ERR_CAPACITY = 3, /* out_capacity < |J|; *out_count holds the required count */
  TJ_ERR_CUDA = 4,     /* a CUDA runtime call failed (sticky errors included) */
  TJ_ERR_TIMEOUT = 5,  /* a bounded device-side wait ran out (result undefined) */
  TJ_ERR_INTERNAL = 6  /* an internal consistency check failed */
} tj_status;

typedef enum { TJ_I32 = 0, TJ_I64 = 1 } tj_dtype;

/* Per-call counters of the calling thread's last successful call. */
typedef struct {
  int32_t key_bits;        /* significant bits of (key - min) over both inputs */
  int32_t radix_passes;    /* digit passes per sorted array */
  int32_t digit_bits;      /* widest digit used */
  int32_t groups;          /* key-range groups processed (1 = single pass) */
  int64_t scratch_peak;    /* peak bytes of library scratch live at once */
  int64_t staging_bytes;   /* bytes of partitioned relation copies (batches) */
  int64_t out_count;       /* pairs produced (join) */
  int32_t used_hbm_table;  /* 1 if the HBM hash table path ran */
  int32_t learned;         /* 1 if learned routing ran, 2 if it fell back to radix */
} tj_stats;

/*
 * Inner equi-join (Sec. 4.1): J = { (r.id, s.id) : r.key == s.key }.
 *
 * keys_r, ids_r : R's key and row-id columns, n_r rows each (const).
 * keys_s, ids_s : S's key and row-id columns, n_s rows each (const).
 * mem_budget_bytes : cap on the library's device scratch for this call
 *   (0 = unbounded).  The partitioned copies of R and S (the device-resident
 *   batches that replace the relational path's temp files) are counted in
 *   tj_stats.staging_bytes and, when the budget is below the single-pass
 *   working set, every pass's hash tables, sort workspaces, histograms and
 *   look-back state stay within the budget (Sec. 6: no spill regime).
 *   A budget below the smallest pass returns TJ_ERR_BUDGET.
 * out_pairs : device array of out_capacity pairs; pair i is
 *   out_pairs[2i] = r_id, out_pairs[2i+1] = s_id (id width).
 *   Pairs are ordered by key ascending, then by the S row's input position,
 *   then by the R row's input position.
 * out_count : HOST pointer; receives |J|.  If |J| > out_capacity the call
 *   returns TJ_ERR_CAPACITY, *out_count = |J| and out_pairs holds garbage.
 * The call synchronises `stream` twice (plan statistics, final count).
 */
tj_status tj_join_inner(tj_dtype dt, const void* keys_r, const void* ids_r, int64_t n_r,
                        const void* keys_s, const void* ids_s, int64_t n_s,
                        size_t mem_budget_bytes, void* out_pairs, int64_t out_capacity,
                        int64_t* out_count, void* stream);

/*
 * ORDER BY key (Sec. 4.2): stable sort of the rows (keys[i], ids[i]) by key
 * ascending, in place.  n rows; keys and ids are device arrays (read-write).
 * Synchronises `stream` once (key statistics for the digit plan).
 */
tj_status tj_sort(tj_dtype dt, void* keys, void* ids, int64_t n, void* stream);

/*
 * Many independent inner joins in one batch (no counterpart in the paper; it
 * batches Sec. 4.1 joins).  Job j joins R rows [r_off[j], r_off[j+1]) with S
 * rows [s_off[j], s_off[j+1]) of the concatenated device columns; r_off and
 * s_off are HOST arrays of n_jobs + 1 int64 offsets.  The output is the
 * concatenation of the jobs' outputs (each ordered as in tj_join_inner);
 * out_off (DEVICE, n_jobs + 1 int64) receives each job's first output index
 * and the total.  *out_count (HOST) receives the total; TJ_ERR_CAPACITY as in
 * tj_join_inner.  All jobs' kernels run together: one launch per phase for the
 * whole batch, captured once in a CUDA graph and replayed.
 */
tj_status tj_join_batch(tj_dtype dt, int64_t n_jobs, const int64_t* r_off, const int64_t* s_off,
                        const void* keys_r, const void* ids_r, const void* keys_s,
                        const void* ids_s, void* out_pairs, int64_t out_capacity,
                        int64_t* out_off, int64_t* out_count, void* stream);

/* Text of a status code (static storage). */
const char* tj_status_str(tj_status s);

/* One-line detail of the calling thread's last failed call ("" if none). */
const char* tj_last_error(void);

/* Counters of the calling thread's last successful call. */
tj_status tj_get_stats(tj_stats* out);

/*
 * Kernel trace (a profiling aid; no counterpart in the paper).  While enabled,
 * every kernel the library launches is bracketed by CUDA events on the
 * caller's stream; at the end of each call the elapsed times are added to a
 * process-wide table keyed by kernel name, together with the kernel's
 * algorithmic bytes (the reads and writes its algorithm needs, not counters).
 * Calls made while a stream is being captured are not traced.
 */
void tj_trace_enable(int on);
void tj_trace_reset(void);
int tj_trace_count(void);
/* Entry i of the table: name (copied, NUL-terminated, at most name_len bytes),
 * launches, total milliseconds, total algorithmic bytes.  TJ_ERR_INVALID if i
 * is out of range. */
tj_status tj_trace_get(int i, char* name, int name_len, int64_t* launches, double* ms,
                       double* bytes);

/* Library version string (static storage). */
const char* tj_version(void);

#ifdef __cplusplus
}
#endif

#endif /* TJ_H */
