/*
 * CPU oracle for the tensor-path join and sort (TEST INFRASTRUCTURE ONLY).
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
 * leg may load this file's library.  It shares no code, header, table or helper
 * with the CUDA path under paper_2602_21237_gb300/csrc/, and the product never
 * links or calls it.
 *
 * What it computes (plain definitions, written out):
 *
 *  - Inner equi-join (paper Sec. 4.1: "align the key axis of both relations and
 *    combine on it"; Sec. 3.3: the path chosen never changes the result;
 *    Sec. 5.1: results of both paths are checked for consistency):
 *        J = multiset { (r.id, s.id) : r in R, s in S, r.key == s.key }.
 *    The paper fixes no output order.  The order used by the library (and so by
 *    this oracle) is a total order on J:
 *        key ascending, then the input position of the S row, then the input
 *        position of the R row.
 *    That makes the output unique and comparable byte for byte.
 *
 *  - ORDER BY one key (paper Sec. 4.2, "relocation along the sort-key axis"):
 *    a stable permutation of the (key, id) rows by key ascending.  The paper
 *    does not say whether the sort is stable; stable is the reading taken here,
 *    which makes the result unique.
 *
 * Keys are two's-complement signed integers (int32 or int64); every value is a
 * legal key.  Ids share the key width.  Internally everything is widened to
 * int64, which preserves order and equality.
 *
 * Algorithms: nested loop for small inputs (n_r * n_s <= 1e6), otherwise sort
 * both sides by (key, position) with the C library qsort and walk the equal-key
 * runs (a plain sort-merge join).  Both produce the order stated above.  No
 * blocking, fusion or reordering beyond that.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define DT_I32 0
#define DT_I64 1

typedef struct {
  int64_t key;
  int64_t pos;
} kp_t;

typedef struct {
  int64_t key;
  int64_t spos;
  int64_t rpos;
} trip_t;

static int64_t load_val(int dt, const void* p, int64_t i) {
  if (dt == DT_I32) return (int64_t)((const int32_t*)p)[i];
  return ((const int64_t*)p)[i];
}

static void store_val(int dt, void* p, int64_t i, int64_t v) {
  if (dt == DT_I32)
    ((int32_t*)p)[i] = (int32_t)v;
  else
    ((int64_t*)p)[i] = v;
}

/* (key, position) ascending: a total order, so qsort's lack of stability does
 * not matter. */
static int cmp_kp(const void* a, const void* b) {
  const kp_t* x = (const kp_t*)a;
  const kp_t* y = (const kp_t*)b;
  if (x->key != y->key) return x->key < y->key ? -1 : 1;
  if (x->pos != y->pos) return x->pos < y->pos ? -1 : 1;
  return 0;
}

static int cmp_trip(const void* a, const void* b) {
  const trip_t* x = (const trip_t*)a;
  const trip_t* y = (const trip_t*)b;
  if (x->key != y->key) return x->key < y->key ? -1 : 1;
  if (x->spos != y->spos) return x->spos < y->spos ? -1 : 1;
  if (x->rpos != y->rpos) return x->rpos < y->rpos ? -1 : 1;
  return 0;
}

static kp_t* sorted_kp(int dt, const void* keys, int64_t n) {
  kp_t* v = (kp_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(kp_t));
  if (!v) return NULL;
  for (int64_t i = 0; i < n; ++i) {
    v[i].key = load_val(dt, keys, i);
    v[i].pos = i;
  }
  qsort(v, (size_t)n, sizeof(kp_t), cmp_kp);
  return v;
}

/*
 * Inner equi-join.  Writes min(|J|, cap) pairs (r_id, s_id) to out (2 values of
 * the id width per pair, r_id first) in the order stated above and returns |J|,
 * or -1 if host memory ran out.  out may be NULL when cap == 0 (count only).
 */
int64_t oracle_join_inner(int dt, const void* keys_r, const void* ids_r, int64_t n_r,
                          const void* keys_s, const void* ids_s, int64_t n_s, void* out,
                          int64_t cap) {
  int64_t count = 0;
  if (n_r <= 0 || n_s <= 0) return 0;

  if ((double)n_r * (double)n_s <= 1e6) {
    /* Nested loop over every (s, r) pair, then order the matches. */
    int64_t m = 0;
    for (int64_t s = 0; s < n_s; ++s)
      for (int64_t r = 0; r < n_r; ++r)
        if (load_val(dt, keys_s, s) == load_val(dt, keys_r, r)) ++m;
    trip_t* t = (trip_t*)malloc((size_t)(m > 0 ? m : 1) * sizeof(trip_t));
    if (!t) return -1;
    int64_t k = 0;
    for (int64_t s = 0; s < n_s; ++s)
      for (int64_t r = 0; r < n_r; ++r) {
        int64_t ks = load_val(dt, keys_s, s);
        if (ks == load_val(dt, keys_r, r)) {
          t[k].key = ks;
          t[k].spos = s;
          t[k].rpos = r;
          ++k;
        }
      }
    qsort(t, (size_t)m, sizeof(trip_t), cmp_trip);
    for (int64_t i = 0; i < m && i < cap; ++i) {
      store_val(dt, out, 2 * i, load_val(dt, ids_r, t[i].rpos));
      store_val(dt, out, 2 * i + 1, load_val(dt, ids_s, t[i].spos));
    }
    free(t);
    return m;
  }

  /* Sort-merge: both sides ordered by (key, position); walk equal-key runs. */
  kp_t* R = sorted_kp(dt, keys_r, n_r);
  kp_t* S = sorted_kp(dt, keys_s, n_s);
  if (!R || !S) {
    free(R);
    free(S);
    return -1;
  }
  int64_t i = 0, j = 0;
  while (i < n_s && j < n_r) {
    if (S[i].key < R[j].key) {
      ++i;
    } else if (R[j].key < S[i].key) {
      ++j;
    } else {
      int64_t key = S[i].key;
      int64_t i1 = i, j1 = j;
      while (i1 < n_s && S[i1].key == key) ++i1;
      while (j1 < n_r && R[j1].key == key) ++j1;
      for (int64_t a = i; a < i1; ++a)
        for (int64_t b = j; b < j1; ++b) {
          if (count < cap) {
            store_val(dt, out, 2 * count, load_val(dt, ids_r, R[b].pos));
            store_val(dt, out, 2 * count + 1, load_val(dt, ids_s, S[a].pos));
          }
          ++count;
        }
      i = i1;
      j = j1;
    }
  }
  free(R);
  free(S);
  return count;
}

/*
 * Stable ORDER BY key of (keys, ids) in place.  Returns 0, or -1 if host
 * memory ran out.
 */
int oracle_sort(int dt, void* keys, void* ids, int64_t n) {
  if (n <= 1) return 0;
  kp_t* v = sorted_kp(dt, keys, n);
  int64_t* idc = (int64_t*)malloc((size_t)n * sizeof(int64_t));
  if (!v || !idc) {
    free(v);
    free(idc);
    return -1;
  }
  for (int64_t i = 0; i < n; ++i) idc[i] = load_val(dt, ids, i);
  for (int64_t i = 0; i < n; ++i) {
    store_val(dt, keys, i, v[i].key);
    store_val(dt, ids, i, idc[v[i].pos]);
  }
  free(v);
  free(idc);
  return 0;
}

/*
 * Batched joins: job j joins R_j with S_j, where the jobs' rows are stored back
 * to back (job j's R rows start at r_off[j], its S rows at s_off[j]).  The
 * output is the concatenation of the jobs' outputs in job order;
 * out_off[j] receives the first output index of job j (out_off has n_jobs + 1
 * entries, the last is the total).  Returns the total or -1.
 */
int64_t oracle_join_batch(int dt, int64_t n_jobs, const int64_t* r_off, const int64_t* s_off,
                          const void* keys_r, const void* ids_r, const void* keys_s,
                          const void* ids_s, void* out, int64_t cap, int64_t* out_off) {
  size_t w = (dt == DT_I32) ? 4 : 8;
  int64_t total = 0;
  for (int64_t j = 0; j < n_jobs; ++j) {
    int64_t nr = r_off[j + 1] - r_off[j];
    int64_t ns = s_off[j + 1] - s_off[j];
    out_off[j] = total;
    int64_t room = cap - total;
    if (room < 0) room = 0;
    void* dst = out ? (void*)((char*)out + (size_t)(2 * total) * w) : NULL;
    int64_t c = oracle_join_inner(dt, (const char*)keys_r + (size_t)r_off[j] * w,
                                  (const char*)ids_r + (size_t)r_off[j] * w, nr,
                                  (const char*)keys_s + (size_t)s_off[j] * w,
                                  (const char*)ids_s + (size_t)s_off[j] * w, ns,
                                  room > 0 ? dst : NULL, room);
    if (c < 0) return -1;
    total += c;
  }
  out_off[n_jobs] = total;
  return total;
}
