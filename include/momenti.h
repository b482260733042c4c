/*
 * momenti.h - C ABI of the GB300 (sm_103a) LSH top-k multidimensional motif
 * search of MOMENTI (Ceccarello, Monaco, Silvestri; arXiv 2502.14446).
 *
 * Problem (Section 3.1, Definition of the top-k multidimensional motifs):
 * given a D-dimensional series T of length n, a window length w, a motif
 * dimensionality d and a count k, return the k pairs of length-w windows
 * (a, b) with the smallest d-dimensional distance dist_d (Definition
 * distdims: the sum of the d smallest per-dimension z-normalised Euclidean
 * distances, Eq. zned), no two returned windows being trivial matches
 * (|a - b| <= eps, eps = w/2).  The search is Algorithm 1 (MOMENTI) with the
 * stopping rule of Algorithm 2: each returned motif is the exact one with
 * probability at least 1 - delta (Lemma topk), or 1 - delta over all k in the
 * ALL_K mode (Lemma topkdip).
 *
 * Conventions for every entry point:
 *   - return value: MOMENTI_OK (0) or a negative MOMENTI_ERR_* code; no C++
 *     exception crosses the ABI (host memory exhaustion is reported as
 *     MOMENTI_ERR_MEMORY); momenti_last_error() gives a message;
 *   - pointers are host pointers unless a parameter says otherwise; the
 *     caller owns every buffer it passes and the handle owns everything it
 *     allocates (released by momenti_destroy);
 *   - a handle is single-threaded: calls on one handle must not overlap;
 *   - all GPU work of a handle runs on the stream given to momenti_hash_all
 *     (the legacy default stream when NULL); calls return after that stream
 *     has finished the call's work, unless stated otherwise; that stream
 *     must stay valid until the next momenti_hash_all or momenti_destroy
 *     (device buffers are released on it);
 *   - device memory comes from a stream-ordered pool of the library, one per
 *     device, trimmed by momenti_destroy (the batching form's worker
 *     handles are destroyed, so the pool is trimmed when a batch ends).
 */
#ifndef MOMENTI_H
#define MOMENTI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define MOMENTI_OK            0
#define MOMENTI_ERR_ARG      (-1)  /* invalid argument (see each call)          */
#define MOMENTI_ERR_MEMORY   (-2)  /* the memory limit cannot hold one repetition */
#define MOMENTI_ERR_CUDA     (-3)  /* a CUDA runtime call failed               */
#define MOMENTI_ERR_TIMEOUT  (-4)  /* a bounded device wait ran out            */
#define MOMENTI_ERR_OVERFLOW (-5)  /* an internal buffer overflowed            */
#define MOMENTI_ERR_STATE    (-6)  /* call out of order (e.g. topk before hash_all) */

/* ---- enumerations ---------------------------------------------------- */
#define MOMENTI_F32 0              /* series element type float  */
#define MOMENTI_F64 1              /* series element type double */

#define MOMENTI_PREC_FP32  0       /* projections as plain FP32 FMAs on CUDA cores          */
#define MOMENTI_PREC_F16X2 1       /* projections on tcgen05 tensor cores, FP16 hi+lo split
                                      of the z-normalised windows, FP32 accumulation       */

#define MOMENTI_DELTA_PER_MOTIF 0  /* Algorithm 2 with delta (Lemma topk)      */
#define MOMENTI_DELTA_ALL_K     1  /* Algorithm 2 with delta / k (Lemma topkdip) */

#define MOMENTI_MAX_D 64           /* dimensions per series (dims travel as a 64-bit mask) */
#define MOMENTI_MAX_K 8            /* concatenations: one byte each in a 64-bit key */

/* ---- parameters (Algorithm 1's inputs, Section 3.2 and Section 6.1) --- */
typedef struct momenti_params {
  int32_t  w;             /* window length, 2 <= w <= n                          */
  int32_t  d;             /* motif dimensionality, 1 <= d <= D                   */
  int32_t  k;             /* number of motifs, >= 1                              */
  double   delta;         /* failure probability, 0 < delta < 1                  */
  uint64_t mem_limit;     /* device bytes the handle may hold; 0 = 80% of free   */
  int32_t  K;             /* concatenations, 1..8 (paper default 8)              */
  int32_t  L;             /* maximum repetitions (paper default 200); 0 = as many
                             as mem_limit allows, at most 4096. The memory planner
                             may use fewer (momenti_stats.L).                      */
  double   r;             /* quantisation width of Eq. drp; <= 0 selects the
                             heuristic of Section 6.1                              */
  int32_t  excl;          /* exclusion zone eps; < 0 selects w / 2 (Section 3.1) */
  uint64_t seed;          /* seed of the hash functions drawn on the device      */
  int32_t  precision;     /* MOMENTI_PREC_*                                      */
  int32_t  delta_mode;    /* MOMENTI_DELTA_*                                     */
  uint32_t flags;         /* MOMENTI_FLAG_* (0 = defaults)                       */
  uint32_t reserved;
} momenti_params;

/* flags: count collisions at every prefix length with the pair tiles instead
 * of the bucket jobs of prefix lengths 1..3 (same candidates; for tests). */
#define MOMENTI_FLAG_TILES_ONLY 1u
/* flags: follow Algorithm 1's loop to its end before the exact path (no
 * cost switch).  By default each level starts with a one-repetition probe
 * whose work counts predict the rest of the traversal (the rest of the
 * level, and each lower level at least as much); when that prediction
 * exceeds the predicted time of the exact all-pairs path, the traversal
 * stops there and the exact path runs (its result is the exact top-k, the
 * probability-1 branch of Lemma topk). */
#define MOMENTI_FLAG_NO_COST_SWITCH 2u
/* flags: tensoring (Section 6.1).  The L = m^2 repetitions are built from m
 * left and m right hash functions of K/2 values each (K even): repetition
 * j' (0-based) interleaves the values of left function j' div m and right
 * function j' mod m, a left value first.  The projections cover K m hash
 * values per window and dimension instead of K L.  The memory planner
 * keeps L a square (the largest that fits, at most params.L, 4096 when 0).
 * The r heuristic projects the sample windows onto the K/2 vectors of
 * left function 0.  STOP compares the re-derived tensoring bound
 * (momenti_tensoring_failure_bound of P(dist_max)^d) with delta.  Explicit
 * hash functions (momenti_set_hash_params) are then 2 m' half functions of
 * K/2 values, left function l at index 2 l and right function r at
 * 2 r + 1 (m' >= the m the planner uses). */
#define MOMENTI_FLAG_TENSORING 4u

/* One motif: windows a < b (0-based), dist_d (Definition distdims),
 * dist_d^max (Eq. distdmax), the dims_d set as a bit mask (bit f = dim f),
 * and fail_bound = the miss-probability bound of Lemma stop at return
 * (0 when Algorithm 1's exact all-pairs fallback produced it). */
typedef struct momenti_motif {
  int64_t  a, b;
  double   dist_d;
  double   dist_max;
  double   fail_bound;
  uint64_t dims_mask;
} momenti_motif;

/* Counters of one momenti_topk call. */
typedef struct momenti_stats {
  int32_t  stop_i, stop_j;   /* (i, j) at which STOP held, 1-based; 0, 0 = exact path */
  int32_t  K, L;             /* concatenations and repetitions used                   */
  double   r;                /* quantisation width used                               */
  int64_t  n_windows;        /* M = n - w + 1                                         */
  int64_t  n_candidates;     /* (pair, repetition) events with W >= d, first dim only */
  int64_t  n_verified;       /* distinct pairs whose distances were computed          */
  int64_t  n_pool;           /* distinct verified pairs held by TOP's pool            */
  int32_t  fallback;         /* 1 if Algorithm 1's exact fallback (all pairs) ran    */
  int32_t  n_chunks;         /* device round trips of the traversal                   */
  double   t_hash_ms;        /* momenti_hash_all: stats, r, projections, hashes       */
  double   t_sort_ms;        /*   of which the index sort                             */
  double   t_traverse_ms;    /* momenti_topk: collision counting, verification, STOP  */
  double   t_fallback_ms;    /* momenti_topk: exact all-pairs path                     */
  double   max_rel_err_fp32; /* max |FP32 - FP64| / FP64 of dist_d over the result    */
  uint64_t device_bytes;     /* device bytes held by the handle                        */
  int32_t  precision_used;   /* MOMENTI_PREC_* of the projections that ran            */
  int32_t  reserved;
  uint64_t n_rehashed;       /* tensor-core values re-hashed in FP32 (near a boundary) */
  int64_t  n_lb_pruned;      /* candidates dropped by the segment-mean lower bound    */
  double   t_host_ms;        /* host time replaying TOP and STOP in the traversal     */
  int32_t  switch_level;     /* level i at which the cost switch chose the exact path, 0 = none */
  int32_t  reserved2;
  int64_t  n_pair_checks;    /* bucket pairs compared by collision counting           */
  double   predicted_rest_ms;  /* cost model at the switch: rest of the traversal     */
  double   predicted_exact_ms; /*   and the exact path                                */
} momenti_stats;

typedef struct momenti_handle momenti_handle;

/* Fills *p with the paper's defaults (Section 7, default parameter values:
 * K = 8, L = 200, delta = 0.01, r automatic) and w = 100, d = 1, k = 1,
 * eps = w/2, FP16x2 tensor-core projections.  Returns MOMENTI_ERR_ARG if p
 * is NULL. */
int momenti_default_params(momenti_params* p);

/* Validates *p and creates a handle (no device memory yet).
 * MOMENTI_ERR_ARG: out or p NULL, w < 2, d < 1, k < 1, delta not in (0,1),
 * K not in 1..8, L < 0, unknown precision or delta_mode, or
 * MOMENTI_FLAG_TENSORING with an odd K. */
int momenti_create(momenti_handle** out, const momenti_params* p);

/* Releases the handle and every device buffer it holds.  NULL is a no-op. */
void momenti_destroy(momenti_handle* h);

/* Message of the last failing call on h (static text when h is NULL). */
const char* momenti_last_error(const momenti_handle* h);

/* Optional: the random numbers of the D * L * K hash functions of Eq. drp,
 * h(x) = floor((a . x + b) / r), instead of drawing them on the device.
 * a: D*L*K*w floats, layout [f][j][k][t], N(0,1) draws; they are used
 * rounded to IEEE half precision (pass half-representable values to make
 * the rounding exact).  u: D*L*K floats in [0, 1), layout [f][j][k];
 * b = u * r.  L here is the number of repetitions supplied; the memory
 * planner uses the first L_used <= L of them.  With MOMENTI_FLAG_TENSORING,
 * L counts half functions (even; left l at 2 l, right r at 2 r + 1) and K
 * is their K/2 values.  Copied by the call.
 * MOMENTI_ERR_ARG on NULL pointers, w / K mismatch with the parameters,
 * D not in 1..64, an odd L under tensoring, or u outside [0, 1). */
int momenti_set_hash_params(momenti_handle* h, int32_t D, int32_t L, int32_t K, int32_t w,
                            const float* a, const float* u);

/* The hashing step of Algorithm 1 and the index of Section 4 ("Index construction"):
 * rolling mean / std of every window (population sigma, float64 running
 * sums), r by the heuristic of Section 6.1 unless fixed, the composite hash
 * h_{K,j}^f of every window, dimension and repetition, and for every (j, f)
 * the windows sorted lexicographically by hash string.
 *   series : D rows of n elements, row f at series + f * ld (elements), of
 *            type dtype (MOMENTI_F32 / MOMENTI_F64); a device pointer if
 *            on_device != 0 (borrowed only during the call), else host.
 *   stream : cudaStream_t for all work of this handle, or NULL.
 * The index stays on the device, owned by the handle; a later call
 * replaces it.  MOMENTI_ERR_ARG: NULL series, D not in 1..64 or not the D
 * of set_hash_params, d > D, n < w, ld < n, n - w + 1 >= 65535 * 2048
 * (134,215,680 windows).
 * MOMENTI_ERR_MEMORY: the limit cannot hold the series, its statistics and
 * one repetition. */
int momenti_hash_all(momenti_handle* h, const void* series, int32_t dtype, int64_t n,
                     int32_t D, int64_t ld, int32_t on_device, void* stream);

/* Algorithm 1 after hashing, with Algorithm 2: traverses prefixes i = K..1 and
 * repetitions j = 1..L, counts per pair the dimensions sharing the length-i
 * prefix (W), verifies pairs with W >= d, keeps TOP and stops when STOP
 * holds; otherwise returns the exact top-k over all pairs — after the
 * whole loop, or (by default) as soon as the work model predicts the rest
 * of the traversal to cost more than the exact path (MOMENTI_FLAG_NO_COST_
 * SWITCH; stats->switch_level).  Distances of the result are re-verified
 * in float64.
 *   out   : room for k motifs, sorted by (dist_d, a, b);
 *   n_out : number written (k unless fewer than k non-trivial pairs exist);
 *   stats : optional counters (may be NULL).
 * MOMENTI_ERR_STATE before momenti_hash_all. */
int momenti_topk(momenti_handle* h, momenti_motif* out, int32_t* n_out, momenti_stats* stats);

/* Section 6.3, motifs of several dimensionalities: the top-k motifs of
 * every d in [d_low, d_high] from one traversal.  One TOP per d; the
 * collision condition W >= d uses the smallest d not yet confirmed; every
 * verified pair is offered to the TOP of every unconfirmed d (its
 * per-dimension distances give dist_d for all d); after each repetition
 * every unconfirmed d whose TOP passes STOP (Algorithm 2 with its own d) is
 * confirmed at that (i, j); each d still unconfirmed when the loop ends
 * (or when the cost switch chooses it) gets the exact top-k.  Each d's
 * result carries the guarantee of Lemma topk for that d.  params.d of the
 * handle is not used.
 *   out   : (d_high - d_low + 1) * k motifs, row q for d = d_low + q, each
 *           sorted by (dist_d, a, b) and float64 re-verified;
 *   n_out : d_high - d_low + 1 counts;
 *   stops : optional, 2 per d: the (i, j) at which d was confirmed, 0 0 for
 *           the exact path;
 *   stats : optional counters (stop_i, stop_j of d_low; fallback = 1 if
 *           any d took the exact path).
 * MOMENTI_ERR_ARG unless 1 <= d_low <= d_high <= D; MOMENTI_ERR_STATE
 * before momenti_hash_all. */
int momenti_topk_multi(momenti_handle* h, int32_t d_low, int32_t d_high, momenti_motif* out,
                       int32_t* n_out, int32_t* stops, momenti_stats* stats);

/* ---- anytime search (Section 4, the remark after Algorithm 1) ---------
 * The traversal of momenti_topk / momenti_topk_multi as a search that can
 * be advanced, inspected and resumed: TOP only ever admits better pairs, so
 * at any point it holds candidate motifs whose miss probability the bound
 * of Lemma stop gives for the repetitions done so far.
 *   momenti_search_begin   starts a search for d_low..d_high (one d for the
 *                          plain problem) on the current index, replacing
 *                          any search in progress;
 *   momenti_search_step    advances it by at least one and at most max_reps
 *                          repetitions (fewer at the end); *ended (may be
 *                          NULL) becomes 1 once STOP held for every d, the
 *                          cost switch chose the exact path, or the loop
 *                          ran out; further steps are no-ops;
 *   momenti_search_current the current TOP of every d: out (k per d, as
 *                          momenti_topk_multi), n_out per d; each motif's
 *                          fail_bound is the bound of Lemma stop for its own
 *                          dist_d^max after the last repetition processed
 *                          (1 before any; the confirming value for a d that
 *                          STOP confirmed); distances are the traversal's
 *                          float32 form; cursor (3 ints, may be NULL): the
 *                          last (i, j) processed and the ended flag;
 *   momenti_search_finish  completes it (the rest of the traversal, the
 *                          float64 re-verification, the exact top-k of any d
 *                          STOP did not confirm) with the outputs of
 *                          momenti_topk_multi, and ends the search.
 * momenti_hash_all ends a search in progress.  MOMENTI_ERR_STATE without a
 * search (or before momenti_hash_all); MOMENTI_ERR_ARG for bad d bounds or
 * max_reps < 1. */
int momenti_search_begin(momenti_handle* h, int32_t d_low, int32_t d_high);
int momenti_search_step(momenti_handle* h, int64_t max_reps, int32_t* ended);
int momenti_search_current(momenti_handle* h, momenti_motif* out, int32_t* n_out, int32_t* cursor);
int momenti_search_finish(momenti_handle* h, momenti_motif* out, int32_t* n_out, int32_t* stops,
                          momenti_stats* stats);

/* The final fallback of Algorithm 1 alone: the exact top-k over all pairs (the quantity
 * of Definition top-k), on the GPU, float64 re-verified.  Same outputs and
 * errors as momenti_topk.
 *
 * For a float32 series the all-pairs sweep has several forms that record
 * the same pairs; the first sweep of an index times them on a part of the
 * grid and keeps the fastest per (device, padded D, log2 w, log2 M) for the
 * process.  Environment: MOMENTI_AUTOTUNE=0 takes the default form,
 * MOMENTI_SWEEP_VARIANT=v (a digit) forces form v, MOMENTI_TRACE=1 prints
 * the choice, one line per traversal chunk and one per exact-path sweep to
 * stderr. */
int momenti_topk_exact(momenti_handle* h, momenti_motif* out, int32_t* n_out);

/* Eq. zned per dimension and Definition distdims for m given pairs
 * (pairs[2q], pairs[2q+1]), 0 <= a, b < M.  Outputs (host, caller-owned,
 * any may be NULL): per_dim m*D distances [q][f], dist_d m values, dims_mask
 * m masks of the d best dims.  fp64 != 0 computes in float64, else in the
 * float32 form the traversal uses.  MOMENTI_ERR_ARG on an index outside
 * [0, M); MOMENTI_ERR_STATE before momenti_hash_all. */
int momenti_verify(momenti_handle* h, const int64_t* pairs, int64_t m, double* per_dim,
                   double* dist_d, uint64_t* dims_mask, int32_t fp64);

/* ---- batching form ----------------------------------------------------- */

/* Many independent searches at once: B series, each with its own
 * parameters, length and dimension count (the batching form: series of
 * uneven lengths and widths).  Series b is searched exactly as
 *   momenti_create(&h, &params[b]);
 *   momenti_hash_all(h, series[b], dtype[b], n[b], D[b], n[b], on_device, s);
 *   momenti_topk(h, out + b * out_stride, &n_out[b], stats + b);
 * would, and gives the same result (no arithmetic differs).  The work is
 * spread over `threads` worker handles (8 when <= 0), each on its own
 * non-blocking CUDA stream and host thread, taking the series longest first
 * (by n * D), so the GPU interleaves the searches; device memory is held by
 * at most `threads` series at a time.
 *   params   : B parameter records, each checked as momenti_create checks one;
 *              a zero mem_limit means 80% of the free memory / threads
 *   series   : B pointers to D[b] x n[b] row-major arrays (row stride n[b]),
 *              host memory, or device memory when on_device != 0 (already
 *              written: the workers' streams do not wait for other streams)
 *   out      : B * out_stride motifs; out_stride >= every params[b].k
 *   n_out    : B counts; stats (B entries) and rc (B statuses) may be NULL
 *   err      : optional buffer (err_len bytes) for the first failure's
 *              message, "series <b>: <text>"
 * Returns MOMENTI_OK, MOMENTI_ERR_ARG for bad batch arguments (nothing
 * run), or the status of the lowest-numbered failing series; a failing
 * series does not stop the others. */
int momenti_topk_batch(int32_t B, const momenti_params* params, const void* const* series,
                       const int32_t* dtype, const int64_t* n, const int32_t* D, int32_t on_device,
                       int32_t threads, momenti_motif* out, int32_t out_stride, int32_t* n_out,
                       momenti_stats* stats, int32_t* rc, char* err, int32_t err_len);

/* ---- inspection of the index (for tests and tools) ------------------- */

/* Sizes of the current index: M windows, D dims, L_used repetitions, K, r. */
int momenti_get_info(const momenti_handle* h, int64_t* M, int32_t* D, int32_t* L, int32_t* K,
                     double* r);

/* Window statistics, host arrays of D*M doubles, layout [f][a]. */
int momenti_get_window_stats(momenti_handle* h, double* mu, double* sigma);

/* Composite keys of repetition j (0-based): M*D uint64 [a][f]; byte 7-k
 * (k = 0 most significant) holds h_k + 128, bytes beyond K are zero. */
int momenti_get_keys(momenti_handle* h, int32_t j, uint64_t* keys);

/* The random numbers of the hash functions the index was built with
 * (Eq. drp: a ~ N(0,1)^w, b = u r with u ~ U[0,1)), for the first L_used
 * repetitions (momenti_get_info's L; under MOMENTI_FLAG_TENSORING the 2 m
 * half functions of K/2 values, m^2 = L, laid out as for
 * momenti_set_hash_params): a D*L*K*w floats, layout [f][j][k][t],
 * as the projections use them (rounded to half precision); u D*L*K floats,
 * layout [f][j][k].  Drawn on the device from seed (Philox4x32-10, Salmon
 * et al. SC'11: counter {q, q >> 32, stream, 0}, key {seed, seed >> 32};
 * element 4q + e of a takes Box-Muller on outputs (2h, 2h + 1) of counter q,
 * stream 0, h = e / 2, cos for even e, sin for odd, with u1 = ((x >> 8) + 1)
 * 2^-24 and u2 = (x >> 8) 2^-24; element 4q + e of u is output e of counter
 * q, stream 1, as (x >> 8) 2^-24), or the values given to
 * momenti_set_hash_params.  Either output may be NULL (not both).
 * MOMENTI_ERR_STATE before momenti_hash_all. */
int momenti_get_hash_draws(momenti_handle* h, float* a, float* u);

/* Sorted index of (j, f): order[p] = window at rank p (ties by window
 * index), lcp[p] = hash values shared with rank p - 1 (lcp[0] = 0). */
int momenti_get_index(momenti_handle* h, int32_t j, int32_t f, uint32_t* order, uint8_t* lcp);

/* The collision count of Algorithm 1 for one (i, j), 1-based i and 0-based j: the
 * non-trivial pairs (a < b) with W >= d at prefix length i in repetition j,
 * each once, without the cross-level and cross-repetition de-duplication
 * of the traversal.  pairs: room for 2*cap int64; *count = total found
 * (may exceed cap; only cap are written). */
int momenti_collide(momenti_handle* h, int32_t i, int32_t j, int64_t* pairs, int64_t cap,
                    int64_t* count);

/* ---- host arithmetic of the search (no device needed) ----------------- */

/* Eq. (eucl-collision-probability): the probability that one hash function
 * h(x) = floor((a . x + b) / r) gives two vectors at Euclidean distance R
 * the same value; 1 for R <= 0, NaN for r <= 0 or a NaN R.  The function
 * momenti_topk uses. */
double momenti_collision_probability(double R, double r);

/* The miss-probability bound of Lemma stop (Eq. probnotcolliding) that
 * Algorithm 2 compares with delta, for a pair with dist_d^max = dist_max
 * after repetition j of prefix length i (both 1-based, 1 <= i <= K,
 * 0 <= j <= L): with p = P(dist_max)^d, (1 - p^i)^j when i = K, else
 * (1 - p^i)^j (1 - p^(i+1))^(L - j).  The function momenti_topk uses;
 * NaN for arguments outside those ranges, d < 1, r <= 0 or a NaN dist_max. */
double momenti_failure_bound(double dist_max, int32_t i, int32_t j, int32_t K, int32_t L,
                             int32_t d, double r);

/* Tensoring (Section 6.1), its miss-probability bound re-derived: the
 * probability that a pair whose hash values collide independently with
 * probability p (pass P(dist_max)^d) was missed after j repetitions at
 * prefix length i, when the L = m^2 repetitions pair m left and m right
 * functions of K/2 values each (repetition j', 0-based: left j' div m,
 * right j' mod m) and keys interleave their values, left first; for i < K
 * every repetition has also been seen at length i + 1.  Exact under that
 * model, so an upper bound for any p at most the true one.  NaN unless
 * 0 <= p <= 1, K even >= 2, 1 <= i <= K, L a square, 0 <= j <= L. */
double momenti_tensoring_failure_bound(double p, int32_t i, int32_t j, int32_t K, int32_t L);

/* TOP of Algorithm 1 over given candidates, through the pool momenti_topk
 * keeps: the m pairs (a[q] < b[q]) with distances dd[q] (float, as the
 * device records them) enter in order, batch at a time, as verified pairs
 * enter the pool during the search (a pair seen before keeps its first
 * distance); afterwards TOP is the top-k motif set of Section 3.1 (trivial-
 * match exclusion eps) over the distinct pairs: taken in ascending
 * (dd, a, b) order, a pair is accepted iff b - a > eps and both of its
 * indices are more than eps away from both indices of every accepted
 * pair, until k are accepted.  idx (room for k) receives the positions q
 * (first occurrences) of TOP's pairs in order, *n_out their number.  Host
 * arrays, caller-owned; nothing is kept; no device is used.
 * MOMENTI_ERR_ARG: NULL arrays (m > 0), idx or n_out NULL, m < 0, k < 1,
 * eps < 0, batch < 1, a NaN distance, or an index outside 0 .. 2^32 - 1
 * or a >= b. */
int momenti_top_select(const float* dd, const int64_t* a, const int64_t* b, int64_t m,
                       int32_t k, int64_t eps, int64_t batch, int64_t* idx, int32_t* n_out);

/* ---- index sort without allocation ------------------------------------ */

/* Largest key count momenti_index_sort_noalloc accepts. */
#define MOMENTI_NOALLOC_MAX_KEYS 262144

/* The paper has no counterpart: this is a service for callers that must
 * not allocate device memory, for example code that runs under a fixed
 * device-memory budget reserved at start-up, or code called from inside
 * another allocator (a caching allocator or an out-of-memory handler),
 * where a nested cudaMalloc could fail or recurse.
 *
 * Sorts m composite hash keys (device array keys, the layout of one
 * (repetition, dimension) column of momenti_get_keys) the way the index of
 * momenti_hash_all is sorted: order[p] = position of the key at rank p
 * (ties by position), lcp[p] = leading bytes shared with rank p - 1, at
 * most K (lcp[0] = 0).  order (m uint32) and lcp (m uint8) are caller-owned
 * device arrays.  Work is queued on stream (cudaStream_t, NULL = legacy
 * default stream) and the call returns without waiting for it.
 *
 * It allocates nothing: its scratch is a fixed array inside the library
 * (about 6.4 MB per device that loads the library, held until the process
 * exits).  The first call on a device looks up that array's device address
 * (cudaGetSymbolAddress, with that device current) and keeps it with the
 * id of the current CUDA context; a call made in another context (after
 * cudaDeviceReset, for instance, which invalidates the kept address) looks
 * it up again.  Make the first call on a device, and the first after a
 * reset, before any stream capture.  Every call on a device shares the
 * array and leaves the last call's contents in it; calls whose work
 * overlaps on the GPU race on it, so serialise them (one stream, or
 * events).
 * Errors: MOMENTI_ERR_OVERFLOW if m > MOMENTI_NOALLOC_MAX_KEYS;
 * MOMENTI_ERR_ARG for NULL arrays (m > 0), m < 0 or K outside 1..8;
 * MOMENTI_ERR_CUDA if a CUDA error is already pending in the calling
 * thread (left by earlier work; it is not cleared and nothing is
 * launched), or if the address lookup or a launch fails. */
int momenti_index_sort_noalloc(const uint64_t* keys, int64_t m, int32_t K, uint32_t* order,
                               uint8_t* lcp, void* stream);

/* ---- launch accounting (for benchmarks) ------------------------------ */

/* Number of CUDA kernels this library has launched in the process.
 * (The paper has no counterpart: this is instrumentation.) */
uint64_t momenti_launch_count(void);

/* Starts timing every launch of the kernel called name with CUDA events on
 * the launching stream, and clears the accumulated time; NULL stops timing.
 * A name ending in '*' selects every kernel whose name starts with the part
 * before it (for example "sort_*": all kernels of the index sort).
 * Kernel names: split_f32, split_f64, point_major, window_stats,
 * stats_pm, col_prep, mean16, r_sample, draw, layout_hash, layout_boff,
 * proj_hash_fp32, proj_hash_tc, rehash, sort_init, sort_hist, sort_scan,
 * sort_scatter, sort_local, tensor_keys, chunk_agg, chunk_scan, scan_local, scan_top,
 * scan_add, collide, bucket_jobs, subbucket, subwarp, hs_clear,
 * verify_events, verify_pairs, allpairs, allpairs_batch, select_pairs. */
int momenti_time_kernel(const char* name);

/* Device time in milliseconds accumulated by the timed kernel since the
 * last momenti_time_kernel call, and the number of timed launches.  Waits
 * for the recorded events. */
int momenti_kernel_time(double* total_ms, uint64_t* launches);

#ifdef __cplusplus
}
#endif

#endif /* MOMENTI_H */
