/*
 * fbn.h -- C ABI of the GB300 PC-stable skeleton engine (Fast-BNS method,
 * arXiv 2212.04259) for discrete data with the G^2 conditional-independence
 * test.
 *
 * Every entry point returns an int status: FBN_OK (0) on success, a negative
 * FBN_E* code otherwise; fbn_last_error() then gives a one-line reason.  A
 * handle is not thread-safe: calls on one handle must not overlap.  Outputs go
 * to caller-provided buffers.  Pointers documented as "host or device" are
 * classified with cudaPointerGetAttributes; device pointers must belong to the
 * handle's device.  No function falls back to the CPU: without a usable CUDA
 * device, fbn_create returns FBN_ECUDA.
 *
 * Notation: n variables V_0..V_{n-1}, N samples, r_v = arity of V_v.  A CI test
 * I(X, Y | S) builds the contingency table N_xyz over all samples and reduces
 * it to G^2, df and a chi-square p-value (Section III-B).
 */
#ifndef FBN_H
#define FBN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define FBN_OK        0
#define FBN_EINVAL   (-1)  /* bad argument (null pointer, size or index out of range) */
#define FBN_EDATA    (-2)  /* a data value is >= its variable's arity */
#define FBN_ENOMEM   (-3)  /* device or host allocation failed */
#define FBN_ECUDA    (-4)  /* a CUDA runtime call or kernel failed */
#define FBN_ETOOBIG  (-5)  /* a contingency table exceeds the supported cell count */
#define FBN_ETIMEOUT (-6)  /* a bounded device wait gave up */
#define FBN_ENUMERIC (-7)  /* the p-value iteration did not converge */

/* ---- options ----------------------------------------------------------- */
#define FBN_FORM_POOL  0   /* CI-level work pool: persistent kernel, atomic chunk claims (Section IV-B) */
#define FBN_FORM_PLAIN 1   /* edge-level form: one CTA per edge, one launch per depth (Section IV-A) */

#define FBN_DEPTH0_AUTO 0  /* tensor-core one-hot Gram when the problem is large enough, else histogram */
#define FBN_DEPTH0_HIST 1  /* depth 0 through the shared-memory histogram path */
#define FBN_DEPTH0_GRAM 2  /* depth 0 through the tcgen05 one-hot Gram */

#define FBN_DEPTH1_AUTO   0  /* the work pool (the faster of the two on the measured workloads) */
#define FBN_DEPTH1_POOL   1  /* depth 1 through the work pool */
#define FBN_DEPTH1_TENSOR 2  /* depth 1 through the tcgen05 neighbourhood product (arities <= 8, else FBN_EINVAL) */

#define FBN_STAT_G2 0      /* G^2 = 2 sum N ln(N / E) (Section III-B) */
#define FBN_STAT_X2 1      /* Pearson's X^2 = sum (N - E)^2 / E over cells with E > 0, same table and df */

#define FBN_DF_FIXED    0  /* df = (r_x - 1)(r_y - 1) prod r_z from the declared arities */
#define FBN_DF_ADJUSTED 1  /* df = sum over strata with N_++z > 0 of (values of X seen - 1)(values of Y seen - 1);
                              a test with df = 0 cannot reject (p = 1) */

#define FBN_COUNT_AUTO 0   /* tables of small tests (every arity <= 4, at most 2 conditioning variables, few
                              cells) counted from bit planes with popcounts, the others by byte histograms */
#define FBN_COUNT_HIST 1   /* every table by the byte histogram (shared-memory reductions, or a global table) */
#define FBN_COUNT_BITS 2   /* bit planes for every test that qualifies and fits shared memory, whatever its size */

#define FBN_TUNE_OFF  0    /* fixed rules: bit planes where every small table qualifies, group size by a cost model,
                              depth 0 on the Gram by problem size */
#define FBN_TUNE_AUTO 1    /* the first skeleton call on a workload shape runs fbn_autotune (or reuses its result
                              for this device and shape from earlier in the process) and applies its choices */

#define FBN_LOOP_DEVICE 0  /* the depths after any launched directly run as one CUDA graph whose while node the
                              device drives (no host round trip between depths) */
#define FBN_LOOP_HOST   1  /* the same kernels, one depth at a time from the host, which reads the loop flag
                              between depths (for tools that profile kernel by kernel) */

typedef struct fbn_options {
    int32_t form;        /* FBN_FORM_POOL (default) or FBN_FORM_PLAIN */
    int32_t group_size;  /* gs >= 1: consecutive conditioning sets taken per claim (Section IV-B); 0 = default (1) */
    int32_t depth0;      /* FBN_DEPTH0_* */
    int32_t device;      /* CUDA device ordinal; -1 = the current device */
    int32_t group_threads; /* threads per CI test in the pool: 32, 64, 128 or 256; 0 = chosen per depth */
    int32_t wait_limit;  /* attempts of each bounded device wait of the depth-0 Gram pipeline; 0 = default
                            (2^22); -1 = give up at once, which exercises the FBN_ETIMEOUT path (also the depth-1
                            tensor-core pipeline) */
    int32_t depth1;      /* FBN_DEPTH1_*: how depth 1 counts its tables (pool form only); every test of a
                            vertex's neighbourhood at once on the tensor cores, or the work pool */
    int32_t statistic;   /* FBN_STAT_G2 (default) or FBN_STAT_X2: the statistic of every CI test */
    int32_t df_mode;     /* FBN_DF_FIXED (default) or FBN_DF_ADJUSTED: degrees of freedom of every CI test */
    int32_t loop;        /* FBN_LOOP_DEVICE (default) or FBN_LOOP_HOST: who drives the depth loop */
    int32_t count;       /* FBN_COUNT_*: how contingency tables are counted (pool form and explicit tests; the
                            plain form always uses byte histograms) */
    int32_t tune;        /* FBN_TUNE_OFF (default) or FBN_TUNE_AUTO */
    int32_t reserved[4]; /* must be zero */
} fbn_options;

/* Per-depth counters of the last fbn_learn_skeleton call. */
#define FBN_MAX_DEPTHS 64
typedef struct fbn_stats {
    int32_t depths;                         /* depths that ran */
    int32_t reserved;
    int64_t launches;                       /* kernels launched by the call */
    int64_t edges[FBN_MAX_DEPTHS];          /* edges with at least one test at depth d */
    int64_t tests[FBN_MAX_DEPTHS];          /* CI tests executed, redundant ones included */
    int64_t tests_oracle[FBN_MAX_DEPTHS];   /* tests the sequential Algorithm 1 runs (gs = 1) */
    int64_t removed[FBN_MAX_DEPTHS];        /* edges removed at depth d */
    double  ms[FBN_MAX_DEPTHS];             /* device time of depth d (device clock, ms) */
    double  test_ms[FBN_MAX_DEPTHS];        /* device time of depth d's CI-test kernels (ms) */
    double  gram_ms;                        /* device time of the one-hot Gram (0 if not used) */
    int64_t gram_rows;                      /* M = sum of arities, when the Gram ran */
    int64_t gram_samples;                   /* padded samples of the Gram */
    int64_t test_samples[FBN_MAX_DEPTHS];   /* sum over the tests_oracle[d] tests of their data set's N
                                               (in a batch each test counts its own problem's samples) */
    int64_t popc_work[FBN_MAX_DEPTHS];      /* counting work executed from bit planes: cells x 32-sample words
                                               (one POPC each) over the tests so counted, redundant ones included */
    int64_t smem_updates[FBN_MAX_DEPTHS];   /* counting work executed by byte histograms: samples of the tests so
                                               counted (one shared-memory reduction each, or a global one for the
                                               largest tables), redundant ones included */
} fbn_stats;

/* The choices of fbn_autotune, per depth of the skeleton. */
typedef struct fbn_tuning {
    int32_t depths;                            /* depths measured */
    int32_t depth0;                            /* FBN_DEPTH0_GRAM or FBN_DEPTH0_HIST: how depth 0 counts */
    int32_t group_threads[FBN_MAX_DEPTHS];     /* threads per test of the small-table class at depth d (32..256) */
    int32_t count[FBN_MAX_DEPTHS];             /* FBN_COUNT_HIST or FBN_COUNT_BITS at depth d */
    double  ms_fixed;                          /* skeleton time under the fixed rules (device events, ms) */
    double  ms_tuned;                          /* skeleton time under the choices */
    int32_t candidates;                        /* configurations timed */
    int32_t reserved;
} fbn_tuning;

typedef struct fbn_handle fbn_handle;

/* fbn_create -- load a discrete data set (Section IV-C, cache-friendly storage:
 * one row per variable).
 *   data     : uint8 [n_vars][n_samples], variable-major, host or device memory;
 *              copied into the handle's padded device store (row stride a
 *              multiple of 256 bytes), the caller keeps ownership.
 *   arities  : uint8 [n_vars], host memory, 2 <= r_v <= 255.
 *   opt      : nullable; zero-initialised fields take defaults.
 *   out      : receives the handle.
 * Errors: FBN_EINVAL (null pointer, n_vars < 2, n_samples < 1 or >= 2^31,
 * arity outside [2, 255], nonzero reserved option), FBN_EDATA (a value >= its
 * arity; the handle is not created), FBN_ENOMEM, FBN_ECUDA.  When the call
 * fails before a handle exists, fbn_last_error(NULL) gives the reason. */
int fbn_create(const uint8_t* data, int32_t n_vars, int64_t n_samples,
               const uint8_t* arities, const fbn_options* opt, fbn_handle** out);

/* fbn_update_data -- replace the handle's samples with a new data set of the
 * same shape (n_vars x n_samples, same arities), host or device memory, as in
 * fbn_create; keeps every device buffer.  Results of earlier calls are
 * dropped.  Errors: FBN_EINVAL, FBN_EDATA (a value >= its arity; the handle's
 * data is then undefined until the next successful update), FBN_ECUDA. */
int fbn_update_data(fbn_handle* h, const uint8_t* data);

/* fbn_update_data_batch -- fbn_update_data on k handles of one device at
 * once (data[p] for handle p, each in its handle's shape, host or device): the
 * copies, the arity checks and the bit-plane builds of every data set are
 * queued on the first handle's stream and end with one synchronisation.
 * Errors: FBN_EINVAL, FBN_EDATA (the first offending data set is named; the
 * data of every handle of the call is then undefined until the next
 * successful update), FBN_ECUDA. */
int fbn_update_data_batch(fbn_handle* const* hs, int32_t k, const uint8_t* const* data);

/* fbn_set_stream -- run the handle's work on a caller-owned cudaStream_t
 * (passed as void*; NULL selects the handle's own stream).  The stream must
 * outlive its use by the handle. */
int fbn_set_stream(fbn_handle* h, void* stream);

/* fbn_ci_test -- one conditional-independence test I(X, Y | Z) (Section III-B):
 * contingency table over all samples, marginals, G^2 = 2 sum N ln(N/E),
 * df = (r_x - 1)(r_y - 1) prod_{k in Z} r_k, p = P(chi^2_df > G^2).
 *   x, y : variable indices, x != y;  z : nz distinct indices (host), none
 *   equal to x or y, nz >= 0 (z may be NULL when nz == 0).
 *   g2, df, p : host outputs (double).
 * Errors: FBN_EINVAL, FBN_ETOOBIG (table over the cell limit), FBN_ENUMERIC,
 * FBN_ECUDA.  Synchronises the handle's stream. */
int fbn_ci_test(fbn_handle* h, int32_t x, int32_t y, const int32_t* z, int32_t nz,
                double* g2, double* df, double* p);

/* fbn_ci_table -- the exact contingency table of I(X, Y | Z) (Section III-B),
 * int32 counts in host memory, layout counts[(zi * r_x + xv) * r_y + yv] where
 * zi is the mixed-radix index of the Z values in the order given, z[0] most
 * significant.  cap is the capacity of counts in elements; the call returns
 * FBN_EINVAL if cap is smaller than the cell count r_x r_y prod r_z. */
int fbn_ci_table(fbn_handle* h, int32_t x, int32_t y, const int32_t* z, int32_t nz,
                 int32_t* counts, int64_t cap);

/* fbn_pairwise_counts -- the depth-0 contingency tables of every pair at once
 * (Section IV-B: depth zero tests each pair of the complete graph), as the
 * one-hot Gram matrix computed on the tensor cores.  With M = sum_v r_v and
 * off_v = sum_{u<v} r_u, counts is an int32 [M][M] host or device buffer and
 * counts[(off_i + x) * M + off_j + y] = #{samples with V_i = x and V_j = y}
 * (symmetric; the diagonal blocks hold the marginal counts of one variable).
 * cap is the capacity of counts in elements (>= M*M).  Errors: FBN_EINVAL,
 * FBN_ENOMEM, FBN_ETIMEOUT, FBN_ECUDA.  Synchronises the handle's stream. */
int fbn_pairwise_counts(fbn_handle* h, int32_t* counts, int64_t cap);

/* fbn_learn_skeleton -- the first step of PC-stable (Algorithm 1): start from
 * the complete graph; at each depth d = 0, 1, ... snapshot the adjacency sets
 * a(V), test every remaining edge i<j against conditioning sets of size d
 * drawn from a(V_i)\{V_j} and then a(V_j)\{V_i} (the two endpoints grouped,
 * Section IV-C), remove the edge at the end of the depth if some test accepts
 * independence (p > alpha) and keep the first accepting set (lowest rank in
 * that order) as its separating set; stop when no edge has a side with at
 * least d candidates or when d > max_depth (max_depth = -1: unbounded).
 *   adj_out : uint8 [n][n], host or device, receives the symmetric 0/1
 *             adjacency of the skeleton (zero diagonal).  Nullable.
 * Separating sets stay in the handle until the next call or fbn_destroy; read
 * them with fbn_get_sepset / fbn_export_sepsets (the first such read compacts
 * them on the device and copies the compact form to the host; for a handle of
 * a batch, every member's sets at once).
 * Errors: FBN_EINVAL (alpha outside (0, 1), max_depth < -1), FBN_ETOOBIG,
 * FBN_ENOMEM, FBN_ENUMERIC, FBN_ECUDA. */
int fbn_learn_skeleton(fbn_handle* h, double alpha, int32_t max_depth, uint8_t* adj_out);

/* fbn_learn_skeleton_batch -- fbn_learn_skeleton on k independent handles that
 * share one device and one stream (the first handle's): each depth runs one
 * work pool over the edges of every problem still active.  Results are the
 * same as k separate calls.  adj_out: array of k nullable pointers, each as in
 * fbn_learn_skeleton.  Errors as fbn_learn_skeleton; the handles' devices must
 * match. */
int fbn_learn_skeleton_batch(fbn_handle* const* hs, int32_t k, double alpha, int32_t max_depth,
                             uint8_t* const* adj_out);

/* Callbacks of fbn_learn_skeleton_sharded, called on the calling thread.
 * own: fill owned (uint8 [n][n], host, zeroed) with 1 at [i][j], i < j, for
 *   every edge of adj (the graph every process shares at the start of depth
 *   `depth`, uint8 [n][n] host, read-only) that this process tests.  Every
 *   process's sets must partition the edges.  Return 0, nonzero to abort.
 * exchange: gather the removal records of every process for this depth --
 *   local: int64 [n_local][3] (i, j, rank), this process's -- into all (int64
 *   [cap][3], host, library-owned, cap = n(n-1)/2) and set *n_all; every
 *   process must receive the same records (in any order).  Return 0, nonzero
 *   to abort. */
typedef int (*fbn_shard_own_fn)(void* ctx, int32_t depth, int32_t n, const uint8_t* adj, uint8_t* owned);
typedef int (*fbn_shard_exchange_fn)(void* ctx, int32_t depth, const int64_t* local, int64_t n_local, int64_t* all,
                                     int64_t cap, int64_t* n_all);

/* fbn_learn_skeleton_sharded -- fbn_learn_skeleton learnt by several
 * processes together, each on its own device with its own handle on the same
 * data, by the edge-level partition of Section IV-A across devices: at each
 * depth every process takes the edges `own` gives it, tests them (the work
 * pool, the same kernels), and exports its removals as (i, j, rank) records,
 * rank the edge's lowest accepting rank in the order of Algorithm 1 with the
 * grouping of Section IV-C; `exchange` gathers every process's records, and
 * every process removes all of them from the same snapshot, keeping as
 * separating set the conditioning set of the rank.  So every process ends
 * with the adjacency and separating sets fbn_learn_skeleton gives.  One data
 * set per handle; depth 0 runs on the work pool.  Records that name no edge
 * of the shared graph, twice the same edge, or a rank outside the edge's
 * rank space are refused (FBN_EINVAL).  adj_out as in fbn_learn_skeleton.
 * Errors as fbn_learn_skeleton, FBN_EINVAL when a callback fails. */
int fbn_learn_skeleton_sharded(fbn_handle* h, double alpha, int32_t max_depth, fbn_shard_own_fn own,
                               fbn_shard_exchange_fn exchange, void* ctx, uint8_t* adj_out);

/* fbn_autotune -- choose how each depth of fbn_learn_skeleton(_batch) on these
 * handles counts its tables, by measurement instead of fixed rules (the
 * paper's group-size study, Section V-D, is such a measured trade-off).  Runs
 * the skeleton (same results as fbn_learn_skeleton_batch) once per candidate
 * configuration -- byte histograms with 32, 64, 128 or 256 threads per test,
 * bit planes where every small table qualifies, and, where the one-hot Gram
 * applies, depth 0 on the Gram or on the histogram -- timing every depth with
 * the device clock, and keeps per depth the fastest.  The choices are stored
 * in every handle (later skeleton calls use them) and in a process-wide cache
 * keyed by the device and the workload shape (used by handles created with
 * FBN_TUNE_AUTO).  A choice the caller fixed in the options (group_threads,
 * count, depth0) is not changed.  out: nullable.  The handles' results are
 * those of the last run.  Errors as fbn_learn_skeleton_batch. */
int fbn_autotune(fbn_handle* const* hs, int32_t k, double alpha, int32_t max_depth, fbn_tuning* out);

/* fbn_get_sepset -- separating set of the pair (i, j) from the last skeleton
 * (Algorithm 1, SepSet): returns |S| (0 for an empty set) and writes up to cap
 * members, ascending, into buf (host); returns -1 if i and j are still
 * adjacent, FBN_EINVAL for bad indices or before any skeleton was learnt. */
int32_t fbn_get_sepset(const fbn_handle* h, int32_t i, int32_t j, int32_t* buf, int32_t cap);

/* fbn_export_sepsets -- every separating set at once, in CSR form (host):
 *   pairs   : int32 [n_removed][2] (i < j), ascending by (i, j);
 *   offsets : int64 [n_removed + 1];  members : int32 [offsets[n_removed]].
 * Call with NULL buffers to get the sizes in *n_removed and *n_members. */
int fbn_export_sepsets(const fbn_handle* h, int64_t* n_removed, int64_t* n_members,
                       int32_t* pairs, int64_t* offsets, int32_t* members);

/* fbn_orient_cpdag -- steps 2 and 3 of PC-stable (Section II-C) on the last
 * skeleton: v-structures from the separating sets, then Meek's orientation
 * rules, giving the completed partially directed graph (host code; the
 * skeleton is the hot path).
 *   cpdag_out : uint8 [n][n], host, caller-owned.  cpdag_out[a][b] = 1 and
 *               cpdag_out[b][a] = 0 for a directed edge a -> b; both 1 for an
 *               undirected edge; both 0 for no edge.
 * v-structures: every unshielded triple a - k - b (a, b not adjacent) with k
 * outside SepSet(a, b) marks a -> k and b -> k, all triples judged on the
 * skeleton alone; an edge marked both ways stays undirected.  Meek rules
 * R1-R3 then run in rounds, each round applying at once every orientation a
 * rule implies on the current graph except those implied both ways, until a
 * round changes nothing.  The result does not depend on variable order.
 * Errors: FBN_EINVAL (NULL, or no skeleton learnt yet). */
int fbn_orient_cpdag(const fbn_handle* h, uint8_t* cpdag_out);

/* fbn_get_stats -- per-depth counters of the last skeleton call. */
int fbn_get_stats(const fbn_handle* h, fbn_stats* out);

/* fbn_last_error -- reason for the last failure on h (or of the last failed
 * fbn_create when h is NULL).  The string lives until the next call on h. */
const char* fbn_last_error(const fbn_handle* h);

/* fbn_destroy -- free the handle and its device memory (NULL is a no-op). */
void fbn_destroy(fbn_handle* h);

/* fbn_measure_unit_rates -- measured throughput of the two units that bound
 * the contingency counts, for reporting the counting kernels against a
 * measured peak (the paper has no counterpart: a measurement utility).
 *   device : CUDA device ordinal, -1 = the current device (restored after).
 *   out    : host, n_out >= 4 doubles:
 *            out[0] shared-memory 32-bit reductions per second (red.shared.add,
 *                   each thread on its own column: no conflicts), whole device;
 *            out[1] POPC per second, whole device;
 *            out[2] SMs;  out[3] the device's reported SM clock (Hz).
 * Runs two kernels of a few milliseconds each, allocates a few kilobytes and
 * synchronises.  Errors: FBN_EINVAL (out NULL or n_out < 4), FBN_ENOMEM,
 * FBN_ECUDA, with the reason in fbn_last_error(NULL). */
int fbn_measure_unit_rates(int32_t device, double* out, int32_t n_out);

/* fbn_ci_test_noalloc -- the test of fbn_ci_test for callers that cannot
 * allocate device memory: a process whose device memory belongs to another
 * allocator (a framework's caching allocator, or a server that reserves a
 * fixed budget at start-up) or a latency-critical loop where cudaMalloc and
 * cudaFree would stall the device.  The paper has no counterpart: this is an
 * interface for such callers, not a step of the method.
 *   data     : device, uint8 [n_vars][ld] variable-major, 16-byte aligned,
 *              ld >= n_samples and a multiple of 16.  The d + 2 rows of the
 *              test are checked on the device before counting: if a value is
 *              >= its arity, nothing is counted, table_out is not written and
 *              all three outputs are NaN.
 *   arities  : host, uint8 [n_vars], each >= 2.
 *   x, y, z, nz : as in fbn_ci_test (z in host memory).
 *   out      : device, 3 doubles written in stream order: G^2, df, p
 *              (p alone NaN: the p-value iteration failed; all three NaN: a
 *              data value out of range).
 *   table_out: device, nullable; int32 counts in the fbn_ci_table layout.
 *   stream   : cudaStream_t (NULL = the legacy default stream).
 * The call is asynchronous and allocates nothing: it calls no cudaMalloc,
 * cudaFree or allocating library routine.  Its scratch is one fixed 3 MiB
 * device array inside the library, which every GPU that loads the library
 * holds until the process exits; tables above 2^18 = 262,144 cells are
 * rejected with FBN_ETOOBIG.  The first call on a device looks up that
 * array's device address (cudaGetSymbolAddress) and sets the kernel's
 * shared-memory limit, so make that first call before any stream capture.
 * That set-up is kept per device ordinal for the life of the process and does
 * not survive cudaDeviceReset: do not reset a device between calls.
 * All calls on a device share the one scratch array: calls that overlap on
 * the GPU (different streams, or other host threads) race and must be
 * serialised by the caller.  Errors: FBN_EINVAL, FBN_ETOOBIG, FBN_ECUDA, with
 * the reason in fbn_last_error(NULL). */
int fbn_ci_test_noalloc(const uint8_t* data, int64_t ld, int32_t n_vars, int64_t n_samples,
                        const uint8_t* arities, int32_t x, int32_t y, const int32_t* z, int32_t nz,
                        double* out, int32_t* table_out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* FBN_H */
