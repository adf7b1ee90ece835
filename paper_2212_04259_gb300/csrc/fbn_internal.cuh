// fbn_internal.cuh -- device-side data structures shared by the kernels and the
// host engine of the GB300 PC-stable skeleton library.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace fbn {

constexpr int kMaxD = 30;                 // largest conditioning set supported
constexpr int kMaxRows = kMaxD + 2;       // S rows + X row + Y row
constexpr int kBinomCols = kMaxD + 2;     // binomial table columns k = 0..kMaxD+1
constexpr long long kBinomSat = 1LL << 62;
constexpr long long kMaxCells = 1LL << 24;  // largest contingency table (cells)
constexpr int kMaxVars = 32767;           // neighbour positions are stored in 16 bits
constexpr int kTestThreads = 256;         // threads of a test CTA
constexpr int kBaseSmem = 512;            // pass bases cached in shared memory

// device status bits
constexpr unsigned kStatusTooBig = 1u;    // table over kMaxCells or scratch too small
constexpr unsigned kStatusNumeric = 2u;   // p-value iteration hit its cap
constexpr unsigned kStatusSepPool = 4u;   // separating-set pool overflow
constexpr unsigned kStatusEdges = 8u;     // edge list overflow
constexpr unsigned kStatusTimeout = 16u;  // a bounded device wait gave up
constexpr unsigned kStatusScratch = 32u;  // a table needed more global scratch than allocated
constexpr int kMaxArityPairs = 256;       // arity bound of the depth-0 pair epilogue
// Bit-plane counting: every variable of a test has arity <= kBitsMaxArity (two
// bit planes per variable) and at most kBitsMaxD conditioning variables.
constexpr int kBitsMaxArity = 4;
constexpr int kBitsMaxD = 1;
constexpr long long kBitsMaxN = 2000000;   // samples within the 16-bit counters of the bit-plane count

// Whether a test can be counted from the bit planes (all arities <= 4, d <= 1,
// N within the 16-bit counters).  The same rule, applied to an edge's bound on
// its tables, puts the edge into the bit-plane pool.
__host__ __device__ __forceinline__ bool bits_shape_ok(int d, int max_arity, long long N)
{
    return d <= kBitsMaxD && max_arity <= kBitsMaxArity && N <= kBitsMaxN;
}

// One learning problem (one data set).  Arrays are device pointers.
struct ProblemDev {
    const uint8_t* data;   // [n][ld] uint8, variable-major, zero padded
    const uint8_t* ar;     // [n] arities
    uint8_t* adj;          // [n][n] current graph, 0/1
    int32_t* nbr;          // [n][n] snapshot a(v), ascending, deg[v] valid entries
    int32_t* deg;          // [n]
    int32_t* sep_len;      // [n][n] (entry i<j), -1 while adjacent
    int64_t* sep_off;      // [n][n] offset of the members in the shared pool
    int64_t ld;            // row stride (bytes), multiple of 256
    int32_t n;
    int32_t N;
    int32_t max_arity;
    int32_t pad;
    // one-hot Gram of depth 0 (unused when depth 0 runs on the histogram path)
    const int32_t* off;    // [n] first one-hot row of each variable
    uint8_t* onehot;       // [gram_ld][onehot_ld] E4M3 one-hot rows
    int32_t* gram;         // [gram_ld][gram_ld] INT32 Gram (upper tile triangle)
    int64_t onehot_ld;     // padded samples (multiple of 128)
    int64_t gram_ld;       // padded rows Mp (multiple of 128)
    int32_t* eid;          // [n][n] edge of the current depth at each snapshot slot nbr[v][t]
    int32_t* npos;         // [n][n] npos[v][u] = index of u in nbr[v] (u adjacent to v in the snapshot)
    uint8_t* pk;           // [n][pk_ld] samples 4 bits each (depth-1 tensor-core path; arities <= 8)
    int64_t pk_ld;         // ld / 2
    // bit planes: plane b of variable v, word w = bit b of the values of
    // samples 32 w .. 32 w + 31 (bit i = sample 32 w + i); planes[(2 v + b) *
    // plane_ld + w].  plane_ld is a multiple of 4 words; words past the samples
    // are zero.  Meaningful for variables of arity <= kBitsMaxArity.
    const uint32_t* planes;
    int64_t plane_ld;
};

// One edge i<j of the current depth with its rank space: ranks [0, cnt_i) are
// the X-side conditioning sets (subsets of a(i)\{j}), ranks [cnt_i, total) the
// Y-side ones (subsets of a(j)\{i}), each side in lexicographic order.
// posj = index of j in a(i), posi = index of i in a(j).
struct EdgeWork {
    int32_t prob, i, j;
    int16_t posj, posi;
    int64_t cnt_i, total;
};

// Per-depth codes of the autotuner (DepthCounters::tune).
constexpr int kTuneGroupMask = 0x3FF;
constexpr int kTuneNoBits = 0x400;

__host__ __device__ __forceinline__ int tune_code(const int* tune, int d)
{
    return tune && d >= 0 && d < 64 ? tune[d] : 0;
}

// Edge classes: tables that fit a warp's share of shared memory run on warp
// workers, the others on CTA workers.
constexpr int kClassWarp = 0;
constexpr int kClassCta = 1;
constexpr int kClassBits = 2;   // not an edge class: the small-table class run on the bit-plane pool

// Device-side state of the depth loop.  Per-depth fields are cleared by
// k_depth_begin; d, active, status and sep_used persist across depths.
// Per-depth record written by k_depth_end.
constexpr int kMaxDepthRecords = 64;
struct DepthRecord {
    long long edges, tests, tests_oracle, removed;
    long long test_samples;   // sum of N over the sequential order's tests (their problems' sample counts)
    long long popc_work;      // popcounts of the tests counted from bit planes (cells x 32-sample words)
    long long smem_updates;   // shared-memory histogram updates (samples of the tests counted by histogram)
    // device clock (ns): depth start (snapshot), test kernels start and end,
    // depth end; 0 where a kernel of the depth did not run
    unsigned long long t_begin, t_tests, t_tests_end, t_end;
};

struct DepthCounters {
    unsigned long long n_edges[2];      // edges per class
    unsigned long long maxc[2];         // largest chunk count per class
    unsigned long long next_item[2];    // work-pool claim counters
    unsigned long long total_items[2];  // work items per class
    unsigned long long tests;           // CI tests executed
    unsigned long long tests_oracle;    // tests of the sequential order (gs = 1)
    unsigned long long test_samples;    // sum over those tests of their problem's N
    unsigned long long popc_work;       // executed counting work: popcounts (bit planes)
    unsigned long long smem_updates;    // executed counting work: histogram updates (samples)
    unsigned long long removed;         // edges removed
    unsigned long long max_cells[2];    // upper bound of table cells per class
    unsigned long long sep_used;        // separating-set pool entries in use (persists)
    unsigned int status;                // error bits (persists)
    int d;                              // current depth (persists)
    int active;                         // 1 while Algorithm 1 continues (persists)
    int gsel;                           // group size of the small-table class this depth
    int need_cells;                     // largest table that missed the global scratch (persists)
    int gs;                             // ranks per chunk this depth (set by k_edges)
    unsigned long long adj_ends;        // sum of the snapshot degrees (twice the live edges)
    unsigned long long nbr_claim;       // vertex claims of the depth-1 tensor-core kernel
    unsigned long long max_total[2];    // largest rank count of an edge per class
    int split[2];                       // sample parts per test per class (1 = whole tests)
    int bits_ok;                        // 1 while every small-table edge of the depth can be counted from bit
                                        // planes (k_edges clears it); 1 again for the next depth
    int pad_bits;
    DepthRecord* rec;                   // per-depth records (persists)
    const int* tune;                    // per-depth choices of the autotuner, or nullptr (persists):
                                        // kTuneGroupMask = threads per test of the small-table class (0: cost
                                        // model), kTuneNoBits = byte histograms only at that depth
};

// Tests split by samples: when a depth has few tests against the groups, every
// test is counted by `split` groups over disjoint sample ranges; each part adds
// its table into a zero global table of the test, and the part that finishes
// last decides and zeroes the table again.
constexpr int kMaxSplit = 16;
constexpr long long kSplitMinSamples = 4096;   // samples per part at least
constexpr long long kSplitItems = 4096;        // tests split at once at most

// Passes of the work pool are capped: an edge with more ranks than
// kMaxPasses * gs takes chunks of ceil(total / kMaxPasses) ranks.
constexpr long long kMaxPasses = 4096;

__host__ __device__ __forceinline__ long long chunk_ranks(long long total, int gs)
{
    const long long c = (total + kMaxPasses - 1) / kMaxPasses;
    return c > gs ? c : gs;
}

__host__ __device__ __forceinline__ long long chunk_count(long long total, int gs)
{
    const long long c = chunk_ranks(total, gs);
    return (total + c - 1) / c;
}

// Per-class arguments of the ordering scan.
struct ScanClass {
    const unsigned long long* hist;   // chunk-count histogram of the class
    unsigned long long* alive;        // [maxc + 1] edges with more than k chunks
    unsigned long long* base;         // [maxc + 1] first item of pass k
    long long groups[4];              // groups of 32, 64, 128, 256 threads the class's pool runs
    long long smem_ints;              // shared ints of one pool CTA of the class
    long long groups_bits[4];         // the same for the bit-plane pool (class 0 when every edge qualifies)
    long long smem_ints_bits;
};

// Cache of critical values, see fbn_device.cuh.
struct CritTableDev {
    long long* keys;
    double* vals;
    int cap;
    int dense_n;           // df < dense_n: dense[df], 0 until a test computes it
    double* dense;
    float2* dense_f;       // df < dense_n: the float bracket (largest float <= crit, smallest >= crit), 0 until set
};

// Work pool of one depth and one edge class.  Sizes, the depth and the class
// sub-array come from the DepthCounters on the device.
struct PoolArgs {
    const ProblemDev* probs;
    const EdgeWork* edges;            // whole edge array (class 0 from the front, class 1 from the back)
    unsigned long long* min_accept;   // per edge, lowest accepting rank, init = total
    long long edge_cap;
    const int32_t* sorted;            // class edges by chunk count, descending
    const unsigned long long* base;   // [maxc + 1] first item of pass k
    DepthCounters* ctr;
    const long long* binom;           // [binom_rows][kBinomCols]
    int* gscratch;                    // global tables, gscratch_ints per group
    long long gscratch_ints;
    CritTableDev crit;
    int32_t cls;
    int32_t pad;
    int32_t smem_ints;
    int32_t binom_rows;
    double alpha;
    int* split_tab;                   // [kSplitItems][split_stride] zero global tables of split tests
    unsigned* split_ticket;           // [kSplitItems] parts finished per test, zero between uses
    long long split_stride;           // ints per split table
    int32_t stat;                     // CI statistic: 0 = G^2, 1 = Pearson X^2
    int32_t df_mode;                  // degrees of freedom: 0 = declared arities, 1 = observed table
};

}  // namespace fbn
