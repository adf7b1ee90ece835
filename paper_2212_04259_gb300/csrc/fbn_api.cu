// fbn_api.cu -- host engine and C ABI (include/fbn.h) of the GB300 PC-stable
// skeleton library.  The depth loop of Algorithm 1 runs here; every step of a
// depth (snapshot, edge list, CI tests, removal) is a kernel in fbn_kernels.cu.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/fbn.h"
#include "fbn_gram.h"
#include "fbn_nbr.h"
#include "fbn_sepsets.h"
#include "fbn_launch.h"

using namespace fbn;

namespace {

thread_local std::string g_create_error;

constexpr size_t kSmemBytes = 100 * 1024;     // dynamic shared memory of a CTA test group: 2 CTAs / SM with the ~9 KB static
constexpr long long kSplitStride = 4096;        // cells of a split test's global table at most
constexpr size_t kWarpSmemBytes = 56 * 1024;  // dynamic shared memory of a CTA of 8 warp groups (3 CTAs / SM)
constexpr size_t kBitsSmemBytes = 36 * 1024;  // the bit-plane pool: 8 groups of 32 x 32 counter words, table and
                                              // marginals (4 CTAs / SM)
constexpr int kCritCap = 8192;                // critical-value cache slots (power of two)
constexpr int kCritDense = 8192;              // critical values kept in a dense table: df < kCritDense
constexpr int kBitsCellsAuto = 64;            // largest table counted from bit planes by default

template <typename T>
cudaError_t dalloc(T** p, size_t count)
{
    *p = nullptr;
    if (count == 0) count = 1;
    return cudaMalloc((void**)p, count * sizeof(T));
}

void dfree(void* p)
{
    if (p) cudaFree(p);
}

// ---- small kernels of the host engine ------------------------------------
__global__ void k_validate(const uint8_t* data, int64_t ld, int n, int64_t N, const uint8_t* ar,
                           unsigned long long* first_bad)
{
    const int v = blockIdx.y;
    const uint8_t r = ar[v];
    const uint8_t* row = data + (long long)v * ld;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < N;
         s += (long long)gridDim.x * blockDim.x) {
        if (row[s] >= r) atomicMin(first_bad, (unsigned long long)v * (unsigned long long)N + s);
    }
}

// Bit planes of the samples: word w of plane b of variable v holds bit b of
// the values of samples 32 w .. 32 w + 31.  One thread per word reads its 32
// bytes (two 16-byte loads; the zero padding of the rows covers the words
// past the samples, which therefore stay zero).
__global__ void k_planes(const uint8_t* __restrict__ data, int64_t ld, int64_t wp, uint32_t* __restrict__ planes)
{
    const int v = blockIdx.y;
    const uint8_t* row = data + (long long)v * ld;
    for (long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x; w < wp; w += (long long)gridDim.x * blockDim.x) {
        const uint4* p = reinterpret_cast<const uint4*>(row + w * 32);
        const uint4 a = p[0], b = p[1];
        const unsigned q[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
        unsigned m0 = 0, m1 = 0;
#pragma unroll
        for (int k = 0; k < 32; ++k) {
            const unsigned val = (q[k >> 2] >> ((k & 3) * 8)) & 0xFFu;
            m0 |= (val & 1u) << k;
            m1 |= ((val >> 1) & 1u) << k;
        }
        planes[(2LL * v) * wp + w] = m0;
        planes[(2LL * v + 1) * wp + w] = m1;
    }
}

__global__ void k_init_graph(const ProblemDev* probs, const int32_t* vtx_prob, const int32_t* vtx_first,
                             int total_vertices)
{
    const int g = blockIdx.x;
    if (g >= total_vertices) return;
    const int p = vtx_prob[g];
    const ProblemDev P = probs[p];
    const int i = g - vtx_first[p];
    for (int j = threadIdx.x; j < P.n; j += blockDim.x) {
        P.adj[(long long)i * P.n + j] = (uint8_t)(i != j);
        P.sep_len[(long long)i * P.n + j] = -1;
        P.sep_off[(long long)i * P.n + j] = 0;
    }
}

}  // namespace

// ---- workspace shared by the depth loop ----------------------------------
struct Workspace {
    long long edge_cap = 0;
    EdgeWork* edges = nullptr;
    unsigned long long* min_accept = nullptr;
    int32_t* sorted = nullptr;
    long long ord_cap = 0;
    unsigned long long *hist = nullptr, *alive = nullptr, *base = nullptr, *cursor = nullptr;
    DepthCounters* d_ctr = nullptr;
    DepthCounters* h_ctr = nullptr;   // pinned
    long long* binom = nullptr;
    int brows = 0;
    int vtx_cap = 0, prob_cap = 0;
    int32_t *vtx_prob = nullptr, *vtx_first = nullptr;
    ProblemDev* probs = nullptr;
    int32_t* sep_pool = nullptr;
    long long sep_cap = 0;
    int* gscratch = nullptr;
    long long gscratch_total = 0;
    long long* crit_keys = nullptr;
    double* crit_vals = nullptr;
    double* crit_dense = nullptr;
    float2* crit_dense_f = nullptr;
    double crit_alpha = -1.0;
    cudaEvent_t kev[2 * FBN_MAX_DEPTHS + 2] = {};   // the Gram's window at the end
    DepthRecord* d_rec = nullptr;
    DepthRecord* h_rec = nullptr;                   // pinned
    long long gs_cells = 0;                         // cells per group of the global scratch
    // one-hot Gram of a whole batch
    uint8_t* gram_E = nullptr;                      // one-hot matrices, problem after problem
    long long gram_E_cap = 0;
    int32_t* gram_G = nullptr;                      // Grams, problem after problem
    long long gram_G_cap = 0;
    uint8_t* gram_maps = nullptr;                   // tensor maps, one per problem
    long long gram_maps_cap = 0;
    int4* gram_units = nullptr;
    long long gram_units_cap = 0;
    // samples 4 bits each, problem after problem (depth 1 on the tensor cores)
    uint8_t* pk = nullptr;
    long long pk_cap = 0;
    // global tables of tests split by samples; zero between uses (cleared
    // again when a call did not run to its end)
    int* split_tab = nullptr;
    unsigned* split_ticket = nullptr;
    bool split_dirty = false;
    // per-depth choices of the autotuner on the device, as last uploaded
    int* d_tune = nullptr;
    std::vector<int> tune_loaded;
    // sharded skeletons: this process's edges, removal records, their count
    uint8_t* d_owned = nullptr;
    long long owned_cap = 0;
    long long* d_shard = nullptr;
    long long shard_cap = 0;
    unsigned long long* d_shard_count = nullptr;
    // launch geometry of the device, fixed once (kernel attributes set)
    int dev_sms = 0, grid_small = 0, grid_big = 0, grid_bits = 0;
    // the problem descriptors and vertex maps as last uploaded (skipped when
    // unchanged), staged through pinned memory
    std::vector<uint8_t> up_last;
    uint8_t* h_up = nullptr;
    size_t h_up_cap = 0;
    // pinned staging of the separating-set export: totals, then the arrays
    long long* h_tot = nullptr;
    size_t h_tot_cap = 0;
    uint8_t* h_stage = nullptr;
    size_t h_stage_cap = 0;
    int gram_n_units = 0;
    std::vector<uint8_t> h_maps;
    // one-hot layout of the last prepare_gram and the last one whose pad rows
    // were zeroed (k_onehot writes only the rows below M)
    std::vector<long long> gram_layout, gram_zeroed;
    // the graph of the generic depths (a device-driven while loop)
    cudaGraphExec_t loop = nullptr;
    std::vector<uint8_t> graph_key;
    cudaEvent_t tev[2][2] = {};   // test-kernel windows of depths 0 and 1 when launched directly
    bool events = false;

    void release()
    {
        dfree(edges); dfree(min_accept); dfree(sorted);
        dfree(hist); dfree(alive); dfree(base); dfree(cursor);
        dfree(d_ctr);
        if (h_ctr) cudaFreeHost(h_ctr);
        dfree(binom); dfree(vtx_prob); dfree(vtx_first); dfree(probs);
        dfree(sep_pool); dfree(gscratch); dfree(crit_keys); dfree(crit_vals); dfree(crit_dense);
        dfree(crit_dense_f);
        dfree(gram_E); dfree(gram_G); dfree(gram_maps); dfree(gram_units); dfree(pk);
        dfree(split_tab); dfree(split_ticket); dfree(d_tune);
        dfree(d_owned); dfree(d_shard); dfree(d_shard_count);
        if (events) {
            for (auto& e : kev) cudaEventDestroy(e);
            for (auto& row : tev)
                for (auto& e : row) cudaEventDestroy(e);
        }
        if (loop) cudaGraphExecDestroy(loop);
        dfree(d_rec);
        if (h_rec) cudaFreeHost(h_rec);
        if (h_up) cudaFreeHost(h_up);
        if (h_tot) cudaFreeHost(h_tot);
        if (h_stage) cudaFreeHost(h_stage);
        h_maps.clear();
        gram_E = nullptr; gram_G = nullptr; gram_maps = nullptr; gram_units = nullptr; pk = nullptr;
        split_tab = nullptr; split_ticket = nullptr;
        *this = Workspace();
    }
};

// A device array released when its last holder lets go.
struct DeviceInts {
    int32_t* d = nullptr;
    long long n = 0;
    std::vector<fbn_handle*> members;   // the handles whose sets live here (a batch)
    ~DeviceInts()
    {
        if (d) cudaFree(d);
    }
};

struct fbn_handle {
    int device = 0;
    cudaStream_t own_stream = nullptr;
    cudaStream_t stream = nullptr;
    fbn_options opt{};
    int n = 0;
    int64_t N = 0, ld = 0;
    int max_arity = 0;
    std::vector<uint8_t> h_ar;
    uint8_t* d_data = nullptr;
    uint32_t* d_planes = nullptr;       // two bit planes per variable (see k_planes)
    int64_t plane_ld = 0;               // words per plane, a multiple of 4
    uint8_t* d_ar = nullptr;
    uint8_t* d_adj = nullptr;
    int32_t* d_nbr = nullptr;
    int32_t* d_eid = nullptr;
    int32_t* d_npos = nullptr;
    int32_t* d_deg = nullptr;
    int32_t* d_sep_len = nullptr;
    int64_t* d_sep_off = nullptr;
    ProblemDev* d_prob = nullptr;
    // single-test scratch
    CiTestDesc* d_ci = nullptr;
    double* d_ci_out = nullptr;
    unsigned* d_status = nullptr;
    int32_t* d_table = nullptr;
    long long table_cap = 0;
    int* d_gscratch = nullptr;
    long long gscratch_ints = 0;
    CiTestDesc* h_ci = nullptr;   // pinned
    double* h_ci_out = nullptr;   // pinned
    unsigned* h_status = nullptr; // pinned
    // one-hot Gram (depth 0 on tensor cores)
    int M = 0;                          // sum of arities
    int Mp = 0;                         // M padded to the tile
    long long K = 0;                    // samples padded to the stage width
    int32_t* d_off = nullptr;           // [n] first one-hot row of each variable
    // results of the last skeleton
    bool learnt = false;
    bool sep_pending = false;           // separating sets still only on the device
    unsigned long long sep_pool_used = 0;
    // members of a batch's separating sets: a device copy of the batch's
    // shared pool, held by every handle of that batch until it learns again
    std::shared_ptr<DeviceInts> sep_snap;
    // separating sets on the host, CSR: removed pairs (i < j) ascending, their
    // member offsets (one more than pairs), the members
    std::vector<int32_t> csr_pairs;
    std::vector<int64_t> csr_offs;
    std::vector<int32_t> csr_members;
    // row counts of the compaction on the device: [2n] counts, then [2][n + 1] row offsets
    long long* d_sep_cnt = nullptr;
    fbn_stats stats{};
    // the autotuner's choices (empty: the fixed rules): a per-depth code
    // (kTuneGroupMask, kTuneNoBits) and how depth 0 counts (0: the rule)
    std::vector<int> tune;
    int tune_depth0 = 0;
    Workspace ws;
    std::string err;
};

namespace {

int fail(fbn_handle* h, int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (h) h->err = buf; else g_create_error = buf;
    return code;
}

#define CK(call)                                                                       \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess)                                                         \
            return fail(h, e_ == cudaErrorMemoryAllocation ? FBN_ENOMEM : FBN_ECUDA,   \
                        "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)


int ensure_order(fbn_handle* h, Workspace& ws, long long maxc);

int grow_workspace(fbn_handle* h, Workspace& ws, long long edge_cap, int max_n, int nprob, int total_vtx)
{
    if (!ws.d_ctr) {
        CK(dalloc(&ws.d_ctr, 1));
        CK(cudaMallocHost((void**)&ws.h_ctr, sizeof(DepthCounters)));
        for (auto& e : ws.kev) CK(cudaEventCreate(&e));
        for (auto& row : ws.tev)
            for (auto& e : row) CK(cudaEventCreate(&e));
        ws.events = true;
        CK(dalloc(&ws.d_rec, kMaxDepthRecords));
        CK(cudaMallocHost((void**)&ws.h_rec, kMaxDepthRecords * sizeof(DepthRecord)));
        const int orc = ensure_order(h, ws, kMaxPasses);
        if (orc) return orc;
        CK(dalloc(&ws.crit_keys, kCritCap));
        CK(dalloc(&ws.crit_vals, kCritCap));
        CK(dalloc(&ws.crit_dense, kCritDense));
        CK(dalloc(&ws.crit_dense_f, kCritDense));
        CK(dalloc(&ws.split_tab, kSplitItems * kSplitStride));
        CK(dalloc(&ws.split_ticket, kSplitItems));
        ws.split_dirty = true;
        CK(dalloc(&ws.d_tune, kMaxDepthRecords));
    }
    if (edge_cap > ws.edge_cap) {
        dfree(ws.edges); dfree(ws.min_accept); dfree(ws.sorted);
        ws.edges = nullptr; ws.min_accept = nullptr; ws.sorted = nullptr; ws.edge_cap = 0;
        CK(dalloc(&ws.edges, edge_cap));
        CK(dalloc(&ws.min_accept, edge_cap));
        CK(dalloc(&ws.sorted, edge_cap));
        ws.edge_cap = edge_cap;
    }
    if (max_n + 1 > ws.brows) {
        dfree(ws.binom);
        ws.binom = nullptr;
        const int rows = max_n + 1;
        std::vector<long long> B((size_t)rows * kBinomCols, 0);
        for (int nn = 0; nn < rows; ++nn) {
            B[(size_t)nn * kBinomCols] = 1;
            for (int k = 1; k < kBinomCols; ++k) {
                if (nn == 0) break;
                const long long a = B[(size_t)(nn - 1) * kBinomCols + k - 1];
                const long long b = B[(size_t)(nn - 1) * kBinomCols + k];
                long long s = a + b;
                if (s > kBinomSat || s < 0) s = kBinomSat;
                B[(size_t)nn * kBinomCols + k] = s;
            }
        }
        CK(dalloc(&ws.binom, B.size()));
        CK(cudaMemcpy(ws.binom, B.data(), B.size() * sizeof(long long), cudaMemcpyHostToDevice));
        ws.brows = rows;
    }
    if (total_vtx > ws.vtx_cap) {
        dfree(ws.vtx_prob); dfree(ws.vtx_first);
        ws.vtx_prob = nullptr; ws.vtx_first = nullptr; ws.vtx_cap = 0;
        CK(dalloc(&ws.vtx_prob, total_vtx));
        CK(dalloc(&ws.vtx_first, std::max(nprob, total_vtx)));
        ws.vtx_cap = total_vtx;
    }
    if (nprob > ws.prob_cap) {
        dfree(ws.probs);
        ws.probs = nullptr; ws.prob_cap = 0;
        CK(dalloc(&ws.probs, nprob));
        ws.prob_cap = nprob;
    }
    return FBN_OK;
}

int ensure_order(fbn_handle* h, Workspace& ws, long long maxc)
{
    if (maxc + 1 <= ws.ord_cap) return FBN_OK;
    dfree(ws.hist); dfree(ws.alive); dfree(ws.base); dfree(ws.cursor);
    ws.hist = ws.alive = ws.base = ws.cursor = nullptr;
    ws.ord_cap = 0;
    const long long cap = maxc + 1;   // per class; both classes side by side
    CK(dalloc(&ws.hist, 2 * cap));
    CK(dalloc(&ws.alive, 2 * cap));
    CK(dalloc(&ws.base, 2 * cap));
    CK(dalloc(&ws.cursor, 2 * cap));
    ws.ord_cap = cap;
    return FBN_OK;
}

int ensure_sep_pool(fbn_handle* h, Workspace& ws, long long need, long long used, cudaStream_t st)
{
    if (need <= ws.sep_cap) return FBN_OK;
    const long long cap = std::max(need, 2 * ws.sep_cap);
    int32_t* p = nullptr;
    CK(dalloc(&p, cap));
    if (ws.sep_pool && used > 0)
        CK(cudaMemcpyAsync(p, ws.sep_pool, used * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
    CK(cudaStreamSynchronize(st));
    dfree(ws.sep_pool);
    ws.sep_pool = p;
    ws.sep_cap = cap;
    return FBN_OK;
}

int ensure_gscratch(fbn_handle* h, Workspace& ws, long long total_ints)
{
    if (total_ints <= ws.gscratch_total) return FBN_OK;
    dfree(ws.gscratch);
    ws.gscratch = nullptr;
    ws.gscratch_total = 0;
    CK(dalloc(&ws.gscratch, total_ints));
    ws.gscratch_total = total_ints;
    return FBN_OK;
}

// Whether a table of C cells (plus its marginals, at most 1.25 C entries as
// r_x, r_y >= 2) fits a shared-memory budget without a global table.
bool fits_smem(long long C, size_t bytes = kSmemBytes)
{
    return C + (C * 5) / 4 + 8 <= (long long)(bytes / 4);
}

// Largest table a warp group takes: its eighth of the CTA's shared memory.
long long warp_cells_cap()
{
    const long long slice = (long long)(kWarpSmemBytes / 4) / (kTestThreads / 32);
    return (slice - 8) * 4 / 9;   // C + 1.25 C <= slice - 8
}

int check_status(fbn_handle* h, unsigned status)
{
    if (status & kStatusTooBig) return fail(h, FBN_ETOOBIG, "a contingency table exceeds %lld cells", kMaxCells);
    if (status & kStatusNumeric) return fail(h, FBN_ENUMERIC, "p-value iteration did not converge");
    if (status & kStatusSepPool) return fail(h, FBN_ECUDA, "separating-set pool overflow");
    if (status & kStatusEdges) return fail(h, FBN_ECUDA, "edge list overflow");
    if (status & kStatusTimeout) return fail(h, FBN_ETIMEOUT, "a bounded device wait gave up");
    if (status & kStatusScratch) return fail(h, FBN_ENOMEM, "global table scratch too small");
    return FBN_OK;
}

// Largest table a test of h counts from the bit planes (0: none): the
// option's choice; the plain edge-level form keeps the byte histogram.
int bits_cells(const fbn_handle* h)
{
    if (h->opt.form == FBN_FORM_PLAIN || h->opt.count == FBN_COUNT_HIST) return 0;
    return h->opt.count == FBN_COUNT_BITS ? (int)kMaxCells : kBitsCellsAuto;
}

// Whether the explicit test of (x, y | z) is counted from the bit planes.
bool test_uses_bits(const fbn_handle* h, int32_t x, int32_t y, const int32_t* z, int32_t nz, long long cells)
{
    int mx = std::max(h->h_ar[x], h->h_ar[y]);
    for (int k = 0; k < nz; ++k) mx = std::max<int>(mx, h->h_ar[z[k]]);
    return bits_shape_ok(nz, mx, h->N) && cells <= bits_cells(h);
}

int launch_planes(fbn_handle* h, cudaStream_t st)
{
    dim3 grid((unsigned)std::min<long long>((h->plane_ld + 255) / 256, 64), h->n);
    k_planes<<<grid, 256, 0, st>>>(h->d_data, h->ld, h->plane_ld, h->d_planes);
    CK(cudaGetLastError());
    return FBN_OK;
}

// Whether depth 0 runs as the one-hot Gram on tensor cores.
bool use_gram(fbn_handle* const* hs, int k, bool rule_only = false)
{
    const fbn_handle* h = hs[0];
    if (h->opt.depth0 == FBN_DEPTH0_GRAM) return true;
    if (h->opt.depth0 == FBN_DEPTH0_HIST) return false;
    if (!rule_only && h->tune_depth0) return h->tune_depth0 == FBN_DEPTH0_GRAM;
    long long M = 0, Nmax = 0;
    for (int p = 0; p < k; ++p) {
        M += hs[p]->M;
        Nmax = std::max<long long>(Nmax, hs[p]->N);
    }
    return M >= 512 && Nmax >= 4096;
}

// Depth 1 on the tensor cores: pool form, asked for, every arity within the
// kernel's bound.  The work pool stays the default: on the measured workloads
// it is faster, its early exit running about a quarter of the tests the
// neighbourhood product evaluates.
bool use_nbr1(fbn_handle* const* hs, int k)
{
    const fbn_handle* h = hs[0];
    if (h->opt.form == FBN_FORM_PLAIN || h->opt.depth1 != FBN_DEPTH1_TENSOR) return false;
    if (h->opt.statistic != FBN_STAT_G2 || h->opt.df_mode != FBN_DF_FIXED) return false;
    for (int p = 0; p < k; ++p)
        if (hs[p]->max_arity > nbr1_max_arity()) return false;
    return true;
}

// Room for every problem's samples at 4 bits each; sets the problems' pk rows.
int prepare_pack(fbn_handle* const* hs, int k, Workspace& ws, ProblemDev* P)
{
    fbn_handle* h = hs[0];
    long long total = 0;
    for (int p = 0; p < k; ++p) total += (long long)hs[p]->n * (hs[p]->ld / 2);
    if (total > ws.pk_cap) {
        dfree(ws.pk);
        ws.pk = nullptr;
        ws.pk_cap = 0;
        CK(dalloc(&ws.pk, total));
        ws.pk_cap = total;
    }
    long long off = 0;
    for (int p = 0; p < k; ++p) {
        P[p].pk = ws.pk + off;
        P[p].pk_ld = hs[p]->ld / 2;
        off += (long long)hs[p]->n * (hs[p]->ld / 2);
    }
    return FBN_OK;
}

// Lay out the one-hot matrices and Grams of every problem in the workspace,
// set the problems' pointers, and upload one tensor map per problem and the
// work units (problem, tile pair, chunk), problem-major.
int prepare_gram(fbn_handle* const* hs, int k, Workspace& ws, ProblemDev* P)
{
    fbn_handle* h = hs[0];
    cudaStream_t st = h->stream;
    long long e_total = 0, g_total = 0;
    for (int p = 0; p < k; ++p) {
        e_total += (long long)hs[p]->Mp * hs[p]->K;
        g_total += (long long)hs[p]->Mp * hs[p]->Mp;
    }
    if (e_total > ws.gram_E_cap) {
        dfree(ws.gram_E);
        ws.gram_E = nullptr;
        ws.gram_E_cap = 0;
        CK(dalloc(&ws.gram_E, e_total));
        ws.gram_E_cap = e_total;
    }
    if (g_total > ws.gram_G_cap) {
        dfree(ws.gram_G);
        ws.gram_G = nullptr;
        ws.gram_G_cap = 0;
        CK(dalloc(&ws.gram_G, g_total));
        ws.gram_G_cap = g_total;
    }
    const size_t mb = tensor_map_bytes();
    if ((long long)(k * mb) > ws.gram_maps_cap) {
        dfree(ws.gram_maps);
        ws.gram_maps = nullptr;
        ws.gram_maps_cap = 0;
        CK(dalloc(&ws.gram_maps, k * mb));
        ws.gram_maps_cap = (long long)(k * mb);
    }
    ws.h_maps.assign(k * mb, 0);
    std::vector<int4> units;
    long long eo = 0, go = 0;
    ws.gram_layout.assign(1, (long long)(uintptr_t)ws.gram_E);
    for (int p = 0; p < k; ++p) {
        const fbn_handle* q = hs[p];
        P[p].off = q->d_off;
        P[p].onehot = ws.gram_E + eo;
        P[p].gram = ws.gram_G + go;
        P[p].onehot_ld = q->K;
        P[p].gram_ld = q->Mp;
        CK(encode_onehot_map(ws.h_maps.data() + p * mb, P[p].onehot, q->Mp, q->K));
        // 128-row tiles a against 256-row tiles b that reach the upper triangle
        const int T = q->Mp / 128, T2 = (T + 1) / 2, C = gram_chunks(q->K);
        for (int c = 0; c < C; ++c)
            for (int a = 0; a < T; ++a)
                for (int b = a / 2; b < T2; ++b) units.push_back(make_int4(p, a, b, c));
        ws.gram_layout.push_back(eo);
        ws.gram_layout.push_back(q->M);
        ws.gram_layout.push_back(q->Mp);
        ws.gram_layout.push_back(q->K);
        eo += (long long)q->Mp * q->K;
        go += (long long)q->Mp * q->Mp;
    }
    if ((long long)units.size() > ws.gram_units_cap) {
        dfree(ws.gram_units);
        ws.gram_units = nullptr;
        ws.gram_units_cap = 0;
        CK(dalloc(&ws.gram_units, units.size()));
        ws.gram_units_cap = (long long)units.size();
    }
    ws.gram_n_units = (int)units.size();
    CK(cudaMemcpyAsync(ws.gram_maps, ws.h_maps.data(), k * mb, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(ws.gram_units, units.data(), units.size() * sizeof(int4), cudaMemcpyHostToDevice, st));
    return FBN_OK;
}

// One-hot matrices and their INT32 Grams (upper tile triangle) for the
// problems already in ws.probs (prepared by prepare_gram).
int run_gram(fbn_handle* h, Workspace& ws, int k, int total_vtx, unsigned* d_status, cudaEvent_t ev0 = nullptr,
             cudaEvent_t ev1 = nullptr)
{
    cudaStream_t st = h->stream;
    int sms = 0;
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
    if (ws.gram_layout != ws.gram_zeroed) {   // pad rows stay zero while the layout holds
        CK(launch_zero_pad(ws.probs, k, st));
        ws.gram_zeroed = ws.gram_layout;
    }
    CK(launch_onehot(ws.probs, ws.vtx_prob, ws.vtx_first, total_vtx, st));
    CK(cudaMemsetAsync(ws.gram_G, 0, ws.gram_G_cap * sizeof(int32_t), st));
    if (ev0) CK(cudaEventRecord(ev0, st));
    CK(launch_gram(ws.gram_maps, ws.gram_units, ws.gram_n_units, ws.probs, sms, d_status, h->opt.wait_limit, st));
    if (ev1) CK(cudaEventRecord(ev1, st));
    return FBN_OK;
}

// Copy the separating sets of h (in the pool of workspace ws) to the host,
// as CSR rows per removed pair.
// Move a handle to another separating-set snapshot (or to none).
void set_snapshot(fbn_handle* h, std::shared_ptr<DeviceInts> snap)
{
    if (h->sep_snap) {
        auto& m = h->sep_snap->members;
        m.erase(std::remove(m.begin(), m.end(), h), m.end());
    }
    h->sep_snap = std::move(snap);
    if (h->sep_snap) h->sep_snap->members.push_back(h);
}

// Grow a pinned host buffer (contents not kept).
template <class T>
cudaError_t grow_pinned(T** p, size_t* cap, size_t n)
{
    if (n <= *cap) return cudaSuccess;
    if (*p) cudaFreeHost(*p);
    *p = nullptr;
    *cap = 0;
    const cudaError_t e = cudaMallocHost((void**)p, std::max<size_t>(n, 1) * sizeof(T));
    if (e == cudaSuccess) *cap = n;
    return e;
}

// The handle's separating sets as host CSR, compacted on the device by a
// kernel that writes the compact arrays straight into pinned host staging
// (device-addressable). One handle: staging sized by bounds known on the
// host (every pair removed; every pool entry its own), one synchronisation.
// A handle of a batch: every member whose sets are still on the device, in
// two passes (row counts and totals; then the arrays), one synchronisation
// each.
int materialize_sepsets(fbn_handle* h, Workspace& ws)
{
    if (!h->sep_pending) return FBN_OK;
    CK(cudaSetDevice(h->device));
    cudaStream_t st = h->stream;
    std::vector<fbn_handle*> todo;
    if (h->sep_snap) {
        for (fbn_handle* q : h->sep_snap->members)
            if (q->sep_pending && q->device == h->device) todo.push_back(q);
    } else {
        todo.push_back(h);
    }
    const size_t k = todo.size();
    auto align16 = [](size_t b) { return (b + 15) & ~(size_t)15; };
    // staging of one handle laid out for L pairs: pairs int32 [2L], offsets
    // int64 [L], members int32
    auto place = [](uint8_t* base, long long L, int32_t** pr, int64_t** of, int32_t** mb) {
        *pr = reinterpret_cast<int32_t*>(base);
        *of = reinterpret_cast<int64_t*>(base + 2 * (size_t)L * sizeof(int32_t));
        *mb = reinterpret_cast<int32_t*>(base + (size_t)L * (2 * sizeof(int32_t) + sizeof(int64_t)));
    };
    auto count = [&](fbn_handle* q, long long* tot) -> int {
        const int n = q->n;
        if (!q->d_sep_cnt) CK(dalloc(&q->d_sep_cnt, 4 * (size_t)n + 4));
        long long* roff_p = q->d_sep_cnt + 2 * (size_t)n;
        long long* roff_m = roff_p + n + 1;
        CK(launch_sep_count(q->d_sep_len, n, q->d_sep_cnt, roff_p, roff_m, st));
        CK(cudaMemcpyAsync(tot, roff_p + n, sizeof(long long), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(tot + 1, roff_m + n, sizeof(long long), cudaMemcpyDeviceToHost, st));
        return FBN_OK;
    };
    auto write = [&](fbn_handle* q, uint8_t* base, long long L) -> int {
        const int n = q->n;
        const int32_t* pool = q->sep_snap ? q->sep_snap->d : q->ws.sep_pool;
        long long* roff_p = q->d_sep_cnt + 2 * (size_t)n;
        long long* roff_m = roff_p + n + 1;
        int32_t* pr = nullptr;
        int64_t* of = nullptr;
        int32_t* mb = nullptr;
        place(base, L, &pr, &of, &mb);
        CK(launch_sep_write(q->d_sep_len, q->d_sep_off, pool, n, roff_p, roff_m, pr, of, mb, st));
        return FBN_OK;
    };
    auto unpack = [&](fbn_handle* q, uint8_t* base, long long L, long long R, long long Mtot) {
        int32_t* pr = nullptr;
        int64_t* of = nullptr;
        int32_t* mb = nullptr;
        place(base, L, &pr, &of, &mb);
        q->csr_pairs.assign(pr, pr + 2 * (size_t)R);
        q->csr_offs.assign(of, of + (size_t)R);
        q->csr_offs.push_back(Mtot);
        q->csr_members.assign(mb, mb + (size_t)Mtot);
        q->sep_pending = false;
    };
    int rc = FBN_OK;
    if (k == 1) {
        fbn_handle* q = todo[0];
        const long long Rmax = (long long)q->n * (q->n - 1) / 2;
        const long long Mmax = (long long)q->sep_pool_used;
        const size_t bytes = align16((size_t)Rmax * (2 * sizeof(int32_t) + sizeof(int64_t)) +
                                     (size_t)Mmax * sizeof(int32_t));
        CK(grow_pinned(&ws.h_stage, &ws.h_stage_cap, bytes + 16));
        uint8_t* dstage = nullptr;   // the staging as the device addresses it
        CK(cudaHostGetDevicePointer((void**)&dstage, ws.h_stage, 0));
        long long* tot = reinterpret_cast<long long*>(ws.h_stage + bytes);
        if ((rc = count(q, tot)) || (rc = write(q, dstage, Rmax))) return rc;
        CK(cudaStreamSynchronize(st));
        if (tot[0] > Rmax || tot[1] > Mmax) return fail(h, FBN_ECUDA, "separating-set export over its bounds");
        unpack(q, ws.h_stage, Rmax, tot[0], tot[1]);
        return FBN_OK;
    }
    CK(grow_pinned(&ws.h_tot, &ws.h_tot_cap, 2 * k));
    for (size_t i = 0; i < k; ++i)   // pass 1: row counts and offsets, totals to the host
        if ((rc = count(todo[i], ws.h_tot + 2 * i))) return rc;
    CK(cudaStreamSynchronize(st));
    std::vector<size_t> at(k + 1, 0);   // staging offsets (bytes, 16-aligned)
    for (size_t i = 0; i < k; ++i) {
        const long long R = ws.h_tot[2 * i], Mtot = ws.h_tot[2 * i + 1];
        at[i + 1] = at[i] + align16((size_t)R * (2 * sizeof(int32_t) + sizeof(int64_t)) +
                                    (size_t)Mtot * sizeof(int32_t));
    }
    CK(grow_pinned(&ws.h_stage, &ws.h_stage_cap, std::max<size_t>(at[k], 16)));
    uint8_t* dstage = nullptr;
    CK(cudaHostGetDevicePointer((void**)&dstage, ws.h_stage, 0));
    for (size_t i = 0; i < k; ++i)   // pass 2: the compact arrays into the staging
        if (ws.h_tot[2 * i] > 0 && (rc = write(todo[i], dstage + at[i], ws.h_tot[2 * i]))) return rc;
    CK(cudaStreamSynchronize(st));
    for (size_t i = 0; i < k; ++i)
        unpack(todo[i], ws.h_stage + at[i], ws.h_tot[2 * i], ws.h_tot[2 * i], ws.h_tot[2 * i + 1]);
    return FBN_OK;
}

// Index of the removed pair (i < j) in the handle's CSR, or -1.
long long find_sepset(const fbn_handle* h, int i, int j)
{
    long long lo = 0, hi = (long long)h->csr_offs.size() - 1;   // pairs [0, R)
    while (lo < hi) {
        const long long mid = (lo + hi) >> 1;
        const int a = h->csr_pairs[2 * mid], b = h->csr_pairs[2 * mid + 1];
        if (a < i || (a == i && b < j)) lo = mid + 1; else hi = mid;
    }
    if (lo < (long long)h->csr_offs.size() - 1 && h->csr_pairs[2 * lo] == i && h->csr_pairs[2 * lo + 1] == j) return lo;
    return -1;
}

// Callbacks of a sharded skeleton (fbn_learn_skeleton_sharded).
struct ShardHooks {
    fbn_shard_own_fn own;
    fbn_shard_exchange_fn exchange;
    void* ctx;
};

// The depth loop of Algorithm 1 over one or more problems sharing a stream,
// one attempt.  Every kernel of a depth takes the depth and the sizes from the
// device counters, so the host queues depth d+1 before depth d has finished
// and only waits for the loop flag of depth d-1.  *retry is set when a
// separating-set pool or global-table scratch turned out too small (both are
// grown before returning).
int run_skeleton_once(fbn_handle* const* hs, int k, double alpha, int32_t max_depth, bool* retry,
                      uint8_t* const* adj_out, const ShardHooks* shard = nullptr)
{
    fbn_handle* h = hs[0];
    Workspace& ws = h->ws;
    cudaStream_t st = h->stream;
    *retry = false;
    CK(cudaSetDevice(h->device));
    long long edge_cap = 0;
    int max_n = 0, total_vtx = 0;
    std::vector<ProblemDev> P(k);
    std::vector<int32_t> vtx_prob, vtx_first(k);
    for (int p = 0; p < k; ++p) {
        const fbn_handle* q = hs[p];
        edge_cap += (long long)q->n * (q->n - 1) / 2;
        max_n = std::max(max_n, q->n);
        vtx_first[p] = total_vtx;
        total_vtx += q->n;
        for (int v = 0; v < q->n; ++v) vtx_prob.push_back(p);
        ProblemDev& d = P[p];
        d.data = q->d_data; d.ar = q->d_ar; d.adj = q->d_adj; d.nbr = q->d_nbr; d.eid = q->d_eid; d.npos = q->d_npos; d.deg = q->d_deg;
        d.sep_len = q->d_sep_len; d.sep_off = q->d_sep_off; d.ld = q->ld; d.n = q->n; d.N = (int32_t)q->N;
        d.max_arity = q->max_arity; d.pad = 0;
        d.planes = q->d_planes; d.plane_ld = q->plane_ld;
    }
    int rc = grow_workspace(h, ws, edge_cap, max_n, k, total_vtx);
    if (rc) return rc;
    const bool plain = h->opt.form == FBN_FORM_PLAIN;
    if (shard && k != 1) return fail(h, FBN_EINVAL, "a sharded skeleton learns one problem");
    const bool gram = !plain && !shard && use_gram(hs, k);
    const bool nbr1 = !shard && use_nbr1(hs, k);
    if (shard) {   // this process's edges (n x n) and the depth's removal records (3 per edge at most)
        const long long nn = (long long)h->n * h->n;
        if (nn > ws.owned_cap) {
            dfree(ws.d_owned);
            ws.d_owned = nullptr;
            ws.owned_cap = 0;
            CK(dalloc(&ws.d_owned, nn));
            ws.owned_cap = nn;
        }
        if (edge_cap > ws.shard_cap) {
            dfree(ws.d_shard);
            ws.d_shard = nullptr;
            ws.shard_cap = 0;
            CK(dalloc(&ws.d_shard, 3 * edge_cap));
            ws.shard_cap = edge_cap;
        }
        if (!ws.d_shard_count) CK(dalloc(&ws.d_shard_count, 1));
    }
    if (nbr1) {
        rc = prepare_pack(hs, k, ws, P.data());
        if (rc) return rc;
    }
    if (gram) {
        rc = prepare_gram(hs, k, ws, P.data());
        if (rc) return rc;
    }
    if (ws.sep_cap == 0) {
        rc = ensure_sep_pool(h, ws, 2 * edge_cap + 1024, 0, st);
        if (rc) return rc;
    }
    {   // problem descriptors and vertex maps: uploaded only when they changed
        const size_t nk = (size_t)std::max(k, 1), nv = (size_t)std::max(total_vtx, 0);
        const size_t b0 = nk * sizeof(ProblemDev), b1 = nv * sizeof(int32_t), b2 = nk * sizeof(int32_t);
        const void* dst[3] = {ws.probs, ws.vtx_prob, ws.vtx_first};
        std::vector<uint8_t> blob(sizeof dst + b0 + b1 + b2);
        std::memcpy(blob.data(), dst, sizeof dst);
        std::memcpy(blob.data() + sizeof dst, P.data(), b0);
        std::memcpy(blob.data() + sizeof dst + b0, vtx_prob.data(), b1);
        std::memcpy(blob.data() + sizeof dst + b0 + b1, vtx_first.data(), b2);
        if (blob != ws.up_last) {
            if (blob.size() > ws.h_up_cap) {
                if (ws.h_up) cudaFreeHost(ws.h_up);
                ws.h_up = nullptr;
                ws.h_up_cap = 0;
                CK(cudaMallocHost((void**)&ws.h_up, blob.size()));
                ws.h_up_cap = blob.size();
            }
            // the staging buffer is free: every call ends with its stream drained
            std::memcpy(ws.h_up, blob.data(), blob.size());
            const uint8_t* src = ws.h_up + sizeof dst;
            CK(cudaMemcpyAsync(ws.probs, src, b0, cudaMemcpyHostToDevice, st));
            CK(cudaMemcpyAsync(ws.vtx_prob, src + b0, b1, cudaMemcpyHostToDevice, st));
            CK(cudaMemcpyAsync(ws.vtx_first, src + b0 + b1, b2, cudaMemcpyHostToDevice, st));
            ws.up_last.swap(blob);
        }
    }
    k_init_graph<<<total_vtx, 256, 0, st>>>(ws.probs, ws.vtx_prob, ws.vtx_first, total_vtx);
    CK(cudaGetLastError());
    long long launches = 1;
    if (nbr1) {
        CK(launch_pack4(ws.probs, ws.vtx_prob, ws.vtx_first, total_vtx, st));
        launches += 1;
    }

    if (!ws.dev_sms) {
        int sms = 0;
        CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
        CK(set_kernel_smem(kSmemBytes));
        // CTAs of the small-table pool (any group size) and of the big-table pool
        ws.grid_small = sms * std::max(1, pool_blocks_per_sm(kClassWarp, kWarpSmemBytes));
        ws.grid_big = sms * std::max(1, pool_blocks_per_sm(kClassCta, kSmemBytes));
        ws.grid_bits = sms * std::max(1, pool_blocks_per_sm(kClassBits, kBitsSmemBytes));
        ws.dev_sms = sms;
    }
    const int dev_sms = ws.dev_sms, grid_small = ws.grid_small, grid_big = ws.grid_big, grid_bits = ws.grid_bits;
    const long long groups[4] = {(long long)grid_small * 8, (long long)grid_small * 4, (long long)grid_small * 2,
                                 (long long)grid_small};
    const long long groups_big[4] = {(long long)grid_big * 8, (long long)grid_big * 4, (long long)grid_big * 2,
                                     (long long)grid_big};
    double mean_n = 0;
    for (int p = 0; p < k; ++p) mean_n += (double)hs[p]->N / k;
    const int grid_aux = dev_sms * 4;   // grid-stride helpers (ordering, removal)
    // ranks per chunk: fixed by the option, else chosen on the device per depth
    const int gs_forced = plain ? 1 : h->opt.group_size;
    const long long gs_edges = 8LL * grid_small * 8;   // live edges from which 4 ranks per claim pay
    const long long wcap = plain ? 0 : warp_cells_cap();   // the plain form runs every edge on a CTA
    const int forced = h->opt.group_threads;
    if (ws.crit_alpha != alpha) {
        CK(cudaMemsetAsync(ws.crit_keys, 0, kCritCap * sizeof(long long), st));
        CK(cudaMemsetAsync(ws.crit_dense, 0, kCritDense * sizeof(double), st));
        CK(cudaMemsetAsync(ws.crit_dense_f, 0, kCritDense * sizeof(float2), st));
        ws.crit_alpha = alpha;
    }
    CritTableDev ct{ws.crit_keys, ws.crit_vals, kCritCap, kCritDense, ws.crit_dense, ws.crit_dense_f};

    CK(cudaMemsetAsync(ws.d_rec, 0, kMaxDepthRecords * sizeof(DepthRecord), st));
    CK(cudaMemsetAsync(ws.hist, 0, 2 * ws.ord_cap * sizeof(unsigned long long), st));
    CK(cudaMemsetAsync(ws.cursor, 0, 2 * ws.ord_cap * sizeof(unsigned long long), st));
    if (h->tune != ws.tune_loaded) {   // the autotuner's per-depth choices
        std::vector<int> t(kMaxDepthRecords, 0);
        for (size_t d = 0; d < h->tune.size() && d < t.size(); ++d) t[d] = h->tune[d];
        CK(cudaMemcpy(ws.d_tune, t.data(), t.size() * sizeof(int), cudaMemcpyHostToDevice));
        ws.tune_loaded = h->tune;
    }
    DepthCounters c0{};
    c0.active = 1;
    c0.bits_ok = 1;
    c0.tune = h->tune.empty() ? nullptr : ws.d_tune;
    c0.rec = ws.d_rec;
    *ws.h_ctr = c0;
    CK(cudaMemcpyAsync(ws.d_ctr, ws.h_ctr, sizeof(DepthCounters), cudaMemcpyHostToDevice, st));

    PoolArgs base{};
    base.probs = ws.probs;
    base.edges = ws.edges;
    base.min_accept = ws.min_accept;
    base.edge_cap = ws.edge_cap;
    base.sorted = ws.sorted;
    base.ctr = ws.d_ctr;
    base.binom = ws.binom;
    base.binom_rows = ws.brows;
    base.crit = ct;
    base.alpha = alpha;
    base.stat = h->opt.statistic;
    base.df_mode = h->opt.df_mode;
    base.split_tab = ws.split_tab;
    base.split_ticket = ws.split_ticket;
    base.split_stride = kSplitStride;

    if (ws.split_dirty) {
        CK(cudaMemsetAsync(ws.split_tab, 0, kSplitItems * kSplitStride * sizeof(int), st));
        CK(cudaMemsetAsync(ws.split_ticket, 0, kSplitItems * sizeof(unsigned), st));
    }
    ws.split_dirty = true;   // until this call completes its loop

    // The kernels of one depth after the edge list: ordering and the pool of
    // each class; then removal and the end of the depth.
    auto enqueue_tests = [&]() {
        const int nclass = 2;
        if (!plain) {   // both classes ordered up front: their sorted orders do not overlap
            ScanClass sc[2];
            for (int cls = 0; cls < 2; ++cls) {
                sc[cls].hist = ws.hist + cls * ws.ord_cap;
                sc[cls].alive = ws.alive + cls * ws.ord_cap;
                sc[cls].base = ws.base + cls * ws.ord_cap;
                for (int k = 0; k < 4; ++k) {
                    sc[cls].groups[k] = cls == 0 ? groups[k] : groups_big[k];
                    sc[cls].groups_bits[k] = ((long long)grid_bits * 8) >> k;
                }
                sc[cls].smem_ints = (long long)((cls == 0 ? kWarpSmemBytes : kSmemBytes) / 4);
                sc[cls].smem_ints_bits = (long long)(kBitsSmemBytes / 4);
            }
            launch_order(ws.edges, ws.edge_cap, nclass, ws.d_ctr, sc, ws.cursor, ws.cursor + ws.ord_cap, ws.sorted,
                         mean_n, forced, kSplitStride, 1, grid_aux, st);
        }
        for (int cls = 0; cls < nclass; ++cls) {
            PoolArgs a = base;
            a.cls = cls;
            const bool small = cls == kClassWarp && !plain;
            const size_t smem = small ? kWarpSmemBytes : kSmemBytes;
            a.smem_ints = (int)(smem / 4);
            if (!small && ws.gs_cells > 0) {
                a.gscratch = ws.gscratch;
                a.gscratch_ints = 3 * ws.gs_cells + 64;
            }
            if (plain) {
                launch_plain(a, grid_big, kSmemBytes, st);
                continue;
            }
            a.base = ws.base + cls * ws.ord_cap;
            a.sorted = ws.sorted;
            if (small) {   // the bit-plane pool first; exactly one of the two runs the class
                PoolArgs b = a;
                b.smem_ints = (int)(kBitsSmemBytes / 4);
                launch_pool_bits(b, grid_bits, kBitsSmemBytes, st);
            }
            launch_pool(a, cls, small ? grid_small : grid_big, smem, st);
        }
    };
    auto enqueue_head = [&]() {
        launch_snapshot(ws.probs, ws.vtx_prob, ws.vtx_first, total_vtx, ws.d_ctr, st);
        launch_edges(ws.probs, ws.vtx_prob, ws.vtx_first, total_vtx, gs_forced, gs_edges, ws.binom, ws.brows, wcap,
                     bits_cells(h), shard ? ws.d_owned : nullptr, ws.edges, ws.min_accept, ws.edge_cap, ws.d_ctr,
                     ws.hist, st);
    };
    auto enqueue_tail = [&]() {
        launch_apply(ws.probs, ws.edges, ws.min_accept, ws.edge_cap, ws.binom, ws.sep_pool, ws.sep_cap, ws.d_ctr,
                     grid_aux, st);
        launch_depth_end(ws.d_ctr, ws.d_rec, max_depth, ws.hist, ws.cursor, st);
    };
    const int body_launches = plain ? 7 : 10;
    auto capture_loop = [&]() -> cudaError_t {
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaGraphCreate(&g, 0);
        if (e != cudaSuccess) return e;
        auto give_up = [&](cudaError_t err) {
            cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
            if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
                cudaGraph_t tmp = nullptr;
                cudaStreamEndCapture(st, &tmp);
            }
            cudaGetLastError();
            cudaGraphDestroy(g);
            return err;
        };
        cudaGraphConditionalHandle cond{};
        if ((e = cudaGraphConditionalHandleCreate(&cond, g, 0, 0)) != cudaSuccess) return give_up(e);
        // top level: the first depth's edge list and the loop condition
        if ((e = cudaStreamBeginCaptureToGraph(st, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) !=
            cudaSuccess)
            return give_up(e);
        enqueue_head();
        launch_gate(ws.d_ctr, cond, st);
        cudaGraphNode_t gate_node = nullptr;
        {
            cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
            const cudaGraphNode_t* deps = nullptr;
            size_t nd = 0;
            if ((e = cudaStreamGetCaptureInfo(st, &cs, nullptr, nullptr, &deps, nullptr, &nd)) != cudaSuccess)
                return give_up(e);
            if (cs != cudaStreamCaptureStatusActive || nd != 1) return give_up(cudaErrorStreamCaptureInvalidated);
            gate_node = deps[0];
        }
        cudaGraph_t out = nullptr;
        if ((e = cudaStreamEndCapture(st, &out)) != cudaSuccess) return give_up(e);
        // the while node and its body: one depth, then the next one's edge list
        cudaGraphNodeParams cp{};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = cond;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t cn = nullptr;
        if ((e = cudaGraphAddNode(&cn, g, &gate_node, nullptr, 1, &cp)) != cudaSuccess) return give_up(e);
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        if ((e = cudaStreamBeginCaptureToGraph(st, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) !=
            cudaSuccess)
            return give_up(e);
        enqueue_tests();
        enqueue_tail();
        enqueue_head();
        launch_gate(ws.d_ctr, cond, st);
        if ((e = cudaStreamEndCapture(st, &out)) != cudaSuccess) return give_up(e);
        e = cudaGraphInstantiate(&ws.loop, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            ws.loop = nullptr;
            cudaGetLastError();
        }
        return e;
    };

    // The generic depths as one graph: the edge list of the first one, then a
    // device-driven while loop whose body tests a depth, removes its edges,
    // ends it and lists the next depth's edges (k_gate: go on or stop).
    // Captured once per configuration: every argument it holds is in the key.
    if (!shard) {
        std::vector<uint8_t> key;
        auto put = [&](const void* p, size_t n) {
            const uint8_t* b = (const uint8_t*)p;
            key.insert(key.end(), b, b + n);
        };
        const void* ptrs[] = {ws.probs, ws.vtx_prob, ws.vtx_first, ws.binom, ws.edges, ws.min_accept, ws.d_ctr,
                              ws.hist, ws.alive, ws.base, ws.cursor, ws.sorted, ws.gscratch, ws.sep_pool, ws.d_rec,
                              ws.crit_keys, ws.crit_vals, ws.crit_dense, ws.crit_dense_f, ws.split_tab,
                              ws.split_ticket};
        put(ptrs, sizeof ptrs);
        const long long ints[] = {total_vtx, gs_forced, gs_edges, ws.brows, wcap, ws.edge_cap, ws.ord_cap, forced,
                                  grid_aux, grid_small, grid_big, grid_bits, ws.gs_cells, ws.sep_cap, max_depth, plain,
                                  h->opt.statistic, h->opt.df_mode, bits_cells(h),
                                  groups[0], groups[1], groups[2], groups[3]};
        put(ints, sizeof ints);
        put(&mean_n, sizeof mean_n);
        put(&alpha, sizeof alpha);
        if (key != ws.graph_key) {
            if (ws.loop) cudaGraphExecDestroy(ws.loop);
            ws.loop = nullptr;
            ws.graph_key.clear();
            // with programmatic launches first, else without (bodies of
            // conditional nodes may refuse programmatic edges)
            cudaError_t err = cudaSuccess;
            for (int pdl = 1; pdl >= 0 && !ws.loop; --pdl) {
                set_pdl(pdl != 0);
                err = capture_loop();
            }
            set_pdl(true);
            if (!ws.loop) return fail(h, FBN_ECUDA, "depth loop graph: %s", cudaGetErrorString(err));
            ws.graph_key = key;
        }
    }

    fbn_stats stats{};
    int d_loop = 0;   // first depth of the graph loop
    bool direct[2] = {false, false};   // depths 0 and 1 launched directly (timed by events)
    if (gram) {
        enqueue_head();
        CK(cudaEventRecord(ws.tev[0][0], st));
        rc = run_gram(h, ws, k, total_vtx, &ws.d_ctr->status, ws.kev[2 * FBN_MAX_DEPTHS],
                      ws.kev[2 * FBN_MAX_DEPTHS + 1]);
        if (rc) return rc;
        CK(launch_pairs_decide(ws.edges, ws.edge_cap, ws.probs, ws.min_accept, ct, alpha, ws.d_ctr,
                               h->opt.statistic, h->opt.df_mode, grid_aux, st));
        CK(cudaEventRecord(ws.tev[0][1], st));
        enqueue_tail();
        launches += 6;
        direct[0] = true;
        d_loop = 1;
    }
    if (nbr1 && (max_depth < 0 || max_depth >= 1)) {
        if (d_loop == 0) {   // depth 0 on the pool, launched directly
            enqueue_head();
            CK(cudaEventRecord(ws.tev[0][0], st));
            enqueue_tests();
            CK(cudaEventRecord(ws.tev[0][1], st));
            enqueue_tail();
            launches += body_launches - 1;
            direct[0] = true;
        }
        enqueue_head();
        CK(cudaEventRecord(ws.tev[1][0], st));
        CK(launch_nbr1(ws.probs, ws.vtx_prob, ws.vtx_first, total_vtx, ws.edges, ws.min_accept, ct, alpha, ws.d_ctr,
                       dev_sms, h->opt.wait_limit, st));
        CK(cudaEventRecord(ws.tev[1][1], st));
        enqueue_tail();
        launches += 5;
        direct[1] = true;
        d_loop = 2;
    }
    const bool loop = max_depth < 0 || d_loop <= max_depth;
    const bool host_loop = h->opt.loop == FBN_LOOP_HOST || shard;
    if (shard) {
        // Several processes learn this skeleton together (Section IV-A's
        // edge-level partition across devices): every process holds the same
        // graph; per depth, the caller's `own` picks this process's edges, the
        // process tests them and exports its removals as (i, j, rank) records,
        // the caller's `exchange` gathers every process's records, and each
        // process applies all of them to the same snapshot.  The host decides
        // the stop, from the graph every process shares.
        const int n = h->n;
        std::vector<uint8_t> adj_h((size_t)n * n), own_h((size_t)n * n);
        std::vector<int64_t> local, all;
        for (int d = 0;; ++d) {
            if (max_depth >= 0 && d > max_depth) break;
            if (d >= kMaxDepthRecords - 1 || d > kMaxD) break;
            CK(cudaMemcpyAsync(adj_h.data(), h->d_adj, adj_h.size(), cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            std::vector<int> deg(n, 0);
            for (int i = 0; i < n; ++i)
                for (int j = 0; j < n; ++j) deg[i] += adj_h[(size_t)i * n + j] != 0;
            bool any = false;   // an edge with a side of at least d candidates
            for (int i = 0; i < n && !any; ++i)
                for (int j = i + 1; j < n && !any; ++j)
                    any = adj_h[(size_t)i * n + j] && std::max(deg[i], deg[j]) - 1 >= d;
            if (!any) break;
            std::fill(own_h.begin(), own_h.end(), 0);
            if (shard->own(shard->ctx, d, n, adj_h.data(), own_h.data()) != 0)
                return fail(h, FBN_EINVAL, "the own callback failed at depth %d", d);
            CK(cudaMemcpyAsync(ws.d_owned, own_h.data(), own_h.size(), cudaMemcpyHostToDevice, st));
            CK(cudaMemsetAsync(ws.d_shard_count, 0, sizeof(unsigned long long), st));
            enqueue_head();
            enqueue_tests();
            launch_shard_export(ws.probs, ws.edges, ws.min_accept, ws.edge_cap, ws.d_ctr, ws.d_shard, ws.d_shard_count,
                                grid_aux, st);
            unsigned long long m = 0;
            CK(cudaMemcpyAsync(&m, ws.d_shard_count, sizeof m, cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            if ((long long)m > ws.shard_cap) return fail(h, FBN_ECUDA, "removal records over their bound");
            local.resize(3 * m);
            if (m) CK(cudaMemcpy(local.data(), ws.d_shard, 3 * m * sizeof(int64_t), cudaMemcpyDeviceToHost));
            const long long cap = (long long)n * (n - 1) / 2;
            all.assign(3 * (size_t)cap, 0);
            int64_t n_all = 0;
            if (shard->exchange(shard->ctx, d, local.data(), (int64_t)m, all.data(), cap, &n_all) != 0 || n_all < 0 ||
                n_all > cap)
                return fail(h, FBN_EINVAL, "the exchange callback failed at depth %d", d);
            // every record must name an edge of the shared graph once, with a
            // rank inside its rank space (checked here: the kernel trusts them)
            std::vector<uint8_t> seen((size_t)n * n, 0);
            for (long long t = 0; t < n_all; ++t) {
                const long long i = (long long)all[3 * t], j = (long long)all[3 * t + 1], r = (long long)all[3 * t + 2];
                if (i < 0 || j <= i || j >= n || !adj_h[(size_t)i * n + j] || seen[(size_t)i * n + j] || r < 0)
                    return fail(h, FBN_EINVAL, "bad removal record (%lld, %lld, %lld) at depth %d", i, j, r, d);
                seen[(size_t)i * n + j] = 1;
                if (d > 0) {
                    double ti = 1, tj = 1;   // C(deg - 1, d) on each side, in double (no overflow to care about here)
                    for (int q = 0; q < d; ++q) {
                        ti = ti * (deg[i] - 1 - q) / (q + 1);
                        tj = tj * (deg[j] - 1 - q) / (q + 1);
                    }
                    if ((double)r >= std::max(ti, 0.0) + std::max(tj, 0.0))
                        return fail(h, FBN_EINVAL, "removal record rank %lld out of range at depth %d", r, d);
                } else if (r != 0) {
                    return fail(h, FBN_EINVAL, "removal record rank %lld out of range at depth 0", r);
                }
            }
            if (n_all) CK(cudaMemcpyAsync(ws.d_shard, all.data(), 3 * n_all * sizeof(int64_t), cudaMemcpyHostToDevice, st));
            launch_shard_apply(ws.probs, ws.d_shard, n_all, ws.binom, ws.brows, ws.sep_pool, ws.sep_cap, ws.d_ctr,
                               grid_aux, st);
            launch_depth_end(ws.d_ctr, ws.d_rec, -1, ws.hist, ws.cursor, st);
            launch_shard_continue(ws.d_ctr, st);
            launches += body_launches + 1;
        }
    } else if (loop && host_loop) {
        // the same kernels, depth by depth: the edge list, then while the
        // depth has an edge to test, its tests, removal and end, and the next
        // depth's edge list
        enqueue_head();
        launches += 2;
        for (;;) {
            CK(cudaMemcpyAsync(ws.h_ctr, ws.d_ctr, sizeof(DepthCounters), cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            if (!ws.h_ctr->active || ws.h_ctr->n_edges[0] + ws.h_ctr->n_edges[1] == 0) break;
            enqueue_tests();
            enqueue_tail();
            enqueue_head();
        }
    } else if (loop) {
        CK(cudaGraphLaunch(ws.loop, st));
        launches += 3;
    }
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(ws.h_ctr, ws.d_ctr, sizeof(DepthCounters), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(ws.h_rec, ws.d_rec, kMaxDepthRecords * sizeof(DepthRecord), cudaMemcpyDeviceToHost, st));
    if (adj_out)   // the adjacency goes out with the counters (dropped if the call is retried)
        for (int p = 0; p < k; ++p)
            if (adj_out[p])
                CK(cudaMemcpyAsync(adj_out[p], hs[p]->d_adj, (size_t)hs[p]->n * hs[p]->n, cudaMemcpyDefault, st));
    CK(cudaStreamSynchronize(st));
    if (loop && !shard) launches += (long long)(body_launches - (host_loop ? 1 : 0)) * std::max(0, ws.h_ctr->d - d_loop);
    for (int q = 0; q < 2; ++q)
        if (direct[q]) {
            float kms = 0.f;
            CK(cudaEventElapsedTime(&kms, ws.tev[q][0], ws.tev[q][1]));
            stats.test_ms[q] = kms;
        }
    const DepthCounters& c = *ws.h_ctr;
    if (c.status == 0) ws.split_dirty = false;   // every split test's last part zeroed its table
    if (c.status & (kStatusSepPool | kStatusScratch)) {
        if (c.status & kStatusSepPool) {
            rc = ensure_sep_pool(h, ws, 2 * ws.sep_cap + 2 * (long long)c.sep_used, 0, st);
            if (rc) return rc;
        }
        if (c.status & kStatusScratch) {
            if (c.need_cells <= 0 || c.need_cells > kMaxCells) return check_status(h, kStatusTooBig);
            ws.gs_cells = std::max<long long>(2 * ws.gs_cells, c.need_cells);
            rc = ensure_gscratch(h, ws, (3 * ws.gs_cells + 64) * grid_big);
            if (rc) return rc;
        }
        *retry = true;
        return FBN_OK;
    }
    rc = check_status(h, c.status);
    if (rc) return rc;

    for (int d = 0; d < kMaxDepthRecords; ++d) {
        const DepthRecord& r = ws.h_rec[d];
        if (r.edges == 0) break;   // the depth that found no edge: Algorithm 1 stopped before it
        if (d >= FBN_MAX_DEPTHS) break;
        stats.depths = d + 1;
        stats.edges[d] = r.edges;
        stats.tests[d] = r.tests;
        stats.tests_oracle[d] = r.tests_oracle;
        stats.test_samples[d] = r.test_samples;
        stats.popc_work[d] = r.popc_work;
        stats.smem_updates[d] = r.smem_updates;
        stats.removed[d] = r.removed;
        const unsigned long long next = d + 1 < kMaxDepthRecords ? ws.h_rec[d + 1].t_begin : 0;
        const unsigned long long end = next > r.t_begin ? next : r.t_end;
        stats.ms[d] = end > r.t_begin && r.t_begin ? (float)((end - r.t_begin) * 1e-6) : 0.f;
        if (d >= d_loop && r.t_tests_end > r.t_tests && r.t_tests)
            stats.test_ms[d] = (float)((r.t_tests_end - r.t_tests) * 1e-6);
    }
    if (gram) {
        float gms = 0.f;
        CK(cudaEventElapsedTime(&gms, ws.kev[2 * FBN_MAX_DEPTHS], ws.kev[2 * FBN_MAX_DEPTHS + 1]));
        stats.gram_ms = gms;
        for (int p = 0; p < k; ++p) {
            stats.gram_rows += hs[p]->M;
            stats.gram_samples = std::max<int64_t>(stats.gram_samples, hs[p]->K);
        }
    }
    stats.launches = launches;
    // every problem's sets stay on the device until asked for; a batch's
    // members live in the first handle's pool, which its next call reuses, so
    // the batch keeps a device copy of the used part
    std::shared_ptr<DeviceInts> snap;
    if (k > 1) {
        snap = std::make_shared<DeviceInts>();
        snap->n = std::max<long long>(1, (long long)c.sep_used);
        CK(dalloc(&snap->d, snap->n));
        if (c.sep_used)
            CK(cudaMemcpyAsync(snap->d, ws.sep_pool, c.sep_used * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
    }
    for (int p = 0; p < k; ++p) {
        hs[p]->stats = stats;
        hs[p]->learnt = true;
        hs[p]->sep_pending = true;
        hs[p]->sep_pool_used = c.sep_used;
        set_snapshot(hs[p], snap);
    }
    return FBN_OK;
}

int run_skeleton(fbn_handle* const* hs, int k, double alpha, int32_t max_depth, uint8_t* const* adj_out = nullptr,
                 const ShardHooks* shard = nullptr)
{
    for (int attempt = 0; attempt < 6; ++attempt) {
        bool retry = false;
        const int rc = run_skeleton_once(hs, k, alpha, max_depth, &retry, adj_out, shard);
        if (rc || !retry) return rc;
    }
    return fail(hs[0], FBN_ENOMEM, "scratch or separating-set pool kept overflowing");
}

int check_test_args(fbn_handle* h, int32_t x, int32_t y, const int32_t* z, int32_t nz, long long* cells)
{
    if (!h) return FBN_EINVAL;
    if (x < 0 || x >= h->n || y < 0 || y >= h->n || x == y)
        return fail(h, FBN_EINVAL, "bad x=%d y=%d for n=%d", x, y, h->n);
    if (nz < 0 || nz > kMaxD || (nz > 0 && !z))
        return fail(h, FBN_EINVAL, "conditioning set size %d outside [0, %d]", nz, kMaxD);
    long long c = (long long)h->h_ar[x] * h->h_ar[y];
    for (int k = 0; k < nz; ++k) {
        if (z[k] < 0 || z[k] >= h->n || z[k] == x || z[k] == y)
            return fail(h, FBN_EINVAL, "bad conditioning variable %d", z[k]);
        for (int l = 0; l < k; ++l)
            if (z[l] == z[k]) return fail(h, FBN_EINVAL, "conditioning variable %d repeated", z[k]);
        c *= h->h_ar[z[k]];
        if (c > kMaxCells) return fail(h, FBN_ETOOBIG, "table exceeds %lld cells", kMaxCells);
    }
    *cells = c;
    return FBN_OK;
}

int run_ci(fbn_handle* h, int32_t x, int32_t y, const int32_t* z, int32_t nz, long long cells, bool want_table)
{
    CK(cudaSetDevice(h->device));
    cudaStream_t st = h->stream;
    CiTestDesc& q = *h->h_ci;
    std::memset(&q, 0, sizeof q);
    q.x = x; q.y = y; q.d = nz;
    for (int k = 0; k < nz; ++k) q.z[k] = z[k];
    if (want_table && cells > h->table_cap) {
        dfree(h->d_table);
        h->d_table = nullptr;
        h->table_cap = 0;
        CK(dalloc(&h->d_table, cells));
        h->table_cap = cells;
    }
    long long gints = 0;
    if (!fits_smem(cells)) {
        gints = 3 * cells + 64;
        if (gints > h->gscratch_ints) {
            dfree(h->d_gscratch);
            h->d_gscratch = nullptr;
            h->gscratch_ints = 0;
            CK(dalloc(&h->d_gscratch, gints));
            h->gscratch_ints = gints;
        }
    }
    CK(set_kernel_smem(kSmemBytes));
    CK(cudaMemcpyAsync(h->d_ci, h->h_ci, sizeof(CiTestDesc), cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(h->d_status, 0, sizeof(unsigned), st));
    launch_ci_tests(h->d_prob, h->d_ci, 1, h->d_ci_out, want_table ? h->d_table : nullptr,
                    gints ? h->d_gscratch : nullptr, gints, h->d_status, kSmemBytes, h->opt.statistic, h->opt.df_mode,
                    test_uses_bits(h, x, y, z, nz, cells), st);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(h->h_ci_out, h->d_ci_out, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(h->h_status, h->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return check_status(h, *h->h_status);
}

// ---- autotuning --------------------------------------------------------
struct TuneChoice {
    std::vector<int> table;   // per-depth codes (empty: the fixed rules won)
    int depth0 = 0;
    fbn_tuning report{};
};
std::mutex g_tune_mu;
std::map<std::vector<long long>, TuneChoice> g_tune_cache;

// The workload shape a tuning applies to: device, options that shape the
// work, alpha, max depth, and every problem's (n, N, largest arity).
std::vector<long long> tune_key(fbn_handle* const* hs, int k, double alpha, int32_t max_depth)
{
    const fbn_handle* h = hs[0];
    long long abits = 0;
    std::memcpy(&abits, &alpha, sizeof abits);
    std::vector<long long> key = {h->device, k, h->opt.form, h->opt.statistic, h->opt.df_mode, h->opt.count,
                                  h->opt.group_threads, h->opt.depth0, h->opt.depth1, abits, max_depth};
    for (int p = 0; p < k; ++p) {
        key.push_back(hs[p]->n);
        key.push_back(hs[p]->N);
        key.push_back(hs[p]->max_arity);
    }
    return key;
}

void apply_tuning(fbn_handle* const* hs, int k, const std::vector<int>& table, int depth0)
{
    for (int p = 0; p < k; ++p) {
        hs[p]->tune = table;
        hs[p]->tune_depth0 = depth0;
    }
}

// Timed skeletons of the batch under a configuration: a first run warms
// (capture, lazily filled tables), then `reps` runs are timed with events on
// the stream; the whole time and every depth's test window (device clock) are
// the medians over the runs.
int timed_run(fbn_handle* const* hs, int k, double alpha, int32_t max_depth, const std::vector<int>& table,
              int depth0, int reps, float* ms, fbn_stats* st)
{
    fbn_handle* h = hs[0];
    apply_tuning(hs, k, table, depth0);
    int rc = run_skeleton(hs, k, alpha, max_depth);
    if (rc) return rc;
    cudaEvent_t e0 = h->ws.kev[0], e1 = h->ws.kev[1];
    std::vector<float> whole;
    std::vector<std::vector<double>> depth(FBN_MAX_DEPTHS);
    for (int r = 0; r < reps; ++r) {
        CK(cudaEventRecord(e0, h->stream));
        rc = run_skeleton(hs, k, alpha, max_depth);
        if (rc) return rc;
        CK(cudaEventRecord(e1, h->stream));
        CK(cudaEventSynchronize(e1));
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, e0, e1));
        whole.push_back(t);
        for (int d = 0; d < FBN_MAX_DEPTHS; ++d) depth[d].push_back(h->stats.test_ms[d]);
    }
    auto median = [](auto v) {
        std::sort(v.begin(), v.end());
        return v[v.size() / 2];
    };
    *st = h->stats;
    *ms = median(whole);
    for (int d = 0; d < FBN_MAX_DEPTHS; ++d) st->test_ms[d] = median(depth[d]);
    return FBN_OK;
}

int autotune_impl(fbn_handle* const* hs, int k, double alpha, int32_t max_depth, fbn_tuning* out)
{
    fbn_handle* h = hs[0];
    const fbn_options& o = h->opt;
    const bool pool = o.form == FBN_FORM_POOL;
    // candidates for the pool depths: byte histograms at each group size, and
    // bit planes where every small table qualifies (their pool runs warp groups)
    std::vector<int> cands;
    if (pool && o.group_threads == 0) {
        for (int g : {32, 64, 128, kTestThreads}) cands.push_back(g | (o.count == FBN_COUNT_BITS ? 0 : kTuneNoBits));
        if (o.count == FBN_COUNT_AUTO) cands.push_back(0);
    } else {
        cands.push_back(0);
    }
    const bool gram_rule = pool && use_gram(hs, k, true);
    const bool tune_d0 = pool && o.depth0 == FBN_DEPTH0_AUTO && gram_rule;
    const int d0_rule = gram_rule ? FBN_DEPTH0_GRAM : FBN_DEPTH0_HIST;
    fbn_tuning rep{};
    std::vector<std::vector<double>> test_ms;
    fbn_stats st{};
    float ms = 0.f;
    int depths = 0;
    for (int c : cands) {
        std::vector<int> table(kMaxDepthRecords, c);
        const int rc = timed_run(hs, k, alpha, max_depth, table, d0_rule, 3, &ms, &st);
        if (rc) return rc;
        depths = st.depths;
        test_ms.emplace_back(st.test_ms, st.test_ms + FBN_MAX_DEPTHS);
        rep.candidates += 1;
    }
    // depth 0: the Gram against the histogram (the pool at later depths as the
    // first candidate), by the depth's device time
    int d0 = 0;
    if (tune_d0) {
        std::vector<int> table(kMaxDepthRecords, cands[0]);
        fbn_stats sg{}, sh{};
        int rc = timed_run(hs, k, alpha, max_depth, table, FBN_DEPTH0_GRAM, 3, &ms, &sg);
        if (!rc) rc = timed_run(hs, k, alpha, max_depth, table, FBN_DEPTH0_HIST, 3, &ms, &sh);
        if (rc) return rc;
        rep.candidates += 2;
        d0 = sh.ms[0] < sg.ms[0] ? FBN_DEPTH0_HIST : FBN_DEPTH0_GRAM;
    }
    // per depth the fastest candidate
    std::vector<int> best(kMaxDepthRecords, cands[0]);
    for (int d = 0; d < depths && d < FBN_MAX_DEPTHS; ++d) {
        size_t bi = 0;
        for (size_t i = 1; i < cands.size(); ++i)
            if (test_ms[i][d] < test_ms[bi][d]) bi = i;
        best[d] = cands[bi];
    }
    // the whole skeleton under the choices against the fixed rules; keep the faster
    fbn_stats s1{};
    float ms_fixed = 0.f, ms_tuned = 0.f;
    int rc = timed_run(hs, k, alpha, max_depth, {}, 0, 5, &ms_fixed, &s1);
    if (!rc) rc = timed_run(hs, k, alpha, max_depth, best, d0, 5, &ms_tuned, &s1);
    if (rc) return rc;
    rep.candidates += 2;
    TuneChoice choice;
    if (ms_tuned <= ms_fixed) {
        choice.table = best;
        choice.depth0 = d0;
    }
    const bool gram_used = choice.depth0 ? choice.depth0 == FBN_DEPTH0_GRAM : gram_rule;
    rep.depths = depths;
    rep.depth0 = gram_used ? FBN_DEPTH0_GRAM : FBN_DEPTH0_HIST;
    int max_ar = 0;
    long long max_n = 0;
    for (int p = 0; p < k; ++p) {
        max_ar = std::max(max_ar, hs[p]->max_arity);
        max_n = std::max<long long>(max_n, hs[p]->N);
    }
    for (int d = 0; d < depths && d < FBN_MAX_DEPTHS; ++d) {
        const int c = choice.table.empty() ? 0 : choice.table[d];
        // bit planes only where the depth's tables can take them
        const bool bits = !(c & kTuneNoBits) && bits_cells(h) > 0 && bits_shape_ok(d, max_ar, max_n) &&
                          !(d == 0 && gram_used);
        rep.count[d] = bits ? FBN_COUNT_BITS : FBN_COUNT_HIST;
        rep.group_threads[d] = bits ? 32 : o.group_threads ? o.group_threads : (c & kTuneGroupMask);   // 0: cost model
    }
    rep.ms_fixed = ms_fixed;
    rep.ms_tuned = ms_tuned;
    choice.report = rep;
    apply_tuning(hs, k, choice.table, choice.depth0);
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune_cache[tune_key(hs, k, alpha, max_depth)] = choice;
    }
    if (out) *out = rep;
    return FBN_OK;
}

// FBN_TUNE_AUTO: the first skeleton call on a shape takes the cached choices
// of this device and shape, or tunes.
int ensure_tuned(fbn_handle* const* hs, int k, double alpha, int32_t max_depth)
{
    fbn_handle* h = hs[0];
    if (h->opt.tune != FBN_TUNE_AUTO) return FBN_OK;
    const std::vector<long long> key = tune_key(hs, k, alpha, max_depth);
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            apply_tuning(hs, k, it->second.table, it->second.depth0);
            return FBN_OK;
        }
    }
    return autotune_impl(hs, k, alpha, max_depth, nullptr);
}

void free_handle(fbn_handle* h)
{
    if (!h) return;
    cudaSetDevice(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    set_snapshot(h, nullptr);
    h->ws.release();
    dfree(h->d_data); dfree(h->d_planes); dfree(h->d_ar); dfree(h->d_adj); dfree(h->d_nbr); dfree(h->d_eid); dfree(h->d_npos); dfree(h->d_deg);
    dfree(h->d_sep_len); dfree(h->d_sep_off); dfree(h->d_prob);
    dfree(h->d_sep_cnt);
    dfree(h->d_ci); dfree(h->d_ci_out); dfree(h->d_status); dfree(h->d_table); dfree(h->d_gscratch);
    dfree(h->d_off);
    if (h->h_ci) cudaFreeHost(h->h_ci);
    if (h->h_ci_out) cudaFreeHost(h->h_ci_out);
    if (h->h_status) cudaFreeHost(h->h_status);
    if (h->own_stream) cudaStreamDestroy(h->own_stream);
    delete h;
}

}  // namespace

void fbn::fbn_internal_set_error(const char* msg)
{
    g_create_error = msg;
}

// ==========================================================================
extern "C" {

int fbn_create(const uint8_t* data, int32_t n_vars, int64_t n_samples, const uint8_t* arities,
               const fbn_options* opt, fbn_handle** out)
{
    fbn_handle* h = nullptr;
    if (!out) return fail(nullptr, FBN_EINVAL, "out is NULL");
    *out = nullptr;
    if (!data || !arities) return fail(nullptr, FBN_EINVAL, "data or arities is NULL");
    if (n_vars < 2 || n_vars > kMaxVars)
        return fail(nullptr, FBN_EINVAL, "n_vars=%d outside [2, %d]", n_vars, kMaxVars);
    if (n_samples < 1 || n_samples >= (1LL << 31)) return fail(nullptr, FBN_EINVAL, "n_samples=%lld outside [1, 2^31)", (long long)n_samples);
    fbn_options o{};
    o.device = -1;
    if (opt) {
        o = *opt;
        for (int k = 0; k < 4; ++k)
            if (o.reserved[k]) return fail(nullptr, FBN_EINVAL, "reserved option field %d is nonzero", k);
        if (o.loop != FBN_LOOP_DEVICE && o.loop != FBN_LOOP_HOST) return fail(nullptr, FBN_EINVAL, "bad loop %d", o.loop);
        if (o.wait_limit < -1) return fail(nullptr, FBN_EINVAL, "bad wait_limit %d", o.wait_limit);
        if (o.group_threads != 0 && o.group_threads != 32 && o.group_threads != 64 && o.group_threads != 128 &&
            o.group_threads != kTestThreads)
            return fail(nullptr, FBN_EINVAL, "bad group_threads %d", o.group_threads);
        if (o.form != FBN_FORM_POOL && o.form != FBN_FORM_PLAIN) return fail(nullptr, FBN_EINVAL, "bad form %d", o.form);
        if (o.group_size < 0) return fail(nullptr, FBN_EINVAL, "bad group_size %d", o.group_size);
        if (o.depth0 < FBN_DEPTH0_AUTO || o.depth0 > FBN_DEPTH0_GRAM) return fail(nullptr, FBN_EINVAL, "bad depth0 %d", o.depth0);
        if (o.depth1 < FBN_DEPTH1_AUTO || o.depth1 > FBN_DEPTH1_TENSOR) return fail(nullptr, FBN_EINVAL, "bad depth1 %d", o.depth1);
        if (o.statistic != FBN_STAT_G2 && o.statistic != FBN_STAT_X2)
            return fail(nullptr, FBN_EINVAL, "bad statistic %d", o.statistic);
        if (o.df_mode != FBN_DF_FIXED && o.df_mode != FBN_DF_ADJUSTED)
            return fail(nullptr, FBN_EINVAL, "bad df_mode %d", o.df_mode);
        if (o.count < FBN_COUNT_AUTO || o.count > FBN_COUNT_BITS) return fail(nullptr, FBN_EINVAL, "bad count %d", o.count);
        if (o.tune != FBN_TUNE_OFF && o.tune != FBN_TUNE_AUTO) return fail(nullptr, FBN_EINVAL, "bad tune %d", o.tune);
        if (o.depth1 == FBN_DEPTH1_TENSOR && (o.statistic != FBN_STAT_G2 || o.df_mode != FBN_DF_FIXED))
            return fail(nullptr, FBN_EINVAL, "depth1 tensor takes the G^2 statistic with fixed df only");
    }
    int max_ar = 0;
    for (int v = 0; v < n_vars; ++v) {
        if (arities[v] < 2) return fail(nullptr, FBN_EINVAL, "arity of variable %d is %d < 2", v, arities[v]);
        max_ar = std::max(max_ar, (int)arities[v]);
    }
    if (o.depth1 == FBN_DEPTH1_TENSOR && max_ar > nbr1_max_arity())
        return fail(nullptr, FBN_EINVAL, "depth1 tensor takes arities <= %d, not %d", nbr1_max_arity(), max_ar);
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return fail(nullptr, FBN_ECUDA, "no CUDA device available");
    }
    int dev = o.device;
    if (dev < 0) {
        if (cudaGetDevice(&dev) != cudaSuccess) return fail(nullptr, FBN_ECUDA, "cudaGetDevice failed");
    }
    if (dev >= ndev) return fail(nullptr, FBN_EINVAL, "device %d of %d", dev, ndev);
    if (cudaSetDevice(dev) != cudaSuccess) return fail(nullptr, FBN_ECUDA, "cudaSetDevice(%d) failed", dev);

    h = new fbn_handle();
    h->device = dev;
    h->opt = o;
    h->n = n_vars;
    h->N = n_samples;
    h->ld = (n_samples + 255) / 256 * 256;
    h->max_arity = max_ar;
    h->h_ar.assign(arities, arities + n_vars);
    auto bail = [&](int code) {
        std::string m = h->err;
        free_handle(h);
        g_create_error = m;
        return code;
    };
#define CKC(call)                                                                          \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            fail(h, e_ == cudaErrorMemoryAllocation ? FBN_ENOMEM : FBN_ECUDA, "%s: %s", #call, \
                 cudaGetErrorString(e_));                                                  \
            return bail(e_ == cudaErrorMemoryAllocation ? FBN_ENOMEM : FBN_ECUDA);           \
        }                                                                                  \
    } while (0)
    CKC(cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking));
    h->stream = h->own_stream;
    const size_t nn = (size_t)n_vars * n_vars;
    CKC(dalloc(&h->d_data, (size_t)n_vars * h->ld));
    h->plane_ld = ((n_samples + 31) / 32 + 3) / 4 * 4;   // 32-sample words, whole uint4 groups
    CKC(dalloc(&h->d_planes, (size_t)n_vars * 2 * h->plane_ld));
    CKC(dalloc(&h->d_ar, n_vars));
    CKC(dalloc(&h->d_adj, nn));
    CKC(dalloc(&h->d_nbr, nn));
    CKC(dalloc(&h->d_eid, nn));
    CKC(dalloc(&h->d_npos, nn));
    CKC(dalloc(&h->d_deg, n_vars));
    CKC(dalloc(&h->d_sep_len, nn));
    CKC(dalloc(&h->d_sep_off, nn));
    CKC(dalloc(&h->d_prob, 1));
    CKC(dalloc(&h->d_ci, 1));
    CKC(dalloc(&h->d_ci_out, 3));
    CKC(dalloc(&h->d_status, 1));
    CKC(cudaMallocHost((void**)&h->h_ci, sizeof(CiTestDesc)));
    CKC(cudaMallocHost((void**)&h->h_ci_out, 3 * sizeof(double)));
    CKC(cudaMallocHost((void**)&h->h_status, sizeof(unsigned long long)));
    cudaStream_t st = h->stream;
    CKC(cudaMemsetAsync(h->d_data, 0, (size_t)n_vars * h->ld, st));
    CKC(cudaMemsetAsync(h->d_eid, 0, nn * sizeof(int32_t), st));
    CKC(cudaMemcpy2DAsync(h->d_data, h->ld, data, n_samples, n_samples, n_vars, cudaMemcpyDefault, st));
    CKC(cudaMemcpyAsync(h->d_ar, arities, n_vars, cudaMemcpyHostToDevice, st));
    // values must lie below their arity: checked on the device
    unsigned long long* bad = (unsigned long long*)h->d_ci_out;   // scratch, 8 bytes
    CKC(cudaMemsetAsync(bad, 0xff, sizeof(unsigned long long), st));
    {
        dim3 grid((unsigned)std::min<long long>((n_samples + 255) / 256, 64), n_vars);
        k_validate<<<grid, 256, 0, st>>>(h->d_data, h->ld, n_vars, n_samples, h->d_ar, bad);
    }
    CKC(cudaGetLastError());
    if (launch_planes(h, st)) return bail(FBN_ECUDA);
    unsigned long long first_bad = 0;
    CKC(cudaMemcpyAsync(h->h_status, bad, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    CKC(cudaStreamSynchronize(st));
    std::memcpy(&first_bad, h->h_status, sizeof first_bad);
    if (first_bad != ~0ULL) {
        const long long v = (long long)(first_bad / (unsigned long long)n_samples);
        const long long s = (long long)(first_bad % (unsigned long long)n_samples);
        fail(h, FBN_EDATA, "value of variable %lld at sample %lld is >= its arity %d", v, s, (int)arities[v]);
        return bail(FBN_EDATA);
    }
    {
        std::vector<int32_t> off(n_vars);
        int M = 0;
        for (int v = 0; v < n_vars; ++v) {
            off[v] = M;
            M += arities[v];
        }
        h->M = M;
        h->Mp = gram_rows_padded(M);
        h->K = gram_samples_padded(n_samples);
        CKC(dalloc(&h->d_off, n_vars));
        CKC(cudaMemcpy(h->d_off, off.data(), n_vars * sizeof(int32_t), cudaMemcpyHostToDevice));
    }
    ProblemDev P{};
    P.data = h->d_data; P.ar = h->d_ar; P.adj = h->d_adj; P.nbr = h->d_nbr; P.eid = h->d_eid; P.npos = h->d_npos; P.deg = h->d_deg;
    P.sep_len = h->d_sep_len; P.sep_off = h->d_sep_off; P.ld = h->ld; P.n = n_vars; P.N = (int32_t)n_samples;
    P.max_arity = max_ar;
    P.planes = h->d_planes; P.plane_ld = h->plane_ld;
    CKC(cudaMemcpyAsync(h->d_prob, &P, sizeof P, cudaMemcpyHostToDevice, st));
    CKC(cudaStreamSynchronize(st));
#undef CKC
    *out = h;
    return FBN_OK;
}

int fbn_update_data(fbn_handle* h, const uint8_t* data)
{
    if (!h) return FBN_EINVAL;
    if (!data) return fail(h, FBN_EINVAL, "data is NULL");
    CK(cudaSetDevice(h->device));
    cudaStream_t st = h->stream;
    h->learnt = false;
    h->sep_pending = false;
    CK(cudaMemcpy2DAsync(h->d_data, h->ld, data, h->N, h->N, h->n, cudaMemcpyDefault, st));
    unsigned long long* bad = (unsigned long long*)h->d_ci_out;   // 8 bytes of scratch
    CK(cudaMemsetAsync(bad, 0xff, sizeof(unsigned long long), st));
    dim3 grid((unsigned)std::min<long long>((h->N + 255) / 256, 64), h->n);
    k_validate<<<grid, 256, 0, st>>>(h->d_data, h->ld, h->n, h->N, h->d_ar, bad);
    CK(cudaGetLastError());
    const int prc = launch_planes(h, st);
    if (prc) return prc;
    CK(cudaMemcpyAsync(h->h_status, bad, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    unsigned long long first_bad;
    std::memcpy(&first_bad, h->h_status, sizeof first_bad);
    if (first_bad != ~0ULL) {
        const long long v = (long long)(first_bad / (unsigned long long)h->N);
        const long long smp = (long long)(first_bad % (unsigned long long)h->N);
        return fail(h, FBN_EDATA, "value of variable %lld at sample %lld is >= its arity %d", v, smp,
                    (int)h->h_ar[v]);
    }
    return FBN_OK;
}

int fbn_update_data_batch(fbn_handle* const* hs, int32_t k, const uint8_t* const* data)
{
    if (!hs || k < 1 || !hs[0] || !data) return FBN_EINVAL;
    fbn_handle* h = hs[0];
    for (int p = 0; p < k; ++p) {
        if (!hs[p]) return fail(h, FBN_EINVAL, "handle %d is NULL", p);
        if (!data[p]) return fail(h, FBN_EINVAL, "data %d is NULL", p);
        if (hs[p]->device != h->device) return fail(h, FBN_EINVAL, "handle %d is on another device", p);
    }
    CK(cudaSetDevice(h->device));
    cudaStream_t st = h->stream;
    for (int p = 0; p < k; ++p) {   // every copy, check and bit-plane build queued on one stream
        fbn_handle* q = hs[p];
        q->learnt = false;
        q->sep_pending = false;
        CK(cudaMemcpy2DAsync(q->d_data, q->ld, data[p], q->N, q->N, q->n, cudaMemcpyDefault, st));
        unsigned long long* bad = (unsigned long long*)q->d_ci_out;   // 8 bytes of scratch
        CK(cudaMemsetAsync(bad, 0xff, sizeof(unsigned long long), st));
        dim3 grid((unsigned)std::min<long long>((q->N + 255) / 256, 64), q->n);
        k_validate<<<grid, 256, 0, st>>>(q->d_data, q->ld, q->n, q->N, q->d_ar, bad);
        CK(cudaGetLastError());
        const int prc = launch_planes(q, st);
        if (prc) return fail(h, prc, "%s", q->err.c_str());
        CK(cudaMemcpyAsync(q->h_status, bad, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    }
    CK(cudaStreamSynchronize(st));
    for (int p = 0; p < k; ++p) {
        const fbn_handle* q = hs[p];
        unsigned long long first_bad;
        std::memcpy(&first_bad, q->h_status, sizeof first_bad);
        if (first_bad != ~0ULL) {
            const long long v = (long long)(first_bad / (unsigned long long)q->N);
            const long long smp = (long long)(first_bad % (unsigned long long)q->N);
            return fail(h, FBN_EDATA, "data set %d: value of variable %lld at sample %lld is >= its arity %d", p, v, smp,
                        (int)q->h_ar[v]);
        }
    }
    return FBN_OK;
}

int fbn_set_stream(fbn_handle* h, void* stream)
{
    if (!h) return FBN_EINVAL;
    h->stream = stream ? (cudaStream_t)stream : h->own_stream;
    return FBN_OK;
}

int fbn_ci_test(fbn_handle* h, int32_t x, int32_t y, const int32_t* z, int32_t nz, double* g2, double* df,
                double* p)
{
    if (!h) return FBN_EINVAL;
    if (!g2 || !df || !p) return fail(h, FBN_EINVAL, "null output pointer");
    long long cells = 0;
    int rc = check_test_args(h, x, y, z, nz, &cells);
    if (rc) return rc;
    rc = run_ci(h, x, y, z, nz, cells, false);
    if (rc) return rc;
    *g2 = h->h_ci_out[0];
    *df = h->h_ci_out[1];
    *p = h->h_ci_out[2];
    return FBN_OK;
}

int fbn_ci_table(fbn_handle* h, int32_t x, int32_t y, const int32_t* z, int32_t nz, int32_t* counts, int64_t cap)
{
    if (!h) return FBN_EINVAL;
    if (!counts) return fail(h, FBN_EINVAL, "counts is NULL");
    long long cells = 0;
    int rc = check_test_args(h, x, y, z, nz, &cells);
    if (rc) return rc;
    if (cap < cells) return fail(h, FBN_EINVAL, "cap %lld < %lld cells", (long long)cap, cells);
    rc = run_ci(h, x, y, z, nz, cells, true);
    if (rc) return rc;
    CK(cudaMemcpy(counts, h->d_table, cells * sizeof(int32_t), cudaMemcpyDeviceToHost));
    return FBN_OK;
}

int fbn_learn_skeleton(fbn_handle* h, double alpha, int32_t max_depth, uint8_t* adj_out)
{
    if (!h) return FBN_EINVAL;
    h->sep_pending = false;
    if (!(alpha > 0.0 && alpha < 1.0)) return fail(h, FBN_EINVAL, "alpha=%g outside (0, 1)", alpha);
    if (max_depth < -1) return fail(h, FBN_EINVAL, "max_depth=%d < -1", max_depth);
    h->learnt = false;
    fbn_handle* hs[1] = {h};
    uint8_t* outs[1] = {adj_out};
    const int rc = ensure_tuned(hs, 1, alpha, max_depth);
    if (rc) return rc;
    return run_skeleton(hs, 1, alpha, max_depth, outs);
}

int fbn_learn_skeleton_batch(fbn_handle* const* hs, int32_t k, double alpha, int32_t max_depth,
                             uint8_t* const* adj_out)
{
    if (!hs || k < 1) return FBN_EINVAL;
    fbn_handle* h = hs[0];
    for (int p = 0; p < k; ++p) {
        if (!hs[p]) return fail(h, FBN_EINVAL, "handle %d is NULL", p);
        if (hs[p]->device != h->device) return fail(h, FBN_EINVAL, "handle %d is on another device", p);
        hs[p]->learnt = false;
        hs[p]->sep_pending = false;
    }
    if (!(alpha > 0.0 && alpha < 1.0)) return fail(h, FBN_EINVAL, "alpha=%g outside (0, 1)", alpha);
    if (max_depth < -1) return fail(h, FBN_EINVAL, "max_depth=%d < -1", max_depth);
    const int rc = ensure_tuned(hs, k, alpha, max_depth);
    if (rc) return rc;
    return run_skeleton(hs, k, alpha, max_depth, adj_out);
}

int fbn_learn_skeleton_sharded(fbn_handle* h, double alpha, int32_t max_depth, fbn_shard_own_fn own,
                               fbn_shard_exchange_fn exchange, void* ctx, uint8_t* adj_out)
{
    if (!h) return FBN_EINVAL;
    h->sep_pending = false;
    h->learnt = false;
    if (!own || !exchange) return fail(h, FBN_EINVAL, "own and exchange callbacks are required");
    if (!(alpha > 0.0 && alpha < 1.0)) return fail(h, FBN_EINVAL, "alpha=%g outside (0, 1)", alpha);
    if (max_depth < -1) return fail(h, FBN_EINVAL, "max_depth=%d < -1", max_depth);
    fbn_handle* hs[1] = {h};
    uint8_t* outs[1] = {adj_out};
    const ShardHooks hooks{own, exchange, ctx};
    return run_skeleton(hs, 1, alpha, max_depth, outs, &hooks);
}

int fbn_autotune(fbn_handle* const* hs, int32_t k, double alpha, int32_t max_depth, fbn_tuning* out)
{
    if (!hs || k < 1 || !hs[0]) return FBN_EINVAL;
    fbn_handle* h = hs[0];
    for (int p = 0; p < k; ++p) {
        if (!hs[p]) return fail(h, FBN_EINVAL, "handle %d is NULL", p);
        if (hs[p]->device != h->device) return fail(h, FBN_EINVAL, "handle %d is on another device", p);
        hs[p]->learnt = false;
        hs[p]->sep_pending = false;
    }
    if (!(alpha > 0.0 && alpha < 1.0)) return fail(h, FBN_EINVAL, "alpha=%g outside (0, 1)", alpha);
    if (max_depth < -1) return fail(h, FBN_EINVAL, "max_depth=%d < -1", max_depth);
    return autotune_impl(hs, k, alpha, max_depth, out);
}

int fbn_pairwise_counts(fbn_handle* h, int32_t* counts, int64_t cap)
{
    if (!h) return FBN_EINVAL;
    if (!counts) return fail(h, FBN_EINVAL, "counts is NULL");
    const long long MM = (long long)h->M * h->M;
    if (cap < MM) return fail(h, FBN_EINVAL, "cap %lld < M*M = %lld", (long long)cap, MM);
    CK(cudaSetDevice(h->device));
    Workspace& ws = h->ws;
    fbn_handle* hs[1] = {h};
    int rc = grow_workspace(h, ws, (long long)h->n * (h->n - 1) / 2, h->n, 1, h->n);
    if (rc) return rc;
    ProblemDev P{};
    P.data = h->d_data; P.ar = h->d_ar; P.adj = h->d_adj; P.nbr = h->d_nbr; P.eid = h->d_eid; P.npos = h->d_npos; P.deg = h->d_deg;
    P.sep_len = h->d_sep_len; P.sep_off = h->d_sep_off; P.ld = h->ld; P.n = h->n; P.N = (int32_t)h->N;
    P.max_arity = h->max_arity;
    rc = prepare_gram(hs, 1, ws, &P);
    if (rc) return rc;
    std::vector<int32_t> vp(h->n, 0), vf(1, 0);
    ws.up_last.clear();   // the skeleton's next call uploads its own descriptors again
    CK(cudaMemcpyAsync(ws.probs, &P, sizeof P, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(ws.vtx_prob, vp.data(), h->n * sizeof(int32_t), cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(ws.vtx_first, vf.data(), sizeof(int32_t), cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemsetAsync(h->d_status, 0, sizeof(unsigned), h->stream));
    rc = run_gram(h, ws, 1, h->n, h->d_status);
    if (rc) return rc;
    CK(launch_symmetrize(P.gram, h->Mp, h->M, h->stream));
    CK(cudaMemcpy2DAsync(counts, (size_t)h->M * sizeof(int32_t), P.gram, (size_t)h->Mp * sizeof(int32_t),
                         (size_t)h->M * sizeof(int32_t), (size_t)h->M, cudaMemcpyDefault, h->stream));
    CK(cudaMemcpyAsync(h->h_status, h->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return check_status(h, *h->h_status);
}

int32_t fbn_get_sepset(const fbn_handle* hc, int32_t i, int32_t j, int32_t* buf, int32_t cap)
{
    if (!hc || !hc->learnt) return FBN_EINVAL;
    fbn_handle* h = const_cast<fbn_handle*>(hc);   // the host copy is a cache of device results
    if (h->sep_pending) {
        const int rc = materialize_sepsets(h, h->ws);
        if (rc) return rc;
    }
    if (i < 0 || j < 0 || i >= h->n || j >= h->n || i == j) return FBN_EINVAL;
    if (i > j) std::swap(i, j);
    const long long k = find_sepset(h, i, j);
    if (k < 0) return -1;
    const int32_t L = (int32_t)(h->csr_offs[k + 1] - h->csr_offs[k]);
    if (L > 0 && cap > 0 && !buf) return FBN_EINVAL;
    for (int t = 0; t < L && t < cap; ++t) buf[t] = h->csr_members[(size_t)h->csr_offs[k] + t];
    return L;
}

int fbn_export_sepsets(const fbn_handle* hc, int64_t* n_removed, int64_t* n_members, int32_t* pairs,
                       int64_t* offsets, int32_t* members)
{
    if (!hc || !hc->learnt || !n_removed || !n_members) return FBN_EINVAL;
    fbn_handle* h = const_cast<fbn_handle*>(hc);   // the host copy is a cache of device results
    if (h->sep_pending) {
        const int rc = materialize_sepsets(h, h->ws);
        if (rc) return rc;
    }
    const int64_t nr = (int64_t)h->csr_offs.size() - 1, nm = h->csr_offs.back();
    if (pairs && nr > 0) std::memcpy(pairs, h->csr_pairs.data(), 2 * (size_t)nr * sizeof(int32_t));
    if (offsets && nr > 0) std::memcpy(offsets, h->csr_offs.data(), (size_t)nr * sizeof(int64_t));
    if (members && nm > 0) std::memcpy(members, h->csr_members.data(), (size_t)nm * sizeof(int32_t));
    if (offsets) offsets[nr] = nm;
    *n_removed = nr;
    *n_members = nm;
    return FBN_OK;
}

int fbn_orient_cpdag(const fbn_handle* hc, uint8_t* cpdag_out)
{
    if (!hc || !hc->learnt || !cpdag_out) return FBN_EINVAL;
    fbn_handle* h = const_cast<fbn_handle*>(hc);   // the host copy is a cache of device results
    if (h->sep_pending) {
        const int rc = materialize_sepsets(h, h->ws);
        if (rc) return rc;
    }
    const int n = h->n;
    const size_t nn = (size_t)n * n;
    std::vector<uint8_t> A(nn);
    CK(cudaSetDevice(h->device));
    CK(cudaMemcpyAsync(A.data(), h->d_adj, nn, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    std::vector<std::vector<int>> nb(n);
    for (int u = 0; u < n; ++u)
        for (int v = 0; v < n; ++v)
            if (A[(size_t)u * n + v]) nb[u].push_back(v);
    auto adj = [&](int u, int v) { return A[(size_t)u * n + v] != 0; };
    auto in_sepset = [&](int a, int b, int k) {   // a < b, not adjacent
        const long long r = find_sepset(h, a, b);
        if (r < 0) return false;
        for (int64_t t = h->csr_offs[r]; t < h->csr_offs[r + 1]; ++t)
            if (h->csr_members[(size_t)t] == k) return true;
        return false;
    };
    // step 2: arrowheads of the unshielded colliders
    std::vector<uint8_t> head(nn, 0);   // head[a*n+k]: a -> k marked
    for (int k = 0; k < n; ++k) {
        const std::vector<int>& N = nb[k];
        for (size_t x = 0; x < N.size(); ++x)
            for (size_t y = x + 1; y < N.size(); ++y) {
                const int a = N[x], b = N[y];
                if (adj(a, b) || in_sepset(a, b, k)) continue;
                head[(size_t)a * n + k] = 1;
                head[(size_t)b * n + k] = 1;
            }
    }
    std::vector<uint8_t> arc(nn, 0);    // arc[a*n+b]: a -> b oriented
    for (size_t e = 0; e < nn; ++e) {
        const size_t a = e / n, b = e % n;
        if (head[e] && !head[b * n + a]) arc[e] = 1;
    }
    auto open = [&](int u, int v) { return adj(u, v) && !arc[(size_t)u * n + v] && !arc[(size_t)v * n + u]; };
    // step 3: Meek rules in rounds
    std::vector<std::pair<int, int>> found;
    std::vector<uint8_t> want(nn, 0);
    for (;;) {
        found.clear();
        for (int b = 0; b < n; ++b)
            for (int c : nb[b]) {
                if (!open(b, c)) continue;
                bool orient = false;
                for (int a : nb[b]) {
                    if (a != c && arc[(size_t)a * n + b] && !adj(a, c)) orient = true;      // R1
                    if (arc[(size_t)b * n + a] && arc[(size_t)a * n + c]) orient = true;  // R2
                    if (orient) break;
                }
                if (!orient) {   // R3: two non-adjacent m1, m2 with b - m -> c
                    std::vector<int> mids;
                    for (int m : nb[b])
                        if (open(b, m) && arc[(size_t)m * n + c]) mids.push_back(m);
                    for (size_t x = 0; x < mids.size() && !orient; ++x)
                        for (size_t y = x + 1; y < mids.size(); ++y)
                            if (!adj(mids[x], mids[y])) {
                                orient = true;
                                break;
                            }
                }
                if (orient) {
                    found.emplace_back(b, c);
                    want[(size_t)b * n + c] = 1;
                }
            }
        bool changed = false;
        for (const auto& bc : found) {
            const size_t fw = (size_t)bc.first * n + bc.second, bw = (size_t)bc.second * n + bc.first;
            if (!want[bw]) {
                arc[fw] = 1;
                changed = true;
            }
        }
        for (const auto& bc : found) want[(size_t)bc.first * n + bc.second] = 0;
        if (!changed) break;
    }
    for (size_t e = 0; e < nn; ++e) {
        const size_t a = e / n, b = e % n;
        cpdag_out[e] = (A[e] && !arc[b * n + a]) ? 1 : 0;
    }
    return FBN_OK;
}

int fbn_get_stats(const fbn_handle* h, fbn_stats* out)
{
    if (!h || !out) return FBN_EINVAL;
    *out = h->stats;
    return FBN_OK;
}

const char* fbn_last_error(const fbn_handle* h)
{
    return h ? h->err.c_str() : g_create_error.c_str();
}

void fbn_destroy(fbn_handle* h)
{
    free_handle(h);
}

}  // extern "C"
