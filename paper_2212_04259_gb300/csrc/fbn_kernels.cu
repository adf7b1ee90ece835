// fbn_kernels.cu -- per-depth kernels of the PC-stable skeleton (Algorithm 1)
// and the single-test kernel, for sm_103a.
//
// Depth pipeline (every kernel runs over all problems of a batch at once):
//   k_snapshot   a(v) for every vertex: adjacency row -> ascending neighbour list
//   k_edges      edges i<j with at least one test, with their rank space
//                |X-side| + |Y-side|, split into a warp class (tables that fit
//                a warp's share of shared memory) and a CTA class
//   k_chunk_hist / k_scan / k_place
//                order each class by chunk count, so that pass k of the work
//                pool is a prefix of that order
//   k_pool<G>    persistent CI-level work pool (Section IV-B): each group (a
//                warp or a CTA) claims work items -- one chunk of gs
//                consecutive conditioning sets of one edge -- from one atomic
//                counter; items are laid out pass by pass, so every live edge
//                gets its k-th chunk before any edge gets its (k+1)-th; chunks
//                above an edge's lowest accepting rank are skipped
//   k_plain      edge-level form (Section IV-A): one CTA per edge, sequential
//                conditioning sets with early exit
//   k_apply      end-of-depth removal over the snapshot; the separating set is
//                the conditioning set of the lowest accepting rank
#include <cstdint>
#include <cuda_runtime.h>

#include "fbn_device.cuh"
#include "fbn_launch.h"

namespace fbn {

// --------------------------------------------------------------------------
__global__ void k_snapshot(const ProblemDev* __restrict__ probs, const int32_t* __restrict__ vtx_prob,
                           const int32_t* __restrict__ vtx_first, int total_vertices)
{
    const int g = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (g >= total_vertices) return;
    const int p = vtx_prob[g];
    const ProblemDev P = probs[p];
    const int v = g - vtx_first[p];
    const uint8_t* row = P.adj + (long long)v * P.n;
    int32_t* out = P.nbr + (long long)v * P.n;
    int count = 0;
    for (int j0 = 0; j0 < P.n; j0 += 32) {
        const int j = j0 + lane;
        const bool a = j < P.n && row[j];
        const unsigned m = __ballot_sync(0xffffffffu, a);
        if (a) out[count + __popc(m & ((1u << lane) - 1u))] = j;
        count += __popc(m);
    }
    if (lane == 0) P.deg[v] = count;
}

// --------------------------------------------------------------------------
__device__ __forceinline__ long long binom_sat(const long long* B, int brows, int n, int k)
{
    if (k < 0 || n < k) return 0;
    if (n >= brows || k >= kBinomCols) return kBinomSat;
    return B[(long long)n * kBinomCols + k];
}

__global__ void k_edges(const ProblemDev* __restrict__ probs, const int32_t* __restrict__ vtx_prob,
                        const int32_t* __restrict__ vtx_first, int total_vertices, int d, int gs,
                        const long long* __restrict__ binom, int brows, long long warp_cells_cap,
                        EdgeWork* __restrict__ edges, unsigned long long* __restrict__ min_accept,
                        long long edge_cap, DepthCounters* ctr)
{
    const int g = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (g >= total_vertices) return;
    const int p = vtx_prob[g];
    const ProblemDev P = probs[p];
    const int i = g - vtx_first[p];
    const int deg_i = P.deg[i];
    const int32_t* nb = P.nbr + (long long)i * P.n;
    unsigned long long mc[2] = {0, 0}, mcell[2] = {0, 0};
    for (int t0 = 0; t0 < deg_i; t0 += 32) {
        const int t = t0 + lane;
        int j = -1;
        long long cnt_i = 0, total = 0;
        if (t < deg_i) {
            j = nb[t];
            if (j > i) {
                if (d == 0) {
                    cnt_i = 1;
                    total = 1;
                } else {
                    cnt_i = binom_sat(binom, brows, deg_i - 1, d);
                    total = cnt_i + binom_sat(binom, brows, P.deg[j] - 1, d);
                }
            }
        }
        unsigned long long cells = 0;
        if (total > 0) {
            // cells bound r_i r_j max_arity^d
            cells = (unsigned long long)P.ar[i] * P.ar[j];
            for (int k = 0; k < d && cells <= (unsigned long long)kMaxCells; ++k)
                cells *= (unsigned long long)P.max_arity;
        }
        const int cls = cells <= (unsigned long long)warp_cells_cap ? kClassWarp : kClassCta;
        for (int c = 0; c < 2; ++c) {
            const bool take = total > 0 && cls == c;
            const unsigned m = __ballot_sync(0xffffffffu, take);
            unsigned long long base = 0;
            if (lane == 0 && m) base = atomicAdd(&ctr->n_edges[c], (unsigned long long)__popc(m));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (!take) continue;
            const long long k = (long long)base + __popc(m & ((1u << lane) - 1u));
            if (k >= edge_cap) {
                atomicOr(&ctr->status, kStatusEdges);
                continue;
            }
            const long long e = c == kClassWarp ? k : edge_cap - 1 - k;
            // position of i in a(j)
            const int32_t* nj = P.nbr + (long long)j * P.n;
            int lo = 0, hi = P.deg[j];
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (nj[mid] < i) lo = mid + 1; else hi = mid;
            }
            EdgeWork w;
            w.prob = p; w.i = i; w.j = j;
            w.posj = (int16_t)t; w.posi = (int16_t)lo;
            w.cnt_i = cnt_i; w.total = total;
            edges[e] = w;
            min_accept[e] = (unsigned long long)total;
            const unsigned long long ch = (unsigned long long)((total + gs - 1) / gs);
            mc[c] = ch > mc[c] ? ch : mc[c];
            mcell[c] = cells > mcell[c] ? cells : mcell[c];
        }
    }
#pragma unroll
    for (int c = 0; c < 2; ++c) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long a = __shfl_down_sync(0xffffffffu, mc[c], o);
            const unsigned long long b = __shfl_down_sync(0xffffffffu, mcell[c], o);
            mc[c] = a > mc[c] ? a : mc[c];
            mcell[c] = b > mcell[c] ? b : mcell[c];
        }
        if (lane == 0) {
            if (mc[c]) atomicMax(&ctr->maxc[c], mc[c]);
            if (mcell[c]) atomicMax(&ctr->max_cells[c], mcell[c]);
        }
    }
}

// --------------------------------------------------------------------------
__global__ void k_chunk_hist(const EdgeWork* __restrict__ edges, long long E, int gs,
                             unsigned long long* __restrict__ hist)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    const long long ch = (edges[e].total + gs - 1) / gs;
    atomicAdd(&hist[ch], 1ULL);
}

// One CTA: alive[k] = #edges with more than k chunks (k = 0..maxc), base[k] =
// sum_{k' < k} alive[k'] (k = 0..maxc).  base[maxc] is the item count.
// Block-wide scans over contiguous per-thread segments.
__device__ __forceinline__ unsigned long long block_exclusive_scan(unsigned long long v, unsigned long long* sh)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[warp] = x;
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        unsigned long long s = lane < nw ? sh[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < nw) sh[lane] = s;
    }
    __syncthreads();
    const unsigned long long before = warp > 0 ? sh[warp - 1] : 0;
    __syncthreads();
    return before + x - v;
}

__global__ void k_scan(const unsigned long long* __restrict__ hist, long long maxc,
                       unsigned long long* __restrict__ alive, unsigned long long* __restrict__ base,
                       unsigned long long* total_items, unsigned long long* next_item)
{
    __shared__ unsigned long long sh[32];
    const int T = blockDim.x;
    const long long len = maxc + 1;
    const long long seg = (len + T - 1) / T;
    // alive[c] = sum_{c' > c} hist[c']: thread t owns the t-th segment counted
    // from the end of the array, so an exclusive scan in thread order sums the
    // segments that lie after this thread's one
    long long lo = len - (long long)(threadIdx.x + 1) * seg, hi = len - (long long)threadIdx.x * seg;
    if (lo < 0) lo = 0;
    if (hi < 0) hi = 0;
    unsigned long long s = 0;
    for (long long c = lo; c < hi; ++c) s += hist[c];
    unsigned long long run = block_exclusive_scan(s, sh);
    for (long long c = hi - 1; c >= lo; --c) {
        alive[c] = run;
        run += hist[c];
    }
    __syncthreads();
    // base[k] = sum_{k' < k} alive[k'], segments in forward order
    const long long flo = (long long)threadIdx.x * seg, fhi = flo + seg < len ? flo + seg : len;
    s = 0;
    for (long long c = flo; c < fhi; ++c) s += alive[c];
    run = block_exclusive_scan(s, sh);
    for (long long c = flo; c < fhi; ++c) {
        base[c] = run;
        run += alive[c];
    }
    if (fhi == len && flo < fhi) {
        *total_items = base[maxc];
        *next_item = 0;
    }
}

__global__ void k_place(const EdgeWork* __restrict__ edges, long long E, int gs,
                        const unsigned long long* __restrict__ alive, unsigned long long* __restrict__ cursor,
                        int32_t* __restrict__ sorted)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    const long long ch = (edges[e].total + gs - 1) / gs;
    const unsigned long long pos = alive[ch] + atomicAdd(&cursor[ch], 1ULL);
    sorted[pos] = (int32_t)e;
}

// --------------------------------------------------------------------------
// Per-group state of a worker, in shared memory.
struct GroupState {
    long long r0, r1;
    int e;
    int go;
    double crit;
    int pos[kMaxD];
};

// Fill the test of rank rk of edge w into the group's TestSpec.  Rank 0 of
// the group computes the subset positions (unranked when `fresh`, else the
// successor of the previous rank of the same side); one thread per
// conditioning variable then resolves its row.  Returns false (uniformly)
// when the table is over the cell limit.
template <int G>
__device__ __forceinline__ bool setup_rank(const ProblemDev& P, const EdgeWork& w, int d, long long rk, bool fresh,
                                           GroupState& S, const long long* binom, TestSpec& spec, unsigned* status)
{
    const int r = Grp<G>::rank();
    const bool xside = rk < w.cnt_i;
    const int a = xside ? w.i : w.j;
    const int posb = xside ? w.posj : w.posi;
    if (r == 0) {
        if (d > 0) {
            const long long lr = xside ? rk : rk - w.cnt_i;
            const int p = P.deg[a] - 1;
            if (fresh || lr == 0) unrank_lex(lr, p, d, binom, S.pos);
            else next_subset(p, d, S.pos);
        }
        spec.nrows = d + 2;
        spec.N = P.N;
    }
    Grp<G>::sync();
    if (r < d) {
        const int t = S.pos[r];
        const int v = P.nbr[(long long)a * P.n + (t < posb ? t : t + 1)];
        spec.rows[r] = P.data + (long long)v * P.ld;
        spec.rad[r] = P.ar[v];
    } else if (r == d) {
        spec.rows[d] = P.data + (long long)w.i * P.ld;
        spec.rad[d] = spec.rx = P.ar[w.i];
    } else if (r == d + 1) {
        spec.rows[d + 1] = P.data + (long long)w.j * P.ld;
        spec.rad[d + 1] = spec.ry = P.ar[w.j];
    }
    Grp<G>::sync();
    long long cells = 1;
    for (int k = 0; k < d + 2 && cells <= kMaxCells; ++k) cells *= spec.rad[k];
    if (cells > kMaxCells) {
        if (r == 0) atomicOr(status, kStatusTooBig);
        return false;
    }
    if (r == 0) spec.cells = cells;
    Grp<G>::sync();
    return true;
}

// Run one rank: 1 = accepts independence, 0 = rejects, -1 = could not run.
template <int G>
__device__ __forceinline__ int run_rank(const PoolArgs& a, const ProblemDev& P, const EdgeWork& w, long long rk,
                                        bool fresh, GroupState& S, TestSpec& spec, int* slice, long long slice_ints,
                                        int* gtab, double* red)
{
    if (!setup_rank<G>(P, w, a.d, rk, fresh, S, a.binom, spec, a.status)) return -1;
    int* M = nullptr;
    const int* T = grp_table<G>(spec, slice, slice_ints, gtab, a.gscratch_ints, &M);
    if (!T) {
        if (Grp<G>::rank() == 0) atomicOr(a.status, kStatusTooBig);
        return -1;
    }
    grp_marginals<G>(spec, T, M);
    if (Grp<G>::rank() == 0) {
        const long long df = (long long)(spec.rx - 1) * (spec.ry - 1) * (spec.cells / (spec.rx * spec.ry));
        S.crit = crit_get(a.crit, df, a.alpha, a.status);
        atomicAdd(a.tests, 1ULL);
    }
    Grp<G>::sync();
    return grp_decide<G>(spec, T, M, S.crit, red) ? 1 : 0;
}

template <int G>
__global__ void __launch_bounds__(kTestThreads, G == kTestThreads ? 2 : 3) k_pool(PoolArgs a)
{
    extern __shared__ int smem[];
    constexpr int NG = kTestThreads / G;   // groups per CTA
    __shared__ TestSpec spec_s[NG];
    __shared__ GroupState st_s[NG];
    __shared__ double red[32];
    __shared__ unsigned long long base_s[kBaseSmem];
    const int g = Grp<G>::gid();
    const int r = Grp<G>::rank();
    const long long slice_ints = a.smem_ints / NG;
    int* slice = smem + g * slice_ints;
    int* gtab = a.gscratch ? a.gscratch + ((long long)blockIdx.x * NG + g) * a.gscratch_ints : nullptr;
    const unsigned long long total = *a.total_items;
    const bool base_in_smem = a.maxc + 1 <= kBaseSmem;
    if (base_in_smem)
        for (long long k = threadIdx.x; k <= a.maxc; k += blockDim.x) base_s[k] = a.base[k];
    __syncthreads();
    const unsigned long long* base = base_in_smem ? base_s : a.base;
    GroupState& S = st_s[g];
    TestSpec& spec = spec_s[g];

    for (;;) {
        if (r == 0) {
            const unsigned long long w = atomicAdd(a.next_item, 1ULL);
            S.e = -1;
            if (w < total) {
                long long lo = 0, hi = a.maxc - 1;   // pass k: largest k with base[k] <= w
                while (lo < hi) {
                    const long long mid = (lo + hi + 1) >> 1;
                    if (base[mid] <= w) lo = mid; else hi = mid - 1;
                }
                const int e = a.sorted[w - base[lo]];
                const long long r0 = lo * (long long)a.gs;
                const long long tot = a.edges[e].total;
                S.e = e;
                S.r0 = r0;
                S.r1 = r0 + a.gs < tot ? r0 + a.gs : tot;
            }
        }
        Grp<G>::sync();
        const int e = S.e;
        if (e < 0) break;
        const EdgeWork w = a.edges[e];
        const ProblemDev& P = a.probs[w.prob];
        const long long r0 = S.r0, r1 = S.r1;
        for (long long rk = r0; rk < r1; ++rk) {
            if (r == 0) S.go = (unsigned long long)rk <= *((volatile unsigned long long*)&a.min_accept[e]);
            Grp<G>::sync();
            if (!S.go) break;
            const int res = run_rank<G>(a, P, w, rk, rk == r0, S, spec, slice, slice_ints, gtab, red);
            if (res == 1 && r == 0) atomicMin(&a.min_accept[e], (unsigned long long)rk);
            if (res != 0) break;
        }
        Grp<G>::sync();
    }
}

__global__ void __launch_bounds__(kTestThreads, 2) k_plain(PoolArgs a, long long E)
{
    extern __shared__ int smem[];
    __shared__ TestSpec spec;
    __shared__ GroupState S;
    __shared__ double red[32];
    int* gtab = a.gscratch ? a.gscratch + (long long)blockIdx.x * a.gscratch_ints : nullptr;
    for (long long e = blockIdx.x; e < E; e += gridDim.x) {
        const EdgeWork w = a.edges[e];
        const ProblemDev& P = a.probs[w.prob];
        for (long long rk = 0; rk < w.total; ++rk) {
            const int res = run_rank<kTestThreads>(a, P, w, rk, rk == 0, S, spec, smem, a.smem_ints, gtab, red);
            if (res == 1 && threadIdx.x == 0) a.min_accept[e] = (unsigned long long)rk;
            if (res != 0) break;
        }
        __syncthreads();
    }
}

// --------------------------------------------------------------------------
__global__ void k_apply(const ProblemDev* __restrict__ probs, const EdgeWork* __restrict__ edges,
                        const unsigned long long* __restrict__ min_accept, long long E, int d,
                        const long long* __restrict__ binom, int32_t* __restrict__ sep_pool,
                        long long sep_cap, DepthCounters* ctr)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    const EdgeWork w = edges[e];
    const unsigned long long ma = min_accept[e];
    const bool rm = ma < (unsigned long long)w.total;
    atomicAdd(&ctr->tests_oracle, rm ? ma + 1 : (unsigned long long)w.total);
    if (!rm) return;
    atomicAdd(&ctr->removed, 1ULL);
    const ProblemDev P = probs[w.prob];
    const long long n = P.n;
    P.adj[w.i * n + w.j] = 0;
    P.adj[w.j * n + w.i] = 0;
    long long off = 0;
    if (d > 0) {
        off = (long long)atomicAdd(&ctr->sep_used, (unsigned long long)d);
        if (off + d > sep_cap) {
            atomicOr(&ctr->status, kStatusSepPool);
        } else {
            const bool xside = (long long)ma < w.cnt_i;
            const int a = xside ? w.i : w.j;
            const int posb = xside ? w.posj : w.posi;
            const long long lr = xside ? (long long)ma : (long long)ma - w.cnt_i;
            int pos[kMaxD];
            unrank_lex(lr, P.deg[a] - 1, d, binom, pos);
            const int32_t* nb = P.nbr + (long long)a * n;
            for (int k = 0; k < d; ++k) sep_pool[off + k] = nb[pos[k] < posb ? pos[k] : pos[k] + 1];
        }
    }
    P.sep_len[w.i * n + w.j] = d;
    P.sep_off[w.i * n + w.j] = off;
}

// --------------------------------------------------------------------------
// Explicit tests (fbn_ci_test / fbn_ci_table): exact FP64 G^2 and p-value.
__global__ void __launch_bounds__(kTestThreads) k_ci_tests(const ProblemDev* __restrict__ prob,
                                                           const CiTestDesc* __restrict__ tests, int ntests,
                                                           double* __restrict__ out, int32_t* table_out,
                                                           int* gscratch, long long gscratch_ints,
                                                           unsigned* status, int smem_ints)
{
    extern __shared__ int smem[];
    __shared__ TestSpec spec;
    __shared__ double red[32];
    __shared__ int s_ok;
    const int t = blockIdx.x;
    if (t >= ntests) return;
    const ProblemDev P = *prob;
    if (threadIdx.x == 0) {
        const CiTestDesc& q = tests[t];
        const int d = q.d;
        long long cells = 1;
        for (int k = 0; k < d; ++k) {
            spec.rows[k] = P.data + (long long)q.z[k] * P.ld;
            spec.rad[k] = P.ar[q.z[k]];
        }
        spec.rows[d] = P.data + (long long)q.x * P.ld;
        spec.rad[d] = P.ar[q.x];
        spec.rows[d + 1] = P.data + (long long)q.y * P.ld;
        spec.rad[d + 1] = P.ar[q.y];
        spec.nrows = d + 2;
        spec.rx = P.ar[q.x];
        spec.ry = P.ar[q.y];
        spec.N = P.N;
        for (int k = 0; k < d + 2 && cells <= kMaxCells; ++k) cells *= spec.rad[k];
        spec.cells = cells;
        s_ok = cells <= kMaxCells;
        if (!s_ok) atomicOr(status, kStatusTooBig);
    }
    __syncthreads();
    if (!s_ok) return;
    int* gtab = gscratch ? gscratch + (long long)t * gscratch_ints : nullptr;
    int* M = nullptr;
    const int* T = grp_table<kTestThreads>(spec, smem, smem_ints, gtab, gscratch_ints, &M);
    if (!T) {
        if (threadIdx.x == 0) atomicOr(status, kStatusTooBig);
        return;
    }
    grp_marginals<kTestThreads>(spec, T, M);
    const double g2 = grp_g2_exact<kTestThreads>(spec, T, M, red, table_out);
    if (threadIdx.x == 0) {
        const double df = (double)(spec.rx - 1) * (double)(spec.ry - 1) * (double)(spec.cells / (spec.rx * spec.ry));
        out[3 * t + 0] = g2;
        out[3 * t + 1] = df;
        out[3 * t + 2] = chisq_q(df, g2, status);
    }
}

// --------------------------------------------------------------------------
// host launchers
void launch_snapshot(const ProblemDev* probs, const int32_t* vtx_prob, const int32_t* vtx_first,
                     int total_vertices, cudaStream_t st)
{
    const int warps = 8;
    k_snapshot<<<(total_vertices + warps - 1) / warps, warps * 32, 0, st>>>(probs, vtx_prob, vtx_first,
                                                                           total_vertices);
}

void launch_edges(const ProblemDev* probs, const int32_t* vtx_prob, const int32_t* vtx_first,
                  int total_vertices, int d, int gs, const long long* binom, int brows, long long warp_cells_cap,
                  EdgeWork* edges, unsigned long long* min_accept, long long edge_cap, DepthCounters* ctr,
                  cudaStream_t st)
{
    const int warps = 8;
    k_edges<<<(total_vertices + warps - 1) / warps, warps * 32, 0, st>>>(
        probs, vtx_prob, vtx_first, total_vertices, d, gs, binom, brows, warp_cells_cap, edges, min_accept,
        edge_cap, ctr);
}

void launch_order(const EdgeWork* edges, long long E, int gs, long long maxc, unsigned long long* hist,
                  unsigned long long* alive, unsigned long long* base, unsigned long long* cursor,
                  int32_t* sorted, unsigned long long* total_items, unsigned long long* next_item,
                  cudaStream_t st)
{
    cudaMemsetAsync(hist, 0, (maxc + 1) * sizeof(unsigned long long), st);
    cudaMemsetAsync(cursor, 0, (maxc + 1) * sizeof(unsigned long long), st);
    const int T = 256;
    const unsigned blocks = (unsigned)((E + T - 1) / T);
    k_chunk_hist<<<blocks, T, 0, st>>>(edges, E, gs, hist);
    k_scan<<<1, 1024, 0, st>>>(hist, maxc, alive, base, total_items, next_item);
    k_place<<<blocks, T, 0, st>>>(edges, E, gs, alive, cursor, sorted);
}

void launch_pool(const PoolArgs& a, int group, int grid, size_t smem_bytes, cudaStream_t st)
{
    switch (group) {
        case 32: k_pool<32><<<grid, kTestThreads, smem_bytes, st>>>(a); break;
        case 64: k_pool<64><<<grid, kTestThreads, smem_bytes, st>>>(a); break;
        case 128: k_pool<128><<<grid, kTestThreads, smem_bytes, st>>>(a); break;
        default: k_pool<kTestThreads><<<grid, kTestThreads, smem_bytes, st>>>(a); break;
    }
}

void launch_plain(const PoolArgs& a, long long E, int grid, size_t smem_bytes, cudaStream_t st)
{
    k_plain<<<grid, kTestThreads, smem_bytes, st>>>(a, E);
}

void launch_apply(const ProblemDev* probs, const EdgeWork* edges, const unsigned long long* min_accept,
                  long long E, int d, const long long* binom, int32_t* sep_pool, long long sep_cap,
                  DepthCounters* ctr, cudaStream_t st)
{
    const int T = 256;
    k_apply<<<(unsigned)((E + T - 1) / T), T, 0, st>>>(probs, edges, min_accept, E, d, binom, sep_pool,
                                                       sep_cap, ctr);
}

void launch_ci_tests(const ProblemDev* prob, const CiTestDesc* tests, int ntests, double* out,
                     int32_t* table_out, int* gscratch, long long gscratch_ints, unsigned* status,
                     size_t smem_bytes, cudaStream_t st)
{
    k_ci_tests<<<ntests, kTestThreads, smem_bytes, st>>>(prob, tests, ntests, out, table_out, gscratch,
                                                         gscratch_ints, status, (int)(smem_bytes / 4));
}

cudaError_t set_kernel_smem(size_t max_smem)
{
    cudaError_t e;
    const int b = (int)max_smem;
    if ((e = cudaFuncSetAttribute(k_pool<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, b))) return e;
    if ((e = cudaFuncSetAttribute(k_pool<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, b))) return e;
    if ((e = cudaFuncSetAttribute(k_pool<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, b))) return e;
    if ((e = cudaFuncSetAttribute(k_pool<kTestThreads>, cudaFuncAttributeMaxDynamicSharedMemorySize, b))) return e;
    if ((e = cudaFuncSetAttribute(k_plain, cudaFuncAttributeMaxDynamicSharedMemorySize, b))) return e;
    return cudaFuncSetAttribute(k_ci_tests, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
}

int pool_blocks_per_sm(int group, size_t smem_bytes)
{
    int nb = 0;
    switch (group) {
        case 32: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_pool<32>, kTestThreads, smem_bytes); break;
        case 64: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_pool<64>, kTestThreads, smem_bytes); break;
        case 128: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_pool<128>, kTestThreads, smem_bytes); break;
        default:
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_pool<kTestThreads>, kTestThreads, smem_bytes);
            break;
    }
    return nb;
}

}  // namespace fbn
