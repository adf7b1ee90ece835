// fbn_kernels.cu -- per-depth kernels of the PC-stable skeleton (Algorithm 1)
// and the single-test kernel, for sm_103a.
//
// Depth pipeline (every kernel runs over all problems of a batch at once):
//   k_snapshot   a(v) for every vertex: adjacency row -> ascending neighbour list
//   k_edges      edges i<j with at least one test: rank space |X-side| + |Y-side|
//   k_chunk_hist / k_scan / k_place
//                order the edges by chunk count so that pass k of the work pool
//                is a prefix of that order
//   k_pool       persistent CI-level work pool (Section IV-B): each CTA claims
//                work items (one chunk of gs consecutive conditioning sets of one
//                edge) from a single atomic counter; items are laid out pass by
//                pass, so every live edge gets its k-th chunk before any edge
//                gets its (k+1)-th; chunks above an edge's lowest accepting
//                rank are skipped
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
                        const long long* __restrict__ binom, int brows, EdgeWork* __restrict__ edges,
                        unsigned long long* __restrict__ min_accept, long long edge_cap,
                        DepthCounters* ctr)
{
    const int g = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (g >= total_vertices) return;
    const int p = vtx_prob[g];
    const ProblemDev P = probs[p];
    const int i = g - vtx_first[p];
    const int deg_i = P.deg[i];
    const int32_t* nb = P.nbr + (long long)i * P.n;
    unsigned long long local_maxc = 0, local_cells = 0;
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
                    const long long cnt_j = binom_sat(binom, brows, P.deg[j] - 1, d);
                    total = cnt_i + cnt_j;
                }
            }
        }
        const bool take = total > 0;
        const unsigned m = __ballot_sync(0xffffffffu, take);
        unsigned long long base = 0;
        if (lane == 0 && m) base = atomicAdd(&ctr->n_edges, (unsigned long long)__popc(m));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (take) {
            const long long e = (long long)base + __popc(m & ((1u << lane) - 1u));
            if (e < edge_cap) {
                EdgeWork w;
                w.prob = p; w.i = i; w.j = j; w.pad = 0;
                w.cnt_i = cnt_i; w.total = total;
                edges[e] = w;
                min_accept[e] = (unsigned long long)total;
            }
            const unsigned long long ch = (unsigned long long)((total + gs - 1) / gs);
            local_maxc = ch > local_maxc ? ch : local_maxc;
            // cells bound: r_i r_j max_arity^d
            unsigned long long cells = (unsigned long long)P.ar[i] * P.ar[j];
            for (int k = 0; k < d && cells <= (unsigned long long)kMaxCells; ++k) cells *= (unsigned long long)P.max_arity;
            local_cells = cells > local_cells ? cells : local_cells;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long a = __shfl_down_sync(0xffffffffu, local_maxc, o);
        const unsigned long long b = __shfl_down_sync(0xffffffffu, local_cells, o);
        local_maxc = a > local_maxc ? a : local_maxc;
        local_cells = b > local_cells ? b : local_cells;
    }
    if (lane == 0) {
        if (local_maxc) atomicMax(&ctr->maxc, local_maxc);
        if (local_cells) atomicMax(&ctr->max_cells, local_cells);
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
__global__ void k_scan(const unsigned long long* __restrict__ hist, long long maxc,
                       unsigned long long* __restrict__ alive, unsigned long long* __restrict__ base,
                       DepthCounters* ctr)
{
    __shared__ unsigned long long part[1024];
    const int T = blockDim.x;
    const long long len = maxc + 1;
    const long long seg = (len + T - 1) / T;
    // suffix sums of hist: alive[k] = sum_{c > k} hist[c]
    const long long lo = (long long)threadIdx.x * seg, hi = lo + seg < len ? lo + seg : len;
    unsigned long long s = 0;
    for (long long c = lo; c < hi; ++c) s += hist[c];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {  // exclusive suffix scan of the segment sums
        unsigned long long run = 0;
        for (int t = T - 1; t >= 0; --t) {
            const unsigned long long v = part[t];
            part[t] = run;
            run += v;
        }
    }
    __syncthreads();
    unsigned long long run = part[threadIdx.x];   // sum of hist over later segments
    for (long long c = hi - 1; c >= lo; --c) {
        alive[c] = run;                           // sum over c' > c
        run += hist[c];
    }
    __syncthreads();
    // prefix sums of alive: base[k] = sum_{k' < k} alive[k']
    s = 0;
    for (long long c = lo; c < hi; ++c) s += alive[c];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long r = 0;
        for (int t = 0; t < T; ++t) {
            const unsigned long long v = part[t];
            part[t] = r;
            r += v;
        }
    }
    __syncthreads();
    run = part[threadIdx.x];
    for (long long c = lo; c < hi; ++c) {
        base[c] = run;
        run += alive[c];
    }
    if (hi == len && lo < hi) {
        // base[maxc] already written above as the sum over k < maxc; alive[maxc] == 0
        ctr->total_items = base[maxc];
        ctr->next_item = 0;
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
// Fill the test of rank r of edge w into the shared TestSpec (leader only).
// pos holds the subset positions; when `fresh` the positions are unranked,
// otherwise they are advanced from the previous rank of the same side.
__device__ __forceinline__ bool setup_rank(const ProblemDev& P, const EdgeWork& w, int d, long long r,
                                           bool fresh, int* pos, const long long* binom,
                                           TestSpec& s, unsigned* status)
{
    const bool xside = r < w.cnt_i;
    const int a = xside ? w.i : w.j;
    const int b = xside ? w.j : w.i;
    const long long lr = xside ? r : r - w.cnt_i;
    const int deg_a = P.deg[a];
    const int32_t* nb = P.nbr + (long long)a * P.n;
    if (d > 0) {
        const int p = deg_a - 1;
        if (fresh || lr == 0) unrank_lex(lr, p, d, binom, pos);
        else next_subset(p, d, pos);
        // position of b in a's ascending list
        int lo = 0, hi = deg_a;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (nb[mid] < b) lo = mid + 1; else hi = mid;
        }
        const int posb = lo;
        for (int k = 0; k < d; ++k) {
            const int t = pos[k];
            const int v = nb[t < posb ? t : t + 1];
            s.rows[k] = P.data + (long long)v * P.ld;
            s.rad[k] = P.ar[v];
        }
    }
    s.rows[d] = P.data + (long long)w.i * P.ld;
    s.rad[d] = P.ar[w.i];
    s.rows[d + 1] = P.data + (long long)w.j * P.ld;
    s.rad[d + 1] = P.ar[w.j];
    s.nrows = d + 2;
    s.rx = P.ar[w.i];
    s.ry = P.ar[w.j];
    s.N = P.N;
    long long cells = 1;
    for (int k = 0; k < d + 2; ++k) {
        cells *= s.rad[k];
        if (cells > kMaxCells) break;
    }
    s.cells = cells;
    if (cells > kMaxCells) {
        atomicOr(status, kStatusTooBig);
        return false;
    }
    return true;
}

__global__ void __launch_bounds__(kTestThreads) k_pool(PoolArgs a, unsigned long long maxc)
{
    extern __shared__ int smem[];
    __shared__ TestSpec spec;
    __shared__ double red[32];
    __shared__ unsigned long long s_item;
    __shared__ int s_edge;
    __shared__ long long s_r0, s_r1;
    __shared__ int s_go;
    __shared__ int s_pos[kMaxD];
    int* gtab = a.gscratch ? a.gscratch + (long long)blockIdx.x * a.gscratch_ints : nullptr;
    const unsigned long long total_items = a.ctr->total_items;
    unsigned* status = &a.ctr->status;

    for (;;) {
        if (threadIdx.x == 0) {
            const unsigned long long w = atomicAdd(&a.ctr->next_item, 1ULL);
            s_item = w;
            if (w < total_items) {
                // pass k = largest k with base[k] <= w
                long long lo = 0, hi = (long long)maxc - 1;
                while (lo < hi) {
                    const long long mid = (lo + hi + 1) >> 1;
                    if (a.base[mid] <= w) lo = mid; else hi = mid - 1;
                }
                const int e = a.sorted[w - a.base[lo]];
                const long long r0 = lo * (long long)a.gs;
                const long long tot = a.edges[e].total;
                s_edge = e;
                s_r0 = r0;
                s_r1 = r0 + a.gs < tot ? r0 + a.gs : tot;
            }
        }
        __syncthreads();
        if (s_item >= total_items) break;
        const int e = s_edge;
        const EdgeWork w = a.edges[e];
        const ProblemDev& P = a.probs[w.prob];
        for (long long r = s_r0; r < s_r1; ++r) {
            if (threadIdx.x == 0) {
                const unsigned long long ma = *((volatile unsigned long long*)&a.min_accept[e]);
                s_go = ((unsigned long long)r <= ma) &&
                       setup_rank(P, w, a.d, r, r == s_r0, s_pos, a.binom, spec, status);
            }
            __syncthreads();
            if (!s_go) break;
            const TestResult res = run_test(spec, smem, a.smem_ints, gtab, a.gscratch_ints, nullptr, status, red);
            if (threadIdx.x == 0) {
                atomicAdd(&a.ctr->tests, 1ULL);
                s_go = !(res.p > a.alpha);
                if (!s_go) atomicMin(&a.min_accept[e], (unsigned long long)r);
            }
            __syncthreads();
            if (!s_go) break;
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kTestThreads) k_plain(PoolArgs a, long long E)
{
    extern __shared__ int smem[];
    __shared__ TestSpec spec;
    __shared__ double red[32];
    __shared__ int s_go;
    __shared__ int s_pos[kMaxD];
    int* gtab = a.gscratch ? a.gscratch + (long long)blockIdx.x * a.gscratch_ints : nullptr;
    unsigned* status = &a.ctr->status;
    for (long long e = blockIdx.x; e < E; e += gridDim.x) {
        const EdgeWork w = a.edges[e];
        const ProblemDev& P = a.probs[w.prob];
        for (long long r = 0; r < w.total; ++r) {
            if (threadIdx.x == 0) s_go = setup_rank(P, w, a.d, r, r == 0, s_pos, a.binom, spec, status);
            __syncthreads();
            if (!s_go) break;
            const TestResult res = run_test(spec, smem, a.smem_ints, gtab, a.gscratch_ints, nullptr, status, red);
            if (threadIdx.x == 0) {
                atomicAdd(&a.ctr->tests, 1ULL);
                s_go = !(res.p > a.alpha);
                if (!s_go) a.min_accept[e] = (unsigned long long)r;
            }
            __syncthreads();
            if (!s_go) break;
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
            const int a = xside ? w.i : w.j, b = xside ? w.j : w.i;
            const long long lr = xside ? (long long)ma : (long long)ma - w.cnt_i;
            int pos[kMaxD];
            const int deg_a = P.deg[a];
            unrank_lex(lr, deg_a - 1, d, binom, pos);
            const int32_t* nb = P.nbr + (long long)a * n;
            int posb = 0;
            while (posb < deg_a && nb[posb] < b) ++posb;
            for (int k = 0; k < d; ++k) sep_pool[off + k] = nb[pos[k] < posb ? pos[k] : pos[k] + 1];
        }
    }
    P.sep_len[w.i * n + w.j] = d;
    P.sep_off[w.i * n + w.j] = off;
}

// --------------------------------------------------------------------------
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
        for (int k = 0; k < d + 2; ++k) {
            cells *= spec.rad[k];
            if (cells > kMaxCells) break;
        }
        spec.cells = cells;
        s_ok = cells <= kMaxCells;
        if (!s_ok) atomicOr(status, kStatusTooBig);
    }
    __syncthreads();
    if (!s_ok) return;
    int* gtab = gscratch ? gscratch + (long long)t * gscratch_ints : nullptr;
    const TestResult r = run_test(spec, smem, smem_ints, gtab, gscratch_ints, table_out, status, red);
    if (threadIdx.x == 0) {
        out[3 * t + 0] = r.g2;
        out[3 * t + 1] = r.df;
        out[3 * t + 2] = r.p;
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
                  int total_vertices, int d, int gs, const long long* binom, int brows, EdgeWork* edges,
                  unsigned long long* min_accept, long long edge_cap, DepthCounters* ctr, cudaStream_t st)
{
    const int warps = 8;
    k_edges<<<(total_vertices + warps - 1) / warps, warps * 32, 0, st>>>(
        probs, vtx_prob, vtx_first, total_vertices, d, gs, binom, brows, edges, min_accept, edge_cap, ctr);
}

void launch_order(const EdgeWork* edges, long long E, int gs, long long maxc, unsigned long long* hist,
                  unsigned long long* alive, unsigned long long* base, unsigned long long* cursor,
                  int32_t* sorted, DepthCounters* ctr, cudaStream_t st)
{
    cudaMemsetAsync(hist, 0, (maxc + 1) * sizeof(unsigned long long), st);
    cudaMemsetAsync(cursor, 0, (maxc + 1) * sizeof(unsigned long long), st);
    const int T = 256;
    const unsigned blocks = (unsigned)((E + T - 1) / T);
    k_chunk_hist<<<blocks, T, 0, st>>>(edges, E, gs, hist);
    k_scan<<<1, 1024, 0, st>>>(hist, maxc, alive, base, ctr);
    k_place<<<blocks, T, 0, st>>>(edges, E, gs, alive, cursor, sorted);
}

void launch_pool(const PoolArgs& a, unsigned long long maxc, int grid, size_t smem_bytes, cudaStream_t st)
{
    k_pool<<<grid, kTestThreads, smem_bytes, st>>>(a, maxc);
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

cudaError_t set_kernel_smem(size_t smem_bytes)
{
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_pool, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes))) return e;
    if ((e = cudaFuncSetAttribute(k_plain, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes))) return e;
    return cudaFuncSetAttribute(k_ci_tests, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
}

int pool_blocks_per_sm(size_t smem_bytes)
{
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_pool, kTestThreads, smem_bytes);
    return nb;
}

}  // namespace fbn
