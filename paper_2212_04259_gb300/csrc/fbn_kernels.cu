// fbn_kernels.cu -- per-depth kernels of the PC-stable skeleton (Algorithm 1)
// and their host launchers, for sm_103a.  The work-pool kernels live in
// fbn_pool_small.cu, fbn_pool_bits.cu, fbn_pool_big.cu and fbn_plain.cu (device
// code in fbn_pool.cuh); the explicit-test kernel in fbn_ci.cu.
//
// Depth pipeline (every kernel runs over all problems of a batch at once):
//   k_snapshot   a(v) for every vertex: adjacency row -> ascending neighbour list
//   k_edges      edges i<j with at least one test, with their rank space
//                |X-side| + |Y-side|, split into a warp class (tables that fit
//                a warp's share of shared memory) and a CTA class
//   k_scan / k_place
//                order each class by chunk count (counted by k_edges), so that
//                pass k of the work pool is a prefix of that order
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
//   k_depth_end  records the depth, decides whether Algorithm 1 goes on and
//                clears the per-depth counters for the next depth
//   k_gate       the loop's condition after the next depth's edge list
// Every kernel reads the depth and the sizes from the device counters, so one
// captured sequence serves every depth (the body of the depth loop's while
// node); a kernel that runs after the loop ended finds active == 0 and does
// nothing.
#include <cstdint>
#include <cuda_runtime.h>

#include "fbn_depth.cuh"
#include "fbn_launch.h"

namespace fbn {

// Launches of the depth kernels go through launch_pdl; set_pdl(false)
// launches them without the attribute.
static bool g_pdl = true;

// The work-pool kernels, each defined in its own translation unit.
__global__ void k_pool_small(PoolArgs a);
__global__ void k_pool_bits(PoolArgs a);
__global__ void k_pool_big(PoolArgs a);
__global__ void k_plain(PoolArgs a);

// --------------------------------------------------------------------------
__global__ void k_snapshot(const ProblemDev* __restrict__ probs, const int32_t* __restrict__ vtx_prob,
                           const int32_t* __restrict__ vtx_first, int total_vertices, DepthCounters* ctr)
{
    pdl_enter();
    const int g = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (g >= total_vertices || !ctr->active) return;
    if (g == 0 && lane == 0)
        if (DepthRecord* r = depth_rec(ctr, ctr->d)) r->t_begin = gtime();
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
        if (a) {
            const int slot = count + __popc(m & ((1u << lane) - 1u));
            out[slot] = j;
            P.npos[(long long)v * P.n + j] = slot;
        }
        count += __popc(m);
    }
    if (lane == 0) {
        P.deg[v] = count;
        atomicAdd((unsigned long long*)&ctr->adj_ends, (unsigned long long)count);
    }
}

// --------------------------------------------------------------------------
__device__ __forceinline__ long long binom_sat(const long long* B, int brows, int n, int k)
{
    if (k < 0 || n < k) return 0;
    if (n >= brows || k >= kBinomCols) return kBinomSat;
    return B[(long long)n * kBinomCols + k];
}

__global__ void k_edges(const ProblemDev* __restrict__ probs, const int32_t* __restrict__ vtx_prob,
                        const int32_t* __restrict__ vtx_first, int total_vertices, int gs_forced, long long gs_edges,
                        const long long* __restrict__ binom, int brows, long long warp_cells_cap, int bits_cells,
                        const uint8_t* __restrict__ owned, EdgeWork* __restrict__ edges,
                        unsigned long long* __restrict__ min_accept, long long edge_cap, DepthCounters* ctr,
                        unsigned long long* __restrict__ hist)
{
    pdl_enter();
    const int g = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (g >= total_vertices || !ctr->active) return;
    const int d = ctr->d;
    // ranks per chunk: 1 while the live edges are few against the groups
    // (latency of a single test dominates), 4 when there are many (fewer claims)
    const int gs = gs_forced > 0 ? gs_forced : ((long long)(ctr->adj_ends / 2) >= gs_edges ? 4 : 1);
    if (g == 0 && lane == 0) ctr->gs = gs;
    const int p = vtx_prob[g];
    const ProblemDev P = probs[p];
    const int i = g - vtx_first[p];
    const int deg_i = P.deg[i];
    const int32_t* nb = P.nbr + (long long)i * P.n;
    unsigned long long mc[2] = {0, 0}, mcell[2] = {0, 0}, mtot[2] = {0, 0};
    for (int t0 = 0; t0 < deg_i; t0 += 32) {
        const int t = t0 + lane;
        int j = -1;
        long long cnt_i = 0, total = 0;
        if (t < deg_i) {
            j = nb[t];
            // owned: the edges this process tests when several share the
            // skeleton (one problem; entry [i][j], i < j); nullptr: every edge
            if (j > i && (owned == nullptr || owned[(long long)i * P.n + j])) {
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
        // the small-table class runs on the bit-plane pool only if every one
        // of its edges qualifies there (all arities <= 4, d <= 1, table bound
        // within bits_cells)
        const bool bits = bits_cells > 0 && !(tune_code(ctr->tune, d) & kTuneNoBits) && bits_shape_ok(d, P.max_arity, P.N) &&
                          cells <= (unsigned long long)bits_cells;
        if (__any_sync(0xffffffffu, total > 0 && cls == kClassWarp && !bits) && lane == 0) ctr->bits_ok = 0;
        {   // chunk-count histogram of each class: one atomic per distinct bin in the warp
            const long long bin = total > 0 ? (long long)cls * (kMaxPasses + 1) + chunk_count(total, gs) : -1;
            const unsigned same = __match_any_sync(0xffffffffu, bin);
            if (bin >= 0 && lane == __ffs(same) - 1) atomicAdd(&hist[bin], (unsigned long long)__popc(same));
        }
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
            const int lo = P.npos[(long long)j * P.n + i];   // position of i in a(j)
            EdgeWork w;
            w.prob = p; w.i = i; w.j = j;
            w.posj = (int16_t)t; w.posi = (int16_t)lo;
            w.cnt_i = cnt_i; w.total = total;
            edges[e] = w;
            min_accept[e] = (unsigned long long)total;
            P.eid[(long long)i * P.n + t] = (int32_t)e;
            P.eid[(long long)j * P.n + lo] = (int32_t)e;
            const unsigned long long ch = (unsigned long long)chunk_count(total, gs);
            mc[c] = ch > mc[c] ? ch : mc[c];
            mcell[c] = cells > mcell[c] ? cells : mcell[c];
            mtot[c] = (unsigned long long)total > mtot[c] ? (unsigned long long)total : mtot[c];
        }
    }
#pragma unroll
    for (int c = 0; c < 2; ++c) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long a = __shfl_down_sync(0xffffffffu, mc[c], o);
            const unsigned long long b = __shfl_down_sync(0xffffffffu, mcell[c], o);
            const unsigned long long t = __shfl_down_sync(0xffffffffu, mtot[c], o);
            mc[c] = a > mc[c] ? a : mc[c];
            mcell[c] = b > mcell[c] ? b : mcell[c];
            mtot[c] = t > mtot[c] ? t : mtot[c];
        }
        if (lane == 0) {
            if (mc[c]) atomicMax(&ctr->maxc[c], mc[c]);
            if (mcell[c]) atomicMax(&ctr->max_cells[c], mcell[c]);
            if (mtot[c]) atomicMax(&ctr->max_total[c], mtot[c]);
        }
    }
}

// --------------------------------------------------------------------------
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

// One CTA per class.  Also picks the group size of the small-table class
// from a cost model of the depth: with W work items and g(G) groups of G
// threads, the pool runs ceil(W / g(G)) rounds of one test each, a test
// costing a fixed latency (claim, setup, merge, decision; ~kTestOverhead
// cycles) plus the counting of N samples over G threads (~kCyclesPerSample
// per sample and thread).  groups[k] = groups of size 32 << k; the caller
// may force a size.
constexpr double kTestOverhead = 10000.0;
constexpr double kCyclesPerSample = 8.0;
constexpr double kCyclesPerSampleBits = 3.0;   // the bit-plane pool

__global__ void k_scan(ScanClass c0, ScanClass c1, DepthCounters* ctr, double mean_n, int forced_group,
                       long long split_stride, int allow_split)
{
    pdl_enter();
    __shared__ unsigned long long sh[32];
    if (!ctr->active) return;
    if (blockIdx.x == 0 && threadIdx.x == 0)
        if (DepthRecord* r = depth_rec(ctr, ctr->d)) r->t_tests = gtime();
    const int cls = blockIdx.x;   // one CTA per edge class
    const ScanClass& sc = cls == 0 ? c0 : c1;
    const unsigned long long* __restrict__ hist = sc.hist;
    unsigned long long* __restrict__ alive = sc.alive;
    unsigned long long* __restrict__ base = sc.base;
    const bool bits = cls == kClassWarp && ctr->bits_ok;   // the class runs on the bit-plane pool
    const long long* grp = bits ? sc.groups_bits : sc.groups;
    const long long g32 = grp[0], g64 = grp[1], g128 = grp[2], g256 = grp[3];
    const long long smem_ints = bits ? sc.smem_ints_bits : sc.smem_ints;
    const long long maxc = (long long)ctr->maxc[cls];
    if (ctr->n_edges[cls] == 0) return;
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
        const unsigned long long W = base[maxc];
        ctr->total_items[cls] = W;
        ctr->next_item[cls] = 0;
        if (cls == 0) {
            const long long groups[4] = {g32, g64, g128, g256};
            int best = kTestThreads;
            double best_t = 1e300;
            for (int k = 0; k < 4; ++k) {
                const int G = 32 << k;
                const double rounds = (double)((W + groups[k] - 1) / groups[k]);
                const double t = rounds * (kTestOverhead + (bits ? kCyclesPerSampleBits : kCyclesPerSample) * mean_n / G);
                if (t < best_t) {
                    best_t = t;
                    best = G;
                }
            }
            // the bit-plane pool: warp groups; else the caller's choice, the
            // autotuner's for this depth, or the cost model's
            const int tuned = tune_code(ctr->tune, ctr->d) & kTuneGroupMask;
            ctr->gsel = bits ? 32 : forced_group ? forced_group : tuned ? tuned : best;
        }
        // sample split: few single-rank tests against the groups of the class
        const int G = cls == 0 ? ctr->gsel : kTestThreads;
        const long long groups = cls == 0 ? (G == 32 ? g32 : G == 64 ? g64 : G == 128 ? g128 : g256) : g256;
        const long long slice = smem_ints * G / kTestThreads;
        const long long mcell = (long long)ctr->max_cells[cls];
        long long sp = 1;
        if (allow_split && ctr->gs == 1 && ctr->max_total[cls] <= (unsigned long long)kMaxPasses &&
            (long long)W * 2 <= groups && (long long)W <= kSplitItems && mcell <= split_stride &&
                    (mcell * 9) / 4 + 64 <= slice) {
            sp = groups / (long long)W;
            const long long by_n = (long long)mean_n / kSplitMinSamples;
            sp = sp < by_n ? sp : by_n;
            sp = sp < kMaxSplit ? sp : kMaxSplit;
            sp = sp > 1 ? sp : 1;
        }
        ctr->split[cls] = (int)sp;
        ctr->total_items[cls] = W * (unsigned long long)sp;
    }
}

// Both classes at once: class c's order goes to sorted[class_base(c) ..], the
// same region its edges occupy, so the two never overlap.
__global__ void k_place(const EdgeWork* __restrict__ edges, long long edge_cap, int nclass,
                        const DepthCounters* ctr, const unsigned long long* __restrict__ alive0,
                        unsigned long long* __restrict__ cursor0, const unsigned long long* __restrict__ alive1,
                        unsigned long long* __restrict__ cursor1, int32_t* __restrict__ sorted)
{
    pdl_enter();
    if (!ctr->active) return;
    const int gs = ctr->gs;
    const long long E0 = (long long)ctr->n_edges[0];
    const long long E = E0 + (nclass > 1 ? (long long)ctr->n_edges[1] : 0);
    const long long b1 = class_base(ctr, 1, edge_cap);
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < E; k += (long long)gridDim.x * blockDim.x) {
        const bool first = k < E0;
        const long long e = first ? k : k - E0;
        const long long cb = first ? 0 : b1;
        const long long ch = chunk_count(edges[cb + e].total, gs);
        const unsigned long long pos =
            first ? alive0[ch] + atomicAdd(&cursor0[ch], 1ULL) : alive1[ch] + atomicAdd(&cursor1[ch], 1ULL);
        sorted[cb + (long long)pos] = (int32_t)e;
    }
}

// --------------------------------------------------------------------------
__global__ void k_apply(const ProblemDev* __restrict__ probs, const EdgeWork* __restrict__ edges,
                        const unsigned long long* __restrict__ min_accept, long long edge_cap,
                        const long long* __restrict__ binom, int32_t* __restrict__ sep_pool, long long sep_cap,
                        DepthCounters* ctr)
{
    pdl_enter();
    if (!ctr->active) return;
    const int d = ctr->d;
    const long long n0 = (long long)ctr->n_edges[0], n1 = (long long)ctr->n_edges[1];
    unsigned long long my_tests = 0, my_removed = 0, my_samples = 0;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n0 + n1;
         k += (long long)gridDim.x * blockDim.x) {
        const long long e = k < n0 ? k : edge_cap - n1 + (k - n0);
        const EdgeWork w = edges[e];
        const unsigned long long ma = min_accept[e];
        const bool rm = ma < (unsigned long long)w.total;
        const unsigned long long t = rm ? ma + 1 : (unsigned long long)w.total;
        my_tests += t;
        my_samples += t * (unsigned long long)probs[w.prob].N;
        if (!rm) continue;
        my_removed += 1;
        const ProblemDev P = probs[w.prob];
        const long long n = P.n;
        P.adj[w.i * n + w.j] = 0;
        P.adj[w.j * n + w.i] = 0;
        long long off = 0;
        if (d > 0) {
            off = (long long)atomicAdd(&ctr->sep_used, (unsigned long long)d);
            if (off + d > sep_cap) {
                atomicOr(&ctr->status, kStatusSepPool);
                off = 0;
            } else {
                const bool xside = (long long)ma < w.cnt_i;
                const int a = xside ? w.i : w.j;
                const int posb = xside ? w.posj : w.posi;
                const long long lr = xside ? (long long)ma : (long long)ma - w.cnt_i;
                int pos[kMaxD];
                unrank_lex(lr, P.deg[a] - 1, d, binom, pos);
                const int32_t* nb = P.nbr + (long long)a * n;
                for (int q = 0; q < d; ++q) sep_pool[off + q] = nb[pos[q] < posb ? pos[q] : pos[q] + 1];
            }
        }
        P.sep_len[w.i * n + w.j] = d;
        P.sep_off[w.i * n + w.j] = off;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        my_tests += __shfl_xor_sync(0xffffffffu, my_tests, o);
        my_removed += __shfl_xor_sync(0xffffffffu, my_removed, o);
        my_samples += __shfl_xor_sync(0xffffffffu, my_samples, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (my_tests) atomicAdd(&ctr->tests_oracle, my_tests);
        if (my_samples) atomicAdd(&ctr->test_samples, my_samples);
        if (my_removed) atomicAdd(&ctr->removed, my_removed);
    }
}

// Sharded skeletons (several processes test shares of one problem's edges):
// the depth's removals of this process's edges as (i, j, lowest accepting
// rank) records, without applying them; the oracle-equivalent test counts as
// k_apply keeps them.
__global__ void k_export_removed(const ProblemDev* __restrict__ probs, const EdgeWork* __restrict__ edges,
                                 const unsigned long long* __restrict__ min_accept, long long edge_cap,
                                 DepthCounters* ctr, long long* __restrict__ out, unsigned long long* __restrict__ count)
{
    pdl_enter();
    if (!ctr->active) return;
    const long long n0 = (long long)ctr->n_edges[0], n1 = (long long)ctr->n_edges[1];
    unsigned long long my_tests = 0, my_samples = 0;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n0 + n1;
         k += (long long)gridDim.x * blockDim.x) {
        const long long e = k < n0 ? k : edge_cap - n1 + (k - n0);
        const EdgeWork w = edges[e];
        const unsigned long long ma = min_accept[e];
        const bool rm = ma < (unsigned long long)w.total;
        const unsigned long long t = rm ? ma + 1 : (unsigned long long)w.total;
        my_tests += t;
        my_samples += t * (unsigned long long)probs[w.prob].N;
        if (rm) {
            const unsigned long long pos = atomicAdd(count, 1ULL);   // < edges of the depth <= edge_cap
            out[3 * pos] = w.i;
            out[3 * pos + 1] = w.j;
            out[3 * pos + 2] = (long long)ma;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        my_tests += __shfl_xor_sync(0xffffffffu, my_tests, o);
        my_samples += __shfl_xor_sync(0xffffffffu, my_samples, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (my_tests) atomicAdd(&ctr->tests_oracle, my_tests);
        if (my_samples) atomicAdd(&ctr->test_samples, my_samples);
    }
}

// Sharded skeletons: remove every process's records of the depth from the
// snapshot (identical on every process) and keep the separating set of each:
// the conditioning set of its rank in the order of k_edges (X-side subsets of
// a(i)\{j} first, then Y-side subsets of a(j)\{i}, each lexicographic).
// Records were validated on the host (i < j < n, adjacent, rank within the
// edge's rank space).
__global__ void k_apply_list(const ProblemDev* __restrict__ probs, const long long* __restrict__ list, long long n_list,
                             const long long* __restrict__ binom, int brows, int32_t* __restrict__ sep_pool,
                             long long sep_cap, DepthCounters* ctr)
{
    pdl_enter();
    if (!ctr->active) return;
    const int d = ctr->d;
    const ProblemDev P = probs[0];
    const long long n = P.n;
    unsigned long long my_removed = 0;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n_list;
         t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)list[3 * t], j = (int)list[3 * t + 1];
        const long long ma = list[3 * t + 2];
        my_removed += 1;
        P.adj[i * n + j] = 0;
        P.adj[j * n + i] = 0;
        long long off = 0;
        if (d > 0) {
            const long long cnt_i = binom_sat(binom, brows, P.deg[i] - 1, d);
            const bool xside = ma < cnt_i;
            const int a = xside ? i : j;
            const int posb = xside ? P.npos[(long long)i * n + j] : P.npos[(long long)j * n + i];
            const long long lr = xside ? ma : ma - cnt_i;
            off = (long long)atomicAdd(&ctr->sep_used, (unsigned long long)d);
            if (off + d > sep_cap) {
                atomicOr(&ctr->status, kStatusSepPool);
                off = 0;
            } else {
                int pos[kMaxD];
                unrank_lex(lr, P.deg[a] - 1, d, binom, pos);
                const int32_t* nb = P.nbr + (long long)a * n;
                for (int q = 0; q < d; ++q) sep_pool[off + q] = nb[pos[q] < posb ? pos[q] : pos[q] + 1];
            }
        }
        P.sep_len[i * n + j] = d;
        P.sep_off[i * n + j] = off;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) my_removed += __shfl_xor_sync(0xffffffffu, my_removed, o);
    if ((threadIdx.x & 31) == 0 && my_removed) atomicAdd(&ctr->removed, my_removed);
}

// The next depth of a sharded skeleton runs whatever this process's share
// held: the host decides when Algorithm 1 stops.
__global__ void k_shard_continue(DepthCounters* ctr)
{
    pdl_enter();
    if (ctr->status == 0) ctr->active = 1;
}

// End of a depth (one CTA): record it; stop when it had no edge to test (no
// edge has a side with at least d candidates), when an error bit is set, or
// when the next depth exceeds max_depth (>= 0); clear the per-depth counters,
// the chunk histograms and the placement cursors for the next depth.
__global__ void k_depth_end(DepthCounters* ctr, DepthRecord* rec, int max_depth, unsigned long long* hist,
                            unsigned long long* cursor)
{
    pdl_enter();
    __shared__ long long used[2];   // histogram / cursor entries this depth touched per class
    if (!ctr->active) return;
    if (threadIdx.x < 2) used[threadIdx.x] = (long long)ctr->maxc[threadIdx.x] + 1;
    __syncthreads();
    if (threadIdx.x == 0) {
        const int d = ctr->d;
        const long long E = (long long)(ctr->n_edges[0] + ctr->n_edges[1]);
        if (d < kMaxDepthRecords) {
            rec[d].edges = E;
            rec[d].tests = (long long)ctr->tests;
            rec[d].tests_oracle = (long long)ctr->tests_oracle;
            rec[d].test_samples = (long long)ctr->test_samples;
            rec[d].popc_work = (long long)ctr->popc_work;
            rec[d].smem_updates = (long long)ctr->smem_updates;
            rec[d].removed = (long long)ctr->removed;
            rec[d].t_end = gtime();
        }
        const int next = d + 1;
        const bool stop = E == 0 || ctr->status != 0 || (max_depth >= 0 && next > max_depth) || next > kMaxD ||
                          next >= kMaxDepthRecords;
        for (int c = 0; c < 2; ++c)
            ctr->n_edges[c] = ctr->maxc[c] = ctr->next_item[c] = ctr->total_items[c] = ctr->max_cells[c] = 0;
        ctr->tests = ctr->tests_oracle = ctr->removed = ctr->test_samples = ctr->popc_work = ctr->smem_updates = 0;
        ctr->gsel = 0;
        ctr->adj_ends = 0;
        ctr->nbr_claim = 0;
        ctr->max_total[0] = ctr->max_total[1] = 0;
        ctr->split[0] = ctr->split[1] = 1;
        ctr->bits_ok = 1;
        ctr->d = next;
        __threadfence();
        ctr->active = stop ? 0 : 1;
    }
    for (int c = 0; c < 2; ++c) {
        const long long n = used[c] < kMaxPasses + 1 ? used[c] : kMaxPasses + 1;
        unsigned long long* hc = hist + c * (kMaxPasses + 1);
        unsigned long long* cc = cursor + c * (kMaxPasses + 1);
        for (long long k = threadIdx.x; k < n; k += blockDim.x) {
            hc[k] = 0;
            cc[k] = 0;
        }
    }
}

// Condition of the depth loop's graph (one thread), after the edge list of
// the next depth: go on while Algorithm 1 continues and the depth has an edge
// to test (no edge with a side of at least d candidates: the loop ends).
__global__ void k_gate(DepthCounters* ctr, cudaGraphConditionalHandle loop)
{
    pdl_enter();
    const bool go = ctr->active && ctr->n_edges[0] + ctr->n_edges[1] > 0;
    if (!go) ctr->active = 0;
    cudaGraphSetConditional(loop, go ? 1u : 0u);
}

// --------------------------------------------------------------------------
// host launchers

// Launch with programmatic stream serialisation (see pdl_enter).
template <typename... KArgs, typename... Args>
static void launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = g_pdl ? 1 : 0;
    cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

void launch_snapshot(const ProblemDev* probs, const int32_t* vtx_prob, const int32_t* vtx_first,
                     int total_vertices, DepthCounters* ctr, cudaStream_t st)
{
    const int warps = 8;
    launch_pdl(k_snapshot, dim3((total_vertices + warps - 1) / warps), dim3(warps * 32), 0, st, probs, vtx_prob,
               vtx_first, total_vertices, ctr);
}

void launch_edges(const ProblemDev* probs, const int32_t* vtx_prob, const int32_t* vtx_first,
                  int total_vertices, int gs_forced, long long gs_edges, const long long* binom, int brows,
                  long long warp_cells_cap, int bits_cells, const uint8_t* owned,
                  EdgeWork* edges, unsigned long long* min_accept, long long edge_cap, DepthCounters* ctr,
                  unsigned long long* hist, cudaStream_t st)
{
    const int warps = 8;
    launch_pdl(k_edges, dim3((total_vertices + warps - 1) / warps), dim3(warps * 32), 0, st, probs, vtx_prob,
               vtx_first, total_vertices, gs_forced, gs_edges, binom, brows, warp_cells_cap, bits_cells, owned, edges,
               min_accept, edge_cap, ctr, hist);
}

void launch_order(const EdgeWork* edges, long long edge_cap, int nclass, DepthCounters* ctr, const ScanClass* sc,
                  unsigned long long* cursor0, unsigned long long* cursor1, int32_t* sorted, double mean_n,
                  int forced_group, long long split_stride, int allow_split, int grid, cudaStream_t st)
{
    launch_pdl(k_scan, dim3(nclass), dim3(256), 0, st, sc[0], sc[nclass > 1 ? 1 : 0], ctr, mean_n, forced_group,
               split_stride, allow_split);
    launch_pdl(k_place, dim3(grid), dim3(256), 0, st, edges, edge_cap, nclass, ctr, (const unsigned long long*)sc[0].alive,
               cursor0, (const unsigned long long*)sc[nclass > 1 ? 1 : 0].alive, cursor1, sorted);
}

void launch_pool(const PoolArgs& a, int cls, int grid, size_t smem_bytes, cudaStream_t st)
{
    if (cls == kClassWarp) launch_pdl(k_pool_small, dim3(grid), dim3(kTestThreads), smem_bytes, st, a);
    else launch_pdl(k_pool_big, dim3(grid), dim3(kTestThreads), smem_bytes, st, a);
}

void launch_pool_bits(const PoolArgs& a, int grid, size_t smem_bytes, cudaStream_t st)
{
    launch_pdl(k_pool_bits, dim3(grid), dim3(kTestThreads), smem_bytes, st, a);
}

void launch_plain(const PoolArgs& a, int grid, size_t smem_bytes, cudaStream_t st)
{
    launch_pdl(k_plain, dim3(grid), dim3(kTestThreads), smem_bytes, st, a);
}

void launch_apply(const ProblemDev* probs, const EdgeWork* edges, const unsigned long long* min_accept,
                  long long edge_cap, const long long* binom, int32_t* sep_pool, long long sep_cap,
                  DepthCounters* ctr, int grid, cudaStream_t st)
{
    launch_pdl(k_apply, dim3(grid), dim3(256), 0, st, probs, edges, min_accept, edge_cap, binom, sep_pool, sep_cap,
               ctr);
}

void launch_shard_export(const ProblemDev* probs, const EdgeWork* edges, const unsigned long long* min_accept,
                         long long edge_cap, DepthCounters* ctr, long long* out, unsigned long long* count, int grid,
                         cudaStream_t st)
{
    launch_pdl(k_export_removed, dim3(grid), dim3(256), 0, st, probs, edges, min_accept, edge_cap, ctr, out, count);
}

void launch_shard_apply(const ProblemDev* probs, const long long* list, long long n_list, const long long* binom,
                        int brows, int32_t* sep_pool, long long sep_cap, DepthCounters* ctr, int grid, cudaStream_t st)
{
    launch_pdl(k_apply_list, dim3(grid), dim3(256), 0, st, probs, list, n_list, binom, brows, sep_pool, sep_cap, ctr);
}

void launch_shard_continue(DepthCounters* ctr, cudaStream_t st)
{
    launch_pdl(k_shard_continue, dim3(1), dim3(1), 0, st, ctr);
}

void launch_depth_end(DepthCounters* ctr, DepthRecord* rec, int max_depth, unsigned long long* hist,
                      unsigned long long* cursor, cudaStream_t st)
{
    launch_pdl(k_depth_end, dim3(1), dim3(256), 0, st, ctr, rec, max_depth, hist, cursor);
}

void launch_gate(DepthCounters* ctr, cudaGraphConditionalHandle loop, cudaStream_t st)
{
    launch_pdl(k_gate, dim3(1), dim3(1), 0, st, ctr, loop);
}

void set_pdl(bool on)
{
    g_pdl = on;
}

cudaError_t set_kernel_smem(size_t max_smem)
{
    cudaError_t e;
    const int b = (int)max_smem;
    if ((e = cudaFuncSetAttribute(k_pool_small, cudaFuncAttributeMaxDynamicSharedMemorySize, b))) return e;
    if ((e = cudaFuncSetAttribute(k_pool_big, cudaFuncAttributeMaxDynamicSharedMemorySize, b))) return e;
    if ((e = cudaFuncSetAttribute(k_pool_bits, cudaFuncAttributeMaxDynamicSharedMemorySize, b))) return e;
    if ((e = cudaFuncSetAttribute(k_plain, cudaFuncAttributeMaxDynamicSharedMemorySize, b))) return e;
    return set_ci_smem(b);
}

int pool_blocks_per_sm(int cls, size_t smem_bytes)
{
    int nb = 0;
    if (cls == kClassBits)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_pool_bits, kTestThreads, smem_bytes);
    else if (cls == kClassWarp)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_pool_small, kTestThreads, smem_bytes);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_pool_big, kTestThreads, smem_bytes);
    return nb;
}

}  // namespace fbn
