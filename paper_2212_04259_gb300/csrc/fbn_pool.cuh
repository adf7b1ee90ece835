// fbn_pool.cuh -- device code of the per-depth CI-level work pool (Section
// IV-B) and of the edge-level form (Section IV-A): per-group state, the set-up
// of one conditioning set (Section IV-C), counting, the bounded decision,
// sample-split tests and the pool loop.  Each pool kernel is defined in its
// own translation unit (fbn_pool_small.cu, fbn_pool_bits.cu, fbn_pool_big.cu,
// fbn_plain.cu), so that they compile in parallel.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "fbn_depth.cuh"

namespace fbn {

// --------------------------------------------------------------------------
// Per-group state of a worker, in shared memory.
struct GroupState {
    long long r0, r1;
    unsigned long long tests;
    unsigned long long popc_work, smem_updates;   // counting work done, flushed with tests
    unsigned long long item;   // split tests: the test's item and this group's part
    int part;
    unsigned ticket;
    int e;
    int go;
    double crit;       // exact critical value, 0 until the exact decision needs it
    float crit_lo, crit_hi;
    int pos[kMaxD];
};

// Fill the test of rank rk of edge w into the group's TestSpec.  Rank 0 of
// the group computes the subset positions (unranked when `fresh`, else the
// successor of the previous rank of the same side); one thread per
// conditioning variable then resolves its row.  Returns false (uniformly)
// when the table is over the cell limit.
template <int G, bool BITS>
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
        if (BITS) spec.pstride = P.plane_ld >> 2;
    }
    Grp<G>::sync();
    if (r < d + 2) {
        int v;
        if (r < d) {
            const int t = S.pos[r];
            v = P.nbr[(long long)a * P.n + (t < posb ? t : t + 1)];
        } else {
            v = r == d ? w.i : w.j;
            if (r == d) spec.rx = P.ar[v]; else spec.ry = P.ar[v];
        }
        spec.rows[r] = P.data + (long long)v * P.ld;
        spec.rad[r] = P.ar[v];
        if (BITS && r < kBitsMaxD + 2) spec.prow[r] = reinterpret_cast<const uint4*>(P.planes + (long long)v * 2 * P.plane_ld);
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

// The decision of a counted test from its table and marginals: df from the
// declared arities or from the observed table (no degree of freedom left:
// the test cannot reject), crit from the cache, then the bounded statistic.
template <int G>
__device__ __forceinline__ int decide_test(const PoolArgs& a, const TestSpec& spec, const int* T, const int* M,
                                           GroupState& S, double* red, unsigned* status)
{
    const int nz = (int)spec.cells / (spec.rx * spec.ry);   // cells <= kMaxCells < 2^31: 32-bit
    const long long df = a.df_mode ? grp_df_adjusted<G>(spec, M, red)
                                   : (long long)((spec.rx - 1) * (spec.ry - 1)) * nz;
    if (Grp<G>::rank() == 0) {
        // the float bracket of crit when the table has it; else the exact
        // value (computed and stored on first use) and its bracket
        float2 f = make_float2(0.0f, 0.0f);
        if (df > 0 && df < a.crit.dense_n) f = a.crit.dense_f[df];
        S.crit = 0.0;
        if (df > 0 && !(f.y > 0.0f)) {
            const double c = crit_get(a.crit, df, a.alpha, status);
            S.crit = c;
            f = make_float2(__double2float_rd(c), __double2float_ru(c));
        }
        S.crit_lo = f.x;
        S.crit_hi = f.y;
        S.tests += 1;   // flushed to the depth counter when the group leaves the pool
    }
    Grp<G>::sync();
    if (df <= 0) return 1;   // p = 1 > alpha
    const int dec = grp_decide_bound<G>(spec, T, M, S.crit_lo, S.crit_hi, red, a.stat);
    if (dec >= 0) return dec;
    // the band straddles crit: exact FP64 statistic against the exact value
    if (Grp<G>::rank() == 0 && S.crit == 0.0) S.crit = crit_get(a.crit, df, a.alpha, status);
    Grp<G>::sync();
    const double ex = a.stat == kStatX2 ? grp_x2_exact<G>(spec, T, M, red, nullptr) : grp_g2_exact<G>(spec, T, M, red, nullptr);
    return ex < S.crit ? 1 : 0;
}

// Run one rank: 1 = accepts independence, 0 = rejects, -1 = could not run.
// Counting work of one table (rank 0): C popcounts per 32-sample word from
// bit planes, or one shared-memory update per sample by histogram.
template <int G, bool BITS>
__device__ __forceinline__ void note_work(GroupState& S, const TestSpec& spec)
{
    if (Grp<G>::rank() != 0) return;
    if (BITS) S.popc_work += (unsigned long long)spec.cells * (unsigned long long)((spec.N + 31) >> 5);
    else S.smem_updates += (unsigned long long)spec.N;
}

template <int G, bool BITS>
__device__ __forceinline__ int run_rank(const PoolArgs& a, int d, const ProblemDev& P, const EdgeWork& w, long long rk,
                                        bool fresh, GroupState& S, TestSpec& spec, int* slice, long long slice_ints,
                                        int* gtab, double* red)
{
    unsigned* status = &a.ctr->status;
    if (!setup_rank<G, BITS>(P, w, d, rk, fresh, S, a.binom, spec, status)) return -1;
    int* M = nullptr;
    const int* T = grp_table<G, BITS>(spec, slice, slice_ints, gtab, a.gscratch_ints, &M);
    if (!T) {   // the global scratch is too small: the host grows it and starts over
        if (Grp<G>::rank() == 0) {
            atomicOr(status, kStatusScratch);
            atomicMax(&a.ctr->need_cells, (int)spec.cells);
        }
        return -1;
    }
    note_work<G, BITS>(S, spec);
    grp_marginals<G>(spec, T, M);
    return decide_test<G>(a, spec, T, M, S, red, status);
}

// One rank of a bit-plane test on a warp group, finished in registers.  After
// the count, row k of the slice holds counter word k of every lane (the
// bits_word_of layout: cells (z, x, y) and (z, x, y + 1) with z = k / 8,
// x = (k / 2) mod 4, y = 2 (k mod 2)), so lane l folds row l with 128-bit
// loads (rotated by the lane: each quarter-warp phase touches all 32 banks
// once) and ends with the two cells of word l.  Lanes that share z and x, or
// z and y, differ only in the bits of the other coordinate: the marginals are
// shuffles, and every cell's coordinates are the lane's bits (no division).
// Cells outside the table hold zero (values >= an arity never occur; strata
// >= r_z are not counted).  The FP32 terms and the bound are those of
// grp_decide_bound with two terms per thread; without the float bracket of
// crit, with the observed-table df, or when the band straddles crit, the
// table and marginals go to shared memory in the layout of the other paths
// and decide_test decides.
//
// The edge's lowest accepting rank is read before the set-up and checked
// after it (the load's latency hides behind the set-up): returns 2, nothing
// counted, when rk is above it.
__device__ __forceinline__ int run_rank_bits(const PoolArgs& a, int d, const ProblemDev& P, const EdgeWork& w,
                                             long long rk, bool fresh, GroupState& S, TestSpec& spec, int* slice,
                                             double* red, const unsigned long long* min_accept_e)
{
    unsigned* status = &a.ctr->status;
    unsigned long long ma = 0ULL;
    if ((threadIdx.x & 31) == 0) ma = *((volatile const unsigned long long*)min_accept_e);
    __syncwarp();   // the previous rank's readers of spec and S are done
    if (!setup_rank<32, true>(P, w, d, rk, fresh, S, a.binom, spec, status)) return -1;
    if ((unsigned long long)rk > __shfl_sync(0xffffffffu, ma, 0)) return 2;
    count_bits<32>(spec, slice + (threadIdx.x & 31));
    __syncwarp();
    // the shape is read back from shared memory: nothing of it stays live
    // across the call
    const int lane = threadIdx.x & 31;
    const int rx = spec.rx, ry = spec.ry, N = spec.N;
    const int rz = d ? spec.rad[0] : 1;
    const int df = (rx - 1) * (ry - 1) * rz;   // declared arities: >= 1
    const bool fast = a.df_mode == 0 && df < a.crit.dense_n;
    // the bracket is read by lane 0 and broadcast: another warp may be
    // storing it right now, and every lane must take the same branch below
    // (the branches end in full-warp shuffles)
    float2 f = make_float2(0.0f, 0.0f);
    if (fast && lane == 0) f = a.crit.dense_f[df];   // in flight during the fold
    const int z = lane >> 3, x = (lane >> 1) & 3, y = (lane & 1) * 2;
    unsigned lo = 0u, hi = 0u;
    if (z < rz) {
        const uint4* row = reinterpret_cast<const uint4*>(slice + lane * 32);   // 32 lane columns, 8 uint4
        if (N < 65536) {   // each half of the sum counts one cell (<= N): packed adds cannot carry
            unsigned s2 = 0u;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const uint4 v = row[(q + lane) & 7];
                s2 += v.x + v.y + v.z + v.w;
            }
            lo = s2 & 0xFFFFu;
            hi = s2 >> 16;
        } else {
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const uint4 v = row[(q + lane) & 7];
                lo += (v.x & 0xFFFFu) + (v.y & 0xFFFFu) + (v.z & 0xFFFFu) + (v.w & 0xFFFFu);
                hi += (v.x >> 16) + (v.y >> 16) + (v.z >> 16) + (v.w >> 16);
            }
        }
    }
    // N_x+z over y (lane bit 0), N_+yz over x (bits 1, 2), N_++z over x
    const unsigned nxz = lo + hi + __shfl_xor_sync(0xffffffffu, lo + hi, 1);
    unsigned nylo = lo + __shfl_xor_sync(0xffffffffu, lo, 2);
    unsigned nyhi = hi + __shfl_xor_sync(0xffffffffu, hi, 2);
    unsigned nzz = nxz + __shfl_xor_sync(0xffffffffu, nxz, 2);
    nylo += __shfl_xor_sync(0xffffffffu, nylo, 4);
    nyhi += __shfl_xor_sync(0xffffffffu, nyhi, 4);
    nzz += __shfl_xor_sync(0xffffffffu, nzz, 4);
    if (lane == 0) S.popc_work += (unsigned long long)spec.cells * (unsigned long long)((N + 31) >> 5);
    f.x = __shfl_sync(0xffffffffu, f.x, 0);
    f.y = __shfl_sync(0xffffffffu, f.y, 0);
    if (fast && f.y > 0.0f) {
        float acc = 0.0f, mag = 0.0f;
        if (a.stat == kStatX2) {
            x2_term((int)lo, (int)nzz, (int)nxz, (int)nylo, acc);
            x2_term((int)hi, (int)nzz, (int)nxz, (int)nyhi, acc);
            mag = acc;
        } else {
            if (lo) g2_term((int)lo, (int)nzz, (int)nxz, (int)nylo, acc, mag);
            if (hi) g2_term((int)hi, (int)nzz, (int)nxz, (int)nyhi, acc, mag);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            acc += __shfl_xor_sync(0xffffffffu, acc, o);
            mag += __shfl_xor_sync(0xffffffffu, mag, o);
        }
        const int dec = __shfl_sync(0xffffffffu, decide_from_sums(acc, mag, 2.0f, 5.0f, a.stat, f.x, f.y), 0);
        if (dec >= 0) {
            if (lane == 0) S.tests += 1;   // flushed to the depth counter when the group leaves the pool
            return dec;
        }
    }
    // shared-memory layout of the other paths: T[(z r_x + x) r_y + y], marginals after it
    int* T = slice + kBitsWords * 32;
    if (z < rz && x < rx) {
        const int c = (z * rx + x) * ry + y;
        if (y < ry) T[c] = (int)lo;
        if (y + 1 < ry) T[c + 1] = (int)hi;
    }
    __syncwarp();
    int* M = T + spec.cells;
    grp_marginals<32>(spec, T, M);
    return decide_test<32>(a, spec, T, M, S, red, status);
}

// One part of a split test: count samples [N p / S, N (p + 1) / S) (16-aligned
// bounds) of rank rk into the test's global table; the part that finishes last
// copies the table into shared memory (L2 reads), zeroes it, decides and
// lowers the edge's rank.  Returns 1 when this group decided an acceptance.
template <int G, bool BITS>
__device__ __noinline__ int run_split_part(const PoolArgs& a, int d, const ProblemDev& P, const EdgeWork& w,
                                              long long rk, int split, GroupState& S, TestSpec& spec, int* slice,
                                              long long slice_ints, int* gtab, double* red,
                                              const unsigned long long* min_accept_e)
{
    unsigned* status = &a.ctr->status;
    const int r = Grp<G>::rank();
    int* Tg = a.split_tab + (long long)S.item * a.split_stride;
    if (r == 0) S.go = (unsigned long long)rk <= *((volatile const unsigned long long*)min_accept_e);
    Grp<G>::sync();
    bool ready = false;   // spec holds this rank's table shape (uniform over the group)
    if (S.go && setup_rank<G, BITS>(P, w, d, rk, true, S, a.binom, spec, status)) {
        ready = true;
        const long long N = P.N;
        // part bounds on 128-sample boundaries: whole 16-byte vectors of the
        // byte rows and whole uint4 groups of the bit planes
        const long long lo = (N * S.part / split) & ~127LL;
        const long long hi = S.part == split - 1 ? N : ((N * (S.part + 1) / split) & ~127LL);
        if (r < d + 2) {
            spec.rows[r] += lo;
            if (BITS && r < kBitsMaxD + 2) spec.prow[r] += lo >> 7;
        }
        Grp<G>::sync();
        if (r == 0) spec.N = (int)(hi - lo);
        Grp<G>::sync();
        int* M = nullptr;
        const int* T = grp_table<G, BITS>(spec, slice, slice_ints, gtab, a.gscratch_ints, &M);
        if (!T) {
            if (r == 0) {
                atomicOr(status, kStatusScratch);
                atomicMax(&a.ctr->need_cells, (int)spec.cells);
            }
        } else {
            note_work<G, BITS>(S, spec);
            for (long long c = r; c < spec.cells; c += G)
                if (T[c]) atomicAdd(Tg + c, T[c]);
        }
    }
    __threadfence();
    Grp<G>::sync();
    if (r == 0) S.ticket = atomicAdd(&a.split_ticket[S.item], 1u);
    Grp<G>::sync();
    if (S.ticket != (unsigned)(split - 1)) return 0;
    // the last part: every other part's adds are in L2; the decision needs
    // the table's shape only (cells, radices), which this part's own setup
    // left in spec when it counted
    __threadfence();
    if (!ready && !setup_rank<G, BITS>(P, w, d, rk, true, S, a.binom, spec, status)) return 0;
    const long long C = spec.cells;
    int* Tl = slice;
    for (long long c = r; c < C; c += G) {
        Tl[c] = __ldcg(Tg + c);
        Tg[c] = 0;
    }
    if (r == 0) {
        a.split_ticket[S.item] = 0;
        S.go = (unsigned long long)rk <= *((volatile const unsigned long long*)min_accept_e);
    }
    Grp<G>::sync();
    if (!S.go) return 0;
    int* M = Tl + C;
    grp_marginals<G>(spec, Tl, M);
    return decide_test<G>(a, spec, Tl, M, S, red, status);
}

// Shared state of a pool CTA, sized for the most groups per CTA (8 warps).
struct PoolShared {
    TestSpec spec[kTestThreads / 32];
    GroupState st[kTestThreads / 32];
    double red[32];
    unsigned long long base[kBaseSmem];
};

template <int G, bool BITS = false>
__device__ __forceinline__ void pool_body(const PoolArgs& a, int* smem, PoolShared& sh)
{
    constexpr int NG = kTestThreads / G;   // groups per CTA
    const DepthCounters* ctr = a.ctr;
    const int d = ctr->d;
    const long long maxc = (long long)ctr->maxc[a.cls];
    const unsigned long long total = ctr->total_items[a.cls];
    if (total == 0) return;
    const long long cb = class_base(ctr, a.cls, a.edge_cap);
    const EdgeWork* edges = a.edges + cb;
    unsigned long long* min_accept = a.min_accept + cb;
    unsigned long long* next_item = &a.ctr->next_item[a.cls];
    const int gs = ctr->gs;
    const int g = Grp<G>::gid();
    const int r = Grp<G>::rank();
    const long long slice_ints = a.smem_ints / NG;
    int* slice = smem + g * slice_ints;
    int* gtab = a.gscratch ? a.gscratch + ((long long)blockIdx.x * NG + g) * a.gscratch_ints : nullptr;
    const bool base_in_smem = maxc + 1 <= kBaseSmem;
    if (base_in_smem)
        for (long long k = threadIdx.x; k <= maxc; k += blockDim.x) sh.base[k] = a.base[k];
    __syncthreads();
    const unsigned long long* base = base_in_smem ? sh.base : a.base;
    GroupState& S = sh.st[g];
    TestSpec& spec = sh.spec[g];
    if (r == 0) S.tests = S.popc_work = S.smem_updates = 0;
    const int split = ctr->split[a.cls] > 1 ? ctr->split[a.cls] : 1;

    for (;;) {
        if (r == 0) {
            const unsigned long long wi = atomicAdd(next_item, 1ULL);
            const unsigned long long w = split == 1 ? wi : wi / (unsigned long long)split;
            S.item = w;
            S.part = (int)(wi - w * (unsigned long long)split);
            S.e = -1;
            if (wi < total) {
                long long lo = 0, hi = maxc - 1;   // pass k: largest k with base[k] <= w
                while (lo < hi) {
                    const long long mid = (lo + hi + 1) >> 1;
                    if (base[mid] <= w) lo = mid; else hi = mid - 1;
                }
                const int e = a.sorted[cb + (long long)(w - base[lo])];
                const long long tot = edges[e].total;
                const long long cr = chunk_ranks(tot, gs);
                const long long r0 = lo * cr;
                S.e = e;
                S.r0 = r0;
                S.r1 = r0 + cr < tot ? r0 + cr : tot;
            }
        }
        Grp<G>::sync();
        const int e = S.e;
        if (e < 0) break;
        const EdgeWork w = edges[e];
        const ProblemDev& P = a.probs[w.prob];
        const long long r0 = S.r0, r1 = S.r1;
        if (split > 1) {   // single-rank items (gs = 1, no edge above kMaxPasses ranks)
            const int res = run_split_part<G, BITS>(a, d, P, w, r0, split, S, spec, slice, slice_ints, gtab, sh.red,
                                                    &min_accept[e]);
            if (res == 1 && r == 0) atomicMin(&min_accept[e], (unsigned long long)r0);
            Grp<G>::sync();
            continue;
        }
        for (long long rk = r0; rk < r1; ++rk) {
            int res;
            if constexpr (BITS) {   // checks the edge's rank itself (res = 2: above it)
                static_assert(G == 32, "the bit-plane pool runs warp groups");
                res = run_rank_bits(a, d, P, w, rk, rk == r0, S, spec, slice, sh.red, &min_accept[e]);
            } else {
                if (r == 0) S.go = (unsigned long long)rk <= *((volatile unsigned long long*)&min_accept[e]);
                Grp<G>::sync();
                if (!S.go) break;
                res = run_rank<G, BITS>(a, d, P, w, rk, rk == r0, S, spec, slice, slice_ints, gtab, sh.red);
            }
            if (res == 1 && r == 0) atomicMin(&min_accept[e], (unsigned long long)rk);
            if (res != 0) break;
        }
        Grp<G>::sync();
    }
    if (r == 0 && S.tests) atomicAdd(&a.ctr->tests, S.tests);
    if (r == 0 && S.popc_work) atomicAdd(&a.ctr->popc_work, S.popc_work);
    if (r == 0 && S.smem_updates) atomicAdd(&a.ctr->smem_updates, S.smem_updates);
}

// The end of a test CTA in the depth's record (the latest over CTAs).
__device__ __forceinline__ void tests_done(const DepthCounters* ctr)
{
    __syncthreads();
    if (threadIdx.x == 0)
        if (DepthRecord* r = depth_rec(ctr, ctr->d)) atomicMax(&r->t_tests_end, gtime());
}

}  // namespace fbn
