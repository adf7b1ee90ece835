// fbn_gram.cu -- depth 0 of Algorithm 1 as a one-hot Gram product on the
// fifth-generation tensor cores of sm_103a (tcgen05), all pairs at once.
//
// For every variable v and value x let e_{v,x} in {0,1}^N mark the samples
// with V_v = x.  The depth-0 contingency table of the pair (i, j) is
// N_ij(x, y) = <e_{i,x}, e_{j,y}>, so all n(n-1)/2 tables (Section IV-B: depth
// zero tests every pair of the complete graph once) are blocks of the Gram
// matrix E E^T of the one-hot matrix E [sum_v r_v][N].
//
// E is built in HBM as FP8 E4M3 (0 and 1 are exact).  The product runs on
// tcgen05.mma.kind::f8f6f4 with FP32 accumulators in tensor memory; every
// accumulation covers at most kChunk = 8192 samples, so each partial sum is an
// integer below 2^13 and exact even if the accumulation kept only 14
// significant bits.  Each chunk's 128x256 tile is added into an INT32 Gram in
// global memory.  (tcgen05.mma.kind::i8 does not assemble for sm_103a with this
// toolkit, hence FP8 0/1 operands.)
//
// A tile is 128 rows of E against 256 rows (M = 128, N = 256 per MMA): each
// 128-sample stage brings 48 KB of operands for 8 MFLOP, a third less operand
// traffic per FLOP than square 128-row tiles.  Work unit = (128-row tile,
// 256-row tile reaching the upper triangle, chunk of samples), chunk-major so
// that the CTAs of a wave stream the same sample range and share it in L2.
// CTA roles: warps 0-3 epilogue (TMEM -> registers -> coalesced INT32 atomic
// adds), warp 4 TMA producer, warp 5 MMA issuer and TMEM owner.
#include <algorithm>
#include <cstdint>

#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include "fbn_device.cuh"
#include "fbn_gram.h"
#include "fbn_tc.cuh"

namespace fbn {
namespace {

using namespace tc;

constexpr int kTile = 128;                           // rows of an A tile = M of one MMA
constexpr int kTileN = 256;                          // rows of a B tile = N of one MMA
constexpr int kKSlice = 128;                         // samples (bytes) per pipeline stage
constexpr int kChunk = 8192;                         // samples per exact accumulation
constexpr int kSlicesPerChunk = kChunk / kKSlice;
constexpr int kStages = 4;
constexpr int kTileBytes = kTile * kKSlice;          // 16 KB
constexpr int kStageBytes = 3 * kTileBytes;          // A + the two 128-row halves of B
constexpr int kGramThreads = 192;
constexpr uint32_t kTmemCols = 512;                  // two 256-column FP32 accumulators
constexpr int kStagePad = 33;                        // epilogue transpose tile row (ints)
constexpr size_t kGramSmem = 1024 /*align*/ + (size_t)kStages * kStageBytes + 4 * 32 * kStagePad * 4 + 256;

constexpr uint32_t kIdesc = tc::idesc_f8(kTile, kTileN);

// Work unit of the Gram: problem, 128-row tile ti, 256-row tile tj covering
// some column >= some row (tj >= ti / 2), chunk of samples.
struct GramArgs {
    const CUtensorMap* maps;    // [problems] tensor maps of the one-hot matrices (global memory)
    const int4* units;          // [n_units] (problem, ti, tj, chunk)
    const ProblemDev* probs;
    int n_units;
    unsigned* status;
    unsigned limit;             // attempts of each role's bounded wait
};

__global__ void __launch_bounds__(kGramThreads, 1) k_gram(GramArgs g)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    int* xpose = reinterpret_cast<int*>(smem + (size_t)kStages * kStageBytes);          // 4 x 32 x 33 ints
    uint64_t* bars = reinterpret_cast<uint64_t*>(xpose + 4 * 32 * kStagePad);
    uint64_t* full = bars;                 // [kStages] TMA -> MMA
    uint64_t* empty = bars + kStages;      // [kStages] MMA -> TMA
    uint64_t* acc_full = bars + 2 * kStages;       // [2] MMA -> epilogue
    uint64_t* acc_empty = bars + 2 * kStages + 2;  // [2] epilogue -> MMA
    uint64_t* drain = bars + 2 * kStages + 4;      // MMA completion before teardown
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * kStages + 5);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    int* issued = reinterpret_cast<int*>(tmem_slot + 2);   // [kStages], producer thread only

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int U = g.n_units;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(smem_u32(&full[s]), 1);
            mbar_init(smem_u32(&empty[s]), 1);
            issued[s] = 0;
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&acc_full[b]), 1);
            mbar_init(smem_u32(&acc_empty[b]), 4);   // one arrive per epilogue warp
        }
        mbar_init(smem_u32(drain), 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 5) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 4) {
        // ---------------- TMA producer
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            int fenced = -1;
            for (int u = blockIdx.x; u < U && !*abort_flag; u += gridDim.x) {
                const int4 t = g.units[u];
                const CUtensorMap* map = g.maps + t.x;
                if (t.x != fenced) {   // the host rewrites the maps between launches
                    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(map) : "memory");
                    fenced = t.x;
                }
                const int slices = (int)(g.probs[t.x].onehot_ld / kKSlice);
                const int kb0 = t.w * kSlicesPerChunk;
                const int kb1 = min(kb0 + kSlicesPerChunk, slices);
                for (int kb = kb0; kb < kb1; ++kb) {
                    if (!mbar_wait(smem_u32(&empty[stage]), phase ^ 1u, abort_flag, g.status, g.limit)) break;
                    const uint32_t fb = smem_u32(&full[stage]);
                    const uint32_t a = smem_u32(smem + (size_t)stage * kStageBytes);
                    mbar_expect_tx(fb, kStageBytes);
                    tma_load_2d(a, map, fb, kb * kKSlice, t.y * kTile);
                    // B: rows beyond the padded matrix (odd tile count) come back as zeros
                    tma_load_2d(a + kTileBytes, map, fb, kb * kKSlice, t.z * kTileN);
                    tma_load_2d(a + 2 * kTileBytes, map, fb, kb * kKSlice, t.z * kTileN + kTile);
                    issued[stage] += 1;
                    if (++stage == kStages) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
        }
    } else if (warp == 5) {
        // ---------------- MMA issuer (one thread)
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            int acc = 0;
            uint32_t acc_phase = 0;
            bool ok = true;
            for (int u = blockIdx.x; u < U && ok; u += gridDim.x) {
                const int4 t = g.units[u];
                const int slices = (int)(g.probs[t.x].onehot_ld / kKSlice);
                const int kb0 = t.w * kSlicesPerChunk;
                const int kb1 = min(kb0 + kSlicesPerChunk, slices);
                if (!mbar_wait(smem_u32(&acc_empty[acc]), acc_phase ^ 1u, abort_flag, g.status, g.limit)) break;
                tc_fence_after();
                const uint32_t d_tmem = tmem + (uint32_t)(acc * kTileN);
                for (int kb = kb0; kb < kb1; ++kb) {
                    if (!mbar_wait(smem_u32(&full[stage]), phase, abort_flag, g.status, g.limit)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t a = smem_u32(smem + (size_t)stage * kStageBytes);
                    const uint64_t da = smem_desc(a), db = smem_desc(a + kTileBytes);
#pragma unroll
                    for (int k = 0; k < kKSlice / 32; ++k)   // 32 E4M3 values = 32 bytes of K per MMA
                        mma_f8(d_tmem, da + (uint64_t)(2 * k), db + (uint64_t)(2 * k), kIdesc, (kb > kb0 || k > 0) ? 1u : 0u);
                    mma_commit(smem_u32(&empty[stage]));
                    if (++stage == kStages) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
                if (!ok) break;
                mma_commit(smem_u32(&acc_full[acc]));
                acc ^= 1;
                if (acc == 0) acc_phase ^= 1u;
            }
            // every MMA this thread issued has finished before TMEM is released
            // (the default bound here, whatever the roles' bound)
            mma_commit(smem_u32(drain));
            for (unsigned it = 0; it < kSpinLimit; ++it)
                if (mbar_try(smem_u32(drain), 0)) break;
        }
    } else {
        // ---------------- epilogue: warps 0-3, TMEM lanes 32w .. 32w+31
        int* xp = xpose + warp * 32 * kStagePad;
        int acc = 0;
        uint32_t acc_phase = 0;
        for (int u = blockIdx.x; u < U; u += gridDim.x) {
            const int4 t = g.units[u];
            int32_t* G = g.probs[t.x].gram;
            const long long ldg = g.probs[t.x].gram_ld;
            if (!mbar_wait(smem_u32(&acc_full[acc]), acc_phase, abort_flag, g.status, g.limit)) break;
            tc_fence_after();
            const uint32_t base = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(acc * kTileN);
            const long long row0 = (long long)t.y * kTile + warp * 32;
            for (int j0 = 0; j0 < kTileN; j0 += 32) {
                if ((long long)t.z * kTileN + j0 >= ldg) break;   // columns past the padded matrix
                uint32_t v[32];
                tmem_ld32(base + (uint32_t)j0, v);
#pragma unroll
                for (int q = 0; q < 32; ++q) xp[lane * kStagePad + q] = __float2int_rn(__uint_as_float(v[q]));
                __syncwarp();
                int32_t* dst = G + row0 * ldg + (long long)t.z * kTileN + j0 + lane;
#pragma unroll 4
                for (int r = 0; r < 32; ++r) {
                    const int val = xp[r * kStagePad + lane];
                    if (val) atomicAdd(dst + (long long)r * ldg, val);
                }
                __syncwarp();
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&acc_empty[acc]));
            acc ^= 1;
            if (acc == 0) acc_phase ^= 1u;
        }
    }

    __syncthreads();
    if (warp == 4 && lane == 0) {
        // no TMA write may land after the CTA exits: wait for the last load of
        // every stage (immediate unless a role gave up)
        for (int s = 0; s < kStages; ++s)
            if (issued[s] > 0) {
                for (unsigned it = 0; it < kSpinLimit; ++it)
                    if (mbar_try(smem_u32(&full[s]), (uint32_t)((issued[s] - 1) & 1))) break;
            }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 5) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
}

// One-hot matrix E of every problem: row off_v + x holds 0x38 (E4M3 1.0)
// where V_v = x, else 0; samples at or beyond N (the padding of the store)
// are 0 for every row.  One CTA per variable of the batch.
__global__ void k_onehot(const ProblemDev* __restrict__ probs, const int32_t* __restrict__ vtx_prob,
                         const int32_t* __restrict__ vtx_first, int total_vertices)
{
    const int g = blockIdx.x;
    if (g >= total_vertices) return;
    const int p = vtx_prob[g];
    const ProblemDev& P = probs[p];
    const int v = g - vtx_first[p];
    const int r = P.ar[v];
    const long long K = P.onehot_ld;
    const int N = P.N;
    const uint4* row = reinterpret_cast<const uint4*>(P.data + (long long)v * P.ld);
    uint8_t* E = P.onehot + (long long)P.off[v] * K;
    const long long nvec = K / 16;
    for (long long q = threadIdx.x; q < nvec; q += blockDim.x) {
        uint4 w = row[q];
        const long long s0 = q * 16;
        uint32_t keep[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {   // byte mask of samples below N
            uint32_t m = 0;
#pragma unroll
            for (int b = 0; b < 4; ++b)
                if (s0 + 4 * k + b < N) m |= 0xFFu << (8 * b);
            keep[k] = m;
        }
        for (int x = 0; x < r; ++x) {
            const uint32_t rep = 0x01010101u * (uint32_t)x;
            uint4 o;
            o.x = __vcmpeq4(w.x, rep) & 0x38383838u & keep[0];
            o.y = __vcmpeq4(w.y, rep) & 0x38383838u & keep[1];
            o.z = __vcmpeq4(w.z, rep) & 0x38383838u & keep[2];
            o.w = __vcmpeq4(w.w, rep) & 0x38383838u & keep[3];
            reinterpret_cast<uint4*>(E + (long long)x * K)[q] = o;
        }
    }
}

// Critical values of df <= kCritLocal, cached per CTA in shared memory (NaN
// until first asked): the pairs of a depth share a handful of df, and the
// global cache's acquire loads would serialise on those few slots.
constexpr int kCritLocal = 64;

__device__ __forceinline__ double crit_local(double* local, const CritTableDev& crit, long long df, double alpha,
                                             unsigned* status)
{
    if (df > kCritLocal) return crit_get(crit, df, alpha, status);
    double c = *((volatile double*)&local[df]);
    if (c != c) {   // not cached yet: every thread that misses stores the same value
        c = crit_get(crit, df, alpha, status);
        *((volatile double*)&local[df]) = c;
    }
    return c;
}

// Decision of one depth-0 pair from its block of the Gram (row sums, column
// sums and the total from the block itself).  R bounds the arities so that
// the sums live in registers.  stat: G^2 or Pearson X^2; df_mode: declared
// arities or the observed table (no degree of freedom left: accept).
template <int R>
__device__ __forceinline__ void pair_decide_r(const int32_t* T, long long Mp, int rx, int ry, long long e,
                                              unsigned long long* __restrict__ min_accept, const CritTableDev& crit,
                                              double alpha, DepthCounters* ctr, int stat, int df_mode, double* local)
{
    int rs[R], cs[R];
    int tot = 0;
#pragma unroll
    for (int q = 0; q < R; ++q) rs[q] = cs[q] = 0;
#pragma unroll
    for (int x = 0; x < R; ++x)
#pragma unroll
        for (int y = 0; y < R; ++y)
            if (x < rx && y < ry) {
                const int nxy = T[(long long)x * Mp + y];
                rs[x] += nxy;
                cs[y] += nxy;
                tot += nxy;
            }
    long long df = (long long)(rx - 1) * (ry - 1);
    if (df_mode) {
        int ax = 0, ay = 0;
#pragma unroll
        for (int q = 0; q < R; ++q) {
            ax += rs[q] > 0;
            ay += cs[q] > 0;
        }
        df = ax > 0 && ay > 0 ? (long long)(ax - 1) * (ay - 1) : 0;
    }
    if (df <= 0) {   // p = 1 > alpha
        min_accept[e] = 0;
        return;
    }
    // terms in FP32 (G^2: within 3.2e-7 of their magnitude; X^2: within 6e-7),
    // summed in FP32 by this thread (at most R*R additions, each within 6e-8 of
    // the running sum of magnitudes); exact FP64 only when crit lies inside the
    // error band
    const double c = crit_local(local, crit, df, alpha, &ctr->status);
    float acc = 0.0f, mag = 0.0f;
#pragma unroll
    for (int x = 0; x < R; ++x)
#pragma unroll
        for (int y = 0; y < R; ++y) {
            if (x >= rx || y >= ry) continue;
            const int n = T[(long long)x * Mp + y];
            if (stat == kStatX2) {
                if (rs[x] == 0 || cs[y] == 0) continue;
                const float fd = (float)((long long)n * tot - (long long)rs[x] * cs[y]);
                const float t = fd * fd / ((float)tot * (float)rs[x] * (float)cs[y]);
                acc += t;
                mag += t;
            } else {
                if (n == 0) continue;
                const long long a = (long long)n * tot, b = (long long)rs[x] * cs[y];
                const float fb = (float)b;
                const float delta = (float)(a - b) / fb;
                const float L = fabsf(delta) < 0.5f ? log1pf(delta) : logf((float)a / fb);
                const float t = (float)n * L;
                acc += t;
                mag += fabsf(t);
            }
        }
    const double scale = stat == kStatX2 ? 1.0 : 2.0;
    const double st = scale * (double)acc;
    const double rel = 2.0 * ((stat == kStatX2 ? 6e-7 : 3.2e-7) + (double)(rx * ry) * 6e-8);
    const double err = scale * rel * (double)mag * 1.0001 + 1e-9;
    bool accept;
    if (st + err < c) {
        accept = true;
    } else if (st - err >= c) {
        accept = false;
    } else {
        double ex = 0.0;
#pragma unroll
        for (int x = 0; x < R; ++x)
#pragma unroll
            for (int y = 0; y < R; ++y) {
                if (x >= rx || y >= ry) continue;
                const int n = T[(long long)x * Mp + y];
                if (stat == kStatX2) {
                    if (rs[x] == 0 || cs[y] == 0) continue;
                    const double dd = (double)((long long)n * tot - (long long)rs[x] * cs[y]);
                    ex += dd * dd / ((double)tot * (double)rs[x] * (double)cs[y]);
                } else {
                    if (n == 0) continue;
                    const long long a = (long long)n * tot, b = (long long)rs[x] * cs[y];
                    ex += (double)n * log1p((double)(a - b) / (double)b);
                }
            }
        accept = scale * ex < c;
    }
    if (accept) min_accept[e] = 0;
}

// Arities above 8: the sums are recomputed from the block (no local arrays),
// the statistic in FP64.
__device__ __forceinline__ void pair_decide_wide(const int32_t* T, long long Mp, int rx, int ry, long long e,
                                                 unsigned long long* __restrict__ min_accept, const CritTableDev& crit,
                                                 double alpha, DepthCounters* ctr, int stat, int df_mode, double* local)
{
    long long tot = 0;
    for (int x = 0; x < rx; ++x)
        for (int y = 0; y < ry; ++y) tot += T[(long long)x * Mp + y];
    long long df = (long long)(rx - 1) * (ry - 1);
    if (df_mode) {
        int ax = 0, ay = 0;
        for (int x = 0; x < rx; ++x) {
            long long s = 0;
            for (int y = 0; y < ry; ++y) s += T[(long long)x * Mp + y];
            ax += s > 0;
        }
        for (int y = 0; y < ry; ++y) {
            long long s = 0;
            for (int x = 0; x < rx; ++x) s += T[(long long)x * Mp + y];
            ay += s > 0;
        }
        df = ax > 0 && ay > 0 ? (long long)(ax - 1) * (ay - 1) : 0;
    }
    if (df <= 0) {
        min_accept[e] = 0;
        return;
    }
    const double c = crit_local(local, crit, df, alpha, &ctr->status);
    double ex = 0.0;
    for (int x = 0; x < rx; ++x) {
        long long rsx = 0;
        for (int y = 0; y < ry; ++y) rsx += T[(long long)x * Mp + y];
        for (int y = 0; y < ry; ++y) {
            const int n = T[(long long)x * Mp + y];
            long long csy = 0;
            for (int xx = 0; xx < rx; ++xx) csy += T[(long long)xx * Mp + y];
            if (stat == kStatX2) {
                if (rsx == 0 || csy == 0) continue;
                const double dd = (double)(n * tot - rsx * csy);
                ex += dd * dd / ((double)tot * (double)rsx * (double)csy);
            } else {
                if (n == 0) continue;
                const long long a = (long long)n * tot, b = rsx * csy;
                ex += (double)n * log1p((double)(a - b) / (double)b);
            }
        }
    }
    if ((stat == kStatX2 ? 1.0 : 2.0) * ex < c) min_accept[e] = 0;
}

__device__ __forceinline__ void pair_decide(const EdgeWork* __restrict__ edges, long long e,
                                            const ProblemDev* __restrict__ probs,
                                            unsigned long long* __restrict__ min_accept, const CritTableDev& crit,
                                            double alpha, DepthCounters* ctr, int stat, int df_mode, double* local)
{
    const EdgeWork w = edges[e];
    const ProblemDev& P = probs[w.prob];
    const int rx = P.ar[w.i], ry = P.ar[w.j];
    const long long Mp = P.gram_ld;
    const int32_t* T = P.gram + (long long)P.off[w.i] * Mp + P.off[w.j];
    if (rx <= 4 && ry <= 4) pair_decide_r<4>(T, Mp, rx, ry, e, min_accept, crit, alpha, ctr, stat, df_mode, local);
    else if (rx <= 8 && ry <= 8) pair_decide_r<8>(T, Mp, rx, ry, e, min_accept, crit, alpha, ctr, stat, df_mode, local);
    else pair_decide_wide(T, Mp, rx, ry, e, min_accept, crit, alpha, ctr, stat, df_mode, local);
}

// Depth-0 decisions from the Gram: one thread per edge (i<j) of both classes
// of the edge list (class 0 at the front of the array, class 1 at the back).
__global__ void k_pairs_decide(const EdgeWork* __restrict__ edges, long long edge_cap,
                               const ProblemDev* __restrict__ probs, unsigned long long* __restrict__ min_accept,
                               CritTableDev crit, double alpha, DepthCounters* ctr, int stat, int df_mode)
{
    __shared__ double local[kCritLocal + 1];
    if (!ctr->active) return;
    for (int k = threadIdx.x; k <= kCritLocal; k += blockDim.x) local[k] = __longlong_as_double(0x7ff8000000000000LL);
    __syncthreads();
    const long long n0 = (long long)ctr->n_edges[0], n1 = (long long)ctr->n_edges[1];
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n0 + n1;
         k += (long long)gridDim.x * blockDim.x)
        pair_decide(edges, k < n0 ? k : edge_cap - n1 + (k - n0), probs, min_accept, crit, alpha, ctr, stat,
                    df_mode, local);
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&ctr->tests, (unsigned long long)(n0 + n1));   // one test per pair
}
// Zero the pad rows M..Mp of every problem's one-hot matrix (one CTA per
// problem); rows below M are rewritten by k_onehot on every call.
__global__ void k_zero_pad(const ProblemDev* __restrict__ probs)
{
    const ProblemDev& P = probs[blockIdx.x];
    const long long M = (long long)P.off[P.n - 1] + P.ar[P.n - 1];
    uint4* E = reinterpret_cast<uint4*>(P.onehot + M * P.onehot_ld);
    const long long n = (P.gram_ld - M) * P.onehot_ld / 16;
    for (long long q = threadIdx.x; q < n; q += blockDim.x) E[q] = make_uint4(0, 0, 0, 0);
}

// Mirror the upper block triangle into the lower one (row < col -> col, row).
__global__ void k_symmetrize(int32_t* G, int Mp, int M)
{
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (long long)M * M) return;
    const int r = (int)(k / M), c = (int)(k - (long long)r * M);
    if (r > c) G[(long long)r * Mp + c] = G[(long long)c * Mp + r];
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

}  // namespace

size_t gram_smem_bytes() { return kGramSmem; }

int gram_rows_padded(int M) { return (M + kTile - 1) / kTile * kTile; }

long long gram_samples_padded(long long N) { return (N + kKSlice - 1) / kKSlice * kKSlice; }

cudaError_t launch_onehot(const ProblemDev* probs, const int32_t* vtx_prob, const int32_t* vtx_first,
                          int total_vertices, cudaStream_t st)
{
    k_onehot<<<total_vertices, 256, 0, st>>>(probs, vtx_prob, vtx_first, total_vertices);
    return cudaGetLastError();
}

cudaError_t launch_zero_pad(const ProblemDev* probs, int nprob, cudaStream_t st)
{
    k_zero_pad<<<nprob, 256, 0, st>>>(probs);
    return cudaGetLastError();
}

cudaError_t encode_onehot_map(void* map, const uint8_t* E, int Mp, long long K)
{
    auto encode = encode_fn();
    if (!encode) return cudaErrorNotSupported;
    cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)Mp};
    cuuint64_t strides[1] = {(cuuint64_t)K};
    cuuint32_t box[2] = {(cuuint32_t)kKSlice, (cuuint32_t)kTile};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = encode(reinterpret_cast<CUtensorMap*>(map), CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<uint8_t*>(E),
                        dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

size_t tensor_map_bytes() { return sizeof(CUtensorMap); }

int gram_chunks(long long K) { return (int)((K / kKSlice + kSlicesPerChunk - 1) / kSlicesPerChunk); }

// Gram of every problem's one-hot matrix over the given work units; each
// problem's Gram must be zero.  maps: device array of tensor maps (one per
// problem, 64-byte aligned).
cudaError_t launch_gram(const void* maps, const int4* units, int n_units, const ProblemDev* probs, int num_sms,
                        unsigned* status, int wait_limit, cudaStream_t st)
{
    GramArgs g;
    g.maps = reinterpret_cast<const CUtensorMap*>(maps);
    g.units = units;
    g.probs = probs;
    g.n_units = n_units;
    g.status = status;
    g.limit = wait_limit < 0 ? 0u : wait_limit == 0 ? kSpinLimit : (unsigned)wait_limit;
    cudaError_t e = cudaFuncSetAttribute(k_gram, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGramSmem);
    if (e != cudaSuccess) return e;
    const int grid = n_units < num_sms ? n_units : num_sms;
    if (grid <= 0) return cudaSuccess;
    k_gram<<<grid, kGramThreads, kGramSmem, st>>>(g);
    return cudaGetLastError();
}

cudaError_t launch_pairs_decide(const EdgeWork* edges, long long edge_cap, const ProblemDev* probs,
                                unsigned long long* min_accept, const CritTableDev& crit, double alpha,
                                DepthCounters* ctr, int stat, int df_mode, int grid, cudaStream_t st)
{
    k_pairs_decide<<<grid, 256, 0, st>>>(edges, edge_cap, probs, min_accept, crit, alpha, ctr, stat, df_mode);
    return cudaGetLastError();
}

cudaError_t launch_symmetrize(int32_t* G, int Mp, int M, cudaStream_t st)
{
    const long long n = (long long)M * M;
    k_symmetrize<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(G, Mp, M);
    return cudaGetLastError();
}

}  // namespace fbn
