// fbn_nbr.cu -- depth 1 of Algorithm 1 on the fifth-generation tensor cores:
// for one vertex x, the tables of all its neighbour pairs at once.
//
// At depth 1 the edge x-y is tested against every single z of a(x)\{y}
// (Section III-A, PC-stable; Section III-B, G^2 on the table of X, Y and Z).
// With e_{v,k} in {0,1}^N marking the samples where V_v = k, that table is
//     N(a, b, c) = #{s : X_s = a, Y_s = b, Z_s = c} = < e_{x,a} * e_{z,c}, e_{y,b} >
// (* the elementwise product), so the tables of every pair (y, z) of x's
// neighbours are blocks of one product D = A B^T with
//     A row (z, c, a) = e_{x,a} * e_{z,c},    B row (y, b) = e_{y,b},
// z and y both running over a(x).  D runs on tcgen05.mma.kind::f8f6f4 with
// 0/1 E4M3 operands (A in tensor memory, B in shared memory) and FP32
// accumulators in tensor memory; an accumulation covers at most 8192 samples,
// so every partial count is an integer below 2^13 and exact, and is added into
// INT32 sums in shared memory.  The work pool's early exit has no counterpart
// here: every test of x's side (|a(x)| (|a(x)| - 1) of them) is evaluated, and
// each edge keeps its lowest accepting rank, as in the pool.
//
// The samples come 4 bits each (k_pack4), so that one byte permutation
// (PRMT) turns 4 samples into their 4 one-hot bytes: the 4-bit value selects
// byte `value` of a table that holds 0x38 (E4M3 1.0) at the wanted value.
//
// Work: CTAs claim vertices from a device counter; a vertex is cut into units
// (a range of z's with at most 128 rows of A, a range of y's with at most 128
// rows of B).  Roles of a CTA (one per SM):
//   warp 12     loader: claims vertices, lays each unit out in a ring of
//               descriptors, streams the packed samples of x and of the
//               unit's neighbours into shared memory with bulk copies
//   warps 4-11  builders: per 128-sample stage, the rows of A into tensor
//               memory (a thread per row and half stage) and the rows of B
//               into the swizzled shared tile
//   warp 13     MMA issuer (one thread)
//   warps 0-3   epilogue: tensor memory -> INT32 sums; at the end of a unit one
//               thread per test forms G^2, decides, and lowers the edge's rank
// Every wait is bounded; a role that gives up raises the CTA's abort flag and
// FBN_ETIMEOUT's status bit, the others leave their loops, and the CTA waits for
// its copies in flight and frees its tensor memory before it exits.
#include <cstdint>

#include <cuda.h>
#include <cuda_runtime.h>

#include "fbn_device.cuh"
#include "fbn_nbr.h"
#include "fbn_tc.cuh"

namespace fbn {
namespace {

using namespace tc;

constexpr int kStageSamples = 128;                 // samples (bytes of K) per pipeline stage
constexpr int kStagePacked = kStageSamples / 2;    // packed bytes of one variable per stage
constexpr int kChunkStages = 64;                   // 8192 samples per exact accumulation
constexpr int kStages = 4;
constexpr int kTileRows = 128;                     // rows of A (= M) and at most rows of B (= N)
constexpr int kTileBytes = kTileRows * kStageSamples;
constexpr int kRawBufs = 4;
constexpr int kRawBufBytes = 16384;                // packed samples of one block of stages
constexpr int kMaxBlockStages = 16;
constexpr int kMaxZ = 32;                          // z's of a unit (each takes >= 4 rows of A)
constexpr int kMaxY = 64;                          // y's of a unit (each takes >= 2 rows of B)
constexpr int kRawVars = 1 + kMaxZ + kMaxY;
constexpr int kSumPitch = kTileRows + 1;           // INT32 sums, one row per TMEM lane
constexpr int kRing = 4;
constexpr int kBuilderWarps = 8;
constexpr int kThreads = 32 * (4 + kBuilderWarps + 2);
constexpr int kLoaderWarp = 4 + kBuilderWarps;
constexpr int kMmaWarp = kLoaderWarp + 1;
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kAccCols = 128;                 // two FP32 accumulators at columns 0 and 128
constexpr uint32_t kACol0 = 2 * kAccCols;          // A stages: 32 columns (128 samples) each
constexpr int kMaxArity = 8;
constexpr uint8_t kNoRow = 0xFF;

static_assert(kACol0 + kStages * (kStageSamples / 4) <= kTmemCols, "tensor memory columns");
static_assert(kRawVars * kStagePacked <= kRawBufBytes, "one stage of every variable fits a raw buffer");

struct NbrUnit {
    const uint8_t* pk;       // packed samples of the problem, row stride pk_ld
    long long pk_ld;
    int p, x, N, nst;        // problem, vertex, samples, stages
    int rx, nz, ny, ncols;   // arity of x, z's, y's, rows of B padded to 16
    int zbeg, ybeg, arows, wide;
    int bstages, nraw, pad0, pad1;   // stages per raw block, variables per raw block
    int16_t zrow[kMaxZ];     // first row of z's block of A (rows c * rx + a)
    int16_t ycol[kMaxY];     // first row of B (= column of D) of y's block
    uint8_t rz[kMaxZ];
    uint8_t ry[kMaxY];
    uint8_t aslot[kTileRows];   // row of A -> raw slot of its z (kNoRow past the last block)
    uint8_t aval[kTileRows];    // row of A -> (c << 4) | a
    uint8_t bslot[kTileRows];   // row of B -> raw slot of its y (kNoRow past the last block)
    uint8_t bval[kTileRows];    // row of B -> b
    int32_t var[kRawVars];      // raw slot -> variable: x, the z's, the y's
};

struct NbrArgs {
    const ProblemDev* probs;
    const int32_t* vtx_prob;
    const int32_t* vtx_first;
    const EdgeWork* edges;
    unsigned long long* min_accept;
    DepthCounters* ctr;
    CritTableDev crit;
    double alpha;
    int total_vertices;
    unsigned limit;
};

constexpr size_t kOffB = 0;
constexpr size_t kOffRaw = kOffB + (size_t)kStages * kTileBytes;
constexpr size_t kOffSum = kOffRaw + (size_t)kRawBufs * kRawBufBytes;
constexpr size_t kOffRing = kOffSum + (size_t)kTileRows * kSumPitch * 4;
constexpr size_t kOffBars = (kOffRing + (size_t)kRing * sizeof(NbrUnit) + 15) / 16 * 16;
constexpr int kNumBars = 2 * kStages + 2 * kRawBufs + 4 + 2 * kRing + 2;
constexpr size_t kNbrSmem = 1024 /*align*/ + kOffBars + kNumBars * 8 + 64;

// One-hot table of value v for a byte permutation: byte v of {hi:lo} is 0x38.
__device__ __forceinline__ void onehot_lut(int v, uint32_t& lo, uint32_t& hi)
{
    lo = v < 4 ? 0x38u << (8 * v) : 0u;
    hi = v >= 4 && v < 8 ? 0x38u << (8 * (v - 4)) : 0u;
}

// Bounded wait taken by every lane of a warp, with one outcome for the warp.
__device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag, unsigned* status,
                                          unsigned limit)
{
    const bool ok = mbar_wait(bar, parity, abort_flag, status, limit);
    const bool all = __all_sync(0xffffffffu, ok);
    if (!all) *abort_flag = 1;
    return all;
}

// Greedy packing of consecutive neighbours from position q0: how many fit in
// `cap` rows at `mult` x arity rows each, at most maxn (warp-collective).
__device__ int pack_count(const int32_t* nb, const uint8_t* ar, int q0, int k, int mult, int cap, int maxn,
                          int lane)
{
    int count = 0, used = 0;
    while (count < maxn && q0 + count < k) {
        const int q = q0 + count + lane;
        const bool valid = q < k && count + lane < maxn;
        const int w = valid ? mult * (int)ar[nb[q]] : (1 << 20);
        int s = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        const int f = __popc(__ballot_sync(0xffffffffu, used + s <= cap));   // a prefix: weights are positive
        if (f == 0) break;
        used += __shfl_sync(0xffffffffu, s, f - 1);
        count += f;
        if (f < 32) break;
    }
    return count;
}

// Inclusive warp scan.
__device__ __forceinline__ int warp_scan(int v, int lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    return v;
}

// G^2 decision of the test (x, y | z) from the INT32 sums: rows
// zrow + c * rx + a, columns ycol + b.  Terms n ln(n n_c / (n_ac n_bc)) with
// FP32 logarithms (each within 3.2e-7 of its magnitude, the ratio formed from
// exact 64-bit integers) summed in FP32 by one thread (cells additions, each
// within 6e-8 of the running sum of magnitudes); recomputed in FP64 only when
// crit lies inside the error band.  Returns true when p > alpha.
template <int R>
__device__ bool test_decide(const int* T0, int rx, int ry, int rz, double crit)
{
    float acc = 0.0f, mag = 0.0f;
    for (int c = 0; c < rz; ++c) {
        const int* Tc = T0 + c * rx * kSumPitch;
        int t[R][R];
        int nac[R], nbc[R];
        int nc = 0;
#pragma unroll
        for (int b = 0; b < R; ++b) nbc[b] = 0;
#pragma unroll
        for (int a = 0; a < R; ++a) {
            nac[a] = 0;
#pragma unroll
            for (int b = 0; b < R; ++b) {
                t[a][b] = (a < rx && b < ry) ? Tc[a * kSumPitch + b] : 0;
                nac[a] += t[a][b];
                nbc[b] += t[a][b];
            }
            nc += nac[a];
        }
#pragma unroll
        for (int a = 0; a < R; ++a)
#pragma unroll
            for (int b = 0; b < R; ++b) {
                const int n = t[a][b];
                if (n == 0) continue;
                const long long A = (long long)n * nc, B = (long long)nac[a] * nbc[b];
                const float fb = (float)B;
                const float delta = (float)(A - B) / fb;
                const float L = fabsf(delta) < 0.5f ? log1pf(delta) : logf((float)A / fb);
                const float term = (float)n * L;
                acc += term;
                mag += fabsf(term);
            }
    }
    const double cells = (double)rx * ry * rz;
    const double rel = 2.0 * (3.2e-7 + cells * 6e-8);
    const double g2 = 2.0 * (double)acc;
    const double err = 2.0 * rel * (double)mag * 1.0001 + 1e-9;
    if (g2 + err < crit) return true;
    if (g2 - err >= crit) return false;
    double ex = 0.0;
    for (int c = 0; c < rz; ++c) {
        const int* Tc = T0 + c * rx * kSumPitch;
        long long nc = 0;
        for (int a = 0; a < rx; ++a)
            for (int b = 0; b < ry; ++b) nc += Tc[a * kSumPitch + b];
        for (int a = 0; a < rx; ++a) {
            long long nac = 0;
            for (int b = 0; b < ry; ++b) nac += Tc[a * kSumPitch + b];
            for (int b = 0; b < ry; ++b) {
                const int n = Tc[a * kSumPitch + b];
                if (n == 0) continue;
                long long nbc = 0;
                for (int aa = 0; aa < rx; ++aa) nbc += Tc[aa * kSumPitch + b];
                const long long A = (long long)n * nc, B = nac * nbc;
                ex += (double)n * log1p((double)(A - B) / (double)B);
            }
        }
    }
    return 2.0 * ex < crit;
}

__global__ void __launch_bounds__(kThreads, 1) k_nbr1(NbrArgs g)
{
    DepthCounters* ctr = g.ctr;
    if (!ctr->active || ctr->d != 1) return;

    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* tileB = smem + kOffB;
    uint8_t* raw = smem + kOffRaw;
    int* sums = reinterpret_cast<int*>(smem + kOffSum);
    NbrUnit* ring = reinterpret_cast<NbrUnit*>(smem + kOffRing);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kOffBars);
    uint64_t* st_full = bars;                           // [kStages] builders -> MMA (one arrival per builder warp)
    uint64_t* st_empty = bars + kStages;                // [kStages] MMA -> builders
    uint64_t* raw_full = bars + 2 * kStages;            // [kRawBufs] bulk copies -> builders
    uint64_t* raw_empty = raw_full + kRawBufs;          // [kRawBufs] builders -> loader
    uint64_t* acc_full = raw_empty + kRawBufs;          // [2] MMA -> epilogue
    uint64_t* acc_empty = acc_full + 2;                 // [2] epilogue -> MMA (4 arrivals)
    uint64_t* ring_full = acc_empty + 2;                // [kRing] loader -> all roles
    uint64_t* ring_empty = ring_full + kRing;           // [kRing] epilogue -> loader
    uint64_t* epi_bar = ring_empty + kRing;             // epilogue-wide barrier (128 arrivals)
    uint64_t* drain = epi_bar + 1;                      // MMA completion before teardown
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + kNumBars);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    int* raw_issued = reinterpret_cast<int*>(tmem_slot + 2);   // [kRawBufs], loader lane 0 only

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned* status = &ctr->status;
    const unsigned limit = g.limit;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(smem_u32(&st_full[s]), kBuilderWarps);
            mbar_init(smem_u32(&st_empty[s]), 1);
        }
        for (int b = 0; b < kRawBufs; ++b) {
            mbar_init(smem_u32(&raw_full[b]), 1);
            mbar_init(smem_u32(&raw_empty[b]), kBuilderWarps);
            raw_issued[b] = 0;
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&acc_full[b]), 1);
            mbar_init(smem_u32(&acc_empty[b]), 4);
        }
        for (int r = 0; r < kRing; ++r) {
            mbar_init(smem_u32(&ring_full[r]), 1);
            mbar_init(smem_u32(&ring_empty[r]), 1);
        }
        mbar_init(smem_u32(epi_bar), 128);
        mbar_init(smem_u32(drain), 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kMmaWarp) tmem_alloc(smem_u32(tmem_slot), kTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == kLoaderWarp) {
        // ------------------------------------------------------------ loader
        int slot = 0, rb = 0;
        uint32_t ring_ph = 0, rb_ph = 0;
        bool ok = true;
        for (;;) {
            int gv = 0;
            if (lane == 0) gv = (int)atomicAdd(&ctr->nbr_claim, 1ULL);
            gv = __shfl_sync(0xffffffffu, gv, 0);
            if (gv >= g.total_vertices || *abort_flag) break;
            const int p = g.vtx_prob[gv];
            const ProblemDev& P = g.probs[p];
            const int x = gv - g.vtx_first[p];
            const int k = P.deg[x];
            if (k < 2) continue;
            const int rx = P.ar[x];
            const int32_t* nb = P.nbr + (long long)x * P.n;
            const int nst = (P.N + kStageSamples - 1) / kStageSamples;
            for (int zb = 0; zb < k && ok;) {
                const int nz = pack_count(nb, P.ar, zb, k, rx, kTileRows, kMaxZ, lane);
                if (nz == 0) {
                    ok = false;
                    break;
                }
                for (int yb = 0; yb < k && ok;) {
                    const int ny = pack_count(nb, P.ar, yb, k, 1, kTileRows, kMaxY, lane);
                    if (ny == 0 || !warp_wait(smem_u32(&ring_empty[slot]), ring_ph ^ 1u, abort_flag, status, limit)) {
                        ok = false;
                        break;
                    }
                    NbrUnit& U = ring[slot];
                    int zr = 0, zv = 0;
                    if (lane < nz) {
                        zv = nb[zb + lane];
                        zr = P.ar[zv];
                    }
                    const int zinc = warp_scan(rx * zr, lane);
                    const int arows = __shfl_sync(0xffffffffu, zinc, 31);
                    if (lane < nz) {
                        const int r0 = zinc - rx * zr;
                        U.zrow[lane] = (int16_t)r0;
                        U.rz[lane] = (uint8_t)zr;
                        U.var[1 + lane] = zv;
                        for (int c = 0; c < zr; ++c)
                            for (int a = 0; a < rx; ++a) {
                                U.aslot[r0 + c * rx + a] = (uint8_t)(1 + lane);
                                U.aval[r0 + c * rx + a] = (uint8_t)((c << 4) | a);
                            }
                    }
                    for (int r = arows + lane; r < kTileRows; r += 32) U.aslot[r] = kNoRow;
                    int carry = 0;
                    for (int t0 = 0; t0 < ny; t0 += 32) {
                        const int t = t0 + lane;
                        int yv = 0, yr = 0;
                        if (t < ny) {
                            yv = nb[yb + t];
                            yr = P.ar[yv];
                        }
                        const int yinc = warp_scan(yr, lane);
                        if (t < ny) {
                            const int c0 = carry + yinc - yr;
                            U.ycol[t] = (int16_t)c0;
                            U.ry[t] = (uint8_t)yr;
                            U.var[1 + nz + t] = yv;
                            for (int b = 0; b < yr; ++b) {
                                U.bslot[c0 + b] = (uint8_t)(1 + nz + t);
                                U.bval[c0 + b] = (uint8_t)b;
                            }
                        }
                        carry += __shfl_sync(0xffffffffu, yinc, 31);
                    }
                    for (int r = carry + lane; r < kTileRows; r += 32) U.bslot[r] = kNoRow;
                    const int nraw = 1 + nz + ny;
                    int bst = kRawBufBytes / (nraw * kStagePacked);
                    bst = bst < kMaxBlockStages ? bst : kMaxBlockStages;
                    if (lane == 0) {
                        U.pk = P.pk;
                        U.pk_ld = P.pk_ld;
                        U.p = p;
                        U.x = x;
                        U.N = P.N;
                        U.nst = nst;
                        U.rx = rx;
                        U.nz = nz;
                        U.ny = ny;
                        U.ncols = (carry + 15) / 16 * 16;
                        U.zbeg = zb;
                        U.ybeg = yb;
                        U.arows = arows;
                        U.wide = P.max_arity > 4;
                        U.bstages = bst;
                        U.nraw = nraw;
                        U.var[0] = x;
                    }
                    __syncwarp();
                    if (lane == 0) mbar_arrive(smem_u32(&ring_full[slot]));
                    // the packed samples of the unit, bst stages at a time
                    const uint8_t* base = P.pk;
                    const long long ld = P.pk_ld;
                    for (int s0 = 0; s0 < nst; s0 += bst) {
                        if (!warp_wait(smem_u32(&raw_empty[rb]), rb_ph ^ 1u, abort_flag, status, limit)) {
                            ok = false;
                            break;
                        }
                        const int ns = nst - s0 < bst ? nst - s0 : bst;
                        const uint32_t bytes = (uint32_t)(ns * kStagePacked);
                        const uint32_t fb = smem_u32(&raw_full[rb]);
                        if (lane == 0) {
                            mbar_expect_tx(fb, (uint32_t)nraw * bytes);
                            raw_issued[rb] += 1;
                        }
                        __syncwarp();
                        uint8_t* dst = raw + (size_t)rb * kRawBufBytes;
                        for (int v = lane; v < nraw; v += 32)
                            bulk_load(smem_u32(dst + (size_t)v * bst * kStagePacked),
                                      base + (long long)U.var[v] * ld + (long long)s0 * kStagePacked, bytes, fb);
                        if (++rb == kRawBufs) {
                            rb = 0;
                            rb_ph ^= 1u;
                        }
                    }
                    if (++slot == kRing) {
                        slot = 0;
                        ring_ph ^= 1u;
                    }
                    yb += ny;
                }
                zb += nz;
            }
            if (!ok) break;
        }
        if (!ok && !*abort_flag) {   // a unit could not be laid out
            *abort_flag = 1;
            if (lane == 0) atomicOr(status, kStatusTooBig);
        }
        if (ok && !*abort_flag && warp_wait(smem_u32(&ring_empty[slot]), ring_ph ^ 1u, abort_flag, status, limit)) {
            if (lane == 0) {
                ring[slot].p = -1;   // no more units
                mbar_arrive(smem_u32(&ring_full[slot]));
            }
        }
    } else if (warp >= 4 && warp < kLoaderWarp) {
        // ------------------------------------------------------------ builders
        // Thread bt owns one row of A over half a stage (TMEM lane quarter*32 +
        // lane, samples 64*half ..) and up to four (row, 16-sample chunk) pieces
        // of B; all of it is laid out once per unit.  Per stage the loads and
        // the one-hot arithmetic run before the wait for a free stage, the
        // stores after it.
        const int bt = threadIdx.x - 128;            // 0 .. 255
        const int quarter = warp & 3;                // TMEM lanes 32 * quarter ..
        const int half = (warp - 4) >> 2;            // samples 64 * half .. of the stage
        const int arow = quarter * 32 + lane;
        constexpr int kBTasks = kTileRows * 8 / (32 * kBuilderWarps);   // 4
        int slot = 0, st = 0, rb = 0;
        uint32_t ring_ph = 0, st_ph = 0, rb_ph = 0;
        for (;;) {
            if (!warp_wait(smem_u32(&ring_full[slot]), ring_ph, abort_flag, status, limit)) break;
            const NbrUnit& U = ring[slot];
            if (U.p < 0) break;
            const int nst = U.nst, N = U.N, bst = U.bstages;
            const int vstride = bst * kStagePacked;   // bytes of one variable in a raw block
            // row of A: z's raw slot and the one-hot tables of a and c
            const int zslot = U.aslot[arow];
            uint32_t xl = 0, xh = 0, zl = 0, zh = 0;
            if (zslot != kNoRow) {
                onehot_lut(U.aval[arow] & 15, xl, xh);
                onehot_lut(U.aval[arow] >> 4, zl, zh);
            }
            const int xoff = half * 32;
            const int zoff = (zslot != kNoRow ? zslot : 0) * vstride + half * 32;
            // pieces of B: raw offset, one-hot table, swizzled tile offset
            int boff[kBTasks], bdst[kBTasks];
            uint32_t blo[kBTasks], bhi[kBTasks];
            unsigned bmask = 0;
#pragma unroll
            for (int i = 0; i < kBTasks; ++i) {
                const int task = bt + i * 32 * kBuilderWarps;
                const int row = task >> 3, j = task & 7;
                const int ys = U.bslot[row];
                boff[i] = 0;
                bdst[i] = row * 128 + ((j ^ (row & 7)) << 4);
                blo[i] = bhi[i] = 0;
                if (ys != kNoRow) {
                    bmask |= 1u << i;
                    boff[i] = ys * vstride + j * 8;
                    onehot_lut(U.bval[row], blo[i], bhi[i]);
                }
            }
            bool ok = true;
            int sb = 0;
            for (int s = 0; s < nst; ++s) {
                if (sb == 0 && !warp_wait(smem_u32(&raw_full[rb]), rb_ph, abort_flag, status, limit)) {
                    ok = false;
                    break;
                }
                const uint8_t* rw = raw + (size_t)rb * kRawBufBytes + sb * kStagePacked;
                // loads
                const uint4 xv0 = *reinterpret_cast<const uint4*>(rw + xoff);
                const uint4 xv1 = *reinterpret_cast<const uint4*>(rw + xoff + 16);
                const uint4 zv0 = *reinterpret_cast<const uint4*>(rw + zoff);
                const uint4 zv1 = *reinterpret_cast<const uint4*>(rw + zoff + 16);
                uint2 bw[kBTasks];
#pragma unroll
                for (int i = 0; i < kBTasks; ++i)
                    bw[i] = (bmask >> i) & 1u ? *reinterpret_cast<const uint2*>(rw + boff[i]) : make_uint2(0, 0);
                // one-hot arithmetic
                uint32_t out[16];
                {
                    const uint32_t xw[8] = {xv0.x, xv0.y, xv0.z, xv0.w, xv1.x, xv1.y, xv1.z, xv1.w};
                    const uint32_t zw[8] = {zv0.x, zv0.y, zv0.z, zv0.w, zv1.x, zv1.y, zv1.z, zv1.w};
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        out[2 * q] = __byte_perm(xl, xh, xw[q]) & __byte_perm(zl, zh, zw[q]);
                        out[2 * q + 1] = __byte_perm(xl, xh, xw[q] >> 16) & __byte_perm(zl, zh, zw[q] >> 16);
                    }
                }
                const int sfirst = s * kStageSamples + half * 64;
                if (sfirst + 64 > N) {   // samples at or beyond N count nowhere
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        uint32_t m = 0;
#pragma unroll
                        for (int b = 0; b < 4; ++b)
                            if (sfirst + 4 * q + b < N) m |= 0xFFu << (8 * b);
                        out[q] &= m;
                    }
                }
                uint4 bo[kBTasks];
#pragma unroll
                for (int i = 0; i < kBTasks; ++i)
                    bo[i] = make_uint4(__byte_perm(blo[i], bhi[i], bw[i].x), __byte_perm(blo[i], bhi[i], bw[i].x >> 16),
                                       __byte_perm(blo[i], bhi[i], bw[i].y), __byte_perm(blo[i], bhi[i], bw[i].y >> 16));
                // the raw block is consumed once its last stage is in registers
                const bool last_in_block = sb == bst - 1 || s == nst - 1;
                if (last_in_block) {
                    __syncwarp();
                    if (lane == 0) mbar_arrive(smem_u32(&raw_empty[rb]));
                }
                // stores into a free stage
                if (!warp_wait(smem_u32(&st_empty[st]), st_ph ^ 1u, abort_flag, status, limit)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                uint8_t* B = tileB + (size_t)st * kTileBytes;
#pragma unroll
                for (int i = 0; i < kBTasks; ++i)
                    if ((bmask >> i) & 1u) *reinterpret_cast<uint4*>(B + bdst[i]) = bo[i];
                tmem_st16(tmem + ((uint32_t)(quarter * 32) << 16) + kACol0 + (uint32_t)st * 32 + half * 16, out);
                fence_async_smem();
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&st_full[st]));
                if (++st == kStages) {
                    st = 0;
                    st_ph ^= 1u;
                }
                if (last_in_block) {
                    sb = 0;
                    if (++rb == kRawBufs) {
                        rb = 0;
                        rb_ph ^= 1u;
                    }
                } else {
                    ++sb;
                }
            }
            if (!ok) break;
            if (++slot == kRing) {
                slot = 0;
                ring_ph ^= 1u;
            }
        }
    } else if (warp == kMmaWarp) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            int slot = 0, st = 0, ab = 0;
            uint32_t ring_ph = 0, st_ph = 0, ab_ph = 0;
            bool ok = true;
            for (;;) {
                if (!mbar_wait(smem_u32(&ring_full[slot]), ring_ph, abort_flag, status, limit)) break;
                const NbrUnit& U = ring[slot];
                if (U.p < 0) break;
                const int nst = U.nst;
                const uint32_t idesc = idesc_f8(kTileRows, U.ncols);
                for (int c0 = 0; c0 < nst && ok; c0 += kChunkStages) {
                    if (!mbar_wait(smem_u32(&acc_empty[ab]), ab_ph ^ 1u, abort_flag, status, limit)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t d_tmem = tmem + (uint32_t)ab * kAccCols;
                    const int c1 = min(nst, c0 + kChunkStages);
                    for (int s = c0; s < c1; ++s) {
                        if (!mbar_wait(smem_u32(&st_full[st]), st_ph, abort_flag, status, limit)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t a_tmem = tmem + kACol0 + (uint32_t)st * 32;
                        const uint64_t db = smem_desc(smem_u32(tileB + (size_t)st * kTileBytes));
#pragma unroll
                        for (int k = 0; k < kStageSamples / 32; ++k)   // 32 samples per MMA: 8 columns of A, 32 bytes of B
                            mma_f8_tmem_a(d_tmem, a_tmem + (uint32_t)(8 * k), db + (uint64_t)(2 * k), idesc,
                                          (s > c0 || k > 0) ? 1u : 0u);
                        mma_commit(smem_u32(&st_empty[st]));
                        if (++st == kStages) {
                            st = 0;
                            st_ph ^= 1u;
                        }
                    }
                    if (!ok) break;
                    mma_commit(smem_u32(&acc_full[ab]));
                    if (++ab == 2) {
                        ab = 0;
                        ab_ph ^= 1u;
                    }
                }
                if (!ok) break;
                if (++slot == kRing) {
                    slot = 0;
                    ring_ph ^= 1u;
                }
            }
            // every MMA issued has finished before tensor memory is released
            mma_commit(smem_u32(drain));
            mbar_drain(smem_u32(drain), 0);
        }
    } else {
        // ------------------------------------------------------------ epilogue (warps 0-3)
        const int row = threadIdx.x;   // TMEM lane = row of A = row of the sums
        int slot = 0, ab = 0;
        uint32_t ring_ph = 0, ab_ph = 0, epi_ph = 0;
        unsigned long long my_tests = 0;
        for (;;) {
            if (!warp_wait(smem_u32(&ring_full[slot]), ring_ph, abort_flag, status, limit)) break;
            const NbrUnit& U = ring[slot];
            if (U.p < 0) break;
            const int nst = U.nst, ncols = U.ncols;
            bool ok = true;
            for (int c0 = 0; c0 < nst; c0 += kChunkStages) {
                if (!warp_wait(smem_u32(&acc_full[ab]), ab_ph, abort_flag, status, limit)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t base = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)ab * kAccCols;
                int* srow = sums + row * kSumPitch;
                for (int q0 = 0; q0 < ncols; q0 += 32) {
                    uint32_t v[32];
                    tmem_ld32(base + (uint32_t)q0, v);
                    if (c0 == 0) {
#pragma unroll
                        for (int q = 0; q < 32; ++q) srow[q0 + q] = __float2int_rn(__uint_as_float(v[q]));
                    } else {
#pragma unroll
                        for (int q = 0; q < 32; ++q) srow[q0 + q] += __float2int_rn(__uint_as_float(v[q]));
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&acc_empty[ab]));
                if (++ab == 2) {
                    ab = 0;
                    ab_ph ^= 1u;
                }
            }
            if (!ok) break;
            // every row of the sums is final: epilogue-wide barrier
            mbar_arrive(smem_u32(epi_bar));
            if (!warp_wait(smem_u32(epi_bar), epi_ph, abort_flag, status, limit)) break;
            epi_ph ^= 1u;
            {
                const ProblemDev& P = g.probs[U.p];
                const int x = U.x, rx = U.rx, nz = U.nz, ny = U.ny;
                const int zbeg = U.zbeg, ybeg = U.ybeg;
                const long long n = P.n;
                for (int t = threadIdx.x; t < nz * ny; t += 128) {
                    const int zi = t / ny, yi = t - zi * ny;
                    const int qz = zbeg + zi, qy = ybeg + yi;
                    if (qz == qy) continue;
                    const int rz = U.rz[zi], ry = U.ry[yi];
                    const int* T0 = sums + U.zrow[zi] * kSumPitch + U.ycol[yi];
                    const long long df = (long long)(rx - 1) * (ry - 1) * rz;
                    const double crit = crit_get(g.crit, df, g.alpha, status);
                    const bool accept = U.wide ? test_decide<kMaxArity>(T0, rx, ry, rz, crit)
                                               : test_decide<4>(T0, rx, ry, rz, crit);
                    my_tests += 1;
                    if (accept) {
                        const int e = P.eid[(long long)x * n + qy];
                        const EdgeWork w = g.edges[e];
                        const long long local = qz - (qz > qy ? 1 : 0);
                        const long long rank = (x == w.i ? 0 : w.cnt_i) + local;
                        atomicMin(&g.min_accept[e], (unsigned long long)rank);
                    }
                }
            }
            // the sums are read: the next unit may overwrite them
            mbar_arrive(smem_u32(epi_bar));
            if (!warp_wait(smem_u32(epi_bar), epi_ph, abort_flag, status, limit)) break;
            epi_ph ^= 1u;
            if (threadIdx.x == 0) mbar_arrive(smem_u32(&ring_empty[slot]));
            if (++slot == kRing) {
                slot = 0;
                ring_ph ^= 1u;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) my_tests += __shfl_xor_sync(0xffffffffu, my_tests, o);
        if (lane == 0 && my_tests) atomicAdd(&ctr->tests, my_tests);
    }

    __syncthreads();
    if (warp == kLoaderWarp && lane == 0) {
        // no bulk copy may land after the CTA exits: wait for the last block of
        // every raw buffer (immediate unless a role gave up)
        for (int b = 0; b < kRawBufs; ++b)
            if (raw_issued[b] > 0) mbar_drain(smem_u32(&raw_full[b]), (uint32_t)((raw_issued[b] - 1) & 1));
    }
    tc_fence_before();
    __syncthreads();
    if (warp == kMmaWarp) {
        tc_fence_after();
        tmem_dealloc(tmem, kTmemCols);
    }
}

// Samples 4 bits each: byte q of a row holds samples 2q (low nibble) and
// 2q + 1 (high nibble); arities are at most 8, so bit 3 of every nibble is 0.
// One CTA per variable of the batch.
__global__ void k_pack4(const ProblemDev* __restrict__ probs, const int32_t* __restrict__ vtx_prob,
                        const int32_t* __restrict__ vtx_first, int total_vertices)
{
    const int gv = blockIdx.x;
    if (gv >= total_vertices) return;
    const int p = vtx_prob[gv];
    const ProblemDev& P = probs[p];
    const int v = gv - vtx_first[p];
    const uint4* src = reinterpret_cast<const uint4*>(P.data + (long long)v * P.ld);
    uint2* dst = reinterpret_cast<uint2*>(P.pk + (long long)v * P.pk_ld);
    const long long nvec = P.ld / 16;
    for (long long q = threadIdx.x; q < nvec; q += blockDim.x) {
        const uint4 w = src[q];
        const uint32_t in[4] = {w.x, w.y, w.z, w.w};
        uint32_t o[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            // bytes b0 b1 b2 b3 | b4 b5 b6 b7 -> nibbles b0..b7
            const uint32_t a = in[2 * h], b = in[2 * h + 1];
            const uint32_t a2 = (a | (a >> 4)) & 0x00FF00FFu;   // (b1 b0) in byte 0, (b3 b2) in byte 2
            const uint32_t b2 = (b | (b >> 4)) & 0x00FF00FFu;
            const uint32_t a3 = (a2 | (a2 >> 8)) & 0xFFFFu;
            const uint32_t b3 = (b2 | (b2 >> 8)) & 0xFFFFu;
            o[h] = a3 | (b3 << 16);
        }
        dst[q] = make_uint2(o[0], o[1]);
    }
}

}  // namespace

size_t nbr1_smem_bytes() { return kNbrSmem; }

int nbr1_max_arity() { return kMaxArity; }

cudaError_t launch_pack4(const ProblemDev* probs, const int32_t* vtx_prob, const int32_t* vtx_first,
                         int total_vertices, cudaStream_t st)
{
    if (total_vertices <= 0) return cudaSuccess;
    k_pack4<<<total_vertices, 256, 0, st>>>(probs, vtx_prob, vtx_first, total_vertices);
    return cudaGetLastError();
}

cudaError_t launch_nbr1(const ProblemDev* probs, const int32_t* vtx_prob, const int32_t* vtx_first,
                        int total_vertices, const EdgeWork* edges, unsigned long long* min_accept,
                        const CritTableDev& crit, double alpha, DepthCounters* ctr, int num_sms, int wait_limit,
                        cudaStream_t st)
{
    NbrArgs g;
    g.probs = probs;
    g.vtx_prob = vtx_prob;
    g.vtx_first = vtx_first;
    g.edges = edges;
    g.min_accept = min_accept;
    g.ctr = ctr;
    g.crit = crit;
    g.alpha = alpha;
    g.total_vertices = total_vertices;
    g.limit = wait_limit < 0 ? 0u : wait_limit == 0 ? kSpinLimit : (unsigned)wait_limit;
    cudaError_t e = cudaFuncSetAttribute(k_nbr1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kNbrSmem);
    if (e != cudaSuccess) return e;
    const int grid = total_vertices < num_sms ? total_vertices : num_sms;
    if (grid <= 0) return cudaSuccess;
    k_nbr1<<<grid, kThreads, kNbrSmem, st>>>(g);
    return cudaGetLastError();
}

}  // namespace fbn
