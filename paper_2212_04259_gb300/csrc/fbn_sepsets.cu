// fbn_sepsets.cu -- the separating sets of a learnt skeleton (Algorithm 1,
// SepSet) compacted on the device into CSR form: the removed pairs i < j in
// ascending (i, j), one offset per pair, the members in pair order.  The
// writer's outputs may be pinned host memory (device-addressable): only the
// compact arrays cross to the host.
#include <cstdint>
#include <cuda_runtime.h>

#include "fbn_sepsets.h"

namespace fbn {
namespace {

// Per row i (one warp): removed pairs (i, j > i) and their member total.
__global__ void k_sep_count(const int32_t* __restrict__ sep_len, int n, long long* __restrict__ cnt)
{
    const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= n) return;
    long long pairs = 0, members = 0;
    for (int j = i + 1 + lane; j < n; j += 32) {
        const int32_t L = sep_len[(long long)i * n + j];
        if (L >= 0) {
            pairs += 1;
            members += L;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        pairs += __shfl_xor_sync(0xffffffffu, pairs, o);
        members += __shfl_xor_sync(0xffffffffu, members, o);
    }
    if (lane == 0) {
        cnt[i] = pairs;
        cnt[n + i] = members;
    }
}

// One CTA: exclusive row offsets of pairs and members; totals at index n.
__global__ void k_sep_scan(const long long* __restrict__ cnt, int n, long long* __restrict__ roff_p,
                           long long* __restrict__ roff_m)
{
    __shared__ long long sp[1024], sm[1024];
    const int t = threadIdx.x, T = blockDim.x;
    const int per = (n + T - 1) / T;
    const int lo = t * per, hi = lo + per < n ? lo + per : n;
    long long p = 0, m = 0;
    for (int i = lo; i < hi; ++i) {
        p += cnt[i];
        m += cnt[n + i];
    }
    sp[t] = p;
    sm[t] = m;
    __syncthreads();
    for (int o = 1; o < T; o <<= 1) {   // inclusive Hillis-Steele scan of the thread sums
        const long long ap = t >= o ? sp[t - o] : 0, am = t >= o ? sm[t - o] : 0;
        __syncthreads();
        sp[t] += ap;
        sm[t] += am;
        __syncthreads();
    }
    long long bp = sp[t] - p, bm = sm[t] - m;
    for (int i = lo; i < hi; ++i) {
        roff_p[i] = bp;
        roff_m[i] = bm;
        bp += cnt[i];
        bm += cnt[n + i];
    }
    if (t == T - 1) {
        roff_p[n] = sp[T - 1];
        roff_m[n] = sm[T - 1];
    }
}

// Per row i (one warp): the row's pairs, offsets and members at its offsets.
__global__ void k_sep_write(const int32_t* __restrict__ sep_len, const int64_t* __restrict__ sep_off,
                            const int32_t* __restrict__ pool, int n, const long long* __restrict__ roff_p,
                            const long long* __restrict__ roff_m, int32_t* __restrict__ pairs,
                            int64_t* __restrict__ offs, int32_t* __restrict__ members)
{
    const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= n) return;
    long long p = roff_p[i], m = roff_m[i];
    for (int j0 = i + 1; j0 < n; j0 += 32) {
        const int j = j0 + lane;
        const int32_t L = j < n ? sep_len[(long long)i * n + j] : -1;
        const bool take = L >= 0;
        const unsigned ballot = __ballot_sync(0xffffffffu, take);
        long long inc = take ? L : 0;   // inclusive scan of the lengths
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (take) {
            const long long k = p + __popc(ballot & ((1u << lane) - 1u));
            const long long mo = m + inc - L;
            pairs[2 * k] = i;
            pairs[2 * k + 1] = j;
            offs[k] = mo;
            const int64_t src = sep_off[(long long)i * n + j];
            for (int t = 0; t < L; ++t) members[mo + t] = pool[src + t];
        }
        p += __popc(ballot);
        m += __shfl_sync(0xffffffffu, inc, 31);
    }
}

}  // namespace

cudaError_t launch_sep_count(const int32_t* sep_len, int n, long long* cnt, long long* roff_p, long long* roff_m,
                             cudaStream_t st)
{
    const int warps = 8;
    k_sep_count<<<(n + warps - 1) / warps, warps * 32, 0, st>>>(sep_len, n, cnt);
    k_sep_scan<<<1, 1024, 0, st>>>(cnt, n, roff_p, roff_m);
    return cudaGetLastError();
}

cudaError_t launch_sep_write(const int32_t* sep_len, const int64_t* sep_off, const int32_t* pool, int n,
                             const long long* roff_p, const long long* roff_m, int32_t* pairs, int64_t* offs,
                             int32_t* members, cudaStream_t st)
{
    const int warps = 8;
    k_sep_write<<<(n + warps - 1) / warps, warps * 32, 0, st>>>(sep_len, sep_off, pool, n, roff_p, roff_m, pairs,
                                                               offs, members);
    return cudaGetLastError();
}

}  // namespace fbn
