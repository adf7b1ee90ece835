// fbn_ci.cu -- explicit CI tests (fbn_ci_test / fbn_ci_table): one CTA per test,
// exact FP64 G^2 and p-value (Section III-B).
#include <cstdint>
#include <cuda_runtime.h>

#include "fbn_device.cuh"
#include "fbn_launch.h"

namespace fbn {

// --------------------------------------------------------------------------
// Explicit tests (fbn_ci_test / fbn_ci_table): exact FP64 G^2 and p-value.
template <bool BITS>
__global__ void __launch_bounds__(kTestThreads) k_ci_tests(const ProblemDev* __restrict__ prob,
                                                           const CiTestDesc* __restrict__ tests, int ntests,
                                                           double* __restrict__ out, int32_t* table_out,
                                                           int* gscratch, long long gscratch_ints,
                                                           unsigned* status, int smem_ints, int stat, int df_mode)
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
        for (int k = 0; k < d + 2; ++k) {
            const int v = k < d ? q.z[k] : k == d ? q.x : q.y;
            spec.rows[k] = P.data + (long long)v * P.ld;
            spec.rad[k] = P.ar[v];
            if (BITS && k < kBitsMaxD + 2) spec.prow[k] = reinterpret_cast<const uint4*>(P.planes + (long long)v * 2 * P.plane_ld);
        }
        spec.pstride = P.plane_ld >> 2;
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
    const int* T = grp_table<kTestThreads, BITS>(spec, smem, smem_ints, gtab, gscratch_ints, &M);
    if (!T) {
        if (threadIdx.x == 0) atomicOr(status, kStatusTooBig);
        return;
    }
    grp_marginals<kTestThreads>(spec, T, M);
    const double st = stat == kStatX2 ? grp_x2_exact<kTestThreads>(spec, T, M, red, table_out)
                                      : grp_g2_exact<kTestThreads>(spec, T, M, red, table_out);
    const double df = df_mode ? (double)grp_df_adjusted<kTestThreads>(spec, M, red)
                              : (double)(spec.rx - 1) * (double)(spec.ry - 1) * (double)(spec.cells / (spec.rx * spec.ry));
    if (threadIdx.x == 0) {
        out[3 * t + 0] = st;
        out[3 * t + 1] = df;
        out[3 * t + 2] = df > 0.0 ? chisq_q(df, st, status) : 1.0;
    }
}

void launch_ci_tests(const ProblemDev* prob, const CiTestDesc* tests, int ntests, double* out,
                     int32_t* table_out, int* gscratch, long long gscratch_ints, unsigned* status,
                     size_t smem_bytes, int stat, int df_mode, bool bits, cudaStream_t st)
{
    auto kern = bits ? k_ci_tests<true> : k_ci_tests<false>;
    kern<<<ntests, kTestThreads, smem_bytes, st>>>(prob, tests, ntests, out, table_out, gscratch, gscratch_ints,
                                                   status, (int)(smem_bytes / 4), stat, df_mode);
}

cudaError_t set_ci_smem(int max_smem)
{
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_ci_tests<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem))) return e;
    return cudaFuncSetAttribute(k_ci_tests<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
}

}  // namespace fbn
