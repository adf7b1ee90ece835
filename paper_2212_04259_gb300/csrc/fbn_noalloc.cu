// fbn_noalloc.cu -- fbn_ci_test_noalloc: one CI test that allocates nothing.
//
// Some callers cannot allocate device memory: a process whose device memory
// is owned by another allocator (a framework's caching allocator, or a
// serving process that reserves a fixed budget at start-up and must not
// exceed it), or a latency-critical loop where cudaMalloc/cudaFree stall the
// device.  This entry point runs the same test as fbn_ci_test on buffers the
// caller already owns and keeps its only scratch -- the global contingency
// table for tables too big for shared memory, its marginals and a status
// word -- in a fixed array compiled into the library.
#include <cstdarg>
#include <cmath>
#include <cstdio>
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/fbn.h"
#include "fbn_device.cuh"
#include "fbn_launch.h"

using namespace fbn;

namespace {

constexpr long long kNoAllocMaxCells = 1LL << 18;                    // largest table accepted
constexpr long long kNoAllocTableInts = 3 * kNoAllocMaxCells + 64;   // table + marginals (<= 1.25 C) + slack
constexpr size_t kNoAllocSmem = 108 * 1024;
constexpr int kNoAllocMaxDevices = 64;

// 3 MiB per device that loads the library, held until the process exits.
// Every call on a device shares it; the last call's contents stay in it.
static __device__ __align__(256) int g_noalloc_scratch[kNoAllocTableInts + 64];

std::mutex g_mu;
bool g_ready[kNoAllocMaxDevices];
int* g_scratch[kNoAllocMaxDevices];   // device address of g_noalloc_scratch on each device

// Whether some sample value of the test's rows is not below its variable's
// arity (block-wide, every thread gets the answer).  The other entry points
// validate data when it enters a handle; this one reads caller-owned rows
// directly, and an out-of-range value would index past the table (in shared
// memory or in the scratch array), so the rows are checked before counting:
// 16 samples per 16-byte load, four byte comparisons per 32-bit word.
__device__ bool rows_out_of_range(const TestSpec& s)
{
    bool bad = false;
    const int nvec = s.N >> 4;
    for (int k = 0; k < s.nrows; ++k) {
        const unsigned rr = (unsigned)s.rad[k] * 0x01010101u;   // the arity in each byte
        const uint4* row = reinterpret_cast<const uint4*>(s.rows[k]);
        for (int v = threadIdx.x; v < nvec; v += blockDim.x) {
            const uint4 w = __ldg(row + v);
            bad |= (__vcmpgeu4(w.x, rr) | __vcmpgeu4(w.y, rr) | __vcmpgeu4(w.z, rr) | __vcmpgeu4(w.w, rr)) != 0u;
        }
        for (int t = (nvec << 4) + threadIdx.x; t < s.N; t += blockDim.x) bad |= s.rows[k][t] >= s.rad[k];
    }
    return __syncthreads_or(bad) != 0;
}

__global__ void __launch_bounds__(kTestThreads) k_ci_noalloc(TestSpec spec, int* scratch, double* out,
                                                             int32_t* table_out, int smem_ints)
{
    extern __shared__ int smem[];
    __shared__ TestSpec s;
    __shared__ double red[32];
    unsigned* status = reinterpret_cast<unsigned*>(scratch + kNoAllocTableInts);
    if (threadIdx.x == 0) {
        s = spec;
        *status = 0;   // the previous call's status must not leak into this one
    }
    __syncthreads();
    if (rows_out_of_range(s)) {   // a value >= its arity: no table, every output NaN
        if (threadIdx.x == 0) out[0] = out[1] = out[2] = nan("");
        return;
    }
    int* M = nullptr;
    const int* T = grp_table<kTestThreads>(s, smem, smem_ints, scratch, kNoAllocTableInts, &M);
    if (!T) {   // not reached: the host admits only tables that fit the scratch
        if (threadIdx.x == 0) out[0] = out[1] = out[2] = nan("");
        return;
    }
    grp_marginals<kTestThreads>(s, T, M);
    const double g2 = grp_g2_exact<kTestThreads>(s, T, M, red, table_out);
    if (threadIdx.x == 0) {
        const double df = (double)(s.rx - 1) * (double)(s.ry - 1) * (double)(s.cells / (s.rx * s.ry));
        const double p = chisq_q(df, g2, status);
        out[0] = g2;
        out[1] = df;
        out[2] = *status ? nan("") : p;
    }
}

int nfail(int code, const char* fmt, ...)
{
    char buf[256];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    fbn_internal_set_error(buf);
    return code;
}

}  // namespace

extern "C" int fbn_ci_test_noalloc(const uint8_t* data, int64_t ld, int32_t n_vars, int64_t n_samples,
                                   const uint8_t* arities, int32_t x, int32_t y, const int32_t* z, int32_t nz,
                                   double* out, int32_t* table_out, void* stream)
{
    if (!data || !arities || !out || (nz > 0 && !z)) return nfail(FBN_EINVAL, "null pointer argument");
    if (((uintptr_t)data & 15) || ld % 16 != 0 || ld < n_samples)
        return nfail(FBN_EINVAL, "data must be 16-byte aligned with a row stride ld >= n_samples, ld %% 16 == 0");
    if (n_vars < 2 || n_samples < 1 || n_samples >= (1LL << 31))
        return nfail(FBN_EINVAL, "n_vars=%d or n_samples=%lld out of range", n_vars, (long long)n_samples);
    if (x < 0 || x >= n_vars || y < 0 || y >= n_vars || x == y) return nfail(FBN_EINVAL, "bad x=%d y=%d", x, y);
    if (nz < 0 || nz > kMaxD) return nfail(FBN_EINVAL, "conditioning set size %d outside [0, %d]", nz, kMaxD);
    TestSpec spec{};
    long long cells = 1;
    for (int k = 0; k < nz; ++k) {
        if (z[k] < 0 || z[k] >= n_vars || z[k] == x || z[k] == y) return nfail(FBN_EINVAL, "bad conditioning variable %d", z[k]);
        for (int l = 0; l < k; ++l)
            if (z[l] == z[k]) return nfail(FBN_EINVAL, "conditioning variable %d repeated", z[k]);
        spec.rows[k] = data + (long long)z[k] * ld;
        spec.rad[k] = arities[z[k]];
    }
    spec.rows[nz] = data + (long long)x * ld;
    spec.rad[nz] = arities[x];
    spec.rows[nz + 1] = data + (long long)y * ld;
    spec.rad[nz + 1] = arities[y];
    for (int k = 0; k < nz + 2; ++k) {
        if (spec.rad[k] < 2) return nfail(FBN_EINVAL, "arity below 2");
        cells *= spec.rad[k];
        if (cells > kNoAllocMaxCells)
            return nfail(FBN_ETOOBIG, "table of more than %lld cells: fbn_ci_test_noalloc takes at most %lld",
                         cells, kNoAllocMaxCells);
    }
    spec.nrows = nz + 2;
    spec.rx = arities[x];
    spec.ry = arities[y];
    spec.N = (int)n_samples;
    spec.cells = cells;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices)
        return nfail(FBN_ECUDA, "no usable current CUDA device");
    int* scratch = nullptr;
    {
        // first call on this device: look up the device address of the scratch
        // array and raise the kernel's shared-memory limit
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_ready[dev]) {
            cudaError_t e = cudaGetSymbolAddress((void**)&g_scratch[dev], g_noalloc_scratch);
            if (e != cudaSuccess) return nfail(FBN_ECUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
            e = cudaFuncSetAttribute(k_ci_noalloc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kNoAllocSmem);
            if (e != cudaSuccess) return nfail(FBN_ECUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
            g_ready[dev] = true;
        }
        scratch = g_scratch[dev];
    }
    k_ci_noalloc<<<1, kTestThreads, kNoAllocSmem, (cudaStream_t)stream>>>(spec, scratch, out, table_out,
                                                                         (int)(kNoAllocSmem / 4));
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return nfail(FBN_ECUDA, "launch: %s", cudaGetErrorString(e));
    return FBN_OK;
}
