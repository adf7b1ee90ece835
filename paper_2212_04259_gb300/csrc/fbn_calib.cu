// fbn_calib.cu -- fbn_measure_unit_rates: the throughput of the two units that
// bound the contingency counts, measured on the device, so that the counting
// kernels can be reported against a measured peak instead of a nominal one.
//
//   * shared-memory reductions: red.shared.add on 32-bit words, every thread
//     on its own column (no bank conflicts, no contention) -- the operation the
//     byte histograms of the work pool issue once per sample;
//   * POPC: independent population counts -- the operation the bit-plane
//     count issues once per cell and 32 samples.
//
// Each kernel runs a few milliseconds over every SM (8 CTAs of 256 threads per
// SM), timed with CUDA events after a warm-up launch; the reductions are
// timed for tables of 8 and 32 cells and the faster rate is the peak.  Every
// index stays inside its buffer: the reduction kernel's columns are warp * C *
// 32 + lane + cell * 32 with cell < C, inside C * 256 words.
#include <cstdio>

#include <cuda_runtime.h>

#include "../../include/fbn.h"
#include "fbn_launch.h"

namespace {

constexpr int kCalThreads = 256;
constexpr int kCalMaxCells = 32;   // table sizes tried: 8 and 32 cells (powers of two)

// cells: run-time table size, a power of two <= kCalMaxCells; dynamic shared
// memory of cells * kCalThreads words.  The cells come from the bytes of two
// xorshift words (8 independent reductions per step, a few integer
// instructions each), so the reductions, not the index arithmetic, bound it.
__global__ void __launch_bounds__(kCalThreads) k_cal_red(const unsigned* seed, unsigned* out, int iters, int cells)
{
    extern __shared__ int col[];
    for (int k = threadIdx.x; k < cells * kCalThreads; k += blockDim.x) col[k] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int* base = col + warp * cells * 32 + lane;
    const unsigned mask = (unsigned)cells - 1u;
    unsigned x = (seed[lane] ^ blockIdx.x) | 1u, y = x * 2654435761u + 1u;
    for (int i = 0; i < iters; ++i) {
        x ^= x << 13; x ^= x >> 17; x ^= x << 5;
        y ^= y << 13; y ^= y >> 17; y ^= y << 5;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            atomicAdd(base + ((x >> (8 * k)) & mask) * 32, 1);
            atomicAdd(base + ((y >> (8 * k)) & mask) * 32, 1);
        }
    }
    __syncthreads();
    int s = 0;
    for (int k = threadIdx.x; k < cells * kCalThreads; k += blockDim.x) s += col[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = (unsigned)s;
}

__global__ void __launch_bounds__(kCalThreads) k_cal_popc(const unsigned* seed, unsigned* out, int iters)
{
    unsigned v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = seed[(threadIdx.x + k) & 31] ^ (blockIdx.x * 131u + (unsigned)k);
    unsigned s = 0;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            s += (unsigned)__popc(v[k]);
            v[k] = v[k] * 0x9E3779B9u + (unsigned)i;
        }
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

int cal_fail(const char* what, cudaError_t e)
{
    char buf[256];
    snprintf(buf, sizeof buf, "fbn_measure_unit_rates: %s: %s", what, cudaGetErrorString(e));
    fbn::fbn_internal_set_error(buf);
    return e == cudaErrorMemoryAllocation ? FBN_ENOMEM : FBN_ECUDA;
}

}  // namespace

extern "C" int fbn_measure_unit_rates(int32_t device, double* out, int32_t n_out)
{
    if (!out || n_out < 4) {
        fbn::fbn_internal_set_error("fbn_measure_unit_rates: out must hold 4 doubles");
        return FBN_EINVAL;
    }
    int prev = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&prev)) != cudaSuccess) return cal_fail("cudaGetDevice", e);
    if (device >= 0 && (e = cudaSetDevice(device)) != cudaSuccess) return cal_fail("cudaSetDevice", e);
    int dev = 0, sms = 0, khz = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev);
    const int blocks = sms * 8;
    unsigned *seed = nullptr, *sink = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = FBN_OK;
    float ms_red = 0.f, ms_popc = 0.f, best_red = 1e30f;
    const int it_red = 4000, it_popc = 8000;
    do {
        if ((e = cudaMalloc(&seed, 32 * sizeof(unsigned))) != cudaSuccess) { rc = cal_fail("cudaMalloc", e); break; }
        if ((e = cudaMalloc(&sink, (size_t)blocks * kCalThreads * sizeof(unsigned))) != cudaSuccess) {
            rc = cal_fail("cudaMalloc", e);
            break;
        }
        if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess) { rc = cal_fail("stream", e); break; }
        if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
            rc = cal_fail("event", e);
            break;
        }
        cudaMemsetAsync(seed, 0x5A, 32 * sizeof(unsigned), st);
        if ((e = cudaFuncSetAttribute(k_cal_red, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      kCalMaxCells * kCalThreads * (int)sizeof(int))) != cudaSuccess) {
            rc = cal_fail("cudaFuncSetAttribute", e);
            break;
        }
        for (int rep = 0; rep < 2; ++rep) {   // the first pass warms up
            for (int cells : {8, kCalMaxCells}) {
                cudaEventRecord(e0, st);
                k_cal_red<<<blocks, kCalThreads, cells * kCalThreads * sizeof(int), st>>>(seed, sink, it_red, cells);
                cudaEventRecord(e1, st);
                cudaEventSynchronize(e1);
                cudaEventElapsedTime(&ms_red, e0, e1);
                if (rep == 1 && ms_red < best_red) best_red = ms_red;
            }
            cudaEventRecord(e0, st);
            k_cal_popc<<<blocks, kCalThreads, 0, st>>>(seed, sink, it_popc);
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
            cudaEventElapsedTime(&ms_popc, e0, e1);
        }
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess || (e = cudaGetLastError()) != cudaSuccess) {
            rc = cal_fail("kernels", e);
            break;
        }
        const double threads = (double)blocks * kCalThreads;
        out[0] = threads * it_red * 8.0 / (best_red * 1e-3);   // shared-memory reductions per second
        out[1] = threads * it_popc * 8.0 / (ms_popc * 1e-3);   // POPC per second
        out[2] = (double)sms;
        out[3] = (double)khz * 1e3;                            // the device's reported SM clock (Hz)
    } while (0);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    cudaFree(seed);
    cudaFree(sink);
    cudaSetDevice(prev);
    return rc;
}
