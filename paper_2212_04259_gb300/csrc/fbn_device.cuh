// fbn_device.cuh -- CTA-level conditional-independence test for sm_103a:
// contingency counts over all samples, marginals, G^2 (FP64 terms) and the
// chi-square p-value, plus the lexicographic unranking of conditioning sets.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "fbn_internal.cuh"

namespace fbn {

// --------------------------------------------------------------------------
// Chi-square survival function Q(df/2, g2/2) in FP64.
// Series for the lower regularised gamma P (Abramowitz & Stegun 6.5.29) when
// x < a + 1, else the continued fraction for the upper one (A&S 6.5.31)
// evaluated with the modified Lentz method.  lgamma/log/exp are CUDA's.
__device__ __forceinline__ double chisq_q(double df, double g2, unsigned* status)
{
    if (!(g2 > 0.0)) return 1.0;
    const double a = 0.5 * df, x = 0.5 * g2;
    const double log_pref = a * log(x) - x - lgamma(a);   // ln(x^a e^-x / Gamma(a))
    const int kMaxIt = 1 << 20;
    const double kEps = 5e-16, kTiny = 1e-300;
    if (x < a + 1.0) {
        double term = 1.0 / a, sum = term, den = a;
        int it = 0;
        for (; it < kMaxIt; ++it) {
            den += 1.0;
            term *= x / den;
            sum += term;
            if (term < sum * kEps) break;
        }
        if (it == kMaxIt) atomicOr(status, kStatusNumeric);
        const double q = 1.0 - sum * exp(log_pref);
        return q < 0.0 ? 0.0 : q;
    }
    double b = x + 1.0 - a, c = 1.0 / kTiny, d = 1.0 / b, h = d;
    int i = 1;
    for (; i < kMaxIt; ++i) {
        const double an = -(double)i * ((double)i - a);
        b += 2.0;
        d = an * d + b;
        if (fabs(d) < kTiny) d = kTiny;
        c = b + an / c;
        if (fabs(c) < kTiny) c = kTiny;
        d = 1.0 / d;
        const double del = d * c;
        h *= del;
        if (fabs(del - 1.0) < kEps) break;
    }
    if (i == kMaxIt) atomicOr(status, kStatusNumeric);
    const double q = exp(log_pref) * h;
    return q > 1.0 ? 1.0 : q;
}

// --------------------------------------------------------------------------
// Conditioning sets on the fly (Section IV-C): the r-th q-subset of {0..p-1}
// in lexicographic order, from a table of binomials B[n][k] = C(n, k).
__device__ __forceinline__ long long binom_at(const long long* B, int n, int k)
{
    if (k < 0 || n < k) return 0;
    return B[(long long)n * kBinomCols + k];
}

__device__ __forceinline__ void unrank_lex(long long r, int p, int q, const long long* B, int* out)
{
    int c = 0;
    for (int k = 0; k < q; ++k) {
        if (k == q - 1) {            // last position: one subset per candidate
            out[k] = c + (int)r;
            return;
        }
        for (;;) {
            const long long cnt = binom_at(B, p - c - 1, q - k - 1);
            if (r < cnt) break;
            r -= cnt;
            ++c;
        }
        out[k] = c++;
    }
}

// Next q-subset of {0..p-1} in lexicographic order; false after the last.
__device__ __forceinline__ bool next_subset(int p, int q, int* c)
{
    int k = q - 1;
    while (k >= 0 && c[k] == p - q + k) --k;
    if (k < 0) return false;
    c[k] += 1;
    for (int l = k + 1; l < q; ++l) c[l] = c[l - 1] + 1;
    return true;
}

// --------------------------------------------------------------------------
// One CI test, described in shared memory by the CTA's leader.
// rows = [S_0 .. S_{d-1}, X, Y]; the cell of a sample is the mixed-radix
// number of its values in that order: ((z * r_x + x) * r_y + y).
struct TestSpec {
    const uint8_t* rows[kMaxRows];
    int rad[kMaxRows];
    int nrows;        // d + 2
    int rx, ry;
    int N;
    long long cells;  // prod of all radices
};

struct TestResult {
    double g2, df, p;
};

enum CountMode { kLane = 0, kWarp = 1, kCta = 2, kGlobal = 3 };

__device__ __forceinline__ unsigned byte_of(const uint4& w, int b)
{
    const unsigned word = (b < 4) ? w.x : (b < 8) ? w.y : (b < 12) ? w.z : w.w;
    return (word >> ((b & 3) * 8)) & 0xFFu;
}

template <int MODE>
__device__ __forceinline__ void bump(int* base, unsigned idx)
{
    if (MODE == kLane) base[idx * 32u] += 1;        // lane-private column: no race, no atomic
    else atomicAdd(base + idx, 1);
}

// Count 16-sample vectors (16-byte loads of every row) plus the ragged tail.
// NR > 0: number of rows known at compile time; NR == 0: runtime s.nrows.
template <int NR, int MODE>
__device__ __forceinline__ void count_samples(const TestSpec& s, int* base)
{
    const int nvec = s.N >> 4;
    if (NR > 0) {
        const uint4* r[NR > 0 ? NR : 1];
        unsigned rad[NR > 0 ? NR : 1];
#pragma unroll
        for (int k = 0; k < NR; ++k) {
            r[k] = reinterpret_cast<const uint4*>(s.rows[k]);
            rad[k] = (unsigned)s.rad[k];
        }
        for (int v = threadIdx.x; v < nvec; v += blockDim.x) {
            uint4 w[NR > 0 ? NR : 1];
#pragma unroll
            for (int k = 0; k < NR; ++k) w[k] = __ldg(r[k] + v);
            unsigned idx[16];
#pragma unroll
            for (int b = 0; b < 16; ++b) idx[b] = byte_of(w[0], b);
#pragma unroll
            for (int k = 1; k < NR; ++k)
#pragma unroll
                for (int b = 0; b < 16; ++b) idx[b] = idx[b] * rad[k] + byte_of(w[k], b);
#pragma unroll
            for (int b = 0; b < 16; ++b) bump<MODE>(base, idx[b]);
        }
    } else {
        const int nr = s.nrows;
        for (int v = threadIdx.x; v < nvec; v += blockDim.x) {
            uint4 w = __ldg(reinterpret_cast<const uint4*>(s.rows[0]) + v);
            unsigned idx[16];
#pragma unroll
            for (int b = 0; b < 16; ++b) idx[b] = byte_of(w, b);
            for (int k = 1; k < nr; ++k) {
                w = __ldg(reinterpret_cast<const uint4*>(s.rows[k]) + v);
                const unsigned rk = (unsigned)s.rad[k];
#pragma unroll
                for (int b = 0; b < 16; ++b) idx[b] = idx[b] * rk + byte_of(w, b);
            }
#pragma unroll
            for (int b = 0; b < 16; ++b) bump<MODE>(base, idx[b]);
        }
    }
    for (int t = (nvec << 4) + threadIdx.x; t < s.N; t += blockDim.x) {
        unsigned idx = s.rows[0][t];
        for (int k = 1; k < s.nrows; ++k) idx = idx * (unsigned)s.rad[k] + s.rows[k][t];
        bump<MODE>(base, idx);
    }
}

template <int MODE>
__device__ __forceinline__ void count_dispatch(const TestSpec& s, int* base)
{
    switch (s.nrows) {
        case 2: count_samples<2, MODE>(s, base); break;
        case 3: count_samples<3, MODE>(s, base); break;
        case 4: count_samples<4, MODE>(s, base); break;
        case 5: count_samples<5, MODE>(s, base); break;
        case 6: count_samples<6, MODE>(s, base); break;
        default: count_samples<0, MODE>(s, base); break;
    }
}

__device__ __forceinline__ double block_sum(double v, double* red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (warp == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        t = lane < nw ? red[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    }
    return t;  // valid in thread 0
}

// Pick the counting strategy from the table size and the shared-memory budget.
__device__ __forceinline__ int pick_mode(long long C, long long marg, int smem_ints, int nwarps)
{
    if (C * 32 * nwarps + C + marg <= smem_ints) return kLane;
    if (C * nwarps + marg <= smem_ints) return kWarp;
    if (C + marg <= smem_ints) return kCta;
    return kGlobal;
}

// The whole test, run by every thread of the CTA.  smem: smem_ints ints of
// dynamic shared memory; gtab: this CTA's global scratch (gtab_ints ints) for
// tables that do not fit; table_out: optional copy of the final counts.
// Returns the result in thread 0 (and writes it to *res when non-null).
__device__ TestResult run_test(const TestSpec& s, int* smem, int smem_ints, int* gtab,
                               long long gtab_ints, int32_t* table_out, unsigned* status,
                               double* red)
{
    const long long C = s.cells;
    const int rxy = s.rx * s.ry;
    const long long nz = C / rxy;
    const long long marg = nz * (s.rx + s.ry + 1);
    const int nw = blockDim.x >> 5;
    int mode = pick_mode(C, marg, smem_ints, nw);
    if (mode == kGlobal && C + marg > gtab_ints) {
        if (threadIdx.x == 0) atomicOr(status, kStatusTooBig);
        TestResult bad = {0.0, 0.0, 0.0};
        return bad;
    }
    int* cnt;
    long long zero_n;
    if (mode == kLane) { cnt = smem; zero_n = C * 32 * nw; }
    else if (mode == kWarp) { cnt = smem; zero_n = C * nw; }
    else if (mode == kCta) { cnt = smem; zero_n = C; }
    else { cnt = gtab; zero_n = C; }
    for (long long k = threadIdx.x; k < zero_n; k += blockDim.x) cnt[k] = 0;
    __syncthreads();

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    switch (mode) {
        case kLane: count_dispatch<kLane>(s, cnt + (long long)warp * C * 32 + lane); break;
        case kWarp: count_dispatch<kWarp>(s, cnt + (long long)warp * C); break;
        default: count_dispatch<kCta>(s, cnt); break;   // shared or global table
    }
    __syncthreads();

    // Merge the private copies into one table T.
    int* T;
    int* M;   // marginals: Nxz [nz*rx], Nyz [nz*ry], Nzz [nz]
    if (mode == kLane) {
        T = smem + C * 32 * nw;
        for (long long c = threadIdx.x; c < C; c += blockDim.x) {
            int sum = 0;
            for (int w = 0; w < nw; ++w) {
                const int* col = cnt + ((long long)w * C + c) * 32;
#pragma unroll 8
                for (int l = 0; l < 32; ++l) sum += col[(l + (int)c) & 31];
            }
            T[c] = sum;
        }
        M = T + C;
    } else if (mode == kWarp) {
        T = cnt;
        for (long long c = threadIdx.x; c < C; c += blockDim.x) {
            int sum = 0;
            for (int w = 0; w < nw; ++w) sum += cnt[(long long)w * C + c];
            T[c] = sum;
        }
        M = smem + C * nw;
    } else if (mode == kCta) {
        T = cnt;
        M = smem + C;
    } else {
        T = cnt;
        M = (marg <= smem_ints) ? smem : gtab + C;
    }
    __syncthreads();

    int* Nxz = M;
    int* Nyz = M + nz * s.rx;
    int* Nzz = Nyz + nz * s.ry;
    for (long long k = threadIdx.x; k < nz * s.rx; k += blockDim.x) {
        int sum = 0;
        for (int y = 0; y < s.ry; ++y) sum += T[k * s.ry + y];
        Nxz[k] = sum;
    }
    for (long long k = threadIdx.x; k < nz * s.ry; k += blockDim.x) {
        const long long z = k / s.ry;
        const int y = (int)(k - z * s.ry);
        int sum = 0;
        for (int x = 0; x < s.rx; ++x) sum += T[(z * s.rx + x) * s.ry + y];
        Nyz[k] = sum;
    }
    __syncthreads();
    for (long long z = threadIdx.x; z < nz; z += blockDim.x) {
        int sum = 0;
        for (int x = 0; x < s.rx; ++x) sum += Nxz[z * s.rx + x];
        Nzz[z] = sum;
    }
    __syncthreads();

    // G^2 = 2 sum N ln(N / E): the ratio N / E = (N_xyz N_++z) / (N_x+z N_+yz)
    // is formed in exact 64-bit integers and its log taken as log1p of the
    // exact difference over the denominator.
    double acc = 0.0;
    for (long long c = threadIdx.x; c < C; c += blockDim.x) {
        const int n = T[c];
        if (table_out) table_out[c] = n;
        if (n == 0) continue;
        const long long z = c / rxy;
        const int rem = (int)(c - z * rxy);
        const int x = rem / s.ry, y = rem - x * s.ry;
        const long long a = (long long)n * Nzz[z];
        const long long b = (long long)Nxz[z * s.rx + x] * Nyz[z * s.ry + y];
        acc += (double)n * log1p((double)(a - b) / (double)b);
    }
    const double tot = block_sum(acc, red);
    TestResult r = {0.0, 0.0, 1.0};
    if (threadIdx.x == 0) {
        r.g2 = 2.0 * tot;
        r.df = (double)(s.rx - 1) * (double)(s.ry - 1) * (double)nz;
        r.p = chisq_q(r.df, r.g2, status);
    }
    return r;
}

}  // namespace fbn
