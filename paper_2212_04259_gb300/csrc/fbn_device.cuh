// fbn_device.cuh -- group-level conditional-independence test for sm_103a:
// contingency counts over all samples, marginals, G^2 and the decision
// against alpha, plus the lexicographic unranking of conditioning sets.
//
// A "group" is the set of threads that runs one test: one warp (G = 32) or a
// whole CTA (G = kTestThreads).  Warp groups let many small tests run
// concurrently on an SM so that the latency of one test's setup and epilogue
// is hidden by the others; CTA groups serve tables too big for a warp's share
// of shared memory.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "fbn_internal.cuh"

namespace fbn {

// --------------------------------------------------------------------------
// Chi-square survival function Q(df/2, g2/2) in FP64.
// Series for the lower regularised gamma P (Abramowitz & Stegun 6.5.29) when
// x < a + 1, else the continued fraction for the upper one (A&S 6.5.31)
// evaluated with the modified Lentz method.  lgamma/log/exp are CUDA's.  An
// iteration cap sets kStatusNumeric in *status (and *capped when given).
__device__ __forceinline__ double chisq_q(double df, double g2, unsigned* status, bool* capped = nullptr)
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
        if (it == kMaxIt) {
            atomicOr(status, kStatusNumeric);
            if (capped) *capped = true;
        }
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
    if (i == kMaxIt) {
        atomicOr(status, kStatusNumeric);
        if (capped) *capped = true;
    }
    const double q = exp(log_pref) * h;
    return q > 1.0 ? 1.0 : q;
}

// Critical value of the test: the G^2 at which Q(df/2, G^2/2) = alpha.  Q is
// strictly decreasing in G^2, so "p > alpha" is exactly "G^2 < crit".  Found
// by a safeguarded Newton iteration inside a bracket [lo, hi] with Q(lo) >
// alpha >= Q(hi); the derivative of Q in G^2 is minus the chi-square density.
__device__ __forceinline__ double chisq_crit(double df, double alpha, unsigned* status, bool* capped = nullptr)
{
    const double a = 0.5 * df;
    double lo = 0.0, hi = df + 10.0 * sqrt(2.0 * df) + 40.0;
    for (int k = 0; k < 64 && chisq_q(df, hi, status, capped) > alpha; ++k) {
        lo = hi;
        hi *= 2.0;
    }
    double x = 0.5 * (lo + hi);
    for (int it = 0; it < 200; ++it) {
        const double q = chisq_q(df, x, status, capped);
        if (q > alpha) lo = x; else hi = x;
        // density of chi^2_df at x: x^{a-1} e^{-x/2} / (2^a Gamma(a))
        const double lpdf = (a - 1.0) * log(x) - 0.5 * x - a * 0.6931471805599453 - lgamma(a);
        const double pdf = exp(lpdf);
        double nx = pdf > 0.0 ? x + (q - alpha) / pdf : 0.5 * (lo + hi);
        if (!(nx > lo && nx < hi)) nx = 0.5 * (lo + hi);
        if (fabs(nx - x) <= 1e-15 * x || hi - lo <= 1e-15 * hi) {
            x = nx;
            break;
        }
        x = nx;
    }
    return x;
}

// Critical values for one alpha.  Small df: a dense table whose slot holds 0
// until a test computes the value and stores it (the value is its own
// payload: a reader sees 0 or the value, and one that sees 0 computes it
// too; a value whose computation hit an iteration cap is never stored).
// Larger df: an open-addressing cache keyed by df; a slot is claimed with a
// CAS to -1, filled, then published with a release store of the key; readers
// that see -1 compute the value themselves.  No thread waits on another.
using CritTable = CritTableDev;

__device__ __forceinline__ long long ld_acquire(const long long* p)
{
    long long v;
    asm volatile("ld.acquire.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(long long* p, long long v)
{
    asm volatile("st.release.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ double crit_get(const CritTable& t, long long df, double alpha, unsigned* status)
{
    if (df < t.dense_n) {
        const double v = t.dense[df];
        if (v > 0.0) return v;
        bool capped = false;
        const double c = chisq_crit((double)df, alpha, status, &capped);
        if (!capped) {
            t.dense[df] = c;
            if (t.dense_f) t.dense_f[df] = make_float2(__double2float_rd(c), __double2float_ru(c));
        }
        return c;
    }
    unsigned h = (unsigned)(df * 0x9E3779B97F4A7C15ULL >> 40) & (unsigned)(t.cap - 1);
    for (int probe = 0; probe < 32; ++probe, h = (h + 1) & (unsigned)(t.cap - 1)) {
        const long long k = ld_acquire(t.keys + h);
        if (k == df) return t.vals[h];
        if (k == 0) {
            const double c = chisq_crit((double)df, alpha, status);
            if (atomicCAS((unsigned long long*)(t.keys + h), 0ULL, (unsigned long long)-1LL) == 0ULL) {
                t.vals[h] = c;
                st_release(t.keys + h, df);
            }
            return c;
        }
        if (k == -1) return chisq_crit((double)df, alpha, status);
    }
    return chisq_crit((double)df, alpha, status);
}

// --------------------------------------------------------------------------
// Conditioning sets on the fly (Section IV-C): the r-th q-subset of {0..p-1}
// in lexicographic order, from a table of binomials B[n][k] = C(n, k).
__device__ __forceinline__ long long binom_at(const long long* B, int n, int k)
{
    if (k < 0 || n < k) return 0;
    return __ldg(B + (long long)n * kBinomCols + k);
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
// One CI test as seen by its group, in shared memory.
// rows = [S_0 .. S_{d-1}, X, Y]; the cell of a sample is the mixed-radix
// number of its values in that order: ((z * r_x + x) * r_y + y).
struct TestSpec {
    const uint8_t* rows[kMaxRows];
    int rad[kMaxRows];
    int nrows;        // d + 2
    int rx, ry;
    int N;
    long long cells;  // product of all radices
    // bit planes of the first kBitsMaxD + 2 rows, at the test's first sample
    // (plane 0; plane 1 pstride uint4 further), or nullptr without planes
    const uint4* prow[kBitsMaxD + 2];
    long long pstride;
};

template <int G>
struct Grp {
    static_assert(G == 32 || G == 64 || G == 128 || G == kTestThreads, "group size");
    static constexpr int kWarps = G / 32;
    static __device__ __forceinline__ int rank() { return (int)(threadIdx.x % G); }
    static __device__ __forceinline__ int gid() { return (int)(threadIdx.x / G); }
    static __device__ __forceinline__ void sync()
    {
        if (G == 32) {
            __syncwarp();
        } else if (G == kTestThreads) {
            __syncthreads();
        } else {   // named barrier 1 + group index, G threads
            asm volatile("bar.sync %0, %1;" ::"r"(1 + gid()), "r"(G) : "memory");
        }
    }
};

// Sum over the group; every thread of the group gets the total.  red: the
// CTA's scratch of 32 entries, of which the group uses kWarps.
template <int G, typename T>
__device__ __forceinline__ T grp_sum(T v, T* red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (G == 32) return v;
    T* r = red + Grp<G>::gid() * Grp<G>::kWarps;
    Grp<G>::sync();
    if ((threadIdx.x & 31) == 0) r[Grp<G>::rank() >> 5] = v;
    Grp<G>::sync();
    T t = 0;
#pragma unroll
    for (int w = 0; w < Grp<G>::kWarps; ++w) t += r[w];
    return t;
}

// Two sums in one pass (red: the CTA's scratch of 32 doubles).
template <int G>
__device__ __forceinline__ void grp_sum2(double& a, double& b, double* red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if (G == 32) return;
    double* r = red + Grp<G>::gid() * 2 * Grp<G>::kWarps;
    Grp<G>::sync();
    if ((threadIdx.x & 31) == 0) {
        r[2 * (Grp<G>::rank() >> 5)] = a;
        r[2 * (Grp<G>::rank() >> 5) + 1] = b;
    }
    Grp<G>::sync();
    a = 0.0;
    b = 0.0;
#pragma unroll
    for (int w = 0; w < Grp<G>::kWarps; ++w) {
        a += r[2 * w];
        b += r[2 * w + 1];
    }
}

enum CountMode { kLane = 0, kWarp = 1, kShared = 2, kGlobal = 3, kLane16 = 4, kBits = 5 };

template <int MODE>
__device__ __forceinline__ void bump(int* base, unsigned idx)
{
    // kLane: this lane's private column, so no other thread touches the word;
    // the update is still a shared-memory reduction (red.shared.add) rather
    // than load-add-store, so consecutive samples do not wait on each other
    if (MODE == kLane) atomicAdd(base + idx * 32u, 1);
    else if (MODE == kLane16) atomicAdd(base + (idx >> 1) * 32u, 1 << ((idx & 1u) << 4));   // two 16-bit counters
    else atomicAdd(base + idx, 1);
}

// Count 16-sample vectors (one 16-byte load per row) plus the ragged tail.
// The cell index of two samples is carried in the two 16-bit halves of one
// 32-bit register (every partial index is below cells <= 65536), so one IMAD
// advances two samples.  NR > 0: rows known at compile time; NR == 0: runtime.
template <int NR>
__device__ __forceinline__ void pack_vector(const TestSpec& s, const uint4* w, unsigned* acc)
{
    {
        const unsigned ws[4] = {w[0].x, w[0].y, w[0].z, w[0].w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            acc[2 * q] = __byte_perm(ws[q], 0u, 0x4140);      // bytes 0,1 -> halves
            acc[2 * q + 1] = __byte_perm(ws[q], 0u, 0x4342);  // bytes 2,3 -> halves
        }
    }
#pragma unroll
    for (int k = 1; k < NR; ++k) {
        const unsigned rk = (unsigned)s.rad[k];
        const unsigned ws[4] = {w[k].x, w[k].y, w[k].z, w[k].w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            acc[2 * q] = acc[2 * q] * rk + __byte_perm(ws[q], 0u, 0x4140);
            acc[2 * q + 1] = acc[2 * q + 1] * rk + __byte_perm(ws[q], 0u, 0x4342);
        }
    }
}

template <int MODE>
__device__ __forceinline__ void bump_packed(int* base, const unsigned* acc)
{
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        bump<MODE>(base, acc[q] & 0xFFFFu);
        bump<MODE>(base, acc[q] >> 16);
    }
}

// Count 16-sample vectors (one 16-byte load per row) plus the ragged tail.
// The cell index of two samples is carried in the two 16-bit halves of one
// 32-bit register (every partial index is below cells <= 65536), so one IMAD
// advances two samples.  Two vectors are loaded before either is counted, to
// keep 2 (d + 2) loads in flight per thread.  NR > 0: rows known at compile
// time; NR == 0: runtime.
template <int G, int NR, int MODE>
__device__ __forceinline__ void count_packed(const TestSpec& s, int* base)
{
    const int nvec = s.N >> 4;
    const int t0 = Grp<G>::rank();
    const int nr = NR > 0 ? NR : s.nrows;
    if (NR > 0) {
        const uint4* r[NR > 0 ? NR : 1];
#pragma unroll
        for (int k = 0; k < NR; ++k) r[k] = reinterpret_cast<const uint4*>(s.rows[k]);
        int v = t0;
        for (; v + G < nvec; v += 2 * G) {
            uint4 w0[NR > 0 ? NR : 1], w1[NR > 0 ? NR : 1];
#pragma unroll
            for (int k = 0; k < NR; ++k) {
                w0[k] = __ldg(r[k] + v);
                w1[k] = __ldg(r[k] + v + G);
            }
            if (v + 3 * G < nvec) {   // the next iteration's lines into L1 while these are counted
#pragma unroll
                for (int k = 0; k < NR; ++k) {
                    asm volatile("prefetch.global.L1 [%0];" ::"l"(r[k] + v + 2 * G));
                    asm volatile("prefetch.global.L1 [%0];" ::"l"(r[k] + v + 3 * G));
                }
            }
            unsigned acc[8];
            pack_vector<NR>(s, w0, acc);
            bump_packed<MODE>(base, acc);
            pack_vector<NR>(s, w1, acc);
            bump_packed<MODE>(base, acc);
        }
        if (v < nvec) {
            uint4 w0[NR > 0 ? NR : 1];
#pragma unroll
            for (int k = 0; k < NR; ++k) w0[k] = __ldg(r[k] + v);
            unsigned acc[8];
            pack_vector<NR>(s, w0, acc);
            bump_packed<MODE>(base, acc);
        }
    } else {
        for (int v = t0; v < nvec; v += G) {
            unsigned acc[8];
            {
                const uint4 w = __ldg(reinterpret_cast<const uint4*>(s.rows[0]) + v);
                const unsigned ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    acc[2 * q] = __byte_perm(ws[q], 0u, 0x4140);
                    acc[2 * q + 1] = __byte_perm(ws[q], 0u, 0x4342);
                }
            }
            for (int k = 1; k < nr; ++k) {
                const uint4 w = __ldg(reinterpret_cast<const uint4*>(s.rows[k]) + v);
                const unsigned rk = (unsigned)s.rad[k];
                const unsigned ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    acc[2 * q] = acc[2 * q] * rk + __byte_perm(ws[q], 0u, 0x4140);
                    acc[2 * q + 1] = acc[2 * q + 1] * rk + __byte_perm(ws[q], 0u, 0x4342);
                }
            }
            bump_packed<MODE>(base, acc);
        }
    }
    for (int t = (nvec << 4) + t0; t < s.N; t += G) {
        unsigned idx = s.rows[0][t];
        for (int k = 1; k < nr; ++k) idx = idx * (unsigned)s.rad[k] + s.rows[k][t];
        bump<MODE>(base, idx);
    }
}

// Same, one sample per 32-bit index (tables above 65536 cells).
template <int G, int MODE>
__device__ __forceinline__ void count_wide(const TestSpec& s, int* base)
{
    const int nvec = s.N >> 4;
    const int t0 = Grp<G>::rank();
    for (int v = t0; v < nvec; v += G) {
        unsigned idx[16];
        {
            const uint4 w = __ldg(reinterpret_cast<const uint4*>(s.rows[0]) + v);
            const unsigned ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
            for (int b = 0; b < 16; ++b) idx[b] = (ws[b >> 2] >> ((b & 3) * 8)) & 0xFFu;
        }
        for (int k = 1; k < s.nrows; ++k) {
            const uint4 w = __ldg(reinterpret_cast<const uint4*>(s.rows[k]) + v);
            const unsigned rk = (unsigned)s.rad[k];
            const unsigned ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
            for (int b = 0; b < 16; ++b) idx[b] = idx[b] * rk + ((ws[b >> 2] >> ((b & 3) * 8)) & 0xFFu);
        }
#pragma unroll
        for (int b = 0; b < 16; ++b) bump<MODE>(base, idx[b]);
    }
    for (int t = (nvec << 4) + t0; t < s.N; t += G) {
        unsigned idx = s.rows[0][t];
        for (int k = 1; k < s.nrows; ++k) idx = idx * (unsigned)s.rad[k] + s.rows[k][t];
        bump<MODE>(base, idx);
    }
}

// Tables of at most 256 cells: every partial index of a sample fits one byte,
// so the four samples of a 32-bit word advance together in its four bytes --
// acc * r_k + row_k never carries out of a byte because the result stays below
// the cells counted so far.  One IMAD per row and 4 samples, then one byte
// extraction per sample.
template <int MODE>
__device__ __forceinline__ void bump_bytes(int* base, unsigned acc)
{
    bump<MODE>(base, __byte_perm(acc, 0u, 0x4440));
    bump<MODE>(base, __byte_perm(acc, 0u, 0x4441));
    bump<MODE>(base, __byte_perm(acc, 0u, 0x4442));
    bump<MODE>(base, __byte_perm(acc, 0u, 0x4443));
}

template <int G, int NR, int MODE>
__device__ __forceinline__ void count_bytes(const TestSpec& s, int* base)
{
    const int nvec = s.N >> 4;
    const int t0 = Grp<G>::rank();
    const uint4* r[NR];
    unsigned rad[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) {
        r[k] = reinterpret_cast<const uint4*>(s.rows[k]);
        rad[k] = (unsigned)s.rad[k];
    }
    int v = t0;
    for (; v + G < nvec; v += 2 * G) {
        uint4 w0[NR], w1[NR];
#pragma unroll
        for (int k = 0; k < NR; ++k) {
            w0[k] = __ldg(r[k] + v);
            w1[k] = __ldg(r[k] + v + G);
        }
        if (v + 3 * G < nvec) {   // the next iteration's lines into L1 while these are counted
#pragma unroll
            for (int k = 0; k < NR; ++k) {
                asm volatile("prefetch.global.L1 [%0];" ::"l"(r[k] + v + 2 * G));
                asm volatile("prefetch.global.L1 [%0];" ::"l"(r[k] + v + 3 * G));
            }
        }
        uint4 a0 = w0[0], a1 = w1[0];
#pragma unroll
        for (int k = 1; k < NR; ++k) {
            a0.x = a0.x * rad[k] + w0[k].x; a0.y = a0.y * rad[k] + w0[k].y;
            a0.z = a0.z * rad[k] + w0[k].z; a0.w = a0.w * rad[k] + w0[k].w;
            a1.x = a1.x * rad[k] + w1[k].x; a1.y = a1.y * rad[k] + w1[k].y;
            a1.z = a1.z * rad[k] + w1[k].z; a1.w = a1.w * rad[k] + w1[k].w;
        }
        bump_bytes<MODE>(base, a0.x); bump_bytes<MODE>(base, a0.y);
        bump_bytes<MODE>(base, a0.z); bump_bytes<MODE>(base, a0.w);
        bump_bytes<MODE>(base, a1.x); bump_bytes<MODE>(base, a1.y);
        bump_bytes<MODE>(base, a1.z); bump_bytes<MODE>(base, a1.w);
    }
    if (v < nvec) {
        uint4 a = __ldg(r[0] + v);
#pragma unroll
        for (int k = 1; k < NR; ++k) {
            const uint4 w = __ldg(r[k] + v);
            a.x = a.x * rad[k] + w.x; a.y = a.y * rad[k] + w.y;
            a.z = a.z * rad[k] + w.z; a.w = a.w * rad[k] + w.w;
        }
        bump_bytes<MODE>(base, a.x); bump_bytes<MODE>(base, a.y);
        bump_bytes<MODE>(base, a.z); bump_bytes<MODE>(base, a.w);
    }
    for (int t = (nvec << 4) + t0; t < s.N; t += G) {
        unsigned idx = s.rows[0][t];
#pragma unroll
        for (int k = 1; k < NR; ++k) idx = idx * rad[k] + s.rows[k][t];
        bump<MODE>(base, idx);
    }
}

template <int G, int MODE>
__device__ __forceinline__ void count_dispatch(const TestSpec& s, int* base)
{
    if (s.cells > 65536) {
        count_wide<G, MODE>(s, base);
        return;
    }
    if (s.cells <= 256) {
        switch (s.nrows) {
            case 2: count_bytes<G, 2, MODE>(s, base); return;
            case 3: count_bytes<G, 3, MODE>(s, base); return;
            case 4: count_bytes<G, 4, MODE>(s, base); return;
            case 5: count_bytes<G, 5, MODE>(s, base); return;
            default: break;
        }
    }
    switch (s.nrows) {
        case 2: count_packed<G, 2, MODE>(s, base); break;
        case 3: count_packed<G, 3, MODE>(s, base); break;
        case 4: count_packed<G, 4, MODE>(s, base); break;
        case 5: count_packed<G, 5, MODE>(s, base); break;
        case 6: count_packed<G, 6, MODE>(s, base); break;
        default: count_packed<G, 0, MODE>(s, base); break;
    }
}

// --------------------------------------------------------------------------
// Counting from bit planes (every variable of the test has arity <= 4 and at
// most one conditioning variable: C = r_z r_x r_y <= 64 cells).  With the
// values' two bits held as 32-sample words per variable (plane 0: bit 0,
// plane 1: bit 1), the samples of a word that fall in cell (z, x, y) are the
// AND of one minterm of the planes per variable, and their count is one POPC
// of that AND: one LOP3 and one POPC per cell and 32 samples, where the byte
// histogram spends one shared-memory reduction per sample.
//
// A thread takes one 32-sample word of every plane at a time -- the next
// word's planes are loaded while the current one is counted -- and keeps the
// 64 cells of the fixed [z][x][y] = [4][4][4] layout as 16-bit counters packed
// two to a register (32 registers, indices known at compile time), so the
// sample loop touches no shared memory.  The strata and x loops stop at the
// test's arities; the y loop always runs its 4 values (a value the variable
// cannot take pops zero), which keeps the innermost loop free of branches
// (measured: skipping them by predication, or one loop copy per r_y, ran
// slower -- the kernel is sensitive to its code footprint).
// The one partial word at the end of the samples is peeled off with its
// validity mask.  A counter grows by at most 32 per word and a thread sees at
// most ceil(N / 32 / G) words: below 2^16 while N <= kBitsMaxN.
constexpr int kBitsWords = 32;   // counter words per thread: 4 strata x 4 x 2

__device__ __forceinline__ unsigned minterm1(unsigned m, unsigned p0, unsigned p1, int a)
{
    // m & [value == a] from the value's bit planes; a is a compile-time
    // constant wherever this is called from an unrolled loop (one LOP3)
    return m & ((a & 1) ? p0 : ~p0) & ((a & 2) ? p1 : ~p1);
}

// Counter word of cell (z, x, y) (the fold uses the same layout).
__host__ __device__ __forceinline__ int bits_word_of(int z, int x, int y)
{
    return z * 8 + x * 2 + (y >> 1);
}

struct BitsWord {
    unsigned x0, x1, y0, y1, z0, z1;
};

__device__ __forceinline__ BitsWord bits_load(const unsigned* __restrict__ xr, const unsigned* __restrict__ yr,
                                              const unsigned* __restrict__ zr, int ps, int w, int d)
{
    BitsWord b;
    b.x0 = __ldg(xr + w);
    b.x1 = __ldg(xr + ps + w);
    b.y0 = __ldg(yr + w);
    b.y1 = __ldg(yr + ps + w);
    b.z0 = d ? __ldg(zr + w) : 0u;
    b.z1 = d ? __ldg(zr + ps + w) : 0u;
    return b;
}

__device__ __forceinline__ void bits_count(unsigned* acc, const BitsWord& b, unsigned valid, int d, int rz, int rx)
{
#pragma unroll
    for (int c = 0; c < kBitsMaxArity; ++c) {
        if (c >= rz) break;
        const unsigned zm = d ? minterm1(valid, b.z0, b.z1, c) : valid;
#pragma unroll
        for (int a = 0; a < kBitsMaxArity; ++a) {
            if (a >= rx) break;
            const unsigned xa = minterm1(zm, b.x0, b.x1, a);
            const unsigned n0 = (unsigned)__popc(minterm1(xa, b.y0, b.y1, 0));
            const unsigned n1 = (unsigned)__popc(minterm1(xa, b.y0, b.y1, 1));
            const unsigned n2 = (unsigned)__popc(minterm1(xa, b.y0, b.y1, 2));
            const unsigned n3 = (unsigned)__popc(minterm1(xa, b.y0, b.y1, 3));
            acc[c * 8 + a * 2] += n0 + (n1 << 16);
            acc[c * 8 + a * 2 + 1] += n2 + (n3 << 16);
        }
    }
}

// cnt: this thread's column of kBitsWords counter words with stride G
// (bits_word_of layout).  Not inlined: one call per test, and the sample loop
// gets the kernel's whole register budget.  One body for every table shape:
// copies of the loop per arity (measured) ran slower than the POPC they save.
template <int G>
__device__ __noinline__ void count_bits(const TestSpec& s, int* cnt)
{
    const int rx = s.rx, d = s.nrows - 2;
    const int rz = d ? s.rad[0] : 1;
    const int nw = (s.N + 31) >> 5;
    const int full = s.N >> 5;             // words with every sample below N
    const int ps = (int)(4 * s.pstride);   // words per plane (< 2^26 for N <= kBitsMaxN)
    const unsigned* __restrict__ xr = reinterpret_cast<const unsigned*>(s.prow[d]);
    const unsigned* __restrict__ yr = reinterpret_cast<const unsigned*>(s.prow[d + 1]);
    const unsigned* __restrict__ zr = reinterpret_cast<const unsigned*>(s.prow[0]);
    unsigned acc[kBitsWords];
#pragma unroll
    for (int k = 0; k < kBitsWords; ++k) acc[k] = 0u;
    int w = Grp<G>::rank();
    if (w < full) {
        BitsWord cur = bits_load(xr, yr, zr, ps, w, d);
        for (;;) {
            const int wn = w + G;
            const bool more = wn < full;
            BitsWord nxt = cur;
            if (more) nxt = bits_load(xr, yr, zr, ps, wn, d);   // in flight while cur is counted
            bits_count(acc, cur, ~0u, d, rz, rx);
            w = wn;
            if (!more) break;
            cur = nxt;
        }
    }
    if (w == full && full < nw)
        bits_count(acc, bits_load(xr, yr, zr, ps, w, d), (1u << (s.N & 31)) - 1u, d, rz, rx);
#pragma unroll
    for (int k = 0; k < kBitsWords; ++k)
        if ((k >> 3) < rz) cnt[k * G] = (int)acc[k];
}

// Shared-memory ints needed by each counting strategy for a table of C cells
// (marg = marginal entries); kGlobal when none fits.  kLane16 (warp groups)
// packs two lane-private counters per word: a lane counts at most
// N / 32 + 16 samples, which must stay below 2^16.  Its extra zeroing and
// merge only pay off when the sample loop is long (measured: a gain at
// N = 100,000, a loss for the batched problems of 1,000-50,000 samples),
// hence N >= 65536.
template <int G>
__device__ __forceinline__ int pick_mode(long long C, long long marg, long long slice_ints, int N)
{
    // private copies cost their zeroing and folding (C words per copy); they
    // pay only while that stays below the samples counted (short sample
    // ranges: split tests, small problems, take fewer copies)
    if (C * G + C + marg <= slice_ints && C * G <= N) return kLane;
    if (G == 32 && N >= 65536 && N / 32 + 32 < 65536 && (C + 1) / 2 * 32 + C + marg <= slice_ints) return kLane16;
    if (Grp<G>::kWarps > 1 && C * Grp<G>::kWarps + marg <= slice_ints && 2 * C * Grp<G>::kWarps <= N) return kWarp;
    if (C + marg <= slice_ints) return kShared;
    return kGlobal;
}

// Count the table of the test and merge private copies.  Returns the merged
// table T and sets *M to the space for the marginals; returns nullptr when the
// table fits neither the slice nor the global scratch.  bits_cells: largest
// table counted from the bit planes when the test qualifies (0: never).
template <int G, bool BITS = false>
__device__ int* grp_table(const TestSpec& s, int* slice, long long slice_ints, int* gtab, long long gtab_ints,
                          int** M)
{
    const long long C = s.cells;
    const long long nz = C / (s.rx * s.ry);
    const long long marg = nz * (s.rx + s.ry + 1);
    // BITS: the caller admits only tests that bits_shape_ok accepts, whose
    // kBitsWords * G counter words, table and marginals fit the slice
    const int mode = BITS ? kBits : pick_mode<G>(C, marg, slice_ints, s.N);
    if (mode == kGlobal && (gtab == nullptr || C + marg > gtab_ints)) return nullptr;
    const int r = Grp<G>::rank();
    const int lane = threadIdx.x & 31;
    const int warp = r >> 5;                     // warp within the group
    constexpr int W = Grp<G>::kWarps;
    int* cnt = mode == kGlobal ? gtab : slice;
    const long long zero_n = BITS ? 0 : mode == kLane ? C * G : mode == kLane16 ? (C + 1) / 2 * 32
                                    : mode == kWarp ? C * W : C;
    for (int k = r; k < (int)zero_n; k += G) cnt[k] = 0;   // zero_n <= 2^27
    Grp<G>::sync();
    switch (mode) {
        case kLane: count_dispatch<G, kLane>(s, cnt + (long long)warp * C * 32 + lane); break;
        case kLane16: count_dispatch<G, kLane16>(s, cnt + lane); break;
        case kBits:
            if (BITS) count_bits<G>(s, cnt + r);   // writes every counter word the fold reads
            break;
        case kWarp: count_dispatch<G, kWarp>(s, cnt + (long long)warp * C); break;
        default: count_dispatch<G, kShared>(s, cnt); break;
    }
    Grp<G>::sync();
    int* T;
    if (BITS) {   // fold the G 16-bit columns of each cell (rotated start: no bank conflicts)
        T = slice + kBitsWords * G;
        const int rxy = s.rx * s.ry;
        for (int c = r; c < (int)C; c += G) {
            const int z = c / rxy, rem = c - z * rxy, x = rem / s.ry, y = rem - x * s.ry;
            const int* row = cnt + bits_word_of(z, x, y) * G;
            const int sh = (y & 1) * 16;
            int sum = 0;
#pragma unroll 8
            for (int l = 0; l < G; ++l) sum += (row[(l + c) & (G - 1)] >> sh) & 0xFFFF;
            T[c] = sum;
        }
        *M = T + C;
    } else if (mode == kLane16) {   // one warp: lane l folds the 32 columns of cells l, l + 32, ...
        T = slice + (C + 1) / 2 * 32;
        for (int c = lane; c < (int)C; c += 32) {
            const int* row = cnt + (c >> 1) * 32;
            const int sh = (int)(c & 1) * 16;
            int sum = 0;
#pragma unroll 8
            for (int l = 0; l < 32; ++l) sum += (row[(l + (int)c) & 31] >> sh) & 0xFFFF;
            T[c] = sum;
        }
        *M = T + C;
    } else if (mode == kLane) {
        // stage 1: each warp folds its 32 lane columns, lane l taking cells
        // c = l, l + 32, ...; the sum goes to column (c mod 32) of cell c's
        // row, which only that lane touches (and which keeps stage 2 free of
        // bank conflicts).  stage 2: fold the warps' partial sums.
        int* own = cnt + (long long)warp * C * 32;
        for (int c = lane; c < (int)C; c += 32) {
            const int* col = own + c * 32;
            int sum = 0;
#pragma unroll 8
            for (int l = 0; l < 32; ++l) sum += col[(l + (int)c) & 31];
            own[c * 32 + (c & 31)] = sum;
        }
        Grp<G>::sync();
        T = slice + C * G;
        for (int c = r; c < (int)C; c += G) {
            int sum = 0;
            for (int w = 0; w < W; ++w) sum += cnt[(w * (int)C + c) * 32 + (c & 31)];
            T[c] = sum;
        }
        *M = T + C;
    } else if (mode == kWarp) {
        T = cnt;
        for (int c = r; c < (int)C; c += G) {
            int sum = 0;
            for (int w = 0; w < W; ++w) sum += cnt[w * (int)C + c];
            T[c] = sum;
        }
        *M = slice + C * W;
    } else if (mode == kShared) {
        T = cnt;
        *M = slice + C;
    } else {
        T = cnt;
        *M = marg <= slice_ints ? slice : gtab + C;
    }
    Grp<G>::sync();
    return T;
}

// Marginals N_x+z [nz*rx], N_+yz [nz*ry], N_++z [nz] into M.
template <int G>
__device__ __forceinline__ void grp_marginals(const TestSpec& s, const int* T, int* M)
{
    // cells <= kMaxCells < 2^31: 32-bit indices throughout
    const int rx = s.rx, ry = s.ry;
    const int nz = (int)s.cells / (rx * ry);
    int* Nxz = M;
    int* Nyz = M + nz * rx;
    int* Nzz = Nyz + nz * ry;
    const int r = Grp<G>::rank();
    for (int k = r; k < nz * rx; k += G) {
        int sum = 0;
        for (int y = 0; y < ry; ++y) sum += T[k * ry + y];
        Nxz[k] = sum;
    }
    for (int k = r; k < nz * ry; k += G) {
        const int z = k / ry;
        const int y = k - z * ry;
        int sum = 0;
        for (int x = 0; x < rx; ++x) sum += T[(z * rx + x) * ry + y];
        Nyz[k] = sum;
    }
    Grp<G>::sync();
    for (int z = r; z < nz; z += G) {
        int sum = 0;
        for (int x = 0; x < rx; ++x) sum += Nxz[z * rx + x];
        Nzz[z] = sum;
    }
    Grp<G>::sync();
}

// Exact G^2 = 2 sum N ln(N / E) in FP64 (every thread of the group gets it).
// The ratio N / E = (N_xyz N_++z) / (N_x+z N_+yz) is formed in exact 64-bit
// integers and its log taken as log1p of the exact difference over the
// denominator.
template <int G>
__device__ __forceinline__ double grp_g2_exact(const TestSpec& s, const int* T, const int* M, double* red,
                                               int32_t* table_out)
{
    const int rx = s.rx, ry = s.ry, rxy = rx * ry, C = (int)s.cells;
    const int nz = C / rxy;
    const int* Nxz = M;
    const int* Nyz = M + nz * rx;
    const int* Nzz = Nyz + nz * ry;
    double acc = 0.0;
    for (int c = Grp<G>::rank(); c < C; c += G) {
        const int n = T[c];
        if (table_out) table_out[c] = n;
        if (n == 0) continue;
        const int z = c / rxy;
        const int rem = c - z * rxy;
        const int x = rem / ry, y = rem - x * ry;
        const long long a = (long long)n * Nzz[z];
        const long long b = (long long)Nxz[z * rx + x] * Nyz[z * ry + y];
        acc += (double)n * log1p((double)(a - b) / (double)b);
    }
    return 2.0 * grp_sum<G>(acc, red);
}

// CI-test statistics: G^2 (Section III-B) or Pearson's X^2 of the same table.
constexpr int kStatG2 = 0;
constexpr int kStatX2 = 1;

// Exact Pearson X^2 = sum (N - E)^2 / E in FP64 over cells with E > 0 (empty
// cells included), each term (N_xyz N_++z - N_x+z N_+yz)^2 / (N_++z N_x+z
// N_+yz) with the difference an exact 64-bit integer.
template <int G>
__device__ __forceinline__ double grp_x2_exact(const TestSpec& s, const int* T, const int* M, double* red,
                                               int32_t* table_out)
{
    const int rx = s.rx, ry = s.ry, rxy = rx * ry, C = (int)s.cells;
    const int nz = C / rxy;
    const int* Nxz = M;
    const int* Nyz = M + nz * rx;
    const int* Nzz = Nyz + nz * ry;
    double acc = 0.0;
    for (int c = Grp<G>::rank(); c < C; c += G) {
        const int n = T[c];
        if (table_out) table_out[c] = n;
        const int z = c / rxy;
        const int rem = c - z * rxy;
        const int x = rem / ry, y = rem - x * ry;
        const long long nx = Nxz[z * rx + x], ny = Nyz[z * ry + y];
        if (nx == 0 || ny == 0) continue;
        const double dd = (double)((long long)n * Nzz[z] - nx * ny);
        acc += dd * dd / ((double)Nzz[z] * (double)nx * (double)ny);
    }
    return grp_sum<G>(acc, red);
}

// Degrees of freedom of the observed table: sum over strata with N_++z > 0 of
// (values of X with N_x+z > 0 - 1)(values of Y with N_+yz > 0 - 1).
template <int G>
__device__ __forceinline__ long long grp_df_adjusted(const TestSpec& s, const int* M, double* red)
{
    const int rx = s.rx, ry = s.ry;
    const int nz = (int)s.cells / (rx * ry);
    const int* Nxz = M;
    const int* Nyz = M + nz * rx;
    double acc = 0.0;
    for (int z = Grp<G>::rank(); z < nz; z += G) {
        int ax = 0, ay = 0;
        for (int x = 0; x < rx; ++x) ax += Nxz[z * rx + x] > 0;
        for (int y = 0; y < ry; ++y) ay += Nyz[z * ry + y] > 0;
        if (ax > 0 && ay > 0) acc += (double)(ax - 1) * (double)(ay - 1);
    }
    return (long long)(grp_sum<G>(acc, red) + 0.5);
}

// One FP32 term of the bounded decisions.  G^2: n ln(N / E) with the ratio
// N / E = (n N_++z) / (N_x+z N_+yz) from exact 64-bit integers, its log taken
// as log1p of the exact difference over the denominator (n > 0).  X^2:
// (n N_++z - N_x+z N_+yz)^2 / (N_++z N_x+z N_+yz) with the difference exact,
// skipped when a margin is empty.
__device__ __forceinline__ void g2_term(int n, int nzz, int nx, int ny, float& acc, float& mag)
{
    const long long a = (long long)n * nzz;
    const long long b = (long long)nx * ny;
    const float fb = (float)b;
    const float delta = (float)(a - b) / fb;
    const float L = fabsf(delta) < 0.5f ? log1pf(delta) : logf((float)a / fb);
    const float t = (float)n * L;
    acc += t;
    mag += fabsf(t);
}

__device__ __forceinline__ void x2_term(int n, int nzz, int nx, int ny, float& acc)
{
    if (nx == 0 || ny == 0) return;
    const float fd = (float)((long long)n * nzz - (long long)nx * ny);
    acc += fd * fd / ((float)nzz * (float)nx * (float)ny);
}

// The bounded comparison shared by the FP32 decisions: sum = the group's FP32
// sum of the terms, mag = the sum of their magnitudes, per_thread = terms a
// thread added, levels = the depth of the cross-thread addition tree.  The
// error analysis is the one stated for grp_decide_bound below.  Returns 1
// (accept), 0 (reject) or -1 (the band straddles the bracket of crit).
__device__ __forceinline__ int decide_from_sums(float sum, float mag, float per_thread, float levels, int stat,
                                                float crit_lo, float crit_hi)
{
    const float term_rel = stat == kStatX2 ? 6.0e-7f : 3.2e-7f;
    const float rel = __fmul_ru(2.0f, __fadd_ru(term_rel, __fmul_ru(__fadd_ru(per_thread, levels), 6.0e-8f)));
    const float scale = stat == kStatX2 ? 1.0f : 2.0f;   // G^2 = 2 sum; exact scaling
    const float st = scale * sum;
    const float err = __fadd_ru(__fmul_ru(__fmul_ru(__fmul_ru(scale, rel), fabsf(mag)), 1.0001f), 1e-9f);
    if (__fadd_ru(st, err) < crit_lo) return 1;
    if (__fadd_rd(st, -err) >= crit_hi) return 0;
    return -1;
}

// Decision "p > alpha" as "G^2 < crit" from FP32 terms under an error bound,
// all in FP32 (the FP64 pipe of this part is 1/64 of FP32, and every thread
// of a group would otherwise run the bound in it).  The terms are evaluated
// with FP32 logarithms -- each within 3.2e-7 of its own magnitude, CUDA's logf
// and log1pf being within 1 ulp and the ratio formed from exact 64-bit
// integers -- and summed in FP32: a thread adds at most ceil(C/G) terms and
// the group tree adds log2(G) levels, each addition erring by at most 6e-8 of
// the running sum of magnitudes.  G^2 is thus within 2 (3.2e-7 + (ceil(C/G) +
// log2 G) 6e-8) sum|term| of its exact value; the bound is doubled for margin,
// formed with upward rounding, and compared against a float bracket [lo, hi]
// of crit (lo <= crit <= hi): accept when G^2 + err < lo, reject when G^2 -
// err >= hi (both rounded outward).  Returns 1 (accept), 0 (reject) or -1
// when the band straddles the bracket and the caller decides exactly.
//
// X^2 (stat = kStatX2): each term D^2 / (N_++z N_x+z N_+yz) with D the exact
// integer difference, formed in FP32 within 6e-7 of itself (three conversions,
// a square, two products, a quotient); the terms are non-negative, so the
// running sum of magnitudes is the sum itself, and the same summation bound
// applies without the doubling of G^2.
template <int G>
__device__ __forceinline__ int grp_decide_bound(const TestSpec& s, const int* T, const int* M, float crit_lo,
                                                float crit_hi, double* red, int stat = kStatG2)
{
    const int rx = s.rx, ry = s.ry, rxy = rx * ry, C = (int)s.cells;
    const int nz = C / rxy;
    const int* Nxz = M;
    const int* Nyz = M + nz * rx;
    const int* Nzz = Nyz + nz * ry;
    float acc = 0.0f, mag = 0.0f;
    if (stat == kStatX2) {
        for (int c = Grp<G>::rank(); c < C; c += G) {
            const int z = c / rxy;
            const int rem = c - z * rxy;
            const int x = rem / ry, y = rem - x * ry;
            x2_term(T[c], Nzz[z], Nxz[z * rx + x], Nyz[z * ry + y], acc);
        }
        mag = acc;
    } else {
        for (int c = Grp<G>::rank(); c < C; c += G) {
            const int n = T[c];
            if (n == 0) continue;
            const int z = c / rxy;
            const int rem = c - z * rxy;
            const int x = rem / ry, y = rem - x * ry;
            g2_term(n, Nzz[z], Nxz[z * rx + x], Nyz[z * ry + y], acc, mag);
        }
    }
    float2 v = make_float2(acc, mag);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    if (G > 32) {
        float* r = reinterpret_cast<float*>(red) + Grp<G>::gid() * 2 * Grp<G>::kWarps;
        Grp<G>::sync();
        if ((threadIdx.x & 31) == 0) {
            r[2 * (Grp<G>::rank() >> 5)] = v.x;
            r[2 * (Grp<G>::rank() >> 5) + 1] = v.y;
        }
        Grp<G>::sync();
        v.x = 0.0f;
        v.y = 0.0f;
#pragma unroll
        for (int w = 0; w < Grp<G>::kWarps; ++w) {
            v.x += r[2 * w];
            v.y += r[2 * w + 1];
        }
    }
    const float per_thread = (float)((C + G - 1) / G);   // exact: C < 2^24
    const float levels = (G == 32 ? 5.0f : G == 64 ? 6.0f : G == 128 ? 7.0f : 8.0f);
    return decide_from_sums(v.x, v.y, per_thread, levels, stat, crit_lo, crit_hi);
}

}  // namespace fbn
