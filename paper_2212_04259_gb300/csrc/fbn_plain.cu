// fbn_plain.cu -- the edge-level form (Section IV-A): one CTA per edge.
#include "fbn_pool.cuh"

namespace fbn {

__global__ void __launch_bounds__(kTestThreads, 2) k_plain(PoolArgs a)
{
    pdl_enter();
    extern __shared__ int smem[];
    __shared__ TestSpec spec;
    __shared__ GroupState S;
    __shared__ double red[32];
    const DepthCounters* ctr = a.ctr;
    if (!ctr->active) return;
    const int d = ctr->d;
    if (blockIdx.x == 0 && threadIdx.x == 0 && a.cls == 0)
        if (DepthRecord* r = depth_rec(ctr, d)) r->t_tests = gtime();
    const long long E = (long long)ctr->n_edges[a.cls];
    const long long cb = class_base(ctr, a.cls, a.edge_cap);
    int* gtab = a.gscratch ? a.gscratch + (long long)blockIdx.x * a.gscratch_ints : nullptr;
    if (threadIdx.x == 0) S.tests = S.popc_work = S.smem_updates = 0;
    for (long long e = blockIdx.x; e < E; e += gridDim.x) {
        const EdgeWork w = a.edges[cb + e];
        const ProblemDev& P = a.probs[w.prob];
        for (long long rk = 0; rk < w.total; ++rk) {
            const int res = run_rank<kTestThreads, false>(a, d, P, w, rk, rk == 0, S, spec, smem, a.smem_ints, gtab, red);
            if (res == 1 && threadIdx.x == 0) a.min_accept[cb + e] = (unsigned long long)rk;
            if (res != 0) break;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0 && S.tests) atomicAdd(&a.ctr->tests, S.tests);
    if (threadIdx.x == 0 && S.smem_updates) atomicAdd(&a.ctr->smem_updates, S.smem_updates);
    tests_done(ctr);
}

}  // namespace fbn
