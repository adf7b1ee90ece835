// fbn_pool_bits.cu -- the small-table work-pool kernel counted from bit planes.
#include "fbn_pool.cuh"

namespace fbn {

// Small-table class counted from bit planes: the depth's class when every
// edge qualifies (k_edges); otherwise k_pool_small runs it.  Warp groups only:
// the fastest group size at every measured depth, and one copy of the code (the
// kernel is sensitive to its code footprint).  CTAs per SM: 4 (64 registers a
// thread; its 36 KB of shared memory allow it).
#ifndef FBN_BITS_CTAS
#define FBN_BITS_CTAS 4
#endif
__global__ void __launch_bounds__(kTestThreads, FBN_BITS_CTAS) k_pool_bits(PoolArgs a)
{
    pdl_enter();
    extern __shared__ int smem[];
    __shared__ PoolShared sh;
    if (!a.ctr->active || !a.ctr->bits_ok || a.ctr->n_edges[kClassWarp] == 0) return;
    pool_body<32, true>(a, smem, sh);   // warp groups only (k_scan sets gsel = 32): one copy of the code
    tests_done(a.ctr);
}

}  // namespace fbn
