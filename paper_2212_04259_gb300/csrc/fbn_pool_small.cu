// fbn_pool_small.cu -- the small-table work-pool kernel (byte histograms).
#include "fbn_pool.cuh"

namespace fbn {

// Small-table class: the group size k_scan chose for this depth; byte
// histograms (the depth's class when some edge cannot use the bit planes).
__global__ void __launch_bounds__(kTestThreads, 3) k_pool_small(PoolArgs a)
{
    pdl_enter();
    extern __shared__ int smem[];
    __shared__ PoolShared sh;
    if (!a.ctr->active || a.ctr->bits_ok) return;
    switch (a.ctr->gsel) {
        case 32: pool_body<32>(a, smem, sh); break;
        case 64: pool_body<64>(a, smem, sh); break;
        case 128: pool_body<128>(a, smem, sh); break;
        default: pool_body<kTestThreads>(a, smem, sh); break;
    }
    tests_done(a.ctr);
}

}  // namespace fbn
