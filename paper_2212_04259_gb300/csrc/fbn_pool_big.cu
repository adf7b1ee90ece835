// fbn_pool_big.cu -- the big-table work-pool kernel (CTA groups).
#include "fbn_pool.cuh"

namespace fbn {

// Big-table class: CTA groups.
__global__ void __launch_bounds__(kTestThreads, 2) k_pool_big(PoolArgs a)
{
    pdl_enter();
    extern __shared__ int smem[];
    __shared__ PoolShared sh;
    if (!a.ctr->active) return;
    pool_body<kTestThreads>(a, smem, sh);
    tests_done(a.ctr);
}

}  // namespace fbn
