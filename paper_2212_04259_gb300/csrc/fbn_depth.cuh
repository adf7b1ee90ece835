// fbn_depth.cuh -- small device helpers shared by the depth kernels and the
// work-pool kernels: programmatic dependent launch, the device clock, the
// per-depth record and the edge-class sub-array.
#pragma once

#include "fbn_device.cuh"

namespace fbn {

// Programmatic dependent launch: the kernels of a depth are launched so that
// the next one may be scheduled once every CTA of this one has started; it
// then waits here until this one has finished and its writes are visible.
// Launched without the attribute, both instructions do nothing.
__device__ __forceinline__ void pdl_enter()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Device clock in nanoseconds, for the per-depth records.
__device__ __forceinline__ unsigned long long gtime()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ DepthRecord* depth_rec(const DepthCounters* ctr, int d)
{
    return ctr->rec && d < kMaxDepthRecords ? ctr->rec + d : nullptr;
}

// Edges of class cls: class 0 fills the edge array from the front, class 1
// from the back.
__device__ __forceinline__ long long class_base(const DepthCounters* ctr, int cls, long long edge_cap)
{
    return cls == 0 ? 0 : edge_cap - (long long)ctr->n_edges[1];
}

}  // namespace fbn
