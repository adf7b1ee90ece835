// fbn_nbr.h -- host launcher of the depth-1 neighbourhood product on the
// tensor cores (fbn_nbr.cu).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "fbn_internal.cuh"

namespace fbn {

size_t nbr1_smem_bytes();
int nbr1_max_arity();   // largest arity of a problem the kernel takes
// Every problem's samples 4 bits each into its pk rows.
cudaError_t launch_pack4(const ProblemDev* probs, const int32_t* vtx_prob, const int32_t* vtx_first,
                         int total_vertices, cudaStream_t st);
// Every depth-1 test of every vertex with at least two neighbours, lowering
// min_accept of the edges (the edge list and eid of the depth must be built);
// vertices are claimed through ctr->nbr_claim, which must be zero.
cudaError_t launch_nbr1(const ProblemDev* probs, const int32_t* vtx_prob, const int32_t* vtx_first,
                        int total_vertices, const EdgeWork* edges, unsigned long long* min_accept,
                        const CritTableDev& crit, double alpha, DepthCounters* ctr, int num_sms, int wait_limit,
                        cudaStream_t st);

}  // namespace fbn
