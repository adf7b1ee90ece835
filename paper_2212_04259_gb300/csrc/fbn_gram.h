// fbn_gram.h -- host launchers of the tcgen05 one-hot Gram (fbn_gram.cu).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "fbn_internal.cuh"

namespace fbn {

size_t gram_smem_bytes();
int gram_rows_padded(int M);
long long gram_samples_padded(long long N);
cudaError_t launch_onehot(const ProblemDev* probs, const int32_t* vtx_prob, const int32_t* vtx_first,
                          int total_vertices, cudaStream_t st);
cudaError_t launch_zero_pad(const ProblemDev* probs, int nprob, cudaStream_t st);
cudaError_t encode_onehot_map(void* map, const uint8_t* E, int Mp, long long K);
size_t tensor_map_bytes();
int gram_chunks(long long K);
cudaError_t launch_gram(const void* maps, const int4* units, int n_units, const ProblemDev* probs, int num_sms,
                        unsigned* status, int wait_limit, cudaStream_t st);
cudaError_t launch_pairs_decide(const EdgeWork* edges, long long edge_cap, const ProblemDev* probs,
                                unsigned long long* min_accept, const CritTableDev& crit, double alpha,
                                DepthCounters* ctr, int stat, int df_mode, int grid, cudaStream_t st);
cudaError_t launch_symmetrize(int32_t* G, int Mp, int M, cudaStream_t st);

}  // namespace fbn
