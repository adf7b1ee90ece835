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
cudaError_t launch_onehot(const uint8_t* data, long long ld, int n, int N, const uint8_t* ar, const int32_t* off,
                          uint8_t* E, long long K, cudaStream_t st);
cudaError_t launch_gram(const uint8_t* E, int Mp, long long K, int32_t* G, const int2* tiles, int n_tiles,
                        int num_sms, unsigned* status, cudaStream_t st);
cudaError_t launch_pairs_decide(const EdgeWork* edges, long long edge_cap, const ProblemDev* probs, const int32_t* G,
                                int Mp, const int32_t* off, unsigned long long* min_accept, const CritTableDev& crit,
                                double alpha, DepthCounters* ctr, int grid, cudaStream_t st);
cudaError_t launch_symmetrize(int32_t* G, int Mp, int M, cudaStream_t st);

}  // namespace fbn
