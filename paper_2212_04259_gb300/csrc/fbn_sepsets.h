// fbn_sepsets.h -- host launchers of the separating-set compaction (fbn_sepsets.cu).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace fbn {

// Row counts of the removed pairs and their members, and their exclusive row
// offsets (cnt: [2][n]; roff_p, roff_m: [n + 1], totals at index n).
cudaError_t launch_sep_count(const int32_t* sep_len, int n, long long* cnt, long long* roff_p, long long* roff_m,
                             cudaStream_t st);
// The CSR arrays: pairs [R][2] (i < j, ascending), offs [R] (offs[R] is left
// to the caller), members from the pool at the pairs' offsets; the outputs
// may be device or device-addressable pinned host memory.
cudaError_t launch_sep_write(const int32_t* sep_len, const int64_t* sep_off, const int32_t* pool, int n,
                             const long long* roff_p, const long long* roff_m, int32_t* pairs, int64_t* offs,
                             int32_t* members, cudaStream_t st);

}  // namespace fbn
