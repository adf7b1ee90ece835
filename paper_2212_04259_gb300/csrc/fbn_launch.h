// fbn_launch.h -- host-side launchers of the depth, pool and explicit-test kernels.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "fbn_internal.cuh"

namespace fbn {

// One explicit CI test (fbn_ci_test / fbn_ci_table).
struct CiTestDesc {
    int32_t x, y, d, pad;
    int32_t z[kMaxD];
};

void launch_snapshot(const ProblemDev* probs, const int32_t* vtx_prob, const int32_t* vtx_first,
                     int total_vertices, DepthCounters* ctr, cudaStream_t st);
void launch_edges(const ProblemDev* probs, const int32_t* vtx_prob, const int32_t* vtx_first,
                  int total_vertices, int gs_forced, long long gs_edges, const long long* binom, int brows,
                  long long warp_cells_cap, int bits_cells, const uint8_t* owned,
                  EdgeWork* edges, unsigned long long* min_accept, long long edge_cap, DepthCounters* ctr,
                  unsigned long long* hist, cudaStream_t st);
// Ordering of the depth's edges, one CTA per class (nclass = 1: the small-
// table class only), then the placement of both classes.
void launch_order(const EdgeWork* edges, long long edge_cap, int nclass, DepthCounters* ctr, const ScanClass* sc,
                  unsigned long long* cursor0, unsigned long long* cursor1, int32_t* sorted, double mean_n,
                  int forced_group, long long split_stride, int allow_split, int grid, cudaStream_t st);
void launch_pool(const PoolArgs& a, int cls, int grid, size_t smem_bytes, cudaStream_t st);
void launch_pool_bits(const PoolArgs& a, int grid, size_t smem_bytes, cudaStream_t st);
void launch_plain(const PoolArgs& a, int grid, size_t smem_bytes, cudaStream_t st);
void launch_apply(const ProblemDev* probs, const EdgeWork* edges, const unsigned long long* min_accept,
                  long long edge_cap, const long long* binom, int32_t* sep_pool, long long sep_cap,
                  DepthCounters* ctr, int grid, cudaStream_t st);
// Sharded skeletons: this process's removals as (i, j, rank) records; the
// union of every process's records applied to the snapshot.
void launch_shard_export(const ProblemDev* probs, const EdgeWork* edges, const unsigned long long* min_accept,
                         long long edge_cap, DepthCounters* ctr, long long* out, unsigned long long* count, int grid,
                         cudaStream_t st);
void launch_shard_apply(const ProblemDev* probs, const long long* list, long long n_list, const long long* binom,
                        int brows, int32_t* sep_pool, long long sep_cap, DepthCounters* ctr, int grid, cudaStream_t st);
void launch_shard_continue(DepthCounters* ctr, cudaStream_t st);
void launch_depth_end(DepthCounters* ctr, DepthRecord* rec, int max_depth, unsigned long long* hist,
                      unsigned long long* cursor, cudaStream_t st);
// The depth loop's condition: 1 while the next depth has an edge to test.
void launch_gate(DepthCounters* ctr, cudaGraphConditionalHandle loop, cudaStream_t st);
// Programmatic dependent launch for the depth kernels (on by default).
void set_pdl(bool on);
void launch_ci_tests(const ProblemDev* prob, const CiTestDesc* tests, int ntests, double* out,
                     int32_t* table_out, int* gscratch, long long gscratch_ints, unsigned* status,
                     size_t smem_bytes, int stat, int df_mode, bool bits, cudaStream_t st);
cudaError_t set_kernel_smem(size_t max_smem);
// The dynamic shared-memory limit of the explicit-test kernels (fbn_ci.cu).
cudaError_t set_ci_smem(int max_smem);
// Sets the message fbn_last_error(NULL) returns.
void fbn_internal_set_error(const char* msg);
int pool_blocks_per_sm(int cls, size_t smem_bytes);

}  // namespace fbn
