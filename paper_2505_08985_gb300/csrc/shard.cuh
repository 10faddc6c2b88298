// Launchers of the batch-sharding kernels (shard.cu).
#pragma once

#include "common.cuh"

namespace pndf {
cudaError_t launch_shard_work(const pndf_query *q, const uint32_t *order, int64_t nq, int block, double *partial,
                              cudaStream_t s);
cudaError_t launch_gather_queries(const pndf_query *q, const uint32_t *order, int64_t first, int64_t count,
                                  pndf_query *out, cudaStream_t s);
cudaError_t launch_scatter_results(const float *D, const uint32_t *order, int64_t first, int64_t count, float *out,
                                   cudaStream_t s);
}  // namespace pndf
