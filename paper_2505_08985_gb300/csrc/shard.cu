// Sharding one batch over hierarchy replicas (the queries are independent
// and the hierarchy is read-only, Sec. 4.2 / Eq. 5): the batch is put in
// evaluation order once (pndf_sort_queries), cut into contiguous ranges of
// that order with about equal estimated work, each range's records are
// gathered into a contiguous array for its replica, and each replica's
// results are scattered back into caller order.  These kernels are the data
// movement around the evaluation; the split points are chosen on the host
// from per-block work sums.
#include "shard.cuh"

namespace pndf {
namespace {

// Estimated traversal work of one query: the area of its 4-sigma box in
// texel^2 (the leaf blocks the traversal can reach grow with it), plus a
// fixed cost of 64 for the descent from the entry nodes.  Invalid records
// count as the fixed cost only.
__device__ __forceinline__ double query_work(const pndf_query &r)
{
    const float sx = r.sxx > 0.f ? sqrtf(r.sxx) : 0.f, sy = r.syy > 0.f ? sqrtf(r.syy) : 0.f;
    const double a = 64.0 * double(sx) * double(sy);  // (8 sigma_x)(8 sigma_y)
    return 64.0 + (isfinite(a) ? a : 0.0);
}

// One block of 256 threads per `block` positions of the evaluation order:
// the sum of query_work over positions [b * block, (b + 1) * block).
__global__ void shard_work(const pndf_query *__restrict__ q, const uint32_t *__restrict__ order, int64_t nq,
                           int block, double *__restrict__ partial)
{
    __shared__ double red[256];
    const int64_t b0 = int64_t(blockIdx.x) * block;
    double s = 0.0;
    for (int64_t k = b0 + threadIdx.x; k < b0 + block && k < nq; k += blockDim.x) s += query_work(q[order[k]]);
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (int(threadIdx.x) < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void gather_queries(const pndf_query *__restrict__ q, const uint32_t *__restrict__ order, int64_t first,
                               int64_t count, pndf_query *__restrict__ out)
{
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < count; k += int64_t(gridDim.x) * blockDim.x)
        out[k] = q[order[first + k]];
}

__global__ void scatter_results(const float *__restrict__ D, const uint32_t *__restrict__ order, int64_t first,
                                int64_t count, float *__restrict__ out)
{
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < count; k += int64_t(gridDim.x) * blockDim.x)
        out[order[first + k]] = D[k];
}

unsigned grid_for(int64_t n)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t b = (n + 255) / 256;
    const int64_t cap = int64_t(sms > 0 ? sms : 1) * 8;
    return unsigned(b < 1 ? 1 : (b > cap ? cap : b));
}

}  // namespace

cudaError_t launch_shard_work(const pndf_query *q, const uint32_t *order, int64_t nq, int block, double *partial,
                              cudaStream_t s)
{
    const int64_t nb = (nq + block - 1) / block;
    if (nb == 0) return cudaSuccess;
    shard_work<<<unsigned(nb), 256, 0, s>>>(q, order, nq, block, partial);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_gather_queries(const pndf_query *q, const uint32_t *order, int64_t first, int64_t count,
                                  pndf_query *out, cudaStream_t s)
{
    if (count == 0) return cudaSuccess;
    gather_queries<<<grid_for(count), 256, 0, s>>>(q, order, first, count, out);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_scatter_results(const float *D, const uint32_t *order, int64_t first, int64_t count, float *out,
                                   cudaStream_t s)
{
    if (count == 0) return cudaSuccess;
    scatter_results<<<grid_for(count), 256, 0, s>>>(D, order, first, count, out);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace pndf
