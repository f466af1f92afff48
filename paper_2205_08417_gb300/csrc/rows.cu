// Row gather and scatter of state arrays by cell index, for the halo exchange of a step split
// over ranks [Sec. 6: the cells are split over workers that synchronise between the step's
// phases]: the rows a neighbour needs are packed into a contiguous buffer before the send, and
// the received rows are unpacked into the halo. The adjoint's reverse halo adds received rows
// instead (scatter-add). Element-wise, one thread per (row, column).
#include "kitrt_internal.cuh"

namespace {

enum RowsOp { kGather = 0, kScatter = 1, kScatterAdd = 2 };

template <int OP>
__global__ void rows_kernel(const double *__restrict__ src, const int32_t *__restrict__ idx,
                            int count, int width, double *__restrict__ dst)
{
    const size_t total = (size_t)count * width;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(e / width), c = (int)(e - (size_t)k * width);
        const size_t row = (size_t)idx[k];
        if (OP == kGather)
            dst[e] = src[row * width + c];
        else if (OP == kScatter)
            dst[row * width + c] = src[e];
        else
            dst[row * width + c] += src[e];  // indices are distinct: no two threads share a row
    }
}

template <int OP>
int launch_rows(const double *src, const int32_t *idx, int32_t count, int32_t width, double *dst,
                void *stream)
{
    if (count < 0 || width < 1 || (count > 0 && (!src || !idx || !dst))) return KITRT_EINVAL;
    if (count == 0) return KITRT_OK;
    const size_t total = (size_t)count * width;
    const int blocks = (int)std::min<size_t>((total + 255) / 256, 4096);
    rows_kernel<OP><<<blocks, 256, 0, (cudaStream_t)stream>>>(src, idx, count, width, dst);
    return cudaGetLastError() == cudaSuccess ? KITRT_OK : KITRT_ECUDA;
}

}  // namespace

extern "C" int32_t kitrt_gather_rows(const double *src, const int32_t *idx, int32_t count,
                                     int32_t width, double *dst, void *stream)
{
    return launch_rows<kGather>(src, idx, count, width, dst, stream);
}

extern "C" int32_t kitrt_scatter_rows(const double *src, const int32_t *idx, int32_t count,
                                      int32_t width, double *dst, void *stream)
{
    return launch_rows<kScatter>(src, idx, count, width, dst, stream);
}

extern "C" int32_t kitrt_scatter_add_rows(const double *src, const int32_t *idx, int32_t count,
                                          int32_t width, double *dst, void *stream)
{
    return launch_rows<kScatterAdd>(src, idx, count, width, dst, stream);
}
