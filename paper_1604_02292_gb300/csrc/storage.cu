// storage.cu -- conversions between float and the 16-bit storage types of the resident
// sinogram and FBP image (bfloat16, IEEE half; round to nearest even).  The arithmetic of
// every kernel stays float; only what is stored is narrowed.
#include <cuda_runtime.h>

#include "dev_common.cuh"
#include "roi_internal.h"

namespace roi {

namespace {

template <int SD, int DD>
__global__ void k_convert(const void* __restrict__ src, void* __restrict__ dst, size_t n) {
    const auto* s = static_cast<const typename Stor<SD>::T*>(src);
    auto* d = static_cast<typename Stor<DD>::T*>(dst);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        d[i] = from_f32<DD>(to_f32<SD>(s[i]));
}

// dst[r][c] (or dst[c][r] when transposed) = src[r][c], through a 32 x 33 tile.
template <int DD>
__global__ void k_store_padded(const float* __restrict__ src, int src_ld, void* __restrict__ dst, int dst_ld,
                               int rows, int cols, int transpose) {
    __shared__ float t[32][33];
    auto* d = static_cast<typename Stor<DD>::T*>(dst);
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int r = by + y, c = bx + threadIdx.x;
        if (r < rows && c < cols) {
            const float v = src[(size_t)r * src_ld + c];
            if (transpose)
                t[y][threadIdx.x] = v;
            else
                d[(size_t)r * dst_ld + c] = from_f32<DD>(v);
        }
    }
    if (!transpose) return;
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int c = bx + y, r = by + threadIdx.x;
        if (r < rows && c < cols) d[(size_t)c * dst_ld + r] = from_f32<DD>(t[threadIdx.x][y]);
    }
}

template <int SD>
__global__ void k_load_padded(const void* __restrict__ src, int src_ld, float* __restrict__ dst, int dst_ld, int rows,
                              int cols) {
    const auto* s = static_cast<const typename Stor<SD>::T*>(src);
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y * blockDim.y + threadIdx.y;
    if (r < rows && c < cols) dst[(size_t)r * dst_ld + c] = to_f32<SD>(s[(size_t)r * src_ld + c]);
}

// Truncated rows (Sec. 5.6): dst[a][d] = src[a][clamp(d - off, 0, nm - 1)] -- the measured
// central bins, constant (edge-value) padding on both sides, converted to the storage type.
template <int SD, int DD>
__global__ void k_pad_truncated(const void* __restrict__ src, int nm, void* __restrict__ dst, int nd, int off) {
    const auto* s = static_cast<const typename Stor<SD>::T*>(src);
    auto* d = static_cast<typename Stor<DD>::T*>(dst);
    const int a = blockIdx.y;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nd; j += gridDim.x * blockDim.x) {
        const int k = min(max(j - off, 0), nm - 1);
        d[(size_t)a * nd + j] = from_f32<DD>(to_f32<SD>(s[(size_t)a * nm + k]));
    }
}

template <int SD>
void pad_from(const void* src, int nm, void* dst, int dst_dt, int na, int nd, int off, cudaStream_t st) {
    dim3 grid((nd + 255) / 256, na);
    if (dst_dt == 1)
        k_pad_truncated<SD, 1><<<grid, 256, 0, st>>>(src, nm, dst, nd, off);
    else if (dst_dt == 2)
        k_pad_truncated<SD, 2><<<grid, 256, 0, st>>>(src, nm, dst, nd, off);
    else
        k_pad_truncated<SD, 0><<<grid, 256, 0, st>>>(src, nm, dst, nd, off);
}

template <int SD>
void convert_from(const void* src, void* dst, int dst_dt, size_t n, int blocks, cudaStream_t st) {
    if (dst_dt == 1)
        k_convert<SD, 1><<<blocks, 256, 0, st>>>(src, dst, n);
    else if (dst_dt == 2)
        k_convert<SD, 2><<<blocks, 256, 0, st>>>(src, dst, n);
    else
        k_convert<SD, 0><<<blocks, 256, 0, st>>>(src, dst, n);
}

}  // namespace

void launch_convert(const void* src, int src_dt, void* dst, int dst_dt, size_t n, cudaStream_t st) {
    if (n == 0) return;
    const int blocks = (int)((n + 255) / 256 < 152 * 8 ? (n + 255) / 256 : 152 * 8);
    count_launches(1);
    if (src_dt == 1)
        convert_from<1>(src, dst, dst_dt, n, blocks, st);
    else if (src_dt == 2)
        convert_from<2>(src, dst, dst_dt, n, blocks, st);
    else
        convert_from<0>(src, dst, dst_dt, n, blocks, st);
}

void launch_pad_truncated(const void* src, int src_dt, int nm, void* dst, int dst_dt, int na, int nd, int off,
                          cudaStream_t st) {
    if (na <= 0 || nd <= 0 || nm <= 0) return;
    count_launches(1);
    if (src_dt == 1)
        pad_from<1>(src, nm, dst, dst_dt, na, nd, off, st);
    else if (src_dt == 2)
        pad_from<2>(src, nm, dst, dst_dt, na, nd, off, st);
    else
        pad_from<0>(src, nm, dst, dst_dt, na, nd, off, st);
}

void launch_store_padded(const float* src, int src_ld, void* dst, int dst_dt, int dst_ld, int rows, int cols,
                         int transpose, cudaStream_t st) {
    if (rows <= 0 || cols <= 0) return;
    dim3 grid((cols + 31) / 32, (rows + 31) / 32);
    count_launches(1);
    if (dst_dt == 1)
        k_store_padded<1><<<grid, dim3(32, 8), 0, st>>>(src, src_ld, dst, dst_ld, rows, cols, transpose);
    else if (dst_dt == 2)
        k_store_padded<2><<<grid, dim3(32, 8), 0, st>>>(src, src_ld, dst, dst_ld, rows, cols, transpose);
    else
        k_store_padded<0><<<grid, dim3(32, 8), 0, st>>>(src, src_ld, dst, dst_ld, rows, cols, transpose);
}

void launch_load_padded(const void* src, int src_dt, int src_ld, float* dst, int dst_ld, int rows, int cols,
                        cudaStream_t st) {
    if (rows <= 0 || cols <= 0) return;
    dim3 grid((cols + 31) / 32, (rows + 7) / 8);
    count_launches(1);
    if (src_dt == 1)
        k_load_padded<1><<<grid, dim3(32, 8), 0, st>>>(src, src_ld, dst, dst_ld, rows, cols);
    else if (src_dt == 2)
        k_load_padded<2><<<grid, dim3(32, 8), 0, st>>>(src, src_ld, dst, dst_ld, rows, cols);
    else
        k_load_padded<0><<<grid, dim3(32, 8), 0, st>>>(src, src_ld, dst, dst_ld, rows, cols);
}

}  // namespace roi
