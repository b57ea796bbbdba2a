// solve.cu -- per-pixel and reduction kernels of the local solvers.
//
// Chambolle-Pock for min_x ||p' - W_L x||^2 + lambda ||grad x||_{2,1} (paper Eq. priorsys
// with the TV penalty of Sec. 2.3); nonnegative / weighted SIRT (Eq. sirtit, Eq. sirtbox).
// grad = forward differences with a zero last difference; div = -grad^T.
#include <cuda_runtime.h>

#include <algorithm>

#include "roi_internal.h"

namespace roi {

namespace {

__global__ void k_cp_dual_grad(const float* __restrict__ xb, int ld, float* vx, float* vy, int nx, int ny,
                               const float* sigma_dev, float sigma_v, float lambda) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= ny || j >= nx) return;
    const float sv = sigma_dev ? *sigma_dev : sigma_v;
    const size_t o = (size_t)i * nx + j;
    const float* xp = xb + (size_t)i * ld + j;
    const float x0 = xp[0];
    const float gx = j < nx - 1 ? xp[1] - x0 : 0.f;
    const float gy = i < ny - 1 ? xp[ld] - x0 : 0.f;
    const float ax = fmaf(sv, gx, vx[o]);
    const float ay = fmaf(sv, gy, vy[o]);
    const float m = sqrtf(ax * ax + ay * ay);
    const float sc = m > lambda ? lambda / m : 1.f;  // projection onto the lambda-ball
    vx[o] = ax * sc;
    vy[o] = ay * sc;
}

__global__ void k_precond_rows(float* rows, size_t n, int mode) {
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float s = rows[i];
    const float thr = mode == 0 ? 1e-3f : 1e-6f;
    rows[i] = s > thr ? 1.f / s : 0.f;
}

__global__ void k_precond_cols(float* cols, int nx, int ny, int mode) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= ny || j >= nx) return;
    const size_t o = (size_t)i * nx + j;
    const float s = cols[o];
    if (mode == 0) {
        cols[o] = s > 1e-3f ? 1.f / s : 0.f;
    } else {
        const int cnt = (j < nx - 1) + (j > 0) + (i < ny - 1) + (i > 0);
        cols[o] = 1.f / (s + (float)cnt);
    }
}

__global__ void k_crop(const float* __restrict__ x, int ld, float* __restrict__ out, int nx, int ny, double cxl,
                       double cyl, double r, int crop) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= ny || j >= nx) return;
    const size_t o = (size_t)i * nx + j;
    float v = x[(size_t)i * ld + j];
    if (crop) {
        const double dx = j - cxl, dy = i - cyl;
        if (dx * dx + dy * dy > r * r) v = 0.f;
    }
    out[o] = v;
}

// Deterministic two-level reduction: each block reduces a fixed slice with per-thread
// Neumaier-compensated float sums, combined in double in a fixed tree order; a single
// block then adds the block partials in index order.
constexpr int RED_THREADS = 256;

__device__ inline void neumaier_add(float& s, float& c, float v) {
    const float t = s + v;
    if (fabsf(s) >= fabsf(v))
        c += (s - t) + v;
    else
        c += (v - t) + s;
    s = t;
}

__device__ inline double block_sum(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < RED_THREADS / 32; ++k) r += sh[k];
    return r;  // valid in thread 0
}

__global__ void k_objective_partial(const float* __restrict__ wx, const float* __restrict__ pp,
                                    const float* __restrict__ rowsum, int nwin, const float* __restrict__ x, int ld,
                                    int nx, int ny, double* part) {
    __shared__ double sh[RED_THREADS / 32];
    float s0 = 0.f, c0 = 0.f, s1 = 0.f, c1 = 0.f;
    const int stride = gridDim.x * RED_THREADS;
    for (int i = blockIdx.x * RED_THREADS + threadIdx.x; i < nwin; i += stride) {
        if (rowsum[i] > 1e-6f) {
            const float d = wx[i] - pp[i];
            neumaier_add(s0, c0, d * d);
        }
    }
    const int npx = nx * ny;
    for (int o = blockIdx.x * RED_THREADS + threadIdx.x; o < npx; o += stride) {
        const int i = o / nx, j = o - i * nx;
        const float* xp = x + (size_t)i * ld + j;
        const float gx = j < nx - 1 ? xp[1] - xp[0] : 0.f;
        const float gy = i < ny - 1 ? xp[ld] - xp[0] : 0.f;
        neumaier_add(s1, c1, sqrtf(gx * gx + gy * gy));
    }
    const double d0 = block_sum((double)s0 + (double)c0, sh);
    const double d1 = block_sum((double)s1 + (double)c1, sh);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = d0;
        part[2 * blockIdx.x + 1] = d1;
    }
}

__global__ void k_sum_partials(const double* part, int nblocks, double* out2) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int k = 0; k < nblocks; ++k) {
            a += part[2 * k];
            b += part[2 * k + 1];
        }
        out2[0] = a;
        out2[1] = b;
    }
}


// ---- power iteration for ||K||, K = [W_L; grad] (scalar Chambolle-Pock steps)
// y holds W^T W x on entry; adds grad^T grad x = -div(grad x).
__global__ void k_ktk_grad(float* y, const float* __restrict__ x, int ld, int nx, int ny) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= ny || j >= nx) return;
    const size_t o = (size_t)i * nx + j;
    const float* xp = x + (size_t)i * ld + j;
    // grad at (i,j) and at the left / upper neighbours
    const float gx = j < nx - 1 ? xp[1] - xp[0] : 0.f;
    const float gy = i < ny - 1 ? xp[ld] - xp[0] : 0.f;
    const float gxl = j > 0 ? xp[0] - xp[-1] : 0.f;
    const float gyu = i > 0 ? xp[0] - xp[-ld] : 0.f;
    float dv = 0.f;
    if (j < nx - 1) dv += gx;
    if (j > 0) dv -= gxl;
    if (i < ny - 1) dv += gy;
    if (i > 0) dv -= gyu;
    y[o] -= dv;
}

__global__ void k_sumsq_partial(const float* __restrict__ v, int n, double* part) {
    __shared__ double sh[RED_THREADS / 32];
    float s = 0.f, c = 0.f;
    for (int i = blockIdx.x * RED_THREADS + threadIdx.x; i < n; i += gridDim.x * RED_THREADS)
        neumaier_add(s, c, v[i] * v[i]);
    const double d = block_sum((double)s + (double)c, sh);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = d;
        part[2 * blockIdx.x + 1] = 0.0;
    }
}

// x = y / sqrt(n2[0]); xT = transpose (plain strided store: only used by the power iteration)
__global__ void k_normalize(const float* __restrict__ y, float* x, int x_ld, float* xT, int xT_ld, int nx, int ny,
                            const double* n2) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= ny || j >= nx) return;
    const size_t o = (size_t)i * nx + j;
    const double nrm = sqrt(n2[0]);
    const float v = nrm > 0.0 ? (float)(y[o] / nrm) : 0.f;
    x[(size_t)i * x_ld + j] = v;
    xT[(size_t)j * xT_ld + i] = v;
}

// step = 0.99 / L with L = sqrt(||K^T K x||) = n2^(1/4); writes dst[0..n) and, if L_out, L
__global__ void k_fill_step(float* dst, size_t n, const double* n2, double* L_out) {
    const double L = sqrt(sqrt(n2[0]));
    const float step = L > 0.0 ? (float)(0.99 / L) : 0.f;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = step;
    if (L_out && blockIdx.x == 0 && threadIdx.x == 0) *L_out = L;
}

}  // namespace

void launch_cp_dual_grad(const float* xbar, int xbar_ld, float* vx, float* vy, int nx, int ny, float sigma_v,
                         float lambda, cudaStream_t st) {
    if (nx <= 0 || ny <= 0) return;
    dim3 block(32, 8), grid((nx + 31) / 32, (ny + 7) / 8);
    count_launches(1);
    k_cp_dual_grad<<<grid, block, 0, st>>>(xbar, xbar_ld, vx, vy, nx, ny, nullptr, sigma_v, lambda);
}

void launch_cp_dual_grad_dev(const float* xbar, int xbar_ld, float* vx, float* vy, int nx, int ny,
                             const float* sigma_dev, float lambda, cudaStream_t st) {
    if (nx <= 0 || ny <= 0) return;
    dim3 block(32, 8), grid((nx + 31) / 32, (ny + 7) / 8);
    count_launches(1);
    k_cp_dual_grad<<<grid, block, 0, st>>>(xbar, xbar_ld, vx, vy, nx, ny, sigma_dev, 0.f, lambda);
}

void launch_power_ktk_grad(float* y, const float* x, int x_ld, int nx, int ny, cudaStream_t st) {
    dim3 block(32, 8), grid((nx + 31) / 32, (ny + 7) / 8);
    count_launches(1);
    k_ktk_grad<<<grid, block, 0, st>>>(y, x, x_ld, nx, ny);
}

void launch_sumsq(const float* v, int n, double* scratch, int nscratch, double* out2, cudaStream_t st) {
    const int nblocks = std::max(1, std::min(nscratch / 2, 152));
    count_launches(1);
    k_sumsq_partial<<<nblocks, RED_THREADS, 0, st>>>(v, n, scratch);
    count_launches(1);
    k_sum_partials<<<1, 32, 0, st>>>(scratch, nblocks, out2);
}

void launch_normalize(const float* y, float* x, int x_ld, float* xT, int xT_ld, int nx, int ny, const double* n2,
                      cudaStream_t st) {
    dim3 block(32, 8), grid((nx + 31) / 32, (ny + 7) / 8);
    count_launches(1);
    k_normalize<<<grid, block, 0, st>>>(y, x, x_ld, xT, xT_ld, nx, ny, n2);
}

void launch_fill_step(float* dst, size_t n, const double* n2, double* L_out, cudaStream_t st) {
    if (n == 0) return;
    const int blocks = (int)std::min<size_t>((n + 255) / 256, 152 * 4);
    count_launches(1);
    k_fill_step<<<blocks, 256, 0, st>>>(dst, n, n2, L_out);
}

void launch_precond(float* rows, int nrows_total, float* cols, int nx, int ny, int mode, cudaStream_t st) {
    if (rows && nrows_total > 0)
        k_precond_rows<<<(nrows_total + 255) / 256, 256, 0, st>>>(rows, (size_t)nrows_total, mode);
    if (cols && nx > 0 && ny > 0) {
        dim3 block(32, 8), grid((nx + 31) / 32, (ny + 7) / 8);
        k_precond_cols<<<grid, block, 0, st>>>(cols, nx, ny, mode);
    }
}

void launch_crop(const float* x, int x_ld, float* out, int nx, int ny, double cxl, double cyl, double r, int crop,
                 cudaStream_t st) {
    if (nx <= 0 || ny <= 0) return;
    dim3 block(32, 8), grid((nx + 31) / 32, (ny + 7) / 8);
    count_launches(1);
    k_crop<<<grid, block, 0, st>>>(x, x_ld, out, nx, ny, cxl, cyl, r, crop);
}

void launch_objective(const float* wx, const float* pp, const float* rowsum, int nwin, const float* x, int x_ld,
                      int nx, int ny, double* scratch, int nscratch, double* out2, cudaStream_t st) {
    const int nblocks = std::max(1, std::min(nscratch / 2, 152));
    count_launches(1);
    k_objective_partial<<<nblocks, RED_THREADS, 0, st>>>(wx, pp, rowsum, nwin, x, x_ld, nx, ny, scratch);
    count_launches(1);
    k_sum_partials<<<1, 32, 0, st>>>(scratch, nblocks, out2);
}

}  // namespace roi
