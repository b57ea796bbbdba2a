// filtermethod.cu -- kernels of the paper's own local method (Sec. 3): the filters of
// Alg. filtcalc, the disc subtraction of Sec. 3.3, the filtered sinograms C_{u_k} p and
// the per-pixel step of Alg. method.  The projections themselves are the Joseph kernels
// of project.cu.
#include <cuda_runtime.h>

#include "dev_common.cuh"
#include "roi_internal.h"

namespace roi {

namespace {

// D = the disc of diameter N centred on the rotation axis (pixel centres within N/2 of
// it); the padded image and its transpose are the same image.
__global__ void k_disc_image(float* img, float* imgT, int ld, int N) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;
    if (j >= N) return;
    const float half = 0.5f * (float)(N - 1);
    const float x = (float)j - half, y = half - (float)i;
    const float v = (x * x + y * y <= 0.25f * (float)N * (float)N) ? 1.f : 0.f;
    img[(size_t)i * ld + j] = v;
    imgT[(size_t)i * ld + j] = v;
}

// The unit impulse at the grid centre (four pixels at 1/4 for even N) in a padded image
// and its transpose; everything else 0.
__global__ void k_impulse(float* img, float* imgT, int ld, int N) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x - kPad;
    const int i = blockIdx.y;
    if (j >= ld - kPad) return;
    float v = 0.f;
    if (j >= 0 && j < N) {
        if (N & 1) {
            v = (i == N / 2 && j == N / 2) ? 1.f : 0.f;
        } else {
            const int m = N / 2;
            v = ((i == m - 1 || i == m) && (j == m - 1 || j == m)) ? 0.25f : 0.f;
        }
    }
    img[(size_t)i * ld + j] = v;
    imgT[(size_t)i * ld + j] = v;  // symmetric under transposition
}

// Row sums in double, one block of 256 per row.
__global__ void k_row_sums(const float* s, int cols, double* out) {
    __shared__ double red[256];
    const float* r = s + (size_t)blockIdx.x * cols;
    double acc = 0.0;
    for (int c = threadIdx.x; c < cols; c += 256) acc += (double)r[c];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[blockIdx.x] = red[0];
}

template <int DT>
__global__ void k_disc_subtract(const void* p, const float* wd, float g, float* pd, size_t n) {
    const auto* ps = static_cast<const typename Stor<DT>::T*>(p);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        pd[i] = fmaf(-g, wd[i], to_f32<DT>(ps[i]));
}

// hq += hc (double), u_k[a][m] = alpha * (odd nd: hq[a][m]; even nd: (hq[a][m] + hq[a][m+1]) / 2)
__global__ void k_filter_accum(const float* hc, double* hq, float* uk, int na, int nd, int ndp, double alpha) {
    const int a = blockIdx.y;
    const int nd2 = 2 * nd - 1;
    double* hr = hq + (size_t)a * ndp;
    const float* cr = hc + (size_t)a * ndp;
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < ndp; m += gridDim.x * blockDim.x) hr[m] += (double)cr[m];
    __syncthreads();  // one block per row (gridDim.x == 1): the row is complete here
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < nd2; m += gridDim.x * blockDim.x) {
        const double v = (nd & 1) ? hr[m] : 0.5 * (hr[m] + hr[m + 1]);
        uk[(size_t)a * nd2 + m] = (float)(alpha * v);
    }
}

// c (padded) and its transpose -= alpha g (unpadded [N][N])
__global__ void k_axpy_padded(float* c, float* cT, int ld, const float* g, float alpha, int N) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;
    if (j >= N) return;
    const float gv = g[(size_t)i * N + j];
    c[(size_t)i * ld + j] = fmaf(-alpha, gv, c[(size_t)i * ld + j]);
    cT[(size_t)j * ld + i] = fmaf(-alpha, gv, cT[(size_t)j * ld + i]);
}

// Cp[k][a][d] = sum_e u[k][a][d - e + nd - 1] pd[a][e].  Block: 64 threads x 4 outputs
// (256 bins) x 4 filters of one angle; the bins e are taken 256 at a time with the taps
// they meet staged in shared memory.  For output d = dd + j (j < 4) and bin e the tap is
// m = dd + j - e + nd - 1; the block's taps for e in [e0, e0 + 256) and d in [d0, d0 + 256)
// lie in [mlo, mlo + 511) with mlo = d0 - e0 - 255 + nd - 1; a thread keeps the four taps
// of its outputs in registers and slides them by one each step of e.
constexpr int CV_T = 64, CV_D = 4, CV_K = 4, CV_E = 256, CV_TAPS = 516;
__global__ void __launch_bounds__(CV_T) k_filter_conv(const float* __restrict__ u, const float* __restrict__ pd,
                                                      float* __restrict__ Cp, int n, int na, int nd) {
    __shared__ float T[CV_K][CV_TAPS];
    __shared__ float P[CV_E];
    const int a = blockIdx.y;
    const int k0 = blockIdx.z * CV_K;
    const int d0 = blockIdx.x * (CV_T * CV_D);
    const int t = threadIdx.x;
    const int nd2 = 2 * nd - 1;
    float acc[CV_K][CV_D];
#pragma unroll
    for (int k = 0; k < CV_K; ++k)
#pragma unroll
        for (int j = 0; j < CV_D; ++j) acc[k][j] = 0.f;
    for (int e0 = 0; e0 < nd; e0 += CV_E) {
        __syncthreads();
        const int mlo = d0 - e0 - (CV_E - 1) + nd - 1;
        for (int i = t; i < CV_K * CV_TAPS; i += CV_T) {
            const int k = i / CV_TAPS, li = i - k * CV_TAPS, m = mlo + li;
            float v = 0.f;
            if (k0 + k < n && m >= 0 && m < nd2) v = u[((size_t)(k0 + k) * na + a) * nd2 + m];
            T[k][li] = v;
        }
        for (int i = t; i < CV_E; i += CV_T) P[i] = (e0 + i < nd) ? pd[(size_t)a * nd + e0 + i] : 0.f;
        __syncthreads();
        float w[CV_K][CV_D];
#pragma unroll
        for (int k = 0; k < CV_K; ++k)
#pragma unroll
            for (int j = 0; j < CV_D; ++j) w[k][j] = T[k][CV_D * t + j + CV_E - 1];
        for (int i = 0; i < CV_E; ++i) {
            const float pe = P[i];
#pragma unroll
            for (int k = 0; k < CV_K; ++k) {
#pragma unroll
                for (int j = 0; j < CV_D; ++j) acc[k][j] = fmaf(w[k][j], pe, acc[k][j]);
#pragma unroll
                for (int j = CV_D - 1; j > 0; --j) w[k][j] = w[k][j - 1];
                w[k][0] = (i + 1 < CV_E) ? T[k][CV_D * t + CV_E - 2 - i] : 0.f;
            }
        }
    }
#pragma unroll
    for (int k = 0; k < CV_K; ++k) {
        if (k0 + k >= n) continue;
#pragma unroll
        for (int j = 0; j < CV_D; ++j) {
            const int d = d0 + CV_D * t + j;
            if (d < nd) Cp[((size_t)(k0 + k) * na + a) * nd + d] = acc[k][j];
        }
    }
}

// win[a][j] = Cp_k[rec[a].aidx][rec[a].d0 + j] for j < width, 0 up to stride
__global__ void k_window_gather(const float* Cp_k, int nd, const AngleRec* rec, int stride, float* win) {
    const int a = blockIdx.y;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= stride) return;
    const AngleRec& r = rec[a];
    win[(size_t)a * stride + j] = j < r.width ? Cp_k[(size_t)r.aidx * nd + r.d0 + j] : 0.f;
}

// One step of Alg. method per pixel: s = xs + y - alpha g; x = clamp(s + sh, lo, hi) - sh;
// y = x - xs; y also into the padded images the forward projector reads.
__global__ void k_filter_update(const float* xs, const float* g, float* y, float* x, const float* sh, float lo,
                                float hi, float alpha, float* ya, int lda, float* yaT, int ldaT, int nx, int ny) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;
    if (j >= nx) return;
    const size_t o = (size_t)i * nx + j;
    const float s = fmaf(-alpha, g[o], xs[o] + y[o]);
    const float shv = sh[o];
    const float xv = fminf(fmaxf(s + shv, lo), hi) - shv;
    const float yv = xv - xs[o];
    x[o] = xv;
    y[o] = yv;
    ya[(size_t)i * lda + j] = yv;
    yaT[(size_t)j * ldaT + i] = yv;
}

// shift = g * D on the box (the disc added back after the reconstruction)
__global__ void k_disc_box(float* shift, int x0, int y0, int nx, int ny, int N, float g) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;
    if (j >= nx) return;
    const float half = 0.5f * (float)(N - 1);
    const float x = (float)(x0 + j) - half, y = half - (float)(y0 + i);
    shift[(size_t)i * nx + j] = (x * x + y * y <= 0.25f * (float)N * (float)N) ? g : 0.f;
}

// out = x + shift
__global__ void k_add(const float* x, const float* shift, float* out, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = x[i] + shift[i];
}

// Tiling (Sec. 5.5): out[y][x] for the pixels of tile t, copied from that tile's box result.
struct TileSrc {
    const float* box;   // [bh][bw]
    int bw, tx, ty;     // box width; tile origin inside the box
    int gx, gy;         // tile origin on the grid
};
__global__ void k_paste_tiles(const TileSrc* tiles, int T, float* out, int N) {
    const TileSrc t = tiles[blockIdx.z];
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= T || j >= T) return;
    out[(size_t)(t.gy + i) * N + t.gx + j] = t.box[(size_t)(t.ty + i) * t.bw + t.tx + j];
}

int blocks_for(size_t n) { return (int)((n + 255) / 256 < 152 * 8 ? (n + 255) / 256 : 152 * 8); }

}  // namespace

void launch_disc_image(float* img, float* imgT, int ld, int N, cudaStream_t st) {
    count_launches(1);
    k_disc_image<<<dim3((N + 127) / 128, N), 128, 0, st>>>(img, imgT, ld, N);
}

void launch_impulse(float* img, float* imgT, int ld, int N, cudaStream_t st) {
    count_launches(1);
    k_impulse<<<dim3((ld + 127) / 128, N), 128, 0, st>>>(img, imgT, ld, N);
}

void launch_row_sums(const float* s, int rows, int cols, double* out, cudaStream_t st) {
    count_launches(1);
    k_row_sums<<<rows, 256, 0, st>>>(s, cols, out);
}

void launch_disc_subtract(const void* p, int dt, const float* wd, float g, float* pd, size_t n, cudaStream_t st) {
    count_launches(1);
    if (dt == 1)
        k_disc_subtract<1><<<blocks_for(n), 256, 0, st>>>(p, wd, g, pd, n);
    else if (dt == 2)
        k_disc_subtract<2><<<blocks_for(n), 256, 0, st>>>(p, wd, g, pd, n);
    else
        k_disc_subtract<0><<<blocks_for(n), 256, 0, st>>>(p, wd, g, pd, n);
}

void launch_filter_accum(const float* hc, double* hq, float* uk, int na, int nd, int ndp, double alpha,
                         cudaStream_t st) {
    count_launches(1);
    k_filter_accum<<<dim3(1, na), 256, 0, st>>>(hc, hq, uk, na, nd, ndp, alpha);  // one block per row
}

void launch_axpy_padded(float* c, float* cT, int ld, const float* g, float alpha, int N, cudaStream_t st) {
    count_launches(1);
    k_axpy_padded<<<dim3((N + 127) / 128, N), 128, 0, st>>>(c, cT, ld, g, alpha, N);
}

void launch_filter_conv(const float* u, const float* pd, float* Cp, int n, int na, int nd, cudaStream_t st) {
    if (n <= 0 || na <= 0 || nd <= 0) return;
    count_launches(1);
    dim3 grid((nd + CV_T * CV_D - 1) / (CV_T * CV_D), na, (n + CV_K - 1) / CV_K);
    k_filter_conv<<<grid, CV_T, 0, st>>>(u, pd, Cp, n, na, nd);
}

void launch_window_gather(const float* Cp_k, int nd, const AngleRec* rec, int na, int stride, float* win,
                          cudaStream_t st) {
    count_launches(1);
    k_window_gather<<<dim3((stride + 127) / 128, na), 128, 0, st>>>(Cp_k, nd, rec, stride, win);
}

void launch_filter_update(const float* xs, const float* g, float* y, float* x, const float* shift, float lo, float hi,
                          float alpha, float* ya, int lda, float* yaT, int ldaT, int nx, int ny, cudaStream_t st) {
    count_launches(1);
    k_filter_update<<<dim3((nx + 127) / 128, ny), 128, 0, st>>>(xs, g, y, x, shift, lo, hi, alpha, ya, lda, yaT, ldaT,
                                                               nx, ny);
}

void launch_disc_box(float* shift, int x0, int y0, int nx, int ny, int N, float g, cudaStream_t st) {
    count_launches(1);
    k_disc_box<<<dim3((nx + 127) / 128, ny), 128, 0, st>>>(shift, x0, y0, nx, ny, N, g);
}

void launch_paste_tiles(const void* tiles, int ntiles, int T, float* out, int N, cudaStream_t st) {
    if (ntiles <= 0) return;
    count_launches(1);
    dim3 grid((T + 31) / 32, (T + 7) / 8, ntiles);
    k_paste_tiles<<<grid, dim3(32, 8), 0, st>>>(static_cast<const TileSrc*>(tiles), T, out, N);
}
size_t tile_src_bytes() { return sizeof(TileSrc); }
void tile_src_fill(void* dst, int k, const float* box, int bw, int tx, int ty, int gx, int gy) {
    static_cast<TileSrc*>(dst)[k] = TileSrc{box, bw, tx, ty, gx, gy};
}

void launch_add(const float* x, const float* shift, float* out, size_t n, cudaStream_t st) {
    count_launches(1);
    k_add<<<blocks_for(n), 256, 0, st>>>(x, shift, out, n);
}

}  // namespace roi
