// project.cu -- Joseph forward projector W (ray-driven) and its exact transpose W^T
// (pixel-driven gather), on a frame of the grid, with fused solver epilogues.
//
// Paper Sec. 2.1: W maps an N x N image to N_theta N_d line integrals, computed on the
// fly; W_L = W M_L and W_L^T = M_L W^T restrict both to the local part L (Eq. locouter).
//
// Discretisation (Joseph): ray (theta, t) is sampled once per image row when
// |cos| >= |sin| (per column otherwise); at each sample the image is linearly
// interpolated between the two nearest pixels of that row (column); the sum is
// scaled by 1/|cos| (1/|sin|).  Its transpose gives pixel (i, j) at angle theta the
// weight (1 - |t_d - t_ij|/w)/w from every bin d with |t_d - t_ij| < w.
//
// Precision: coordinates are anchored in double precision (per 32-sample segment
// of a ray, per 32 x 32 tile and angle of the gather) and only short offsets
// (|offset| <= 16 samples) are formed in float, so interpolation positions carry
// an error of about 1e-6 pixel whatever the size of the grid.  Sums are formed in
// float over at most 32 terms (one ray segment, one chunk of 32 angles) and carried
// across segments and chunks in double, so a 4096-sample ray or a 1024-angle
// backprojection rounds like a 32-term float sum.
#include <cuda_runtime.h>

#include <algorithm>

#include "roi_internal.h"

namespace roi {

namespace {

constexpr int FWD_THREADS = 64;   // rays per block (one angle per block row)
constexpr int SEG = 32;           // samples per double-precision anchor

template <int MODE>
__global__ void __launch_bounds__(FWD_THREADS) k_forward(FwdArgs A) {
    const int a = blockIdx.y;
    const int k = blockIdx.x * FWD_THREADS + threadIdx.x;
    if (k >= A.stride) return;
    const AngleRec& r = A.rec[a];
    float* out = A.out + (size_t)a * A.stride + k;
    if (k >= r.width) {                       // padding of the window row
        if (MODE != FWD_CP) *out = 0.f;
        return;
    }
    const int row = r.row;
    const int M = row ? A.ny : A.nx;          // samples along the ray
    const int Mm = row ? A.nx : A.ny;         // extent of the interpolation axis
    const float* src = row ? A.img : A.imgT;  // [M][Mm]
    // hole (exterior step): major range [hM0, hM1), minor range [hm0, hm1)
    int hM0 = 0, hM1 = 0, hm0 = 0, hm1 = 0;
    if (MODE == FWD_EXTERIOR && A.hole.w > 0) {
        hM0 = row ? A.hole.y0 : A.hole.x0;
        hM1 = hM0 + (row ? A.hole.h : A.hole.w);
        hm0 = row ? A.hole.x0 : A.hole.y0;
        hm1 = hm0 + (row ? A.hole.w : A.hole.h);
    }
    const double Ak = r.A0 + (double)k * r.a_scale;
    const float slope = (float)r.slope;
    const double halfM = 0.5 * (M - 1);
    double accd = 0.0;
    for (int m0 = 0; m0 < M; m0 += SEG) {
        float acc = 0.f;
        // minor coordinate at the segment's centre sample m0 + 15.5, in double, split
        // into an integer part and a fraction so that float offsets stay small
        const double bd = Ak + ((double)m0 + 0.5 * (SEG - 1) - halfM) * r.slope;
        const double bfl = floor(bd);
        const int bi = (int)bfl;
        const float bf = (float)(bd - bfl);
        const int mend = min(m0 + SEG, M);
        for (int m = m0; m < mend; ++m) {
            const float q = fmaf((float)(m - m0) - 0.5f * (SEG - 1), slope, bf);
            const float fl = floorf(q);
            const int j0 = bi + (int)fl;
            const float f = q - fl;
            const float* rp = src + (size_t)m * Mm;
            bool ok0 = (j0 >= 0) & (j0 < Mm);
            bool ok1 = (j0 + 1 >= 0) & (j0 + 1 < Mm);
            if (MODE == FWD_EXTERIOR) {
                if (m >= hM0 && m < hM1) {
                    ok0 &= !(j0 >= hm0 && j0 < hm1);
                    ok1 &= !(j0 + 1 >= hm0 && j0 + 1 < hm1);
                }
            }
            const float v0 = ok0 ? __ldg(rp + j0) : 0.f;
            const float v1 = ok1 ? __ldg(rp + j0 + 1) : 0.f;
            acc += fmaf(f, v1 - v0, v0);
        }
        accd += (double)acc;
    }
    if (MODE == FWD_EXTERIOR) {
        *out = (float)((double)A.p[(size_t)a * A.nd + r.d0 + k] - accd * (double)r.inv_w);
        return;
    }
    const float acc = (float)(accd * (double)r.inv_w);
    if (MODE == FWD_PLAIN) {
        *out = acc;
    } else if (MODE == FWD_SIRT) {
        const size_t o = (size_t)a * A.stride + k;
        float res = A.pp[o] - acc;
        if (A.R) res *= A.R[o];
        *out = res;
    } else {  // FWD_CP: prox of the conjugate of ||. - p'||^2
        const size_t o = (size_t)a * A.stride + k;
        const float sig = A.R ? A.R[o] : A.sig_scalar;
        *out = (*out + sig * (acc - A.pp[o])) / (1.f + 0.5f * sig);
    }
}

// ----------------------------------------------------------------------------
// Gather backprojector.  Block = 32 x 8 threads, tile = 32 x 32 pixels, 4 pixels
// per thread (rows ty, ty+8, ty+16, ty+24).  For each chunk of CH angles the
// window bins the tile can reach are staged in shared memory: tile pixels lie
// within 15.5 (|c| + |s|) <= 21.93 of the tile centre in window coordinates and
// the hat reaches one more bin, so with kbase = floor(kappa_centre) - 25 every
// index touched is in [3, 48] < SB.
constexpr int BT_X = 32, BT_Y = 8, PPT = 4, TILE = 32;
constexpr int CH = 32;   // angles per staging chunk
constexpr int SB = 52;   // staged bins per angle

template <int MODE>
__global__ void __launch_bounds__(BT_X* BT_Y) k_back(BackArgs A) {
    __shared__ float stage[CH][SB];
    __shared__ float4 cst[CH];   // c, s, inv_w, kappa relative to kbase
    __shared__ int kb[CH];
    __shared__ float tr[TILE][TILE + 1];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * BT_X + tx;
    const int tile_x0 = blockIdx.x * TILE, tile_y0 = blockIdx.y * TILE;
    // tile centre relative to frame centre
    const double xi_t = tile_x0 + 0.5 * (TILE - 1) - 0.5 * (A.nx - 1);
    const double eta_t = 0.5 * (A.ny - 1) - (tile_y0 + 0.5 * (TILE - 1));
    const float dlj = (float)tx - 0.5f * (TILE - 1);
    double accd[PPT];
#pragma unroll
    for (int p = 0; p < PPT; ++p) accd[p] = 0.0;

    for (int a0 = 0; a0 < A.na; a0 += CH) {
        const int nch = min(CH, A.na - a0);
        __syncthreads();
        if (tid < nch) {
            const AngleRec& r = A.rec[a0 + tid];
            const double kt = xi_t * r.c + eta_t * r.s - r.phi;
            const double fb = floor(kt) - 25.0;
            kb[tid] = (int)fb;
            cst[tid] = make_float4((float)r.c, (float)r.s, r.inv_w, (float)(kt - fb));
        }
        __syncthreads();
        for (int e = tid; e < nch * SB; e += BT_X * BT_Y) {
            const int al = e / SB, b = e - al * SB;
            const int kk = kb[al] + b;
            const int wdt = A.rec[a0 + al].width;
            stage[al][b] = (kk >= 0 && kk < wdt) ? __ldg(A.win + (size_t)(a0 + al) * A.stride + kk) : 0.f;
        }
        __syncthreads();
        float acc[PPT];
#pragma unroll
        for (int p = 0; p < PPT; ++p) acc[p] = 0.f;
        for (int al = 0; al < nch; ++al) {
            const float4 cc = cst[al];
            const float iw = cc.z, iw2 = cc.z * cc.z;
            // pixel rows ty + 8p: kappa = kr + dlj c - dli s, dli = ty + 8p - 15.5
            const float k0 = fmaf(dlj, cc.x, fmaf(-((float)ty - 0.5f * (TILE - 1)), cc.y, cc.w));
            const float* srow = stage[al];
#pragma unroll
            for (int p = 0; p < PPT; ++p) {
                const float kap = fmaf(-(float)(BT_Y * p), cc.y, k0);
                const float fl = floorf(kap);
                const int kl = (int)fl;
                const float f = kap - fl;
                const float w0 = fmaxf(0.f, fmaf(-f, iw2, iw));
                const float w1 = fmaxf(0.f, fmaf(f, iw2, iw - iw2));
                acc[p] = fmaf(w0, srow[kl], fmaf(w1, srow[kl + 1], acc[p]));
            }
        }
#pragma unroll
        for (int p = 0; p < PPT; ++p) accd[p] += (double)acc[p];
    }
    float acc[PPT];
#pragma unroll
    for (int p = 0; p < PPT; ++p) acc[p] = (float)accd[p];

    // epilogue
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
        const int li = tile_y0 + ty + BT_Y * p, lj = tile_x0 + tx;
        float val = 0.f;
        if (li < A.ny && lj < A.nx) {
            const size_t o = (size_t)li * A.nx + lj;
            if (MODE == BACK_PLAIN) {
                val = acc[p];
                A.out[o] = val;
            } else if (MODE == BACK_SIRT) {
                const float step = A.C ? A.C[o] : A.step_scalar;
                float xn = fmaf(step, acc[p], A.out[o]);
                if (A.nonneg) xn = fmaxf(xn, 0.f);
                A.out[o] = xn;
                val = xn;
            } else {  // BACK_CP
                // div v = vx[i][j] - vx[i][j-1] + vy[i][j] - vy[i-1][j], terms outside the
                // gradient's range (last column of vx, last row of vy, j-1 < 0, i-1 < 0) left out
                float dv = 0.f;
                if (lj < A.nx - 1) dv += A.vx[o];
                if (lj > 0) dv -= A.vx[o - 1];
                if (li < A.ny - 1) dv += A.vy[o];
                if (li > 0) dv -= A.vy[o - A.nx];
                const float tau = A.C ? A.C[o] : A.step_scalar;
                const float xo = A.out[o];
                const float xn = xo - tau * (acc[p] - dv);
                A.out[o] = xn;
                val = 2.f * xn - xo;
                A.xbar[o] = val;
            }
        }
        tr[ty + BT_Y * p][tx] = val;
    }
    if (A.outT) {
        __syncthreads();
#pragma unroll
        for (int p = 0; p < PPT; ++p) {
            // write outT[lj][li]: lane tx runs along li
            const int lj = tile_x0 + ty + BT_Y * p, li = tile_y0 + tx;
            if (li < A.ny && lj < A.nx) A.outT[(size_t)lj * A.ny + li] = tr[tx][ty + BT_Y * p];
        }
    }
}

__global__ void k_transpose(const float* __restrict__ in, float* __restrict__ out, int rows, int cols) {
    __shared__ float t[32][33];
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int r = by + y, c = bx + threadIdx.x;
        if (r < rows && c < cols) t[y][threadIdx.x] = in[(size_t)r * cols + c];
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int c = bx + y, r = by + threadIdx.x;
        if (r < rows && c < cols) out[(size_t)c * rows + r] = t[threadIdx.x][y];
    }
}

__global__ void k_fill(float* p, float v, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        p[i] = v;
}

__global__ void k_window_ones(float* win, const AngleRec* rec, int na, int stride) {
    const int a = blockIdx.y;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (a < na && k < stride) win[(size_t)a * stride + k] = k < rec[a].width ? 1.f : 0.f;
}

}  // namespace

void launch_forward(FwdMode mode, const FwdArgs& a, cudaStream_t st) {
    if (a.na <= 0 || a.stride <= 0) return;
    dim3 grid((a.stride + FWD_THREADS - 1) / FWD_THREADS, a.na);
    switch (mode) {
        case FWD_PLAIN: count_launches(1); k_forward<FWD_PLAIN><<<grid, FWD_THREADS, 0, st>>>(a); break;
        case FWD_EXTERIOR: count_launches(1); k_forward<FWD_EXTERIOR><<<grid, FWD_THREADS, 0, st>>>(a); break;
        case FWD_SIRT: count_launches(1); k_forward<FWD_SIRT><<<grid, FWD_THREADS, 0, st>>>(a); break;
        case FWD_CP: count_launches(1); k_forward<FWD_CP><<<grid, FWD_THREADS, 0, st>>>(a); break;
    }
}

void launch_back(BackMode mode, const BackArgs& a, cudaStream_t st) {
    if (a.nx <= 0 || a.ny <= 0) return;
    dim3 grid((a.nx + TILE - 1) / TILE, (a.ny + TILE - 1) / TILE);
    dim3 block(BT_X, BT_Y);
    switch (mode) {
        case BACK_PLAIN: count_launches(1); k_back<BACK_PLAIN><<<grid, block, 0, st>>>(a); break;
        case BACK_SIRT: count_launches(1); k_back<BACK_SIRT><<<grid, block, 0, st>>>(a); break;
        case BACK_CP: count_launches(1); k_back<BACK_CP><<<grid, block, 0, st>>>(a); break;
    }
}

void launch_transpose(const float* in, float* out, int rows, int cols, cudaStream_t st) {
    if (rows <= 0 || cols <= 0) return;
    dim3 grid((cols + 31) / 32, (rows + 31) / 32);
    count_launches(1);
    k_transpose<<<grid, dim3(32, 8), 0, st>>>(in, out, rows, cols);
}

void launch_fill(float* p, float v, size_t n, cudaStream_t st) {
    if (n == 0) return;
    int blocks = (int)std::min<size_t>((n + 255) / 256, 152 * 8);
    count_launches(1);
    k_fill<<<blocks, 256, 0, st>>>(p, v, n);
}

void launch_window_ones(float* win, const AngleRec* rec, int na, int stride, cudaStream_t st) {
    if (na <= 0 || stride <= 0) return;
    dim3 grid((stride + 127) / 128, na);
    count_launches(1);
    k_window_ones<<<grid, 128, 0, st>>>(win, rec, na, stride);
}

}  // namespace roi
