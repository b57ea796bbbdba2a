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
// Precision without FP64 (1/64 of the FP32 rate on GB300): coordinates are anchored in
// float-float (per 16-sample segment of a ray, per 32 x 16 tile and angle of the
// gather) and only short offsets are formed in float, so interpolation positions
// carry an error of about 1e-6 pixel whatever the size of the grid.  Sums are formed
// in float over at most 32 terms and carried across segments / angle chunks with
// Neumaier compensation.
//
// Work decomposition (GB300: 152 SMs, up to 2048 resident threads each):
//   forward: a block is 32 consecutive rays of one angle x S segments of the ray;
//            segment partial sums are added in segment order through shared memory.
//   back:    a block is a 32 x 16 pixel tile x one of G contiguous angle groups;
//            with G > 1 each group writes a partial image and k_combine adds the G
//            partials in group order before the solver epilogue.
//   S and G depend only on the sizes (never on other work in flight), so a result
//   is bit-identical however it is scheduled.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "check.cuh"
#include "dev_common.cuh"
#include "roi_internal.h"

namespace roi {

namespace {

constexpr int FWD_RAYS = 32;      // rays per block (one angle per block)
constexpr int FWD_MAXSEG = 8;     // segments per ray (blockDim.y)
constexpr int SEG = 16;           // samples per float-float anchor
constexpr int TARGET_THREADS = 152 * 2048;

// Forward projector.  Images are padded: `src` points at element (0, 0) of rows of
// stride `ld` that carry two zero columns on each side, so minor indices -2 .. Mm+1
// are readable.  The loop visits only the samples whose minor coordinate q lies in
// [-1.5, Mm + 0.5] (range computed per ray in float: its error, ~1e-4 pixel, is far
// below the 0.5 margin), so floor(q) stays in [-2, Mm] and both taps in [-2, Mm + 1];
// every sample outside the range has both taps outside [0, Mm) and contributes 0.
// Positions: each 16-sample segment is anchored in float-float, then offsets
// |m - anchor| <= 8 are formed in float.  Sums: float within a segment, Neumaier
// carry across segments, float-float across the S threads of a ray.
template <int MODE, int DT, int PDT = DT>
__global__ void __launch_bounds__(FWD_RAYS* FWD_MAXSEG) k_forward(const FwdArgs A) {
    using T = typename Stor<DT>::T;   // element of the frame image: float or 16-bit
    using TP = typename Stor<PDT>::T;  // element of p (FWD_EXTERIOR)
    __shared__ float red_s[FWD_MAXSEG][FWD_RAYS];
    __shared__ float red_c[FWD_MAXSEG][FWD_RAYS];
    const int a = blockIdx.y;
    const int k = blockIdx.x * FWD_RAYS + threadIdx.x;
    const int seg = threadIdx.y;
    const AngleRec& r = A.rec[a];
    const bool valid = k < r.width;
    float sum = 0.f, cmp = 0.f;
    if (valid) {
        const int row = r.row;
        const int M = row ? A.ny : A.nx;           // samples along the ray
        const int Mm = row ? A.nx : A.ny;          // extent of the interpolation axis
        const T* src = static_cast<const T*>(row ? A.img : A.imgT);  // [M][ld], element (0,0)
        const int ld = row ? A.img_ld : A.imgT_ld;
        const float halfM = 0.5f * (float)(M - 1);
        const ff Ak = ff_add(r.A0, ff_mul_f((float)k, r.a_scale));
        // samples m with q(m) = Ak + (m - halfM) slope in [-1.5, Mm + 0.5]
        int mlo = 0, mhi = M;
        if (!r.flat) {
            const float ma = (-1.5f - Ak.hi) * r.inv_slope + halfM;
            const float mb = ((float)Mm + 0.5f - Ak.hi) * r.inv_slope + halfM;
            const float lo = fminf(ma, mb), hi = fmaxf(ma, mb);
            mlo = (int)fminf(fmaxf(0.f, ceilf(lo)), (float)M);
            mhi = (int)fmaxf(fminf((float)M, floorf(hi) + 1.f), 0.f);
        } else if (!(Ak.hi >= -1.5f && Ak.hi <= (float)Mm + 0.5f)) {
            mhi = 0;
        }
        // this thread's segment of the ray
        const int s0 = seg * A.seg_len, s1 = min(s0 + A.seg_len, M);
        mlo = max(mlo, s0);
        mhi = min(mhi, s1);
        // hole (exterior step): major range [hM0, hM1), minor range [hm0, hm1)
        int hM0 = 0, hM1 = 0, hm0 = 0, hm1 = 0;
        if (MODE == FWD_EXTERIOR && A.hole.w > 0) {
            hM0 = row ? A.hole.y0 : A.hole.x0;
            hM1 = hM0 + (row ? A.hole.h : A.hole.w);
            hm0 = row ? A.hole.x0 : A.hole.y0;
            hm1 = hm0 + (row ? A.hole.w : A.hole.h);
        }
        const float slope = r.slope.hi;
        for (int m0 = mlo; m0 < mhi; m0 += SEG) {
            // minor coordinate at the anchor m0 + 7.5: Ak + (m0 + 7.5 - halfM) slope
            const ff bd = ff_add(Ak, ff_mul_f((float)m0 + 0.5f * (SEG - 1) - halfM, r.slope));
            const float bfl = floorf(bd.hi);
            const int bi = (int)bfl;
            const float bf = (bd.hi - bfl) + bd.lo;
            const int mend = min(m0 + SEG, mhi);
            float acc = 0.f;
            const T* rp = src + (size_t)m0 * ld + bi;
            const int jlo = -kPad - bi, jhi = ld - 1 - kPad - bi;  // taps j, j + 1 inside the padded row
#pragma unroll 4
            for (int m = m0; m < mend; ++m, rp += ld) {
                const float q = fmaf((float)(m - m0) - 0.5f * (SEG - 1), slope, bf);
                const float fl = floorf(q);
                const int j = chk((int)fl, jlo, jhi, CHK_FORWARD);
                const float f = q - fl;
                float v0 = to_f32<DT>(__ldg(rp + j));
                float v1 = to_f32<DT>(__ldg(rp + j + 1));
                if (MODE == FWD_EXTERIOR) {
                    if (m >= hM0 && m < hM1) {
                        const int j0 = bi + j;
                        if (j0 >= hm0 && j0 < hm1) v0 = 0.f;
                        if (j0 + 1 >= hm0 && j0 + 1 < hm1) v1 = 0.f;
                    }
                }
                acc += fmaf(f, v1 - v0, v0);
            }
            neu_add(sum, cmp, acc);
        }
    }
    ff tot = two_sum(sum, cmp);
    if (blockDim.y > 1) {
        red_s[seg][threadIdx.x] = tot.hi;
        red_c[seg][threadIdx.x] = tot.lo;
        __syncthreads();
        if (seg != 0) return;
        for (int s = 1; s < (int)blockDim.y; ++s) {
            ff o;
            o.hi = red_s[s][threadIdx.x];
            o.lo = red_c[s][threadIdx.x];
            tot = ff_add(tot, o);
        }
    }
    if (k >= A.stride) return;
    float* out = A.out + (size_t)a * A.stride + k;
    if (!valid) {                              // padding of the window row
        if (MODE != FWD_CP) *out = 0.f;
        return;
    }
    tot = ff_mul_f(r.inv_w, tot);
    if (MODE == FWD_EXTERIOR) {  // p - sum, with the float-float sum
        const float pv = to_f32<PDT>(__ldg(static_cast<const TP*>(A.p) + (size_t)r.aidx * A.nd + r.d0 + k));
        const ff d = two_sum(pv, -tot.hi);
        *out = d.hi + (d.lo - tot.lo);
        return;
    }
    const float acc = tot.hi + tot.lo;
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
// Gather backprojector.  Block = 32 x 8 threads, tile = 32 x 16 pixels, 2 pixels per
// thread (rows ty and ty + 8).  For each chunk of CH angles the window bins the tile
// can reach are staged in shared memory: tile pixels lie within
// max(15.5 |c| + 7.5 |s|) = sqrt(15.5^2 + 7.5^2) = 17.22 of the tile centre in window
// coordinates and the hat reaches one bin further, so with kbase = floor(kappa_c) - 19
// every staged index touched is in [1, 38] < SB.
constexpr int BT_X = 32, BT_Y = 8, PPT = 2, TILE_X = 32, TILE_Y = BT_Y * PPT;
constexpr int CH = 32;   // angles per staging chunk
constexpr int KOFF = 19;
constexpr int SB = 40;   // staged bins per angle

// Solver epilogue for pixel (li, lj): returns the value whose transpose is stored.
template <int MODE>
__device__ __forceinline__ float back_epilogue(const BackArgs& A, int li, int lj, float acc) {
    const size_t o = (size_t)li * A.nx + lj;                  // unpadded [ny][nx] arrays
    float* xo = A.out + (size_t)li * A.out_ld + lj;
    if (MODE == BACK_PLAIN) {
        if (A.fov_d > 0) {  // doubled centre coordinates, exact in integers
            const long long X = 2LL * lj - (A.nx - 1), Y = (long long)(A.ny - 1) - 2LL * li;
            if (X * X + Y * Y > (long long)A.fov_d * A.fov_d) acc = 0.f;
        }
        *xo = acc;
        return acc;
    } else if (MODE == BACK_SIRT) {
        const float step = A.C ? A.C[o] : A.step_scalar;
        float xn = fmaf(step, acc, *xo);
        if (A.nonneg) xn = fmaxf(xn, 0.f);
        *xo = xn;
        return xn;
    } else {  // BACK_CP
        // div v = vx[i][j] - vx[i][j-1] + vy[i][j] - vy[i-1][j], terms outside the
        // gradient's range (last column of vx, last row of vy, j-1 < 0, i-1 < 0) left out
        float dv = 0.f;
        if (lj < A.nx - 1) dv += A.vx[o];
        if (lj > 0) dv -= A.vx[o - 1];
        if (li < A.ny - 1) dv += A.vy[o];
        if (li > 0) dv -= A.vy[o - A.nx];
        const float tau = A.C ? A.C[o] : A.step_scalar;
        const float xold = *xo;
        const float xn = xold - tau * (acc - dv);
        *xo = xn;
        const float xb = 2.f * xn - xold;
        A.xbar[(size_t)li * A.xbar_ld + lj] = xb;
        return xb;
    }
}

template <int MODE>
__global__ void __launch_bounds__(BT_X* BT_Y) k_back(BackArgs A) {
    __shared__ float stage[CH][SB];
    __shared__ float4 cst[CH];   // c, s, inv_w, kappa relative to kbase
    __shared__ int kb[CH];
    __shared__ float tr[TILE_Y][TILE_X + 1];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * BT_X + tx;
    const int tile_x0 = blockIdx.x * TILE_X, tile_y0 = blockIdx.y * TILE_Y;
    const int G = gridDim.z, g = blockIdx.z;
    const int a_lo = (int)((long long)A.na * g / G), a_hi = (int)((long long)A.na * (g + 1) / G);
    // tile centre relative to frame centre (half-integers: exact in float)
    const float xi_t = (float)tile_x0 + 0.5f * (TILE_X - 1) - 0.5f * (float)(A.nx - 1);
    const float eta_t = 0.5f * (float)(A.ny - 1) - ((float)tile_y0 + 0.5f * (TILE_Y - 1));
    const float dlj = (float)tx - 0.5f * (TILE_X - 1);
    const float dli0 = (float)ty - 0.5f * (TILE_Y - 1);
    float sum[PPT], cmp[PPT];
#pragma unroll
    for (int p = 0; p < PPT; ++p) sum[p] = cmp[p] = 0.f;

    for (int a0 = a_lo; a0 < a_hi; a0 += CH) {
        const int nch = min(CH, a_hi - a0);
        __syncthreads();
        if (tid < nch) {
            // kappa at the tile centre, xi_t c + eta_t s - phi, in float-float
            const AngleRec& r = A.rec[a0 + tid];
            ff kt = ff_add(ff_mul_f(xi_t, r.c), ff_mul_f(eta_t, r.s));
            kt = ff_add(kt, ff{-r.phi.hi, -r.phi.lo});
            const float fl = floorf(kt.hi);
            kb[tid] = (int)fl - KOFF;
            cst[tid] = make_float4(r.c.hi, r.s.hi, r.inv_w, ((kt.hi - fl) + kt.lo) + (float)KOFF);
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
            const float iw = cc.z, iw2 = cc.z * cc.z, iwm = iw - iw2;
            // kappa = kr + dlj c - dli s for pixel rows dli = dli0 + 8p
            const float k0 = fmaf(dlj, cc.x, fmaf(-dli0, cc.y, cc.w));
            const float* srow = stage[al];
#pragma unroll
            for (int p = 0; p < PPT; ++p) {
                const float kap = p == 0 ? k0 : fmaf(-(float)(BT_Y * p), cc.y, k0);
                const float fl = floorf(kap);
                const int kl = chk((int)fl, 0, SB - 1, CHK_BACK);
                const float f = kap - fl;
                const float w0 = fmaxf(0.f, fmaf(-f, iw2, iw));
                const float w1 = fmaxf(0.f, fmaf(f, iw2, iwm));
                acc[p] = fmaf(w0, srow[kl], fmaf(w1, srow[kl + 1], acc[p]));
            }
        }
#pragma unroll
        for (int p = 0; p < PPT; ++p) neu_add(sum[p], cmp[p], acc[p]);
    }

    if (G > 1) {  // partial of this angle group; k_combine finishes
#pragma unroll
        for (int p = 0; p < PPT; ++p) {
            const int li = tile_y0 + ty + BT_Y * p, lj = tile_x0 + tx;
            if (li < A.ny && lj < A.nx) A.part[((size_t)g * A.ny + li) * A.nx + lj] = sum[p] + cmp[p];
        }
        return;
    }
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
        const int li = tile_y0 + ty + BT_Y * p, lj = tile_x0 + tx;
        float val = 0.f;
        if (li < A.ny && lj < A.nx) val = back_epilogue<MODE>(A, li, lj, sum[p] + cmp[p]);
        tr[ty + BT_Y * p][tx] = val;
    }
    if (A.outT) {
        __syncthreads();
        // outT[lj][li]: 16 consecutive li per lj
        const int lil = tid & (TILE_Y - 1), ljl = tid / TILE_Y;
        for (int c = ljl; c < TILE_X; c += (BT_X * BT_Y) / TILE_Y) {
            const int li = tile_y0 + lil, lj = tile_x0 + c;
            if (li < A.ny && lj < A.nx) A.outT[(size_t)lj * A.outT_ld + li] = tr[lil][c];
        }
    }
}

// Adds the G angle-group partials of each pixel in group order, then applies the
// solver epilogue.  Block 32 x 8, tile 32 x 32, 4 pixels per thread.
template <int MODE>
__global__ void __launch_bounds__(256) k_combine(BackArgs A, int G) {
    __shared__ float tr[32][33];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tile_x0 = blockIdx.x * 32, tile_y0 = blockIdx.y * 32;
    const size_t plane = (size_t)A.nx * A.ny;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const int li = tile_y0 + ty + 8 * p, lj = tile_x0 + tx;
        float val = 0.f;
        if (li < A.ny && lj < A.nx) {
            const size_t o = (size_t)li * A.nx + lj;
            float s = A.part[o], c = 0.f;
            for (int gg = 1; gg < G; ++gg) neu_add(s, c, A.part[gg * plane + o]);
            val = back_epilogue<MODE>(A, li, lj, s + c);
        }
        tr[ty + 8 * p][tx] = val;
    }
    if (A.outT) {
        __syncthreads();
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const int lj = tile_x0 + ty + 8 * p, li = tile_y0 + tx;
            if (li < A.ny && lj < A.nx) A.outT[(size_t)lj * A.outT_ld + li] = tr[tx][ty + 8 * p];
        }
    }
}

// out[r][c] = in[r][c] for a [rows][cols] image; in and out have row strides in_ld, out_ld.
__global__ void k_copy_pad(const float* __restrict__ in, int in_ld, float* __restrict__ out, int out_ld, int rows,
                           int cols) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y * blockDim.y + threadIdx.y;
    if (r < rows && c < cols) out[(size_t)r * out_ld + c] = in[(size_t)r * in_ld + c];
}

// out[c][r] = in[r][c]; in has row stride in_ld, out has row stride out_ld.
__global__ void k_transpose(const float* __restrict__ in, int in_ld, float* __restrict__ out, int out_ld, int rows,
                            int cols) {
    __shared__ float t[32][33];
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int r = by + y, c = bx + threadIdx.x;
        if (r < rows && c < cols) t[y][threadIdx.x] = in[(size_t)r * in_ld + c];
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int c = bx + y, r = by + threadIdx.x;
        if (r < rows && c < cols) out[(size_t)c * out_ld + r] = t[threadIdx.x][y];
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

int forward_segments(int na, int stride, int nx, int ny, int* seg_len) {
    const int M = std::max(nx, ny);
    const int chunks = (M + SEG - 1) / SEG;
    const long rays = (long)na * ((stride + FWD_RAYS - 1) / FWD_RAYS) * FWD_RAYS;
    int S = (int)std::max(1L, (TARGET_THREADS + rays / 2) / std::max(rays, 1L));
    S = std::min(S, std::min(FWD_MAXSEG, chunks));
    S = std::max(S, 1);
    const int cps = (chunks + S - 1) / S;  // anchor chunks per segment
    *seg_len = cps * SEG;
    return (chunks + cps - 1) / cps;
}

int back_groups(int na, int nx, int ny) {
    const long tiles = (long)((nx + TILE_X - 1) / TILE_X) * ((ny + TILE_Y - 1) / TILE_Y);
    const long threads = tiles * BT_X * BT_Y;
    int G = (int)std::max(1L, (TARGET_THREADS + threads / 2) / std::max(threads, 1L));
    G = std::min(G, 8);
    G = std::min(G, std::max(1, na / 16));  // at least 16 angles per group
    return std::max(G, 1);
}

void launch_forward(FwdMode mode, const FwdArgs& a0, cudaStream_t st) {
    if (a0.na <= 0 || a0.stride <= 0) return;
    FwdArgs a = a0;
    const int S = forward_segments(a.na, a.stride, a.nx, a.ny, &a.seg_len);
    dim3 grid((a.stride + FWD_RAYS - 1) / FWD_RAYS, a.na), block(FWD_RAYS, S);
    count_launches(1);
    switch (mode) {
        case FWD_PLAIN: k_forward<FWD_PLAIN, 0><<<grid, block, 0, st>>>(a); break;
        case FWD_EXTERIOR:  // image storage x sinogram storage
            switch (3 * a.dt + a.pdt) {
                case 1: k_forward<FWD_EXTERIOR, 0, 1><<<grid, block, 0, st>>>(a); break;
                case 2: k_forward<FWD_EXTERIOR, 0, 2><<<grid, block, 0, st>>>(a); break;
                case 3: k_forward<FWD_EXTERIOR, 1, 0><<<grid, block, 0, st>>>(a); break;
                case 4: k_forward<FWD_EXTERIOR, 1, 1><<<grid, block, 0, st>>>(a); break;
                case 5: k_forward<FWD_EXTERIOR, 1, 2><<<grid, block, 0, st>>>(a); break;
                case 6: k_forward<FWD_EXTERIOR, 2, 0><<<grid, block, 0, st>>>(a); break;
                case 7: k_forward<FWD_EXTERIOR, 2, 1><<<grid, block, 0, st>>>(a); break;
                case 8: k_forward<FWD_EXTERIOR, 2, 2><<<grid, block, 0, st>>>(a); break;
                default: k_forward<FWD_EXTERIOR, 0, 0><<<grid, block, 0, st>>>(a); break;
            }
            break;
        case FWD_SIRT: k_forward<FWD_SIRT, 0><<<grid, block, 0, st>>>(a); break;
        case FWD_CP: k_forward<FWD_CP, 0><<<grid, block, 0, st>>>(a); break;
    }
}

void launch_back(BackMode mode, const BackArgs& a, cudaStream_t st) {
    if (a.nx <= 0 || a.ny <= 0) return;
    const int G = a.part ? back_groups(a.na, a.nx, a.ny) : 1;
    dim3 grid((a.nx + TILE_X - 1) / TILE_X, (a.ny + TILE_Y - 1) / TILE_Y, G);
    dim3 block(BT_X, BT_Y);
    count_launches(1);
    switch (mode) {
        case BACK_PLAIN: k_back<BACK_PLAIN><<<grid, block, 0, st>>>(a); break;
        case BACK_SIRT: k_back<BACK_SIRT><<<grid, block, 0, st>>>(a); break;
        case BACK_CP: k_back<BACK_CP><<<grid, block, 0, st>>>(a); break;
    }
    if (G > 1) {
        dim3 g2((a.nx + 31) / 32, (a.ny + 31) / 32);
        count_launches(1);
        switch (mode) {
            case BACK_PLAIN: k_combine<BACK_PLAIN><<<g2, dim3(32, 8), 0, st>>>(a, G); break;
            case BACK_SIRT: k_combine<BACK_SIRT><<<g2, dim3(32, 8), 0, st>>>(a, G); break;
            case BACK_CP: k_combine<BACK_CP><<<g2, dim3(32, 8), 0, st>>>(a, G); break;
        }
    }
}

void launch_copy_pad(const float* in, int in_ld, float* out, int out_ld, int rows, int cols, cudaStream_t st) {
    if (rows <= 0 || cols <= 0) return;
    dim3 grid((cols + 31) / 32, (rows + 7) / 8);
    count_launches(1);
    k_copy_pad<<<grid, dim3(32, 8), 0, st>>>(in, in_ld, out, out_ld, rows, cols);
}

void launch_transpose(const float* in, int in_ld, float* out, int out_ld, int rows, int cols, cudaStream_t st) {
    if (rows <= 0 || cols <= 0) return;
    dim3 grid((cols + 31) / 32, (rows + 31) / 32);
    count_launches(1);
    k_transpose<<<grid, dim3(32, 8), 0, st>>>(in, in_ld, out, out_ld, rows, cols);
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

ROI_CHECK_TU(project)

}  // namespace roi
