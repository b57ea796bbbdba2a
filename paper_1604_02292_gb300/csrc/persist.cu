// persist.cu -- one cooperative launch per local solve (boxes whose padded image fits
// in shared memory): all SIRT / Chambolle-Pock iterations run inside one kernel, with
// a grid-wide barrier between the two phases of an iteration.
//
// Iteration (paper Eq. sirtit / Eq. sirtbox for SIRT; Eq. priorsys with TV by
// Chambolle-Pock; the operators W_L, W_L^T of Sec. 2.1):
//   phase A  every block stages the whole padded image it projects (x for SIRT, xbar
//            for CP; rows or columns by the branch of its angles) into shared memory
//            and runs the ray-driven forward W_L on its share of (angle, 32-ray) units,
//            fusing  r = p' - W_L x  (SIRT)  or  u <- (u + sigma (W_L xbar - p'))/(1 + sigma/2)
//            and, for CP, the gradient dual  v <- proj_lambda(v + sigma_v grad xbar)
//            on its share of pixels;
//   barrier
//   phase B  every block takes 16 x 16 pixel tiles, stages the window bins the tile's
//            pixels reach for all angles, gathers W_L^T of r (or u) over all angles and
//            applies  x <- max(0, x + alpha (.))  (SIRT)  or
//            x+ = x - tau (W_L^T u - div v), xbar = 2 x+ - x  (CP),
//            writing the padded row and column copies the next phase A stages;
//   barrier.
// The arithmetic, the summation structure and the work split per ray / pixel are the
// ones of the multi-kernel path (project.cu), so both paths agree to rounding.
//
// The grid barrier spins on a generation counter with a time limit (one second by
// default, wall clock from %globaltimer): a block that waits longer sets the error flag
// and every block leaves at its next barrier; the host reports ROI_ETIMEOUT.  Blocks are co-resident by construction
// (cooperative launch of at most one block per SM).  Data written by other blocks in
// the previous phase are read with ld.global.cg (L2), never through L1.
#include <cuda_runtime.h>

#include <algorithm>

#include "roi_internal.h"

namespace roi {

namespace {

constexpr int PT = 1024;                 // threads per block
constexpr int NWARP = PT / 32;
constexpr int RAYS = 32;                 // rays per unit (one warp-wide ray group)
constexpr int FSEG = 4;                  // segments per ray in phase A
constexpr int UNITS_PER_PASS = NWARP / FSEG;
constexpr int SEGA = 16;                 // samples per float-float anchor
constexpr int BT = 16;                   // phase B tile side
constexpr int BPIX = BT * BT;
constexpr int QUART = PT / BPIX;         // angle groups per pixel in phase B
// tile pixels lie within 7.5 (|c| + |s|) <= 10.61 of the tile centre in window
// coordinates and the hat reaches one bin further: with kbase = floor(kappa_c) - 12
// every staged index touched is in [1, 24] < BSB
constexpr int BKOFF = 12;
constexpr int BSB = 26;

struct PArgs {
    const AngleRec* rec;
    int na, stride, nx, ny;
    int mode;               // 0 SIRT, 1 CP
    int iters;
    // padded images read by phase A: row layout [ny][lda], column layout [nx][ldaT];
    // *_base is the start of the buffer (row 0, column -2), *0 element (0, 0)
    float* xa_base;
    float* xaT_base;
    int lda, ldaT;
    // windows [na][stride]
    float* u;               // SIRT residual / CP dual
    const float* pp;
    const float* R;         // SIRT weights / CP sigma_u (null: scalar)
    float sig_scalar;
    // box arrays [ny][nx]
    float* x;               // CP primal (SIRT iterates in xa)
    float* vx;
    float* vy;
    const float* C;         // SIRT column weights / CP tau (null: scalar)
    float step_scalar;
    const float* sigma_v_dev;
    float sigma_v;
    float lambda;
    int nonneg;
    // grid barrier
    unsigned* bar;          // [0] arrivals, [1] generation
    unsigned expect;        // participants: gridDim.x (+ phantoms when testing the time limit)
    int* err;
    unsigned long long wait_ns;  // time limit of one barrier wait
    // phase A partition
    int nchunk;             // 32-ray chunks per angle
    int units;              // na * nchunk
    int img_floats;         // floats of the larger padded image (smem region size)
};

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Generation-counting grid barrier with a time limit.  Returns 0 (in every thread of
// the block) when this or another block gave up; the caller then returns.
__device__ __forceinline__ int grid_sync(const PArgs& A, int* s_flag) {
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile unsigned* gen = A.bar + 1;
        const unsigned g = *gen;
        __threadfence();
        const unsigned arrived = atomicAdd(A.bar, 1u);
        if (arrived == A.expect - 1) {
            A.bar[0] = 0u;
            __threadfence();
            atomicAdd(A.bar + 1, 1u);
        } else {
            const unsigned long long t0 = global_ns();
            while (*gen == g) {
                if (*(volatile int*)A.err) {
                    ok = 0;
                    break;
                }
                if (global_ns() - t0 > A.wait_ns) {
                    atomicExch(A.err, 1);
                    ok = 0;
                    break;
                }
                __nanosleep(100);
            }
        }
        __threadfence();
        *s_flag = ok;
    }
    __syncthreads();
    return *s_flag;
}

__device__ __forceinline__ void stage_image(float* dst, const float* src, int nfloats) {
    const float4* s4 = reinterpret_cast<const float4*>(src);
    float4* d4 = reinterpret_cast<float4*>(dst);
    for (int i = threadIdx.x; i < nfloats / 4; i += PT) d4[i] = __ldcg(s4 + i);
}

// One (unit, segment) of phase A: partial Joseph sum of ray k of angle a over the
// samples of segment `seg`, image in shared memory (element (0,0) at img, stride ld).
__device__ __forceinline__ ff ray_segment(const AngleRec& r, int k, int seg, int seg_len, int M, int Mm,
                                          const float* img, int ld) {
    float sum = 0.f, cmp = 0.f;
    const float halfM = 0.5f * (float)(M - 1);
    const ff Ak = ff_add(r.A0, ff_mul_f((float)k, r.a_scale));
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
    const int s0 = seg * seg_len;
    mlo = max(mlo, s0);
    mhi = min(mhi, min(s0 + seg_len, M));
    const float slope = r.slope.hi;
    for (int m0 = mlo; m0 < mhi; m0 += SEGA) {
        const ff bd = ff_add(Ak, ff_mul_f((float)m0 + 0.5f * (SEGA - 1) - halfM, r.slope));
        const float bfl = floorf(bd.hi);
        const int bi = (int)bfl;
        const float bf = (bd.hi - bfl) + bd.lo;
        const int mend = min(m0 + SEGA, mhi);
        float acc = 0.f;
        const float* rp = img + m0 * ld + bi;
#pragma unroll 4
        for (int m = m0; m < mend; ++m, rp += ld) {
            const float q = fmaf((float)(m - m0) - 0.5f * (SEGA - 1), slope, bf);
            const float fl = floorf(q);
            const int j = (int)fl;
            const float f = q - fl;
            const float v0 = rp[j], v1 = rp[j + 1];
            acc += fmaf(f, v1 - v0, v0);
        }
        neu_add(sum, cmp, acc);
    }
    return two_sum(sum, cmp);
}

__global__ void __launch_bounds__(PT, 1) k_persist(PArgs A) {
    extern __shared__ float4 smem4[];
    float* smem = reinterpret_cast<float*>(smem4);
    float* img = smem;                                        // phase A image / phase B staging
    float* red_s = smem + A.img_floats;                       // [NWARP][32]
    float* red_c = red_s + NWARP * 32;                        // [NWARP][32]
    __shared__ int s_flag;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int G = gridDim.x, b = blockIdx.x;
    const int nx = A.nx, ny = A.ny;
    const int u0 = (int)((long long)A.units * b / G), u1 = (int)((long long)A.units * (b + 1) / G);
    const int npix = nx * ny;
    const int p0 = (int)((long long)npix * b / G), p1 = (int)((long long)npix * (b + 1) / G);
    const int tiles_x = (nx + BT - 1) / BT, tiles = tiles_x * ((ny + BT - 1) / BT);
    const int t0 = (int)((long long)tiles * b / G), t1 = (int)((long long)tiles * (b + 1) / G);
    float* xa = A.xa_base + kPad;
    float* xaT = A.xaT_base + kPad;
    // phase B shared layout: stage[na][BSB] | cst[na] float4 | kb[na] int
    float* stage = smem;
    float4* cst = reinterpret_cast<float4*>(smem + ((A.na * BSB + 3) & ~3));
    int* kb = reinterpret_cast<int*>(cst + A.na);

    for (int it = 0; it < A.iters; ++it) {
        // ------------------------------------------------------------ phase A
        if (A.mode == 1) {  // gradient dual on this block's pixels (reads xbar^k)
            const float sv = A.sigma_v_dev ? __ldg(A.sigma_v_dev) : A.sigma_v;
            for (int p = p0 + tid; p < p1; p += PT) {
                const int i = p / nx, j = p - i * nx;
                const float* xp = xa + i * A.lda + j;
                const float x0 = __ldcg(xp);
                const float gx = j < nx - 1 ? __ldcg(xp + 1) - x0 : 0.f;
                const float gy = i < ny - 1 ? __ldcg(xp + A.lda) - x0 : 0.f;
                const float ax = fmaf(sv, gx, __ldcg(A.vx + p));
                const float ay = fmaf(sv, gy, __ldcg(A.vy + p));
                const float m = sqrtf(ax * ax + ay * ay);
                const float sc = m > A.lambda ? A.lambda / m : 1.f;
                A.vx[p] = ax * sc;
                A.vy[p] = ay * sc;
            }
        }
        int staged_row = -1;  // orientation in shared memory
        for (int ub = u0; ub < u1;) {
            // a pass takes up to UNITS_PER_PASS units sharing one branch (orientation)
            const int ua = ub;
            const int row_a = A.rec[ua / A.nchunk].row;
            int ue = min(ub + UNITS_PER_PASS, u1);
            for (int uu = ua + 1; uu < ue; ++uu)
                if (A.rec[uu / A.nchunk].row != row_a) {
                    ue = uu;
                    break;
                }
            if (row_a != staged_row) {
                __syncthreads();
                if (row_a)
                    stage_image(img, A.xa_base, ny * A.lda);
                else
                    stage_image(img, A.xaT_base, nx * A.ldaT);
                staged_row = row_a;
                __syncthreads();
            }
            const int M = row_a ? ny : nx, Mm = row_a ? nx : ny, ld = row_a ? A.lda : A.ldaT;
            const int seg_len = ((M + FSEG - 1) / FSEG + SEGA - 1) / SEGA * SEGA;
            const int unit = ua + warp / FSEG, seg = warp % FSEG;
            ff part = {0.f, 0.f};
            if (unit < ue) {
                const int a = unit / A.nchunk;
                const int k = (unit - a * A.nchunk) * RAYS + lane;
                const AngleRec& r = A.rec[a];
                if (k < r.width) part = ray_segment(r, k, seg, seg_len, M, Mm, img + kPad, ld);
            }
            red_s[warp * 32 + lane] = part.hi;
            red_c[warp * 32 + lane] = part.lo;
            __syncthreads();
            if (warp < UNITS_PER_PASS) {  // finish ray (unit ub + warp, lane)
                const int unit2 = ub + warp;
                if (unit2 < ue) {
                    const int a = unit2 / A.nchunk;
                    const int k = (unit2 - a * A.nchunk) * RAYS + lane;
                    const AngleRec& r = A.rec[a];
                    if (k < r.width) {
                        ff tot = {red_s[(warp * FSEG) * 32 + lane], red_c[(warp * FSEG) * 32 + lane]};
                        for (int s = 1; s < FSEG; ++s) {
                            const ff o = {red_s[(warp * FSEG + s) * 32 + lane], red_c[(warp * FSEG + s) * 32 + lane]};
                            tot = ff_add(tot, o);
                        }
                        tot = ff_mul_f(r.inv_w, tot);
                        const float acc = tot.hi + tot.lo;
                        const size_t o = (size_t)a * A.stride + k;
                        if (A.mode == 0) {
                            float res = __ldg(A.pp + o) - acc;
                            if (A.R) res *= __ldg(A.R + o);
                            A.u[o] = res;
                        } else {
                            const float sig = A.R ? __ldg(A.R + o) : A.sig_scalar;
                            A.u[o] = (__ldcg(A.u + o) + sig * (acc - __ldg(A.pp + o))) / (1.f + 0.5f * sig);
                        }
                    }
                }
            }
            __syncthreads();
            ub = ue;
        }
        if (!grid_sync(A, &s_flag)) return;

        // ------------------------------------------------------------ phase B
        for (int t = t0; t < t1; ++t) {
            const int tile_x0 = (t % tiles_x) * BT, tile_y0 = (t / tiles_x) * BT;
            const float xi_t = (float)tile_x0 + 0.5f * (BT - 1) - 0.5f * (float)(nx - 1);
            const float eta_t = 0.5f * (float)(ny - 1) - ((float)tile_y0 + 0.5f * (BT - 1));
            __syncthreads();
            for (int a = tid; a < A.na; a += PT) {
                const AngleRec& r = A.rec[a];
                ff kt = ff_add(ff_mul_f(xi_t, r.c), ff_mul_f(eta_t, r.s));
                kt = ff_add(kt, ff{-r.phi.hi, -r.phi.lo});
                const float fl = floorf(kt.hi);
                kb[a] = (int)fl - BKOFF;
                cst[a] = make_float4(r.c.hi, r.s.hi, r.inv_w, ((kt.hi - fl) + kt.lo) + (float)BKOFF);
            }
            __syncthreads();
            for (int e = tid; e < A.na * BSB; e += PT) {
                const int a = e / BSB, bb = e - a * BSB;
                const int kk = kb[a] + bb;
                stage[e] = (kk >= 0 && kk < A.rec[a].width) ? __ldcg(A.u + (size_t)a * A.stride + kk) : 0.f;
            }
            __syncthreads();
            const int pix = tid % BPIX, q = tid / BPIX;
            const int lj = pix % BT, li = pix / BT;
            const float dlj = (float)lj - 0.5f * (BT - 1), dli = (float)li - 0.5f * (BT - 1);
            const int a_lo = (int)((long long)A.na * q / QUART), a_hi = (int)((long long)A.na * (q + 1) / QUART);
            float sum = 0.f, cmp = 0.f;
            for (int c0 = a_lo; c0 < a_hi; c0 += 32) {
                const int c1 = min(c0 + 32, a_hi);
                float acc = 0.f;
                for (int a = c0; a < c1; ++a) {
                    const float4 cc = cst[a];
                    const float iw = cc.z, iw2 = cc.z * cc.z;
                    const float kap = fmaf(dlj, cc.x, fmaf(-dli, cc.y, cc.w));
                    const float fl = floorf(kap);
                    const int kl = (int)fl;
                    const float f = kap - fl;
                    const float w0 = fmaxf(0.f, fmaf(-f, iw2, iw));
                    const float w1 = fmaxf(0.f, fmaf(f, iw2, iw - iw2));
                    const float* srow = stage + a * BSB;
                    acc = fmaf(w0, srow[kl], fmaf(w1, srow[kl + 1], acc));
                }
                neu_add(sum, cmp, acc);
            }
            red_s[q * BPIX + pix] = sum;
            red_c[q * BPIX + pix] = cmp;
            __syncthreads();
            if (tid < BPIX) {
                const int gi = tile_y0 + li, gj = tile_x0 + lj;
                if (gi < ny && gj < nx) {
                    float s = red_s[pix], c = red_c[pix];
                    for (int qq = 1; qq < QUART; ++qq) {
                        neu_add(s, c, red_s[qq * BPIX + pix]);
                        neu_add(s, c, red_c[qq * BPIX + pix]);
                    }
                    const float acc = s + c;
                    const int o = gi * nx + gj;
                    if (A.mode == 0) {
                        const float step = A.C ? __ldg(A.C + o) : A.step_scalar;
                        float xn = fmaf(step, acc, __ldcg(xa + gi * A.lda + gj));
                        if (A.nonneg) xn = fmaxf(xn, 0.f);
                        xa[gi * A.lda + gj] = xn;
                        xaT[gj * A.ldaT + gi] = xn;
                    } else {
                        float dv = 0.f;
                        if (gj < nx - 1) dv += __ldcg(A.vx + o);
                        if (gj > 0) dv -= __ldcg(A.vx + o - 1);
                        if (gi < ny - 1) dv += __ldcg(A.vy + o);
                        if (gi > 0) dv -= __ldcg(A.vy + o - nx);
                        const float tau = A.C ? __ldg(A.C + o) : A.step_scalar;
                        const float xo = __ldcg(A.x + o);
                        const float xn = xo - tau * (acc - dv);
                        A.x[o] = xn;
                        const float xb = 2.f * xn - xo;
                        xa[gi * A.lda + gj] = xb;
                        xaT[gj * A.ldaT + gi] = xb;
                    }
                }
            }
        }
        if (!grid_sync(A, &s_flag)) return;
    }
}

}  // namespace

size_t persist_smem_bytes(int na, int nx, int ny) {
    const size_t img = std::max((size_t)ny * padded_ld(nx), (size_t)nx * padded_ld(ny));
    const size_t stageB = (size_t)((na * BSB + 3) & ~3) + 4 * (size_t)na + (size_t)na;  // floats
    const size_t region = std::max(img, stageB);
    return sizeof(float) * (region + 2 * NWARP * 32);
}

cudaError_t launch_persist(const PersistLaunch& L, cudaStream_t st) {
    PArgs A{};
    A.rec = L.rec;
    A.na = L.na;
    A.stride = L.stride;
    A.nx = L.nx;
    A.ny = L.ny;
    A.mode = L.mode;
    A.iters = L.iters;
    A.xa_base = L.xa_base;
    A.xaT_base = L.xaT_base;
    A.lda = padded_ld(L.nx);
    A.ldaT = padded_ld(L.ny);
    A.u = L.u;
    A.pp = L.pp;
    A.R = L.R;
    A.sig_scalar = L.sig_scalar;
    A.x = L.x;
    A.vx = L.vx;
    A.vy = L.vy;
    A.C = L.C;
    A.step_scalar = L.step_scalar;
    A.sigma_v_dev = L.sigma_v_dev;
    A.sigma_v = L.sigma_v;
    A.lambda = L.lambda;
    A.nonneg = L.nonneg;
    A.bar = L.bar;
    A.expect = (unsigned)(L.blocks + L.phantoms);
    A.err = L.err;
    A.wait_ns = L.wait_ns;
    A.nchunk = (L.stride + RAYS - 1) / RAYS;
    A.units = L.na * A.nchunk;
    A.img_floats = (int)((persist_smem_bytes(L.na, L.nx, L.ny) / sizeof(float)) - 2 * NWARP * 32);
    const size_t smem = persist_smem_bytes(L.na, L.nx, L.ny);
    cudaError_t e = cudaFuncSetAttribute(k_persist, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(L.bar, 0, 2 * sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    void* args[] = {&A};
    count_launches(1);
    return cudaLaunchCooperativeKernel((const void*)k_persist, dim3(L.blocks), dim3(PT), args, smem, st);
}

int persist_max_blocks(int na, int nx, int ny, int device) {
    const size_t smem = persist_smem_bytes(na, nx, ny);
    if (cudaFuncSetAttribute(k_persist, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_persist, PT, smem) != cudaSuccess) return 0;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 0;
    return std::min(per_sm, 1) * sms;
}

}  // namespace roi
