// batch.cu -- many local solves of uneven size in one persistent launch.
//
// One block per SM pulls regions from a device queue (largest first) and solves each
// one completely (paper Sec. 1 scheme: SIRT, Eq. sirtit + Eq. sirtbox, or TV by
// Chambolle-Pock, Eq. priorsys; operators W_L, W_L^T of Sec. 2.1).  The windows p' of
// every region were computed beforehand by the batched exterior projection.  Per
// region and iteration the block runs
//   phase A  forward W_L: warps pull 32-ray units (one angle); a warp sums whole rays,
//            reading the box image from shared memory (staged by TMA, rows for the
//            per-row branch, then columns) when it fits, else from global memory, and
//            fuses the residual (SIRT) or dual (CP) update; CP also updates the
//            gradient dual on all pixels;
//   phase B  back W_L^T: warps pull 16 x 16 pixel tiles; a lane owns a run of 8 pixels,
//            angles are streamed in chunks of 16 (per-warp staging of the window bins),
//            and the lane applies the primal update to its pixels.
// Only block barriers separate the phases; blocks never wait on one another.  Every ray
// and every tile is computed by one warp in a fixed order, so a region's result does not
// depend on the other regions of the batch nor on which block solved it.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "dev_common.cuh"
#include "roi_internal.h"

namespace roi {

namespace {

constexpr int BPT = 1024;
constexpr int BNW = BPT / 32;
constexpr int SEGB = 24;     // samples per float-float anchor
constexpr int TB = 16;       // tile side
constexpr int RUNB = 8;      // pixels per lane
constexpr int ACH = 16;      // angles per staging chunk (one per lane of the first half-warp)
constexpr int KOFFB = 12;    // see persist.cu: tile pixels within 10.61 bins of the centre
constexpr int SBB = 26;      // staged bins per angle
constexpr int WARP_STAGE = ACH * SBB + 3 * ACH * 2;  // floats per warp in phase B (bins + consts)

enum PassA { A_SOLVE = 0, A_ROWSUM = 1 };
enum PassB { B_SOLVE = 0, B_COLSUM = 1 };

struct BlockCtx {
    const BatchRoi* R;
    const BatchArgs* B;
    // slot buffers of this block
    float* u;      // slot windows [na][stride]
    float* sig;
    float* x;      // slot box arrays [ny][nx]
    float* vx;
    float* vy;
    float* tau;
    float* xa;     // padded row image, element (0,0)
    float* xaT;    // padded column image, element (0,0)
    int lda, ldaT;
    int nchunk;
    bool smem_img;
};

// Whole-ray Joseph sum of ray k (fixed point along the ray; see persist.cu).
template <bool SM>
__device__ __forceinline__ ff ray_full(const AngleRec& r, int k, int M, int Mm, const float* img, int ld) {
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
    const int step = r.slope_q22;
    for (int m0 = mlo; m0 < mhi; m0 += SEGB) {
        int q = to_fixed<22>(ff_add(Ak, ff_mul_f((float)m0 - halfM, r.slope)));
        const int mend = min(m0 + SEGB, mhi);
        float s0 = 0.f, s1 = 0.f;
        const float* rp = img + (size_t)m0 * ld;
#pragma unroll 4
        for (int m = m0; m < mend; ++m, rp += ld, q += step) {
            const int j = q >> 22;
            const float mf = frac_int<22>(q);
            const float v0 = rp[j], v1 = rp[j + 1];
            s0 += v0;
            s1 = fmaf(mf, v1 - v0, s1);
        }
        neu_add(sum, cmp, fmaf(s1, 2.384185791015625e-07f, s0));
    }
    return two_sum(sum, cmp);
}

// Phase A over the units of one branch (row = 1: per-row sampling; the table lists those
// angles first), warps pulling units from *counter (preset to the branch's first unit +
// the number of warps).  img: padded image of that branch (shared or global).
template <bool SM>
__device__ __forceinline__ void phase_a_branch(const BlockCtx& C, int row, const float* img, int ld, int pass,
                                               int* counter) {
    const BatchRoi& R = *C.R;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int M = row ? R.ny : R.nx, Mm = row ? R.nx : R.ny;
    const int u_end = (row ? R.nrow : R.na) * C.nchunk;
    for (int unit = (row ? 0 : R.nrow * C.nchunk) + warp; unit < u_end;) {
        const int a = unit / C.nchunk;
        const int k = (unit - a * C.nchunk) * 32 + lane;
        const AngleRec& r = R.rec[a];
        if (k < r.width) {
            ff tot = ray_full<SM>(r, k, M, Mm, img, ld);
            tot = ff_mul_f(r.inv_w, tot);
            const float acc = tot.hi + tot.lo;
            const size_t o = (size_t)a * R.stride + k;
            if (pass == A_ROWSUM) {
                const float thr = R.reg == 0 ? 1e-3f : 1e-6f;
                C.sig[o] = acc > thr ? 1.f / acc : 0.f;
            } else if (R.reg == 0) {
                float res = R.pp[o] - acc;
                if (R.weighting) res *= C.sig[o];
                C.u[o] = res;
            } else {
                const float sg = C.sig[o];
                C.u[o] = (C.u[o] + sg * (acc - R.pp[o])) / (1.f + 0.5f * sg);
            }
        }
        int nxt = 0;
        if (lane == 0) nxt = atomicAdd(counter, 1);
        unit = __shfl_sync(0xffffffffu, nxt, 0);
    }
}

// Phase B: warps pull tiles; lane = run of 8 pixels.  wstage: this warp's shared area.
__device__ __forceinline__ void phase_b(const BlockCtx& C, int pass, int* counter, float* wstage) {
    const BatchRoi& R = *C.R;
    const BatchArgs& B = *C.B;
    const int lane = threadIdx.x & 31;
    const int nx = R.nx, ny = R.ny;
    const int tiles_x = (nx + TB - 1) / TB, tiles = tiles_x * ((ny + TB - 1) / TB);
    float* st = wstage;                                            // [ACH][SBB]
    int* cb = reinterpret_cast<int*>(wstage + ACH * SBB);          // [ACH] base (Q.23)
    int* cc = cb + ACH;                                            // [ACH] c step
    int* cs = cc + ACH;                                            // [ACH] s step
    float* ciw = reinterpret_cast<float*>(cs + ACH);               // [ACH] 1/w
    int* ckb = reinterpret_cast<int*>(ciw + ACH);                  // [ACH] kbase
    int* cwd = ckb + ACH;                                          // [ACH] width
    const int li = lane >> 1, lj0 = (lane & 1) * RUNB;
    int t = threadIdx.x >> 5;
    while (t < tiles) {
        const int tile_x0 = (t % tiles_x) * TB, tile_y0 = (t / tiles_x) * TB;
        const float xi_t = (float)tile_x0 + 0.5f * (TB - 1) - 0.5f * (float)(nx - 1);
        const float eta_t = 0.5f * (float)(ny - 1) - ((float)tile_y0 + 0.5f * (TB - 1));
        float sum[RUNB], cmp[RUNB];
#pragma unroll
        for (int p = 0; p < RUNB; ++p) sum[p] = cmp[p] = 0.f;
        for (int a0 = 0; a0 < R.na; a0 += ACH) {
            const int nch = min(ACH, R.na - a0);
            __syncwarp();
            if (lane < nch) {
                const AngleRec& r = R.rec[a0 + lane];
                ff kt = ff_add(ff_mul_f(xi_t, r.c), ff_mul_f(eta_t, r.s));
                kt = ff_add(kt, ff{-r.phi.hi, -r.phi.lo});
                const int kbase = (int)floorf(kt.hi) - KOFFB;
                kt = ff_add(kt, ff{-(float)kbase, 0.f});
                kt = ff_add(kt, ff_mul_f(-0.5f * (TB - 1), r.c));
                kt = ff_add(kt, ff_mul_f(0.5f * (TB - 1), r.s));
                cb[lane] = to_fixed<23>(kt);
                cc[lane] = r.c_q23;
                cs[lane] = r.s_q23;
                ciw[lane] = r.inv_w;
                ckb[lane] = kbase;
                cwd[lane] = r.width;
            }
            __syncwarp();
            for (int e = lane; e < nch * SBB; e += 32) {
                const int al = e / SBB, kk = ckb[al] + (e - al * SBB);
                float v = 0.f;
                if (kk >= 0 && kk < cwd[al]) v = pass == B_COLSUM ? 1.f : C.u[(size_t)(a0 + al) * R.stride + kk];
                st[e] = v;
            }
            __syncwarp();
            float acc[RUNB];
#pragma unroll
            for (int p = 0; p < RUNB; ++p) acc[p] = 0.f;
            for (int al = 0; al < nch; ++al) {
                const float iw = ciw[al], iw2 = iw * iw, iwm = iw - iw2;
                const float iw2s = iw2 * 1.1920928955078125e-07f;
                const int c = cc[al];
                int K = cb[al] + lj0 * c - li * cs[al];
                const float* srow = st + al * SBB;
#pragma unroll
                for (int p = 0; p < RUNB; ++p) {
                    const int kl = K >> 23;
                    const float mf = frac_int<23>(K);
                    const float w0 = fmaxf(0.f, fmaf(-mf, iw2s, iw));
                    const float w1 = fmaxf(0.f, fmaf(mf, iw2s, iwm));
                    acc[p] = fmaf(w0, srow[kl], fmaf(w1, srow[kl + 1], acc[p]));
                    K += c;
                }
            }
#pragma unroll
            for (int p = 0; p < RUNB; ++p) neu_add(sum[p], cmp[p], acc[p]);
        }
        // epilogue for this lane's pixels
        const int gi = tile_y0 + li;
#pragma unroll
        for (int p = 0; p < RUNB; ++p) {
            const int gj = tile_x0 + lj0 + p;
            if (gi >= ny || gj >= nx) continue;
            const float acc = sum[p] + cmp[p];
            const int o = gi * nx + gj;
            if (pass == B_COLSUM) {
                if (R.reg == 0) {
                    C.tau[o] = acc > 1e-3f ? 1.f / acc : 0.f;
                } else {
                    const int cnt = (gj < nx - 1) + (gj > 0) + (gi < ny - 1) + (gi > 0);
                    C.tau[o] = 1.f / (acc + (float)cnt);
                }
            } else if (R.reg == 0) {
                const float step = R.weighting ? C.tau[o] : B.alpha;
                float xn = fmaf(step, acc, C.xa[gi * C.lda + gj]);
                xn = fmaxf(xn, 0.f);
                C.xa[gi * C.lda + gj] = xn;
                C.xaT[gj * C.ldaT + gi] = xn;
            } else {
                float dv = 0.f;
                if (gj < nx - 1) dv += C.vx[o];
                if (gj > 0) dv -= C.vx[o - 1];
                if (gi < ny - 1) dv += C.vy[o];
                if (gi > 0) dv -= C.vy[o - nx];
                const float xo = C.x[o];
                const float xn = xo - C.tau[o] * (acc - dv);
                C.x[o] = xn;
                const float xb = 2.f * xn - xo;
                C.xa[gi * C.lda + gj] = xb;
                C.xaT[gj * C.ldaT + gi] = xb;
            }
        }
        int nxt = 0;
        if (lane == 0) nxt = atomicAdd(counter, 1);
        t = __shfl_sync(0xffffffffu, nxt, 0);
    }
}

__device__ void fill_block(float* p, size_t n, float v) {
    for (size_t i = threadIdx.x; i < n; i += BPT) p[i] = v;
}

// Interior of both padded images := v, borders 0.
__device__ void set_images(const BlockCtx& C, float v) {
    const BatchRoi& R = *C.R;
    const int nx = R.nx, ny = R.ny;
    float* xab = C.xa - kPad;
    float* xaTb = C.xaT - kPad;
    for (int i = threadIdx.x; i < ny * C.lda; i += BPT) {
        const int col = i % C.lda - kPad;
        xab[i] = (col >= 0 && col < nx) ? v : 0.f;
    }
    for (int i = threadIdx.x; i < nx * C.ldaT; i += BPT) {
        const int col = i % C.ldaT - kPad;
        xaTb[i] = (col >= 0 && col < ny) ? v : 0.f;
    }
}

__global__ void __launch_bounds__(BPT, 1) k_batch(BatchArgs B) {
    extern __shared__ float4 smem4[];
    float* smem = reinterpret_cast<float*>(smem4);
    __shared__ int s_roi, s_cnt;
    __shared__ __align__(8) uint64_t s_mbar;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int slot = blockIdx.x;
    if (tid == 0) mbar_init(&s_mbar, 1);
    unsigned parity = 0;
    BlockCtx C;
    C.B = &B;
    C.u = B.slot_u + (size_t)slot * B.win_cap;
    C.sig = B.slot_sig + (size_t)slot * B.win_cap;
    C.x = B.slot_x + (size_t)slot * B.img_cap;
    C.vx = B.slot_vx + (size_t)slot * B.img_cap;
    C.vy = B.slot_vy + (size_t)slot * B.img_cap;
    C.tau = B.slot_tau + (size_t)slot * B.img_cap;
    float* xa_base = B.slot_xa + (size_t)slot * B.pad_cap;
    float* xaT_base = B.slot_xaT + (size_t)slot * B.pad_cap;
    for (;;) {
        __syncthreads();
        if (tid == 0) s_roi = atomicAdd(B.queue, 1);
        __syncthreads();
        const int qi = s_roi;
        if (qi >= B.nroi) break;
        const BatchRoi& R = B.rois[B.order[qi]];
        C.R = &R;
        C.lda = padded_ld(R.nx);
        C.ldaT = padded_ld(R.ny);
        C.xa = xa_base + kPad;
        C.xaT = xaT_base + kPad;
        C.nchunk = (R.stride + 31) / 32;
        const size_t nimg = (size_t)R.nx * R.ny, nwin = (size_t)R.na * R.stride;
        const size_t bytes_row = sizeof(float) * (size_t)R.ny * C.lda;
        const size_t bytes_col = sizeof(float) * (size_t)R.nx * C.ldaT;
        C.smem_img = (bytes_row > bytes_col ? bytes_row : bytes_col) <= (size_t)B.smem_img_bytes;
        // ---- set-up: zero state, preconditioners / weights
        fill_block(C.u, nwin, 0.f);
        fill_block(C.x, nimg, 0.f);
        fill_block(C.vx, nimg, 0.f);
        fill_block(C.vy, nimg, 0.f);
        const bool sums = R.reg == 1 || R.weighting;
        if (sums) {
            set_images(C, 1.f);
            __syncthreads();
            for (int row = 1; row >= 0; --row) {
                if (tid == 0) s_cnt = (row ? 0 : R.nrow * C.nchunk) + BNW;
                __syncthreads();
                phase_a_branch<false>(C, row, row ? C.xa : C.xaT, row ? C.lda : C.ldaT, A_ROWSUM, &s_cnt);
                __syncthreads();
            }
            if (tid == 0) s_cnt = BNW;
            __syncthreads();
            phase_b(C, B_COLSUM, &s_cnt, smem + warp * WARP_STAGE);
        }
        __syncthreads();
        set_images(C, 0.f);
        __syncthreads();
        // ---- iterations
        for (int it = 0; it < R.iters; ++it) {
            for (int row = 1; row >= 0; --row) {
                const float* gimg = row ? C.xa : C.xaT;
                const int ld = row ? C.lda : C.ldaT;
                if (C.smem_img && tid == 0)
                    bulk_load(smem, row ? xa_base : xaT_base, (unsigned)(row ? bytes_row : bytes_col), &s_mbar);
                if (row == 1 && R.reg == 1) {  // gradient dual (reads xbar^k) while the copy runs
                    for (int p = tid; p < (int)nimg; p += BPT) {
                        const int i = p / R.nx, j = p - i * R.nx;
                        const float* xp = C.xa + i * C.lda + j;
                        const float x0 = xp[0];
                        const float gx = j < R.nx - 1 ? xp[1] - x0 : 0.f;
                        const float gy = i < R.ny - 1 ? xp[C.lda] - x0 : 0.f;
                        const float ax = fmaf(R.sigma_v, gx, C.vx[p]);
                        const float ay = fmaf(R.sigma_v, gy, C.vy[p]);
                        const float m = sqrtf(ax * ax + ay * ay);
                        const float sc = m > R.lambda ? R.lambda / m : 1.f;
                        C.vx[p] = ax * sc;
                        C.vy[p] = ay * sc;
                    }
                }
                if (tid == 0) s_cnt = (row ? 0 : R.nrow * C.nchunk) + BNW;
                if (C.smem_img) {
                    if (!mbar_wait(&s_mbar, parity, B.wait_ns, B.err)) return;
                    parity ^= 1u;
                }
                __syncthreads();
                if (C.smem_img)
                    phase_a_branch<true>(C, row, smem + kPad, ld, A_SOLVE, &s_cnt);
                else
                    phase_a_branch<false>(C, row, gimg, ld, A_SOLVE, &s_cnt);
                __syncthreads();
            }
            if (tid == 0) s_cnt = BNW;
            __syncthreads();
            phase_b(C, B_SOLVE, &s_cnt, smem + warp * WARP_STAGE);
            __syncthreads();
        }
        // ---- crop into the caller's buffer
        const float* xs = R.reg == 0 ? C.xa : C.x;
        const int xs_ld = R.reg == 0 ? C.lda : R.nx;
        for (int p = tid; p < (int)nimg; p += BPT) {
            const int i = p / R.nx, j = p - i * R.nx;
            float v = xs[i * xs_ld + j];
            if (R.crop) {
                const float dx = (float)j - R.cxl, dy = (float)i - R.cyl;
                if (dx * dx + dy * dy > R.r2) v = 0.f;
            }
            R.out[p] = v;
        }
    }
}

}  // namespace

size_t batch_smem_bytes(size_t max_img_floats) {
    const size_t phase_b = (size_t)BNW * WARP_STAGE;
    return sizeof(float) * std::max(max_img_floats, phase_b);
}

cudaError_t launch_batch(const BatchArgs& B, int blocks, size_t smem, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(B.queue, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    count_launches(1);
    k_batch<<<blocks, BPT, smem, st>>>(B);
    return cudaGetLastError();
}

int batch_threads() { return BPT; }

}  // namespace roi
