// region_solver.cuh -- one whole local solve by a team of blocks (device code shared by
// the batched solver and the serving kernel).
//
// A region (paper Sec. 1 scheme on the extended box L, Sec. 2.1 operators W_L, W_L^T)
// is solved end to end by a team of `size` blocks of 1024 threads:
//   exterior   p' = (p - W x_fbp) + W_L x_fbp|_L  (Eq. locouter: W_F = W - W_L); the
//              residual p - W x_fbp of every ray is computed once per sinogram, so a
//              region costs one local forward projection of the box of x_fbp;
//   set-up     row sums W_L 1 and column sums W_L^T 1 (SIRT weights, CP steps);
//   iterations SIRT (Eq. sirtit with the clamp of Eq. sirtbox) or Chambolle-Pock TV
//              (Eq. priorsys), each as
//     phase A  forward W_L: warps take 32-ray units (one angle); a warp sums whole rays
//              (fixed point along the ray) and fuses the residual (SIRT) or data-dual
//              (CP) update; CP also updates the gradient dual on every pixel;
//     phase B  back W_L^T: 16 x 16 pixel tiles; a lane owns a run of 8 pixels, angles
//              are streamed in chunks of 16 through per-warp staging buffers, a pixel's
//              gather is the chunk partials added in chunk order, and the pixel's primal
//              update follows.  Warps take whole tiles, or, in a block with few tiles,
//              all warps share each tile by chunks (same operations, same bits).
// The units and tiles of a phase are dealt round-robin to the blocks of the team and
// picked up dynamically by the warps of a block.  Every ray and every chunk of a tile is
// computed by one warp in a fixed order, so a region's result is bit-identical whatever
// team solves it, whatever else runs beside it and however the work is dealt.
//
// How phase A reads the box image depends on the box size alone (stage_mode): every block
// stages it whole in shared memory (one TMA bulk copy per branch and iteration), streams
// it in bands, or reads it from global memory.  A team of one block synchronises with
// __syncthreads; larger teams meet at a barrier counter with bounded waits.  Data written
// by one block of a team and read by another is ordered by that barrier's release /
// acquire at GPU scope.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "check.cuh"
#include "dev_common.cuh"
#include "roi_internal.h"

namespace roi {
namespace rs {

constexpr int BPT = 1024;
constexpr int BNW = BPT / 32;
constexpr int SEGB = 48;     // samples per float-float anchor (Q.22 drift < 6e-6 px)
constexpr int ACH = 16;      // angles per staging chunk (one per lane of the first half-warp)

// Phase B tile shapes: X x Y pixels per warp, a lane owning a run of RUN pixels along a
// tile row (X / RUN lanes per row, 32 lanes = Y rows).  Shape 0 (16 x 16, runs of 8) is
// the default; 1 (8 x 8, runs of 2) and 2 (16 x 8, runs of 4) give more tiles per box,
// so more warps are busy on small boxes and in teams, at a higher per-angle cost per
// pixel.  The shape of a region is chosen by the host (a function of its box size and of
// the handle's tile table, so a region gets the same bits wherever it is solved).
constexpr int kShapes = 3;
template <int SH> struct Shape;
template <> struct Shape<0> { static constexpr int X = 16, Y = 16, RUN = 8; };
template <> struct Shape<1> { static constexpr int X = 8, Y = 8, RUN = 2; };
template <> struct Shape<2> { static constexpr int X = 16, Y = 8, RUN = 4; };
// Tile pixels lie within h = sqrt((X-1)^2 + (Y-1)^2) / 2 bins of the tile centre in window
// coordinates and the hat reaches one bin further, so with kbase = floor(kappa_centre) -
// KOFF, KOFF = ceil(h) + 1, every staged index touched is in [1, 2 ceil(h) + 2] < SB.
constexpr int ceil_half_diag(int x, int y) {
    int c = 0;
    while (4 * c * c < (x - 1) * (x - 1) + (y - 1) * (y - 1)) ++c;
    return c;
}
template <int SH> struct ShapeStage {
    static constexpr int X = Shape<SH>::X, Y = Shape<SH>::Y, RUN = Shape<SH>::RUN;
    static constexpr int LPR = X / RUN;                    // lanes per tile row
    static_assert(LPR * Y == 32, "a tile is one warp");
    static constexpr int KOFF = ceil_half_diag(X, Y) + 1;  // 16 x 16: 12
    static constexpr int SB = 2 * KOFF + 2;                // staged bins per angle (16 x 16: 26)
    static constexpr int BUF = ACH * SB + 8 * ACH;          // one buffer: bins + 8 constants per angle
};
// floats per warp in phase B (double-buffered), the largest shape's
constexpr int WARP_STAGE = 2 * ShapeStage<0>::BUF;
static_assert(2 * ShapeStage<1>::BUF <= WARP_STAGE && 2 * ShapeStage<2>::BUF <= WARP_STAGE, "warp area");
constexpr int TB = 16;       // largest tile side (cooperative partial areas are sized by X Y <= TB TB)

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait_group() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

enum PassA { A_SOLVE = 0, A_ROWSUM = 1, A_EXTER = 2 };
enum PassB { B_SOLVE = 0, B_COLSUM = 1, B_XS = 2 };  // B_XS: x_s^k = W_L^T C_{u_k} p (Sec. 3)

// A team of blocks solving one region.
struct Team {
    int member, size;          // this block's index in the team, team size
    unsigned* bar;             // monotonic arrival counter (size > 1), zeroed at launch
    unsigned nbar;             // barriers passed by this block (thread 0's copy is used)
    int* err;
    unsigned long long wait_ns;
    unsigned expect;           // arrivals a barrier waits for: 0 = size; testing only: size plus
                               // participants that never arrive, so every barrier runs out
};

// Team barrier.  false: a wait gave up (error flag set) and the caller must leave.
// SOLO: the team is one block (known at compile time).
template <bool SOLO>
__device__ __forceinline__ bool team_sync(Team& T) {
    __shared__ int s_ok;
    __syncthreads();
    if (SOLO || T.size == 1) return true;
    if (threadIdx.x == 0) {
        int ok = 1;
        ++T.nbar;
        const unsigned target = T.nbar * (T.expect ? T.expect : (unsigned)T.size);
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(T.bar) : "memory");
        unsigned long long t0 = 0;
        for (unsigned polls = 1;; ++polls) {
            unsigned v;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(T.bar) : "memory");
            if ((int)(v - target) >= 0) break;
            if ((polls & 255u) == 0) {
                const unsigned long long now = global_ns();
                if (t0 == 0) {
                    t0 = now;
                } else if (now - t0 > T.wait_ns) {
                    atomicExch(T.err, 1);
                    ok = 0;
                    break;
                }
                if (*(volatile int*)T.err) {
                    ok = 0;
                    break;
                }
            }
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

using roi::RegionBufs;

struct Ctx {
    const BatchRoi* R;
    RegionBufs b;
    void* xa;      // padded row image (storage R.dt), element (0,0)
    void* xaT;     // padded column image, element (0,0)
    int lda, ldaT; // row strides in elements
    int nchunk;
    int member, gthreads; // this block's index in the team, threads of the team
    int stage;            // stage_mode of the box (0 whole image, 1 bands, 2 global)
    // phase A of the iterations in a team of two or more blocks: the blocks are split between
    // the two branches in proportion to their units, so each stages one image; this block's
    // branch (1 rows, 0 columns; -1: both, in turn) and its index / count within it
    int arow, amember, asize;
};
// (A Ctx lives in shared memory: it is uniform over the block, and keeping it out of
// registers leaves them to the inner loops.)

// This thread's index over the team.
__device__ __forceinline__ int team_tid(const Ctx& C) { return C.member * BPT + (int)threadIdx.x; }

// Samples [mlo, mhi) of ray k whose minor coordinate lies in [-1.5, Mm + 0.5] (the others
// contribute 0, so both taps stay inside the padded row), and the ray's coordinate Ak at
// the major-axis centre.
__device__ __forceinline__ ff ray_span(const AngleRec& r, int k, int M, int Mm, int& mlo, int& mhi) {
    const float halfM = 0.5f * (float)(M - 1);
    const ff Ak = ff_add(r.A0, ff_mul_f((float)k, r.a_scale));
    mlo = 0;
    mhi = M;
    if (!r.flat) {
        const float ma = (-1.5f - Ak.hi) * r.inv_slope + halfM;
        const float mb = ((float)Mm + 0.5f - Ak.hi) * r.inv_slope + halfM;
        const float lo = fminf(ma, mb), hi = fmaxf(ma, mb);
        mlo = (int)fminf(fmaxf(0.f, ceilf(lo)), (float)M);
        mhi = (int)fmaxf(fminf((float)M, floorf(hi) + 1.f), 0.f);
    } else if (!(Ak.hi >= -1.5f && Ak.hi <= (float)Mm + 0.5f)) {
        mhi = 0;
    }
    return Ak;
}

// The ray's samples [m0, min(m0 + SEGB, mhi)) from one float-float anchor at m0: an integer
// column plus a Q.22 offset from it, stepped per sample (the offset stays below 2^31
// whatever the box size); returns s0 + s1 2^-22 (the values and their interpolated
// differences, summed apart).
template <int DT>
__device__ __forceinline__ float ray_anchor(const AngleRec& r, ff Ak, int m0, int mhi, int M,
                                            const typename Stor<DT>::T* img, int ld) {
    const float halfM = 0.5f * (float)(M - 1);
    int j0;
    int q = split_fixed22(ff_add(Ak, ff_mul_f((float)m0 - halfM, r.slope)), j0);
    const int step = r.slope_q22;
    const int mend = min(m0 + SEGB, mhi);
    const int jlo = -kPad - j0, jhi = ld - 1 - kPad - j0;  // taps j, j + 1 inside the padded row
    float s0 = 0.f, s1 = 0.f;
    const typename Stor<DT>::T* rp = img + (size_t)m0 * ld + j0;
#pragma unroll 4
    for (int m = m0; m < mend; ++m, rp += ld, q += step) {
        const int j = chk(q >> 22, jlo, jhi, CHK_REGION_RAY);
        const float mf = frac_int<22>(q);
        const float v0 = to_f32<DT>(rp[j]), v1 = to_f32<DT>(rp[j + 1]);
        s0 += v0;
        s1 = fmaf(mf, v1 - v0, s1);
    }
    return fmaf(s1, 2.384185791015625e-07f, s0);
}

// Whole-ray Joseph sum of ray k (fixed point along the ray): the anchors' values every SEGB
// samples, added in order with Neumaier compensation.
template <int DT>
__device__ __forceinline__ ff ray_full(const AngleRec& r, int k, int M, int Mm, const typename Stor<DT>::T* img,
                                       int ld) {
    float sum = 0.f, cmp = 0.f;
    int mlo, mhi;
    const ff Ak = ray_span(r, k, M, Mm, mlo, mhi);
    for (int m0 = mlo; m0 < mhi; m0 += SEGB) neu_add(sum, cmp, ray_anchor<DT>(r, Ak, m0, mhi, M, img, ld));
    return two_sum(sum, cmp);
}

// The pass's use of the sum tot of window ray (a, k) (angle a of the table).
__device__ __forceinline__ void finish_ray(const Ctx& C, const AngleRec& r, int a, int k, ff tot, int pass) {
    const BatchRoi& R = *C.R;
    tot = ff_mul_f(r.inv_w, tot);
    const size_t o = (size_t)a * R.stride + k;
    if (pass == A_EXTER) {  // p' = (p - W x_fbp) + W_L x_fbp
        const ff d = two_sum(R.resid[(size_t)r.aidx * R.resid_ld + r.d0 + k], tot.hi);
        C.b.pp[o] = d.hi + (d.lo + tot.lo);
        return;
    }
    const float acc = tot.hi + tot.lo;
    if (pass == A_ROWSUM) {
        const float thr = R.reg == 0 ? 1e-3f : 1e-6f;
        C.b.sig[o] = acc > thr ? 1.f / acc : 0.f;
    } else if (R.reg == 0) {
        float res = C.b.pp[o] - acc;
        if (R.weighting) res *= C.b.sig[o];
        C.b.u[o] = res;
    } else if (R.reg >= 2) {
        C.b.u[o] = -R.alpha * acc;
    } else {
        const float sg = C.b.sig[o];
        C.b.u[o] = (C.b.u[o] + sg * (acc - C.b.pp[o])) / (1.f + 0.5f * sg);
    }
}

// Phase A over the units of one branch (row = 1: per-row sampling; the table lists those
// angles first).  This block's units are ustart + member + i * size; warps take i from
// *counter (preset to BNW by the caller, warp w starting at i = w) and sum whole rays.  A
// team block with fewer units than warps splits the rays at their float-float anchors
// instead when `part` (part_floats floats of shared memory) holds every anchor value of its
// units: the (unit, anchor) items go round-robin over all warps, each writes its anchor
// value, and one warp per unit adds a ray's anchor values in order -- the same operations
// as the whole-ray sum, so the same bits.
template <bool SOLO, int DT>
__device__ __forceinline__ void phase_a_branch(const Ctx& C, const Team& T, int row, const void* img_v, int ld,
                                               int pass, int* counter, float* part = nullptr, int part_floats = 0) {
    const auto* img = static_cast<const typename Stor<DT>::T*>(img_v);
    const int tm = SOLO ? 0 : T.member, ts = SOLO ? 1 : T.size;
    const BatchRoi& R = *C.R;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int M = row ? R.ny : R.nx, Mm = row ? R.nx : R.ny;
    const int ustart = row ? 0 : R.nrow * C.nchunk;
    const int uend = (row ? R.nrow : R.na) * C.nchunk;
    if (!SOLO) {
        const int total = uend - ustart;
        const int nu = total > tm ? (total - tm + ts - 1) / ts : 0;
        const int J = (M + SEGB - 1) / SEGB;  // anchors of the longest ray
        if (nu > 0 && nu < BNW && part && nu * J * 32 <= part_floats) {
            for (int item = warp; item < nu * J; item += BNW) {
                const int i = item / J, j = item - i * J;
                const int unit = ustart + tm + i * ts;
                const int a = unit / C.nchunk;
                const int k = (unit - a * C.nchunk) * 32 + lane;
                const AngleRec& r = R.rec[a];
                float v = 0.f;
                if (k < r.width) {
                    int mlo, mhi;
                    const ff Ak = ray_span(r, k, M, Mm, mlo, mhi);
                    const int m0 = mlo + j * SEGB;
                    if (m0 < mhi) v = ray_anchor<DT>(r, Ak, m0, mhi, M, img, ld);
                }
                part[item * 32 + lane] = v;
            }
            __syncthreads();
            for (int i = warp; i < nu; i += BNW) {
                const int unit = ustart + tm + i * ts;
                const int a = unit / C.nchunk;
                const int k = (unit - a * C.nchunk) * 32 + lane;
                const AngleRec& r = R.rec[a];
                if (k < r.width) {
                    int mlo, mhi;
                    ray_span(r, k, M, Mm, mlo, mhi);
                    const int n_anchor = mhi > mlo ? (mhi - mlo + SEGB - 1) / SEGB : 0;
                    float sum = 0.f, cmp = 0.f;
                    for (int j = 0; j < n_anchor; ++j) neu_add(sum, cmp, part[(i * J + j) * 32 + lane]);
                    finish_ray(C, r, a, k, two_sum(sum, cmp), pass);
                }
            }
            return;
        }
    }
    for (int i = warp;;) {
        const int unit = ustart + tm + i * ts;
        if (unit >= uend) break;
        const int a = unit / C.nchunk;
        const int k = (unit - a * C.nchunk) * 32 + lane;
        const AngleRec& r = R.rec[a];
        if (k < r.width) finish_ray(C, r, a, k, ray_full<DT>(r, k, M, Mm, img, ld), pass);
        int nxt = 0;
        if (lane == 0) nxt = atomicAdd(counter, 1);
        i = __shfl_sync(0xffffffffu, nxt, 0);
    }
}

// The disc of Sec. 3.3 at box pixel (i, j): grey value g where the grid pixel's centre lies
// within N/2 of the rotation axis, else 0.
__device__ __forceinline__ float disc_value(const BatchRoi& R, int i, int j) {
    const float half = 0.5f * (float)(R.grid_n - 1);
    const float x = (float)(R.box_x0 + j) - half, y = half - (float)(R.box_y0 + i);
    return (x * x + y * y <= 0.25f * (float)R.grid_n * (float)R.grid_n) ? R.disc_g : 0.f;
}

// Phase B with tile shape SH: this block's tiles are member + i * size.  Per tile and pixel
// the gather is the sum, in chunk order with Neumaier compensation, of per-chunk partials
// (each the FMA chain over the chunk's 16 angles in order), then the pass's update.  Two
// ways to run it, with the same operations and so the same bits:
//  - per warp: warps take tiles i from *counter (preset to BNW), lane = run of RUN pixels,
//    chunks streamed through the warp's double buffer;
//  - cooperative, in a team block with fewer tiles than warps when the shared memory past
//    the warp areas holds at least one tile's partials: the block's tiles go in groups,
//    the (tile, chunk) items of a group are dealt over all warps, their partials meet in
//    shared memory and one thread per pixel adds them in chunk order (a team of many
//    blocks, e.g. a lone large box or a solo launch, keeps every warp busy instead of one
//    per tile).
// wstage: this warp's shared area (WARP_STAGE floats at smem + warp * WARP_STAGE).
template <bool SOLO, int DT, int SH>
__device__ __forceinline__ void phase_b_s(const Ctx& C, const Team& T, int pass, int* counter, float* wstage,
                                          int kiter) {
    using SS = ShapeStage<SH>;
    constexpr int TX = SS::X, TY = SS::Y, RUNB = SS::RUN, SBB = SS::SB, KOFFB = SS::KOFF, BUFB = SS::BUF;
    constexpr int TP = TX * TY;
    auto* xa = static_cast<typename Stor<DT>::T*>(C.xa);
    auto* xaT = static_cast<typename Stor<DT>::T*>(C.xaT);
    const int tm = SOLO ? 0 : T.member, ts = SOLO ? 1 : T.size;
    const BatchRoi& R = *C.R;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nx = R.nx, ny = R.ny;
    const int tiles_x = (nx + TX - 1) / TX, tiles = tiles_x * ((ny + TY - 1) / TY);
    // B_XS reads the window bins of the filtered sinogram of iteration kiter + 1
    const float* fk = pass == B_XS ? R.fcp + (size_t)kiter * R.na * R.fcp_nd : nullptr;
    const int li = lane / SS::LPR, lj0 = (lane % SS::LPR) * RUNB;
    const int nchunks = (R.na + ACH - 1) / ACH;

    // Chunk a0 .. a0 + ACH - 1 of tile (xi_t, eta_t) into buffer b of this warp: the tile
    // constants of each angle (one lane per angle), then the window bins by asynchronous
    // copies (zero outside the window; committed as one group).
    // Buffer layout: bins [ACH][SBB] | base (Q.23) | c step | s step | 1/w | kbase | width |
    // sinogram angle index | first window bin, ACH each.
    auto stage = [&](float xi_t, float eta_t, int a0, int b) {
        float* st = wstage + b * BUFB;
        int* cb = reinterpret_cast<int*>(st + ACH * SBB);
        int* cc = cb + ACH;
        int* cs = cc + ACH;
        float* ciw = reinterpret_cast<float*>(cs + ACH);
        int* ckb = reinterpret_cast<int*>(ciw + ACH);
        int* cwd = ckb + ACH;
        int* cai = cwd + ACH;
        int* cd0 = cai + ACH;
        const int nch = min(ACH, R.na - a0);
        if (lane < nch) {
            const AngleRec& r = R.rec[a0 + lane];
            ff kt = ff_add(ff_mul_f(xi_t, r.c), ff_mul_f(eta_t, r.s));
            kt = ff_add(kt, ff{-r.phi.hi, -r.phi.lo});
            const int kbase = (int)floorf(kt.hi) - KOFFB;
            kt = ff_add(kt, ff{-(float)kbase, 0.f});
            kt = ff_add(kt, ff_mul_f(-0.5f * (TX - 1), r.c));
            kt = ff_add(kt, ff_mul_f(0.5f * (TY - 1), r.s));
            cb[lane] = to_fixed<23>(kt);
            cc[lane] = r.c_q23;
            cs[lane] = r.s_q23;
            ciw[lane] = r.inv_w;
            ckb[lane] = kbase;
            cwd[lane] = r.width;
            cai[lane] = r.aidx;
            cd0[lane] = r.d0;
        }
        __syncwarp();
        for (int e = lane; e < nch * SBB; e += 32) {
            const int al = e / SBB, kk = ckb[al] + (e - al * SBB);
            const bool in = kk >= 0 && kk < cwd[al];
            if (pass == B_COLSUM) {
                st[e] = in ? 1.f : 0.f;
            } else {
                const float* row = pass == B_XS ? fk + (size_t)cai[al] * R.fcp_nd + cd0[al]
                                                : C.b.u + (size_t)(a0 + al) * R.stride;
                cp_async4(st + e, in ? row + kk : row, in);
            }
        }
        cp_async_commit();
    };
    // Partials of chunk a0 (in buffer b, bins landed) for this lane's run of 8 pixels.
    auto gather = [&](int a0, int b, float* acc) {
        const int nch = min(ACH, R.na - a0);
        float* st = wstage + b * BUFB;
        const int* cb = reinterpret_cast<const int*>(st + ACH * SBB);
        const int* cc = cb + ACH;
        const int* cs = cc + ACH;
        const float* ciw = reinterpret_cast<const float*>(cs + ACH);
        // bins times 1/w of their angle: the hat weights below are then max(0, 1 - d/w)
        for (int e = lane; e < nch * SBB; e += 32) st[e] *= ciw[e / SBB];
        __syncwarp();
#pragma unroll
        for (int p = 0; p < RUNB; ++p) acc[p] = 0.f;
        for (int al = 0; al < nch; ++al) {
            // weights max(0, 1 - d/w) of the two bins at distances f and 1 - f, f = mf 2^-23,
            // one saturating FMA each
            const float iw = ciw[al];
            const float iws = iw * 1.1920928955078125e-07f, niws = -iws, omiw = 1.f - iw;
            const int c = cc[al];
            int K = cb[al] + lj0 * c - li * cs[al];
            const float* srow = st + al * SBB;
            // two pixels of the run per packed (f32x2) operation: the same fused multiply-adds
            // as one pixel at a time
#pragma unroll
            for (int p = 0; p < RUNB; p += 2) {
                const int K1 = K + c;
                const int kl0 = chk(K >> 23, 0, SBB - 1, CHK_REGION_GATHER);
                const int kl1 = chk(K1 >> 23, 0, SBB - 1, CHK_REGION_GATHER);
                const float2 bits = make_float2(__uint_as_float(0x4B000000u | ((unsigned)K & 0x7FFFFFu)),
                                                __uint_as_float(0x4B000000u | ((unsigned)K1 & 0x7FFFFFu)));
                const float2 mf = __fadd2_rn(bits, make_float2(-8388608.0f, -8388608.0f));
                const float2 w0 = make_float2(fma_sat(mf.x, niws, 1.f), fma_sat(mf.y, niws, 1.f));
                const float2 w1 = make_float2(fma_sat(mf.x, iws, omiw), fma_sat(mf.y, iws, omiw));
                const float2 s0 = make_float2(srow[kl0], srow[kl1]);
                const float2 s1 = make_float2(srow[kl0 + 1], srow[kl1 + 1]);
                const float2 r = __ffma2_rn(w0, s0, __ffma2_rn(w1, s1, make_float2(acc[p], acc[p + 1])));
                acc[p] = r.x;
                acc[p + 1] = r.y;
                K = K1 + c;
            }
        }
    };
    // The pass's update of box pixel (gi, gj) from its gather acc.
    auto update = [&](int gi, int gj, float acc) {
        const int o = gi * nx + gj;
        if (pass == B_XS) {
            C.b.vy[o] = acc;  // x_s^k
        } else if (R.reg >= 3) {  // z = x_s + x_L - alpha W_L^T W_L x_L, disc added (FISTA-TV, Haar-ISTA)
            C.b.vx[o] = C.b.vy[o] + C.b.x[o] + acc + disc_value(R, gi, gj);
        } else if (R.reg == 2) {  // Alg. method, x >= 0 on the final image (disc added back)
            const float xs = C.b.vy[o];
            const float sv = xs + C.b.x[o] + acc;  // acc = -alpha W_L^T W_L y
            const float sh = disc_value(R, gi, gj);
            const float xv = fmaxf(sv + sh, 0.f) - sh;
            const float yn = xv - xs;
            C.b.x[o] = yn;
            C.b.vx[o] = xv;
            const auto ys = from_f32<DT>(yn);
            xa[gi * C.lda + gj] = ys;
            xaT[gj * C.ldaT + gi] = ys;
        } else if (pass == B_COLSUM) {
            if (R.reg == 0) {
                C.b.tau[o] = acc > 1e-3f ? 1.f / acc : 0.f;
            } else {
                const int cnt = (gj < nx - 1) + (gj > 0) + (gi < ny - 1) + (gi > 0);
                C.b.tau[o] = 1.f / (acc + (float)cnt);
            }
        } else if (R.reg == 0) {  // x in float; the projector reads its stored copy
            const float step = R.weighting ? C.b.tau[o] : R.alpha;
            float xn = fmaf(step, acc, C.b.x[o]);
            xn = fmaxf(xn, 0.f);
            C.b.x[o] = xn;
            const auto xs = from_f32<DT>(xn);
            xa[gi * C.lda + gj] = xs;
            xaT[gj * C.ldaT + gi] = xs;
        } else {
            float dv = 0.f;
            if (gj < nx - 1) dv += C.b.vx[o];
            if (gj > 0) dv -= C.b.vx[o - 1];
            if (gi < ny - 1) dv += C.b.vy[o];
            if (gi > 0) dv -= C.b.vy[o - nx];
            const float xo = C.b.x[o];
            const float xn = xo - C.b.tau[o] * (acc - dv);
            C.b.x[o] = xn;
            const auto xb = from_f32<DT>(2.f * xn - xo);
            xa[gi * C.lda + gj] = xb;
            xaT[gj * C.ldaT + gi] = xb;
        }
    };

    // (the single-block batch kernel, SOLO, keeps the per-warp schedule only: the same bits,
    // and fewer registers live in its loops)
    const int my_tiles = tm < tiles ? (tiles - tm + ts - 1) / ts : 0;
    unsigned dyn_bytes;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn_bytes));
    const int room = (int)(dyn_bytes / sizeof(float)) - BNW * WARP_STAGE;  // floats past the warp areas
    const int per_tile = nchunks * TP;                                     // one tile's chunk partials
    if (!SOLO && my_tiles > 0 && my_tiles < BNW && per_tile <= room) {
        // ---- cooperative: fewer tiles than warps.  The block's tiles are taken in groups
        // whose partials fit the shared memory past the warp areas; the (tile, chunk) items
        // of a group are dealt over all warps, and one thread per pixel adds a tile's chunk
        // partials in chunk order.
        float* part = wstage - warp * WARP_STAGE + BNW * WARP_STAGE;  // [group][nchunks][TP]
        const int G = min(my_tiles, room / per_tile);
        // the window bins of a warp's next item are copied while it gathers the current one
        auto stage_item = [&](int g0, int item, int b) {
            const int gt = item / nchunks, c = item - gt * nchunks;
            const int t = tm + (g0 + gt) * ts;
            const int tile_x0 = (t % tiles_x) * TX, tile_y0 = (t / tiles_x) * TY;
            const float xi_t = (float)tile_x0 + 0.5f * (TX - 1) - 0.5f * (float)(nx - 1);
            const float eta_t = 0.5f * (float)(ny - 1) - ((float)tile_y0 + 0.5f * (TY - 1));
            stage(xi_t, eta_t, c * ACH, b);
        };
        for (int g0 = 0; g0 < my_tiles; g0 += G) {
            const int gn = min(G, my_tiles - g0), nitems = gn * nchunks;
            __syncwarp();  // this warp's buffers are free
            if (warp < nitems) stage_item(g0, warp, 0);
            for (int item = warp, b = 0; item < nitems; item += BNW, b ^= 1) {
                if (item + BNW < nitems) {
                    stage_item(g0, item + BNW, b ^ 1);
                    cp_async_wait_group<1>();  // this item's copies have landed
                } else {
                    cp_async_wait_group<0>();
                }
                __syncwarp();
                const int gt = item / nchunks, c = item - gt * nchunks;
                float acc[RUNB];
                gather(c * ACH, b, acc);
#pragma unroll
                for (int p = 0; p < RUNB; ++p) part[(gt * nchunks + c) * TP + li * TX + lj0 + p] = acc[p];
                __syncwarp();  // buffer b is refilled by the item after next
            }
            __syncthreads();
            for (int e = threadIdx.x; e < gn * TP; e += BPT) {  // one thread per pixel: the chunks in order
                const int gt = e / TP, px = e - gt * TP;
                const int t = tm + (g0 + gt) * ts;
                const int tile_x0 = (t % tiles_x) * TX, tile_y0 = (t / tiles_x) * TY;
                float sum = 0.f, cmp = 0.f;
                for (int c = 0; c < nchunks; ++c) neu_add(sum, cmp, part[(gt * nchunks + c) * TP + px]);
                const int gi = tile_y0 + px / TX, gj = tile_x0 + px % TX;
                if (gi < ny && gj < nx) update(gi, gj, sum + cmp);
            }
            __syncthreads();  // the partials area is reused by the next group
        }
        return;
    }
    // ---- per warp
    for (int i = warp;;) {
        const int t = tm + i * ts;
        if (t >= tiles) break;
        const int tile_x0 = (t % tiles_x) * TX, tile_y0 = (t / tiles_x) * TY;
        const float xi_t = (float)tile_x0 + 0.5f * (TX - 1) - 0.5f * (float)(nx - 1);
        const float eta_t = 0.5f * (float)(ny - 1) - ((float)tile_y0 + 0.5f * (TY - 1));
        float sum[RUNB], cmp[RUNB];
#pragma unroll
        for (int p = 0; p < RUNB; ++p) sum[p] = cmp[p] = 0.f;
        __syncwarp();  // the previous tile's reads of both buffers are done
        stage(xi_t, eta_t, 0, 0);
        for (int a0 = 0, b = 0; a0 < R.na; a0 += ACH, b ^= 1) {
            if (a0 + ACH < R.na) {
                stage(xi_t, eta_t, a0 + ACH, b ^ 1);  // the next chunk's bins fly while this one is gathered
                cp_async_wait_group<1>();               // this chunk's copies have landed
            } else {
                cp_async_wait_group<0>();
            }
            __syncwarp();
            float acc[RUNB];
            gather(a0, b, acc);
#pragma unroll
            for (int p = 0; p < RUNB; ++p) neu_add(sum[p], cmp[p], acc[p]);
            __syncwarp();  // buffer b is refilled by the chunk after next
        }
        // update of this lane's pixels
        const int gi = tile_y0 + li;
#pragma unroll
        for (int p = 0; p < RUNB; ++p) {
            const int gj = tile_x0 + lj0 + p;
            if (gi < ny && gj < nx) update(gi, gj, sum[p] + cmp[p]);
        }
        int nxt = 0;
        if (lane == 0) nxt = atomicAdd(counter, 1);
        i = __shfl_sync(0xffffffffu, nxt, 0);
    }
}

// Phase B with the region's tile shape.
template <bool SOLO, int DT>
__device__ __forceinline__ void phase_b(const Ctx& C, const Team& T, int pass, int* counter, float* wstage,
                                        int kiter = 0) {
    if (C.R->shape == 1)
        phase_b_s<SOLO, DT, 1>(C, T, pass, counter, wstage, kiter);
    else if (C.R->shape == 2)
        phase_b_s<SOLO, DT, 2>(C, T, pass, counter, wstage, kiter);
    else
        phase_b_s<SOLO, DT, 0>(C, T, pass, counter, wstage, kiter);
}

__device__ __forceinline__ void fill_team(const Ctx& C, float* p, size_t n, float v) {
    for (size_t i = team_tid(C); i < n; i += C.gthreads) p[i] = v;
}

// Interior of both padded images := v, borders 0.
template <int DT>
__device__ __forceinline__ void set_images(const Ctx& C, float v) {
    const BatchRoi& R = *C.R;
    const int nx = R.nx, ny = R.ny;
    auto* xab = static_cast<typename Stor<DT>::T*>(C.b.xa_base);
    auto* xaTb = static_cast<typename Stor<DT>::T*>(C.b.xaT_base);
    const auto sv = from_f32<DT>(v), zero = from_f32<DT>(0.f);
    for (int i = team_tid(C); i < ny * C.lda; i += C.gthreads) {
        const int col = i % C.lda - kPad;
        xab[i] = (col >= 0 && col < nx) ? sv : zero;
    }
    for (int i = team_tid(C); i < nx * C.ldaT; i += C.gthreads) {
        const int col = i % C.ldaT - kPad;
        xaTb[i] = (col >= 0 && col < ny) ? sv : zero;
    }
}

// Both padded images := the box of x_fbp (rows from the padded grid image, columns
// from its padded transpose), borders 0.
// (The grid image has the region's storage type, so elements are copied as they are.)
template <int DT>
__device__ __forceinline__ void load_fbp_box(const Ctx& C) {
    using T = typename Stor<DT>::T;
    const BatchRoi& R = *C.R;
    const int nx = R.nx, ny = R.ny;
    auto* xab = static_cast<T*>(C.b.xa_base);
    auto* xaTb = static_cast<T*>(C.b.xaT_base);
    const T* g = static_cast<const T*>(R.xfbp);
    const T* gT = static_cast<const T*>(R.xfbpT);
    const T zero = from_f32<DT>(0.f);
    for (int i = team_tid(C); i < ny * C.lda; i += C.gthreads) {
        const int r = i / C.lda, col = i - r * C.lda - kPad;
        xab[i] = (col >= 0 && col < nx) ? g[(size_t)(R.box_y0 + r) * R.xfbp_ld + R.box_x0 + col] : zero;
    }
    for (int i = team_tid(C); i < nx * C.ldaT; i += C.gthreads) {
        const int r = i / C.ldaT, col = i - r * C.ldaT - kPad;
        xaTb[i] = (col >= 0 && col < ny) ? gT[(size_t)(R.box_x0 + r) * R.xfbp_ld + R.box_y0 + col] : zero;
    }
}

// Floats of dynamic shared memory of this launch.
__device__ __forceinline__ int dyn_smem_floats() {
    unsigned dyn_bytes;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn_bytes));
    return (int)(dyn_bytes / sizeof(float));
}

// Both branches of phase A reading the images from global memory (the dynamic shared
// memory, unused meanwhile, holds the anchor values of a split phase A).
template <bool SOLO, int DT>
__device__ __forceinline__ void phase_a_global(const Ctx& C, const Team& T, int pass, int* s_cnt, float* smem) {
    for (int row = 1; row >= 0; --row) {
        if (threadIdx.x == 0) *s_cnt = BNW;
        __syncthreads();
        phase_a_branch<SOLO, DT>(C, T, row, row ? C.xa : C.xaT, row ? C.lda : C.ldaT, pass, s_cnt, smem,
                                 dyn_smem_floats());
        __syncthreads();
    }
}

// Band-streamed phase A of a block with many units (as phase_a_banded, same bits): passes
// of up to per_pass units, each pass walking all bands once; in every band the warps take the
// pass's units round-robin and add each ray's band value to its partial sums, kept in shared
// memory past the band buffers (st_sum, st_cmp: [per_pass][32]).  The image then crosses from
// L2 once per pass instead of once per 32 units.
template <bool SOLO, int DT>
__device__ __noinline__ bool phase_a_banded_passes(const Ctx& C, const Team& T, int row, const void* img_base_v,
                                                   int ld, float* smem_f, uint64_t* mbar, unsigned& parity,
                                                   int nu, int per_pass, float* st_sum, float* st_cmp) {
    using TS = typename Stor<DT>::T;
    constexpr unsigned ES = sizeof(TS);
    const TS* img_base = static_cast<const TS*>(img_base_v);
    TS* smem = reinterpret_cast<TS*>(smem_f);
    const BatchRoi& R = *C.R;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int tm = SOLO ? 0 : T.member, ts = SOLO ? 1 : T.size;
    const int M = row ? R.ny : R.nx, Mm = row ? R.nx : R.ny;
    const int ustart = row ? 0 : R.nrow * C.nchunk;
    const int BR = band_rows(R.nx, R.ny, ES);
    const int nb = (M + BR - 1) / BR;
    const int band_floats = BR * ld;
    const float halfM = 0.5f * (float)(M - 1);
    for (int g0 = 0; g0 < nu; g0 += per_pass) {
        const int np = min(per_pass, nu - g0);
        for (int e = threadIdx.x; e < np * 32; e += BPT) st_sum[e] = st_cmp[e] = 0.f;
        if (threadIdx.x == 0) {
            const int rows0 = M < BR ? M : BR;
            bulk_load(smem, img_base, ES * rows0 * ld, &mbar[0]);
        }
        for (int b = 0; b < nb; ++b) {
            const int bi = b & 1;
            if (threadIdx.x == 0 && b + 1 < nb) {  // the other buffer was released by the last barrier
                const int rows = min(BR, M - (b + 1) * BR);
                bulk_load(smem + (bi ^ 1) * band_floats, img_base + (size_t)(b + 1) * band_floats, ES * rows * ld,
                          &mbar[bi ^ 1]);
            }
            if (!mbar_wait(&mbar[bi], (parity >> bi) & 1u, T.wait_ns, T.err)) return false;
            parity ^= 1u << bi;
            for (int i = warp; i < np; i += BNW) {
                const int unit = ustart + tm + (g0 + i) * ts;
                const int a = unit / C.nchunk;
                const int k = (unit - a * C.nchunk) * 32 + lane;
                const AngleRec& r = R.rec[a];
                if (k >= r.width) continue;
                int mlo, mhi;
                const ff Ak = ray_span(r, k, M, Mm, mlo, mhi);
                const int m0 = max(mlo, b * BR), m1 = min(mhi, (b + 1) * BR);
                if (m0 >= m1) continue;
                int j0;
                int q = split_fixed22(ff_add(Ak, ff_mul_f((float)m0 - halfM, r.slope)), j0);
                const int step = r.slope_q22;
                const TS* rp = smem + bi * band_floats + (m0 - b * BR) * ld + kPad + j0;
                const int jlo = -kPad - j0, jhi = ld - 1 - kPad - j0;
                float s0 = 0.f, s1 = 0.f;
#pragma unroll 4
                for (int m = m0; m < m1; ++m, rp += ld, q += step) {
                    const int j = chk(q >> 22, jlo, jhi, CHK_REGION_BAND);
                    const float mf = frac_int<22>(q);
                    const float v0 = to_f32<DT>(rp[j]), v1 = to_f32<DT>(rp[j + 1]);
                    s0 += v0;
                    s1 = fmaf(mf, v1 - v0, s1);
                }
                neu_add(st_sum[i * 32 + lane], st_cmp[i * 32 + lane], fmaf(s1, 2.384185791015625e-07f, s0));
            }
            __syncthreads();
        }
        for (int i = warp; i < np; i += BNW) {
            const int unit = ustart + tm + (g0 + i) * ts;
            const int a = unit / C.nchunk;
            const int k = (unit - a * C.nchunk) * 32 + lane;
            const AngleRec& r = R.rec[a];
            if (k < r.width) finish_ray(C, r, a, k, two_sum(st_sum[i * 32 + lane], st_cmp[i * 32 + lane]), A_SOLVE);
        }
        __syncthreads();  // the partial sums are reused by the next pass
    }
    return true;
}

// Phase A of one branch with the image streamed through shared memory in bands of
// band_rows() rows (two buffers, one bulk copy each, refilled while the other is read).
// This block's units (ustart + member + i * size) are taken in groups of 32, one per
// warp; each group walks all bands, each lane accumulating its ray over the samples
// that fall in the band (one float-float anchor per band and ray), then finishes the
// ray as phase_a_branch does.  A block with at least 128 units goes by passes instead
// (phase_a_banded_passes) when the shared memory past the band buffers holds the partial
// sums of 64 or more units.  mbar[0..1]: the buffers' barriers, parity: their phase bits
// (bit b for buffer b).  false: a wait gave up.
template <bool SOLO, int DT>
__device__ __forceinline__ bool phase_a_banded(const Ctx& C, const Team& T, int row, const void* img_base_v, int ld,
                                               float* smem_f, uint64_t* mbar, unsigned& parity) {
    using TS = typename Stor<DT>::T;
    constexpr unsigned ES = sizeof(TS);
    const TS* img_base = static_cast<const TS*>(img_base_v);
    TS* smem = reinterpret_cast<TS*>(smem_f);
    const BatchRoi& R = *C.R;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int tm = SOLO ? 0 : T.member, ts = SOLO ? 1 : T.size;
    const int M = row ? R.ny : R.nx, Mm = row ? R.nx : R.ny;
    const int ustart = row ? 0 : R.nrow * C.nchunk;
    const int total = (row ? R.nrow : R.na) * C.nchunk - ustart;
    const int nu = total > tm ? (total - tm + ts - 1) / ts : 0;
    if (nu >= 4 * BNW) {  // many units: passes with the partial sums in shared memory
        const int state_off = (int)((stage_bytes(R.nx, R.ny, ES) + 15) / 16 * 4);
        const int cap = (dyn_smem_floats() - state_off) / 64 / BNW * BNW;
        if (cap >= 2 * BNW) {
            float* st = smem_f + state_off;
            return phase_a_banded_passes<SOLO, DT>(C, T, row, img_base_v, ld, smem_f, mbar, parity, nu, cap, st,
                                                   st + (size_t)cap * 32);
        }
    }
    const int BR = band_rows(R.nx, R.ny, ES);
    const int nb = (M + BR - 1) / BR;
    const int band_floats = BR * ld;
    const float halfM = 0.5f * (float)(M - 1);
    for (int g0 = 0; g0 < nu; g0 += BNW) {
        const int i = g0 + warp;
        int a = 0, k = 0;
        bool valid = i < nu;
        if (valid) {
            const int unit = ustart + tm + i * ts;
            a = unit / C.nchunk;
            k = (unit - a * C.nchunk) * 32 + lane;
            valid = k < R.rec[a].width;
        }
        const AngleRec& r = R.rec[a];
        ff Ak{0.f, 0.f};
        int mlo = 0, mhi = 0;
        if (valid) {
            Ak = ff_add(r.A0, ff_mul_f((float)k, r.a_scale));
            mhi = M;
            if (!r.flat) {
                const float ma = (-1.5f - Ak.hi) * r.inv_slope + halfM;
                const float mb = ((float)Mm + 0.5f - Ak.hi) * r.inv_slope + halfM;
                const float lo = fminf(ma, mb), hi = fmaxf(ma, mb);
                mlo = (int)fminf(fmaxf(0.f, ceilf(lo)), (float)M);
                mhi = (int)fmaxf(fminf((float)M, floorf(hi) + 1.f), 0.f);
            } else if (!(Ak.hi >= -1.5f && Ak.hi <= (float)Mm + 0.5f)) {
                mhi = 0;
            }
        }
        float sum = 0.f, cmp = 0.f;
        if (threadIdx.x == 0) {
            const int rows0 = M < BR ? M : BR;
            bulk_load(smem, img_base, ES * rows0 * ld, &mbar[0]);
        }
        for (int b = 0; b < nb; ++b) {
            const int bi = b & 1;
            if (threadIdx.x == 0 && b + 1 < nb) {  // the other buffer was released by the last barrier
                const int rows = min(BR, M - (b + 1) * BR);
                bulk_load(smem + (bi ^ 1) * band_floats, img_base + (size_t)(b + 1) * band_floats, ES * rows * ld,
                          &mbar[bi ^ 1]);
            }
            if (!mbar_wait(&mbar[bi], (parity >> bi) & 1u, T.wait_ns, T.err)) return false;
            parity ^= 1u << bi;
            const int m0 = max(mlo, b * BR), m1 = min(mhi, (b + 1) * BR);
            if (valid && m0 < m1) {
                int j0;
                int q = split_fixed22(ff_add(Ak, ff_mul_f((float)m0 - halfM, r.slope)), j0);
                const int step = r.slope_q22;
                const TS* rp = smem + bi * band_floats + (m0 - b * BR) * ld + kPad + j0;
                const int jlo = -kPad - j0, jhi = ld - 1 - kPad - j0;
                float s0 = 0.f, s1 = 0.f;
#pragma unroll 4
                for (int m = m0; m < m1; ++m, rp += ld, q += step) {
                    const int j = chk(q >> 22, jlo, jhi, CHK_REGION_BAND);
                    const float mf = frac_int<22>(q);
                    const float v0 = to_f32<DT>(rp[j]), v1 = to_f32<DT>(rp[j + 1]);
                    s0 += v0;
                    s1 = fmaf(mf, v1 - v0, s1);
                }
                neu_add(sum, cmp, fmaf(s1, 2.384185791015625e-07f, s0));
            }
            __syncthreads();
        }
        if (valid) {
            ff tot = ff_mul_f(r.inv_w, two_sum(sum, cmp));
            const float acc = tot.hi + tot.lo;
            const size_t o = (size_t)a * R.stride + k;
            if (R.reg == 0) {
                float res = C.b.pp[o] - acc;
                if (R.weighting) res *= C.b.sig[o];
                C.b.u[o] = res;
            } else if (R.reg >= 2) {
                C.b.u[o] = -R.alpha * acc;
            } else {
                const float sg = C.b.sig[o];
                C.b.u[o] = (C.b.u[o] + sg * (acc - C.b.pp[o])) / (1.f + 0.5f * sg);
            }
        }
    }
    return true;
}

// Band-streamed phase A of a large team (a lone box on every block), decomposed by row band:
// the branch's (band, 32 units) items are split among the branch's blocks in band order, so
// a block stages the one or two bands of its items once and every warp takes a unit; each
// ray's partial over a band -- the same operations as a band of phase_a_banded -- goes to
// C.b.part, and after a team barrier one warp per unit adds the partials of the bands the ray
// crosses in band order and applies the update: the same bits as phase_a_banded.  Every block
// of the team calls this once per iteration (with its own branch).  false: a wait gave up.
template <bool SOLO, int DT>
__device__ __noinline__ bool phase_a_rowband(const Ctx& C, Team& T, int row, const void* img_base_v, int ld,
                                             float* smem_f, uint64_t* mbar, unsigned& parity) {
    using TS = typename Stor<DT>::T;
    constexpr unsigned ES = sizeof(TS);
    const TS* img_base = static_cast<const TS*>(img_base_v);
    TS* smem = reinterpret_cast<TS*>(smem_f);
    const BatchRoi& R = *C.R;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int M = row ? R.ny : R.nx, Mm = row ? R.nx : R.ny;
    const int BR = band_rows(R.nx, R.ny, ES);
    const int nb = (M + BR - 1) / BR;
    const int band_floats = BR * ld;
    const float halfM = 0.5f * (float)(M - 1);
    const int total_r = R.nrow * C.nchunk, total_c = (R.na - R.nrow) * C.nchunk;
    const int total = row ? total_r : total_c;
    const int ustart = row ? 0 : total_r;
    float* P = C.b.part + (row ? 0 : (size_t)((R.ny + BR - 1) / BR) * total_r * 32);
    // ---- partials: items (band, 32 units), band-major, in contiguous ranges per block
    const int nchk = (total + 31) / 32;
    const long items = (long)nb * nchk;
    const long it0 = items * C.amember / C.asize, it1 = items * (C.amember + 1) / C.asize;
    int cur = -1;
    for (long it = it0; it < it1; ++it) {
        const int b = (int)(it / nchk), ch = (int)(it - (long)b * nchk);
        if (b != cur) {
            __syncthreads();  // the buffer's previous band is read
            if (threadIdx.x == 0) {
                const int rows = min(BR, M - b * BR);
                bulk_load(smem, img_base + (size_t)b * band_floats, ES * rows * ld, &mbar[0]);
            }
            if (!mbar_wait(&mbar[0], parity & 1u, T.wait_ns, T.err)) return false;
            parity ^= 1u;
            cur = b;
        }
        const int u = ch * 32 + warp;
        if (u >= total) continue;
        const int unit = ustart + u;
        const int a = unit / C.nchunk;
        const int k = (unit - a * C.nchunk) * 32 + lane;
        const AngleRec& r = R.rec[a];
        float part = 0.f;
        if (k < r.width) {
            int mlo, mhi;
            const ff Ak = ray_span(r, k, M, Mm, mlo, mhi);
            const int m0 = max(mlo, b * BR), m1 = min(mhi, (b + 1) * BR);
            if (m0 < m1) {
                int j0;
                int q = split_fixed22(ff_add(Ak, ff_mul_f((float)m0 - halfM, r.slope)), j0);
                const int step = r.slope_q22;
                const TS* rp = smem + (m0 - b * BR) * ld + kPad + j0;
                const int jlo = -kPad - j0, jhi = ld - 1 - kPad - j0;
                float s0 = 0.f, s1 = 0.f;
#pragma unroll 4
                for (int m = m0; m < m1; ++m, rp += ld, q += step) {
                    const int j = chk(q >> 22, jlo, jhi, CHK_REGION_BAND);
                    const float mf = frac_int<22>(q);
                    const float v0 = to_f32<DT>(rp[j]), v1 = to_f32<DT>(rp[j + 1]);
                    s0 += v0;
                    s1 = fmaf(mf, v1 - v0, s1);
                }
                part = fmaf(s1, 2.384185791015625e-07f, s0);
            }
        }
        P[((size_t)b * total + u) * 32 + lane] = part;
    }
    if (!team_sync<SOLO>(T)) return false;  // every band's partials are in
    // ---- one warp per unit: the bands the ray crosses, in order, then the update
    for (int u = C.amember * 32 + warp; u < total; u += C.asize * 32) {
        const int unit = ustart + u;
        const int a = unit / C.nchunk;
        const int k = (unit - a * C.nchunk) * 32 + lane;
        const AngleRec& r = R.rec[a];
        if (k >= r.width) continue;
        int mlo, mhi;
        ray_span(r, k, M, Mm, mlo, mhi);
        float sum = 0.f, cmp = 0.f;
        for (int b = 0; b < nb; ++b) {
            const int m0 = max(mlo, b * BR), m1 = min(mhi, (b + 1) * BR);
            if (m0 < m1) neu_add(sum, cmp, __ldcg(P + ((size_t)b * total + u) * 32 + lane));
        }
        ff tot = ff_mul_f(r.inv_w, two_sum(sum, cmp));
        const float acc = tot.hi + tot.lo;
        const size_t o = (size_t)a * R.stride + k;
        if (R.reg == 0) {
            float res = C.b.pp[o] - acc;
            if (R.weighting) res *= C.b.sig[o];
            C.b.u[o] = res;
        } else if (R.reg >= 2) {
            C.b.u[o] = -R.alpha * acc;
        } else {
            const float sg = C.b.sig[o];
            C.b.u[o] = (C.b.u[o] + sg * (acc - C.b.pp[o])) / (1.f + 0.5f * sg);
        }
    }
    return true;
}

// CP gradient dual on this thread's pixels: v = proj_{|v| <= lambda}(v + sigma_v grad xbar).
template <int DT>
__device__ __forceinline__ void dual_grad(const Ctx& C) {
    const BatchRoi& R = *C.R;
    const int nimg = R.nx * R.ny;
    const auto* xa = static_cast<const typename Stor<DT>::T*>(C.xa);
    for (int p = team_tid(C); p < nimg; p += C.gthreads) {
        const int i = p / R.nx, j = p - i * R.nx;
        const auto* xp = xa + i * C.lda + j;
        const float x0 = to_f32<DT>(xp[0]);
        const float gx = j < R.nx - 1 ? to_f32<DT>(xp[1]) - x0 : 0.f;
        const float gy = i < R.ny - 1 ? to_f32<DT>(xp[C.lda]) - x0 : 0.f;
        const float ax = fmaf(R.sigma_v, gx, C.b.vx[p]);
        const float ay = fmaf(R.sigma_v, gy, C.b.vy[p]);
        const float m = sqrtf(ax * ax + ay * ay);
        const float sc = m > R.lambda ? R.lambda / m : 1.f;
        C.b.vx[p] = ax * sc;
        C.b.vy[p] = ay * sc;
    }
}

// FGP on the box (Alg. methodfista's TV prox): x = argmin ||x - z||^2 + 2 lam_f TV(x) by
// R.n_fgp accelerated projected-gradient steps on the dual (step 1/(8 lam_f)); z in C.b.vx,
// x into fgp[4].  Pixels are dealt over the team; neighbours are read only across a
// team barrier.  false: a wait gave up.
template <bool SOLO>
__device__ __forceinline__ bool fgp_prox_t(const Ctx& C, Team& T) {
    const BatchRoi& R = *C.R;
    const int nx = R.nx, ny = R.ny, nimg = nx * ny;
    float* vx = C.b.fgp;
    float* vy = vx + nimg;
    float* rx = vy + nimg;
    float* ry = rx + nimg;
    float* fx = ry + nimg;
    const float* z = C.b.vx;
    const float lam = R.lam_f;
    if (!(lam > 0.f) || R.n_fgp <= 0) {
        for (int p = team_tid(C); p < nimg; p += C.gthreads) fx[p] = z[p];
        return team_sync<SOLO>(T);
    }
    for (int p = team_tid(C); p < nimg; p += C.gthreads) vx[p] = vy[p] = rx[p] = ry[p] = 0.f;
    const float inv8 = 1.f / (8.f * lam);
    float t = 1.f;
    for (int k = 0; k <= R.n_fgp; ++k) {
        if (!team_sync<SOLO>(T)) return false;
        const bool last = k == R.n_fgp;
        const float* dx = last ? vx : rx;
        const float* dy = last ? vy : ry;
        for (int p = team_tid(C); p < nimg; p += C.gthreads) {  // x = z + lam div(r), or div(v) at the end
            const int i = p / nx, j = p - i * nx;
            float d = 0.f;
            if (j < nx - 1) d += dx[p];
            if (j > 0) d -= dx[p - 1];
            if (i < ny - 1) d += dy[p];
            if (i > 0) d -= dy[p - nx];
            fx[p] = fmaf(lam, d, z[p]);
        }
        if (last) break;
        if (!team_sync<SOLO>(T)) return false;
        const float tn = 0.5f * (1.f + sqrtf(1.f + 4.f * t * t));
        const float beta = (t - 1.f) / tn;
        for (int p = team_tid(C); p < nimg; p += C.gthreads) {  // v = P(r + grad x / (8 lam)), r extrapolated
            const int i = p / nx, j = p - i * nx;
            const float x0 = fx[p];
            const float gx = j < nx - 1 ? fx[p + 1] - x0 : 0.f;
            const float gy = i < ny - 1 ? fx[p + nx] - x0 : 0.f;
            float ax = fmaf(gx, inv8, rx[p]), ay = fmaf(gy, inv8, ry[p]);
            const float m = sqrtf(ax * ax + ay * ay);
            if (m > 1.f) {
                ax /= m;
                ay /= m;
            }
            rx[p] = fmaf(beta, ax - vx[p], ax);
            ry[p] = fmaf(beta, ay - vy[p], ay);
            vx[p] = ax;
            vy[p] = ay;
        }
        t = tn;
    }
    return team_sync<SOLO>(T);
}

// FISTA step of Alg. methodfista on this thread's pixels (t = t_{k-1}):
//   x^k = FGP result - disc;  r = x^k + ((t - 1) / t_k) (x^k - x^{k-1});  x_L = r - x_s.
template <int DT>
__device__ __forceinline__ void fista_update(const Ctx& C, float t) {
    const BatchRoi& R = *C.R;
    const int nx = R.nx, nimg = nx * R.ny;
    auto* xa = static_cast<typename Stor<DT>::T*>(C.xa);
    auto* xaT = static_cast<typename Stor<DT>::T*>(C.xaT);
    const float* fx = C.b.fgp + 4 * (size_t)nimg;
    const float tn = 0.5f * (1.f + sqrtf(1.f + 4.f * t * t));
    const float beta = (t - 1.f) / tn;
    for (int p = team_tid(C); p < nimg; p += C.gthreads) {
        const int i = p / nx, j = p - i * nx;
        const float xk = fx[p] - disc_value(R, i, j);
        const float r = fmaf(beta, xk - C.b.tau[p], xk);
        const float xl = r - C.b.vy[p];
        C.b.tau[p] = xk;
        C.b.x[p] = xl;
        const auto xs = from_f32<DT>(xl);
        xa[i * C.lda + j] = xs;
        xaT[j * C.ldaT + i] = xs;
    }
}

// One orthonormal Haar step on the leading [hl][wl] block of an image of row stride ld,
// along rows (dir 0) or columns (dir 1): split = pair sums / differences over sqrt(2), an
// odd last entry carried as a sum; merge = its transpose.  Team-split over the block.
__device__ __forceinline__ void haar_pass(const Ctx& C, const float* in, float* out, int ld, int hl, int wl, int dir,
                                          bool merge) {
    const float s = 0.70710678118654752f;
    const int L = dir ? hl : wl, m = L / 2, c = (L + 1) / 2;
    for (int q = team_tid(C); q < hl * wl; q += C.gthreads) {
        const int i = q / wl, j = q - i * wl;
        const int e = dir ? i : j;                          // index along the pass
        const int base = dir ? j : i * ld, st = dir ? ld : 1;  // line start, element stride
        float v;
        if (!merge) {
            if (e < m)
                v = s * (in[base + 2 * e * st] + in[base + (2 * e + 1) * st]);
            else if (e < c)
                v = in[base + (L - 1) * st];
            else
                v = s * (in[base + 2 * (e - c) * st] - in[base + (2 * e - 2 * c + 1) * st]);
        } else {
            const int k = e / 2;
            if ((L & 1) && e == L - 1)
                v = in[base + m * st];
            else if (e & 1)
                v = s * (in[base + k * st] - in[base + (c + k) * st]);
            else
                v = s * (in[base + k * st] + in[base + (c + k) * st]);
        }
        out[i * ld + j] = v;
    }
}

// Haar-ISTA step of Alg. method (Eq. sirtista): x = B^-1 P_tau(B z) - disc with z in
// C.b.vx (transformed in place, fgp[0] as the other buffer), tau = R.lam_f; then
// y = x - x_s into C.b.x and the projector images, x into C.b.tau.
template <bool SOLO, int DT>
__device__ __forceinline__ bool haar_ista_step(const Ctx& C, Team& T) {
    const BatchRoi& R = *C.R;
    const int nx = R.nx, ny = R.ny, nimg = nx * ny;
    float* z = C.b.vx;
    float* t = C.b.fgp;
    // level l works on the leading [ceil(ny / 2^l)][ceil(nx / 2^l)] block (repeated ceil halving)
    int nl = 0;
    while (nl < 30 && ((ny + (1 << nl) - 1) >> nl) >= 2 && ((nx + (1 << nl) - 1) >> nl) >= 2) ++nl;
    for (int l = 0; l < nl; ++l) {
        const int hl = (ny + (1 << l) - 1) >> l, wl = (nx + (1 << l) - 1) >> l;
        haar_pass(C, z, t, nx, hl, wl, 0, false);
        if (!team_sync<SOLO>(T)) return false;
        haar_pass(C, t, z, nx, hl, wl, 1, false);
        if (!team_sync<SOLO>(T)) return false;
    }
    const float tau = R.lam_f;
    for (int p = team_tid(C); p < nimg; p += C.gthreads) {
        const float a = fabsf(z[p]) - tau;
        z[p] = a > 0.f ? copysignf(a, z[p]) : 0.f;
    }
    for (int l = nl - 1; l >= 0; --l) {
        const int hl = (ny + (1 << l) - 1) >> l, wl = (nx + (1 << l) - 1) >> l;
        if (!team_sync<SOLO>(T)) return false;
        haar_pass(C, z, t, nx, hl, wl, 1, true);
        if (!team_sync<SOLO>(T)) return false;
        haar_pass(C, t, z, nx, hl, wl, 0, true);
    }
    if (!team_sync<SOLO>(T)) return false;
    auto* xa = static_cast<typename Stor<DT>::T*>(C.xa);
    auto* xaT = static_cast<typename Stor<DT>::T*>(C.xaT);
    for (int p = team_tid(C); p < nimg; p += C.gthreads) {
        const int i = p / nx, j = p - i * nx;
        const float xv = z[p] - disc_value(R, i, j);
        const float yv = xv - C.b.vy[p];
        C.b.tau[p] = xv;
        C.b.x[p] = yv;
        const auto ys = from_f32<DT>(yv);
        xa[i * C.lda + j] = ys;
        xaT[j * C.ldaT + i] = ys;
    }
    return team_sync<SOLO>(T);
}

// Solve region R into R.out.  DT: storage of x_fbp and of the projector images (R.dt).
// smem: dynamic shared memory, at least stage_bytes(nx, ny, esz) and the per-warp phase-B
// areas; mbar[0..1]: two initialised mbarriers, parity their phase bits.  Returns false
// when a wait gave up (error flag set): leave the kernel.
template <bool SOLO, int DT>
__device__ __forceinline__ bool solve_region(const BatchRoi& R, const RegionBufs& bufs, Team& T, float* smem,
                                             uint64_t* mbar, unsigned& parity, int* s_cnt) {
    using TS = typename Stor<DT>::T;
    constexpr int ES = (int)sizeof(TS);
    const int tid = threadIdx.x, warp = tid >> 5;
    __shared__ Ctx s_ctx;
    if (tid == 0) {
        Ctx& W = s_ctx;
        W.R = &R;
        W.b = bufs;
        W.lda = padded_ld_e(R.nx, ES);
        W.ldaT = padded_ld_e(R.ny, ES);
        W.xa = static_cast<TS*>(bufs.xa_base) + kPad;
        W.xaT = static_cast<TS*>(bufs.xaT_base) + kPad;
        W.nchunk = (R.stride + 31) / 32;
        W.member = SOLO ? 0 : T.member;
        W.gthreads = (SOLO ? 1 : T.size) * BPT;
        W.stage = stage_mode(R.nx, R.ny, ES);  // every block of a team stages the image itself
        W.arow = -1;
        W.amember = W.member;
        W.asize = SOLO ? 1 : T.size;
        if (!SOLO && T.size > 1) {
            const long ur = (long)R.nrow * W.nchunk, uc = (long)(R.na - R.nrow) * W.nchunk;
            int gr = (int)((ur * T.size + (ur + uc) / 2) / max(ur + uc, 1L));
            if (ur > 0 && gr < 1) gr = 1;
            if (uc > 0 && gr > T.size - 1) gr = T.size - 1;
            if (uc == 0) gr = T.size;
            if (ur == 0) gr = 0;
            W.arow = T.member < gr ? 1 : 0;
            W.amember = W.arow ? T.member : T.member - gr;
            W.asize = W.arow ? gr : T.size - gr;
        }
    }
    __syncthreads();
    const Ctx& C = s_ctx;
    const size_t nimg = (size_t)R.nx * R.ny, nwin = (size_t)R.na * R.stride;
    const unsigned bytes_row = (unsigned)(ES * (size_t)R.ny * C.lda);
    const unsigned bytes_col = (unsigned)(ES * (size_t)R.nx * C.ldaT);
    // floats of the whole staged image (stage mode 0), 16-byte aligned: a split phase A keeps
    // its anchor values past it
    const int img_floats = (int)((stage_bytes(R.nx, R.ny, ES) + 15) / 16 * 4);

    // ---- exterior: p' on the window rays, zero state
    fill_team(C, C.b.u, nwin, 0.f);
    fill_team(C, C.b.x, nimg, 0.f);
    fill_team(C, C.b.vx, nimg, 0.f);
    fill_team(C, C.b.vy, nimg, 0.f);
    if (R.reg < 2) {  // the paper's own method (reg 2, 3) needs no exterior step
        load_fbp_box<DT>(C);
        if (!team_sync<SOLO>(T)) return false;
        phase_a_global<SOLO, DT>(C, T, A_EXTER, s_cnt, smem);
    }
    // ---- set-up: preconditioners / weights from the row and column sums
    if (R.reg == 1 || R.weighting) {
        if (!team_sync<SOLO>(T)) return false;  // the exterior pass has read the images
        set_images<DT>(C, 1.f);
        if (!team_sync<SOLO>(T)) return false;
        phase_a_global<SOLO, DT>(C, T, A_ROWSUM, s_cnt, smem);
        if (tid == 0) *s_cnt = BNW;
        __syncthreads();
        phase_b<SOLO, DT>(C, T, B_COLSUM, s_cnt, smem + warp * WARP_STAGE);
    }
    if (!team_sync<SOLO>(T)) return false;
    set_images<DT>(C, 0.f);
    if (!team_sync<SOLO>(T)) return false;

    // ---- iterations
    float fista_t = 1.f;  // FISTA sequence t_{k-1} (reg 3)
    if (R.reg >= 3) fill_team(C, C.b.tau, nimg, 0.f);  // x^0 = 0
    for (int it = 0; it < R.iters; ++it) {
        // a team block works on its branch only (C.arow), as a member of that branch's blocks
        Team TA = T;
        TA.member = C.amember;
        TA.size = C.asize;
        if (C.stage == 0) {
            for (int row = 1; row >= 0; --row) {
                if (C.arow >= 0 && row != C.arow) continue;
                if (tid == 0) bulk_load(smem, row ? bufs.xa_base : bufs.xaT_base, row ? bytes_row : bytes_col, mbar);
                if (row == (C.arow >= 0 ? C.arow : 1) && R.reg == 1) dual_grad<DT>(C);  // reads xbar^k while the copy runs
                if (tid == 0) *s_cnt = BNW;
                if (!mbar_wait(mbar, parity & 1u, T.wait_ns, T.err)) return false;
                parity ^= 1u;
                __syncthreads();
                phase_a_branch<SOLO, DT>(C, TA, row, reinterpret_cast<TS*>(smem) + kPad, row ? C.lda : C.ldaT,
                                         A_SOLVE, s_cnt, smem + img_floats, dyn_smem_floats() - img_floats);
                __syncthreads();
            }
        } else if (C.stage == 1) {
            if (R.reg == 1) dual_grad<DT>(C);
            // a large team whose blocks would take more units than warps (the per-32-unit
            // schedule would stream the image more than once): by row band, the same bits.
            // The test is the same in every block of the team (the path adds a team barrier).
            if (!SOLO && C.b.part && C.arow >= 0 && R.na * C.nchunk > BNW * T.size) {
                if (!phase_a_rowband<SOLO, DT>(C, T, C.arow, C.arow ? bufs.xa_base : bufs.xaT_base,
                                               C.arow ? C.lda : C.ldaT, smem, mbar, parity))
                    return false;
            } else {
                for (int row = 1; row >= 0; --row) {
                    if (C.arow >= 0 && row != C.arow) continue;
                    if (!phase_a_banded<SOLO, DT>(C, TA, row, row ? bufs.xa_base : bufs.xaT_base,
                                                  row ? C.lda : C.ldaT, smem, mbar, parity))
                        return false;
                }
            }
        } else {
            if (R.reg == 1) dual_grad<DT>(C);
            phase_a_global<SOLO, DT>(C, T, A_SOLVE, s_cnt, smem);
        }
        if (!team_sync<SOLO>(T)) return false;  // u, v of this iteration complete
        if (R.reg >= 2) {  // x_s^k first (tiles stay with their block, so a block barrier suffices)
            if (tid == 0) *s_cnt = BNW;
            __syncthreads();
            phase_b<SOLO, DT>(C, T, B_XS, s_cnt, smem + warp * WARP_STAGE, it);
            __syncthreads();
        }
        if (tid == 0) *s_cnt = BNW;
        __syncthreads();
        phase_b<SOLO, DT>(C, T, B_SOLVE, s_cnt, smem + warp * WARP_STAGE);
        if (!team_sync<SOLO>(T)) return false;  // x, xbar complete (reg 3: z complete)
        if (R.reg == 3) {
            if (!fgp_prox_t<SOLO>(C, T)) return false;
            fista_update<DT>(C, fista_t);
            fista_t = 0.5f * (1.f + sqrtf(1.f + 4.f * fista_t * fista_t));
            if (!team_sync<SOLO>(T)) return false;
        } else if (R.reg == 4) {
            if (!haar_ista_step<SOLO, DT>(C, T)) return false;
        }
    }
    // ---- crop into the output buffer (x is kept in float for both solvers)
    for (int p = team_tid(C); p < (int)nimg; p += C.gthreads) {
        const int i = p / R.nx, j = p - i * R.nx;
        float v = R.reg == 2 ? C.b.vx[p] + disc_value(R, i, j)
                  : R.reg >= 3 ? C.b.tau[p] + disc_value(R, i, j) : C.b.x[p];
        if (R.crop) {
            const float dx = (float)j - R.cxl, dy = (float)i - R.cyl;
            if (dx * dx + dy * dy > R.r2) v = 0.f;
        }
        R.out[p] = v;
    }
    return true;
}

// Dispatch on the region's storage type.
template <bool SOLO>
__device__ __forceinline__ bool solve_region_dt(const BatchRoi& R, const RegionBufs& bufs, Team& T, float* smem,
                                                uint64_t* mbar, unsigned& parity, int* s_cnt) {
    if (R.dt == 1) return solve_region<SOLO, 1>(R, bufs, T, smem, mbar, parity, s_cnt);
    if (R.dt == 2) return solve_region<SOLO, 2>(R, bufs, T, smem, mbar, parity, s_cnt);
    return solve_region<SOLO, 0>(R, bufs, T, smem, mbar, parity, s_cnt);
}

}  // namespace rs
}  // namespace roi
