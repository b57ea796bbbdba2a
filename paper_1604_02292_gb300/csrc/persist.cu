// persist.cu -- one cooperative launch per local solve (boxes whose padded image fits
// in shared memory): all SIRT / Chambolle-Pock iterations run inside one kernel, with
// a grid-wide barrier between the two phases of an iteration.
//
// Iteration (paper Eq. sirtit / Eq. sirtbox for SIRT; Eq. priorsys with TV by
// Chambolle-Pock; the operators W_L, W_L^T of Sec. 2.1):
//   phase A  every block stages the whole padded image it projects (x for SIRT, xbar
//            for CP; rows or columns by the branch of its angles) into shared memory
//            with four TMA bulk copies (the rows of the four ray segments) and runs the
//            ray-driven forward W_L on its share of (angle, 32-ray) units, fusing
//            r = p' - W_L x  (SIRT)  or  u <- (u + sigma (W_L xbar - p'))/(1 + sigma/2)
//            (CP); for CP four warps first update the gradient dual
//            v <- proj_lambda(v + sigma_v grad xbar)  on the block's share of pixels
//            while the first copies are in flight;
//   barrier
//   phase B  every block takes 16 x 16 pixel tiles, stages the window bins the tile's
//            pixels reach for all angles, gathers W_L^T of r (or u) over all angles and
//            applies  x <- max(0, x + alpha (.))  (SIRT)  or
//            x+ = x - tau (W_L^T u - div v), xbar = 2 x+ - x  (CP),
//            writing the padded row and column copies the next phase A stages;
//   barrier.
//
// Inner loops run in fixed point, so they need no float-to-integer conversion (a
// quarter-rate instruction on this GPU): along a ray the interpolation coordinate is
// an integer column plus a Q.22 offset, re-anchored from float-float every 48 samples
// and stepped by round(slope 2^22) (drift <= 47 2^-23 < 6e-6 pixel, below the float ulp of
// a coordinate near 192); across a gather tile row the window coordinate is a Q.23 integer
// stepped by round(cos 2^23).  The fraction bits become a float by the exponent trick
// (one logic op and one add).
//
// The grid barrier polls a monotonic arrival counter with a time limit (one second by
// default, wall clock from %globaltimer): a block that waits longer sets the error flag
// and every block leaves at its next barrier; the host reports ROI_ETIMEOUT.  The TMA
// wait has the same limit.  Blocks are co-resident by construction (cooperative launch
// of at most one block per SM).  Data written by other blocks in the previous phase are
// read with ld.global.cg (L2) or by TMA, never through L1.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "check.cuh"
#include "dev_common.cuh"
#include "roi_internal.h"

namespace roi {

namespace {

constexpr int PT = 1024;                 // threads per block
constexpr int NWARP = PT / 32;
constexpr int RAYS = 32;                 // rays per unit (one warp-wide ray group)
constexpr int FSEG = 4;                  // segments per ray in phase A
constexpr int CHUNK_UNITS = 16;          // phase A units whose partials are held at once
constexpr int DG_WARPS = 4;              // warps that update the gradient dual while the others project
constexpr int SEGA = 48;                 // samples per float-float anchor
constexpr int MAXUNITS = 512;            // phase A units per block (checked by the host)
constexpr int NBUCKET = 512;             // cost classes of the phase A balancing sort
constexpr int ITEM_COST = 16;            // fixed cost of one (unit, segment) item, in samples
constexpr int MAXPRE = 2;                // phase B tiles per block with precomputed constants
constexpr int BT = 16;                   // phase B tile side
constexpr int BPIX = BT * BT;
constexpr int RUN = 8;                   // pixels per gather thread (along a tile row)
constexpr int RUNS = BPIX / RUN;         // 32 runs per tile
constexpr int BGROUPS = PT / RUNS;       // 32 angle groups
// tile pixels lie within 7.5 (|c| + |s|) <= 10.61 of the tile centre in window
// coordinates and the hat reaches one bin further: with kbase = floor(kappa_c) - 12
// every staged index touched is in [1, 24] < BSB
constexpr int BKOFF = 12;
constexpr int BSB = 26;
// operands fetched ahead of use: phase A [CHUNK_UNITS][u, p', weight][32]; phase B
// [x, step, vx(o), vx(o-1), vy(o), vy(o-nx)][BPIX]
constexpr int FIN = CHUNK_UNITS * 3 * 32 > 6 * BPIX ? CHUNK_UNITS * 3 * 32 : 6 * BPIX;

struct PArgs {
    const AngleRec* rec;
    int na, stride, nx, ny;
    int mode;               // 0 SIRT, 1 CP
    int iters;
    // padded images read by phase A: row layout [ny][lda], column layout [nx][ldaT];
    // *_base is the start of the buffer (row 0, column -2)
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
    unsigned* bar;          // [0] arrivals (monotonic within a launch)
    unsigned expect;        // participants: gridDim.x (+ absent ones when testing the time limit)
    int* err;
    unsigned long long wait_ns;  // time limit of one wait
    // phase A partition
    int nchunk;             // 32-ray chunks per angle
    int units;              // na * nchunk
    int region_floats;      // floats of the shared region (image / phase B staging)
    int pre_tiles;          // phase B tiles per block whose constants are precomputed (0: none)
};

struct PhaseBConst {
    int base;   // Q.23 window coordinate of tile pixel (0, 0), relative to kb
    int c, s;   // Q.23 steps per column / per row
    float iw;   // 1 / w
};

// Grid barrier on a monotonic arrival counter: barrier number n (1, 2, ...) is passed
// when the counter reaches n * expect.  Thread 0 of each block adds one with release
// semantics (ordering the block's writes, gathered by the block barrier before it) and
// polls the counter with acquire loads; every 256 polls it checks the time limit and the
// error flag.  Returns 0 (in every thread of the block) when
// this or another block gave up; the caller then returns.
__device__ __forceinline__ int grid_sync(const PArgs& A, int* s_flag, unsigned& nbar) {
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        ++nbar;
        const unsigned target = nbar * A.expect;
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(A.bar) : "memory");
        unsigned long long t0 = 0;
        for (unsigned polls = 1;; ++polls) {
            unsigned v;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(A.bar) : "memory");
            if ((int)(v - target) >= 0) break;
            if ((polls & 255u) == 0) {
                const unsigned long long now = global_ns();
                if (t0 == 0) {
                    t0 = now;
                } else if (now - t0 > A.wait_ns) {
                    atomicExch(A.err, 1);
                    ok = 0;
                    break;
                }
                if (*(volatile int*)A.err) {
                    ok = 0;
                    break;
                }
            }
        }
        *s_flag = ok;
    }
    __syncthreads();
    return *s_flag;
}

// Partial Joseph sum of ray k of angle r over the samples of segment `seg`, image in
// shared memory (element (0,0) at img, row stride ld).  Samples whose exact minor
// coordinate q lies in [-1.5, Mm + 0.5] are visited (range in float, error ~1e-4 <<
// 0.5), so the taps stay in [-2, Mm + 1], inside the padded row; samples outside the
// range have both taps outside [0, Mm) and contribute 0.
// Samples [mlo, mhi) of ray k whose minor coordinate lies in [-1.5, Mm + 0.5] (the others
// contribute 0); returns the ray's coordinate A_k at the major-axis centre.
__device__ __forceinline__ ff ray_range(const AngleRec& r, int k, int M, int Mm, int& mlo, int& mhi) {
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

__device__ __forceinline__ ff ray_segment(const AngleRec& r, int k, int seg, int seg_len, int M, int Mm,
                                          const float* img, int ld) {
    float sum = 0.f, cmp = 0.f;
    const float halfM = 0.5f * (float)(M - 1);
    int mlo, mhi;
    const ff Ak = ray_range(r, k, M, Mm, mlo, mhi);
    const int s0 = seg * seg_len;
    mlo = max(mlo, s0);
    mhi = min(mhi, min(s0 + seg_len, M));
    const int step = r.slope_q22;
    for (int m0 = mlo; m0 < mhi; m0 += SEGA) {
        int j0;
        int q = split_fixed22(ff_add(Ak, ff_mul_f((float)m0 - halfM, r.slope)), j0);  // sample m0
        const int mend = min(m0 + SEGA, mhi);
        const int jlo = -kPad - j0, jhi = ld - 1 - kPad - j0;  // taps j, j + 1 inside the padded row
        // sum of v0 + f (v1 - v0) with f = mf 2^-22: the two parts are summed separately,
        // two samples per packed (f32x2) operation (even and odd samples in the two lanes
        // of the pair, added at the end)
        float2 S0 = make_float2(0.f, 0.f), S1 = make_float2(0.f, 0.f);
        const float2 m1 = make_float2(-1.f, -1.f), e23 = make_float2(-8388608.0f, -8388608.0f);
        const float* rp = img + m0 * ld + j0;
        int m = m0;
#pragma unroll 2
        for (; m + 1 < mend; m += 2, rp += 2 * ld, q += 2 * step) {
            const int q1 = q + step;
            const int ja = chk(q >> 22, jlo, jhi, CHK_PERSIST_RAY), jb = chk(q1 >> 22, jlo, jhi, CHK_PERSIST_RAY);
            const float2 bits = make_float2(__uint_as_float(0x4B000000u | ((unsigned)q & 0x3FFFFFu)),
                                            __uint_as_float(0x4B000000u | ((unsigned)q1 & 0x3FFFFFu)));
            const float2 mf = __fadd2_rn(bits, e23);
            const float2 v0 = make_float2(rp[ja], rp[ld + jb]);
            const float2 v1 = make_float2(rp[ja + 1], rp[ld + jb + 1]);
            S0 = __fadd2_rn(S0, v0);
            S1 = __ffma2_rn(mf, __ffma2_rn(v0, m1, v1), S1);  // v1 - v0 exactly as a subtraction
        }
        if (m < mend) {
            const int j = chk(q >> 22, jlo, jhi, CHK_PERSIST_RAY);
            const float mf = frac_int<22>(q);
            const float v0 = rp[j], v1 = rp[j + 1];
            S0.x += v0;
            S1.x = fmaf(mf, v1 - v0, S1.x);
        }
        neu_add(sum, cmp, fmaf(S1.x + S1.y, 2.384185791015625e-07f, S0.x + S0.y));  // s0 + s1 2^-22
    }
    return two_sum(sum, cmp);
}

// Phase B constants of tile t for angle a: kappa at the tile centre (xi_t c + eta_t s -
// phi) in float-float, kbase = floor - BKOFF, and the Q.23 coordinate of tile pixel (0, 0)
// (centre - 7.5 c + 7.5 s) relative to kbase.
__device__ __forceinline__ void tile_consts(const PArgs& A, int t, int tiles_x, int a, PhaseBConst* bcp, int* kbp,
                                            int* wdp) {
    const int tile_x0 = (t % tiles_x) * BT, tile_y0 = (t / tiles_x) * BT;
    const float xi_t = (float)tile_x0 + 0.5f * (BT - 1) - 0.5f * (float)(A.nx - 1);
    const float eta_t = 0.5f * (float)(A.ny - 1) - ((float)tile_y0 + 0.5f * (BT - 1));
    const AngleRec& r = A.rec[a];
    ff kt = ff_add(ff_mul_f(xi_t, r.c), ff_mul_f(eta_t, r.s));
    kt = ff_add(kt, ff{-r.phi.hi, -r.phi.lo});
    const int kbase = (int)floorf(kt.hi) - BKOFF;
    kt = ff_add(kt, ff{-(float)kbase, 0.f});
    kt = ff_add(kt, ff_mul_f(-0.5f * (BT - 1), r.c));
    kt = ff_add(kt, ff_mul_f(0.5f * (BT - 1), r.s));
    PhaseBConst q;
    q.base = to_fixed<23>(kt);
    q.c = r.c_q23;
    q.s = r.s_q23;
    q.iw = r.inv_w;
    *bcp = q;
    *kbp = kbase;
    *wdp = r.width;
}

// Warp ul < nu starts asynchronous copies of the finishing operands of unit cu + ul (the
// old dual for CP, the data p', the weight) into fin[ul] (whole window rows, in bounds of
// the [na][stride] arrays); the same thread waits for them before the finish, and the
// copies overlap the projection.
__device__ __forceinline__ void prefetch_finish(const PArgs& A, const int* units, int cu, int nu, int warp, int lane,
                                                float* fin) {
    if (warp >= nu) return;
    const int unit = units[cu + warp];
    const int a = unit / A.nchunk;
    const int k = (unit - a * A.nchunk) * RAYS + lane;
    if (k >= A.stride) return;
    const size_t o = (size_t)a * A.stride + k;
    float* f = fin + warp * 96 + lane;
    if (A.mode == 1) cp_async4(f, A.u + o);
    cp_async4(f + 32, A.pp + o);
    if (A.R) cp_async4(f + 64, A.R + o);
}

__global__ void __launch_bounds__(PT, 1) k_persist(PArgs A) {
    extern __shared__ float4 smem4[];
    float* smem = reinterpret_cast<float*>(smem4);
    float* img = smem;                              // phase A image
    float* red_s = smem + A.region_floats;          // [CHUNK_UNITS][FSEG][32] phase A partials
    float* red_c = red_s + CHUNK_UNITS * FSEG * 32;
    float* fin = red_c + CHUNK_UNITS * FSEG * 32;   // [FIN] operands fetched ahead of use
    PhaseBConst* pbc = reinterpret_cast<PhaseBConst*>(fin + FIN);  // [pre_tiles][na]
    int* pkb = reinterpret_cast<int*>(pbc + A.pre_tiles * A.na);
    int* pwd = pkb + A.pre_tiles * A.na;
    __shared__ int s_flag;
    __shared__ int s_nunits, s_row, s_gsize, s_next, s_terr;
    __shared__ int s_units[MAXUNITS];               // this block's phase A units (angle * nchunk + chunk)
    __shared__ __align__(8) uint64_t s_mbar[FSEG];  // one per ray segment's rows
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int G = gridDim.x, b = blockIdx.x;
    const int nx = A.nx, ny = A.ny;
    const int npix = nx * ny;
    const int p0 = (int)((long long)npix * b / G), p1 = (int)((long long)npix * (b + 1) / G);
    const int tiles_x = (nx + BT - 1) / BT, tiles = tiles_x * ((ny + BT - 1) / BT);
    const int t0 = (int)((long long)tiles * b / G), t1 = (int)((long long)tiles * (b + 1) / G);
    float* xa = A.xa_base + kPad;
    float* xaT = A.xaT_base + kPad;
    // phase B shared layout: stage[na][BSB] | consts[na] | kb[na] | width[na] | part[BGROUPS][BPIX]
    float* stage = smem;
    PhaseBConst* bc = reinterpret_cast<PhaseBConst*>(smem + ((A.na * BSB + 3) & ~3));
    int* kb = reinterpret_cast<int*>(bc + A.na);
    int* wdt = kb + A.na;
    float* bpart = reinterpret_cast<float*>(wdt + A.na);

    // prologue 1: phase A work.  The blocks are split between the two branches in
    // proportion to their units, so each block stages one orientation.  Within a branch the
    // units are sorted by their cost (samples of the longest ray in each segment plus a fixed
    // cost per item) and dealt in snake order (0 .. g-1, g-1 .. 0, ...), which balances the
    // blocks to within a fraction of a unit; every block computes the same deal.
    int* rank_angle = reinterpret_cast<int*>(smem);  // scratch in the (not yet used) region: [na]
    if (tid == 0) {
        int nrow = 0, ncol = 0;
        for (int a = 0; a < A.na; ++a) (A.rec[a].row ? nrow : ncol)++;
        const long ur = (long)nrow * A.nchunk, uc = (long)ncol * A.nchunk;
        int gr = (int)((ur * G + (ur + uc) / 2) / max(ur + uc, 1L));
        if (ur > 0 && gr < 1) gr = 1;
        if (uc > 0 && gr > G - 1) gr = G - 1;
        if (uc == 0) gr = G;
        if (ur == 0) gr = 0;
        const int mine = b < gr;  // 1: this block takes row-branch units
        int nb = 0;
        for (int a = 0; a < A.na; ++a)
            if (A.rec[a].row == mine) rank_angle[nb++] = a;
        s_nunits = nb;  // angles of the branch, for now
        s_row = mine;
        s_gsize = mine ? gr : G - gr;
        s_next = 0;
        s_terr = 0;
        for (int q = 0; q < FSEG; ++q) mbar_init(&s_mbar[q], 1);
    }
    __syncthreads();
    {
        const int mine = s_row, gsize = s_gsize, bi = mine ? b : b - (G - gsize);
        const int U = s_nunits * A.nchunk;  // units of the branch
        int* ucost = rank_angle + A.na;      // [U]
        int* uorder = ucost + U;             // [U]
        int* ubucket = uorder + U;           // [NBUCKET]
        const int M = mine ? ny : nx, Mm = mine ? nx : ny;
        const int seg_len = ((M + FSEG - 1) / FSEG + SEGA - 1) / SEGA * SEGA;
        for (int j = warp; j < U; j += NWARP) {  // cost of unit j: one warp, a lane per ray
            const int a = rank_angle[j / A.nchunk];
            const int k = (j % A.nchunk) * RAYS + lane;
            const AngleRec& r = A.rec[a];
            int mlo = 0, mhi = 0;
            if (k < r.width) ray_range(r, k, M, Mm, mlo, mhi);
            int cost = 0;
            for (int sg = 0; sg < FSEG; ++sg) {
                const int s0 = sg * seg_len;
                const int cnt = max(0, min(mhi, min(s0 + seg_len, M)) - max(mlo, s0));
                cost += (int)__reduce_max_sync(0xffffffffu, (unsigned)cnt) + ITEM_COST;
            }
            if (lane == 0) ucost[j] = min(cost, NBUCKET - 1);
        }
        for (int i = tid; i < NBUCKET; i += PT) ubucket[i] = 0;
        __syncthreads();
        if (warp == 0) {  // stable counting sort by decreasing cost
            for (int j = lane; j < U; j += 32) atomicAdd(&ubucket[ucost[j]], 1);
            __syncwarp();
            if (lane == 0) {
                int run = 0;
                for (int c = NBUCKET - 1; c >= 0; --c) {
                    const int h = ubucket[c];
                    ubucket[c] = run;
                    run += h;
                }
            }
            __syncwarp();
            for (int j0 = 0; j0 < U; j0 += 32) {  // 32 units at a time, in unit order
                const int j = j0 + lane;
                const int c = j < U ? ucost[j] : -1 - lane;  // distinct keys for idle lanes
                const unsigned peers = __match_any_sync(0xffffffffu, c);
                const int rank = __popc(peers & ((1u << lane) - 1u));
                const int base = j < U ? ubucket[c] : 0;
                if (j < U) uorder[base + rank] = j;
                __syncwarp();
                if (j < U && rank == __popc(peers) - 1) ubucket[c] = base + rank + 1;
                __syncwarp();
            }
        }
        __syncthreads();
        if (tid == 0) {  // this block's units: sorted positions bi and 2 g - 1 - bi of every 2 g
            int nu = 0;
            for (int r0 = 0; r0 < U; r0 += 2 * gsize) {
                const int rs[2] = {r0 + bi, r0 + 2 * gsize - 1 - bi};
                for (int h = 0; h < 2; ++h) {
                    const int r = rs[h];
                    if (r >= U) continue;
                    if (nu == MAXUNITS) {  // the host sizes MAXUNITS; never silently drop work
                        atomicExch(A.err, 1);
                        break;
                    }
                    const int j = uorder[r];
                    s_units[nu++] = rank_angle[j / A.nchunk] * A.nchunk + j % A.nchunk;
                }
            }
            s_nunits = nu;
        }
        __syncthreads();
    }
    const int nunits = s_nunits, my_row = s_row;
    // prologue 2: phase B constants of this block's tiles (they do not change)
    const bool pre = A.pre_tiles > 0 && (t1 - t0) <= A.pre_tiles;
    if (pre) {
        for (int e = tid; e < (t1 - t0) * A.na; e += PT) {
            const int tt = e / A.na, a = e - tt * A.na;
            tile_consts(A, t0 + tt, tiles_x, a, pbc + e, pkb + e, pwd + e);
        }
    }
    __syncthreads();
    unsigned parity = 0;
    unsigned nbar = 0;

    for (int it = 0; it < A.iters; ++it) {
        // ------------------------------------------------------------ phase A
        const int M = my_row ? ny : nx, Mm = my_row ? nx : ny, ld = my_row ? A.lda : A.ldaT;
        const int seg_len = ((M + FSEG - 1) / FSEG + SEGA - 1) / SEGA * SEGA;
        if (nunits > 0 && tid == PT - 32) {
            // one copy per ray segment (rows [q seg_len, (q + 1) seg_len) of the image), so
            // warps start on the first segments while the rest is in flight; issued by the
            // last warp, which projects last (it first updates the gradient dual for CP)
            const float* src = my_row ? A.xa_base : A.xaT_base;
            asm volatile("fence.proxy.async;" ::: "memory");
            for (int q = 0; q < FSEG; ++q) {
                const int r0 = min(q * seg_len, M), r1 = min(r0 + seg_len, M);
                if (r1 > r0)
                    bulk_copy(img + (size_t)r0 * ld, src + (size_t)r0 * ld, sizeof(float) * (r1 - r0) * ld, &s_mbar[q]);
                else
                    mbar_arrive(&s_mbar[q]);
            }
        }
        if (nunits > 0) prefetch_finish(A, s_units, 0, min(CHUNK_UNITS, nunits), warp, lane, fin);
        if (A.mode == 1) {
            // gradient dual on this block's pixels (reads xbar^k) by the last DG_WARPS warps
            // (all warps in a block without rays); they join the projection afterwards
            const int dgw = nunits > 0 ? DG_WARPS : NWARP;
            if (warp >= NWARP - dgw) {
                const float sv = A.sigma_v_dev ? __ldg(A.sigma_v_dev) : A.sigma_v;
                for (int p = p0 + tid - (NWARP - dgw) * 32; p < p1; p += dgw * 32) {
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
        }
        {
            // Items (unit, segment), segment-major, are taken dynamically by warps from a
            // shared counter; each item's partial goes to its own slot, and the slots of a
            // ray are added in segment order, so the result does not depend on which warp
            // took what.
            unsigned ready = 0;  // segments whose rows this warp has seen arrive
            for (int cu = 0; cu < nunits; cu += CHUNK_UNITS) {
                const int nu = min(CHUNK_UNITS, nunits - cu), nitems = nu * FSEG;
                for (;;) {
                    int item = 0;
                    if (lane == 0) item = atomicAdd(&s_next, 1);
                    item = __shfl_sync(0xffffffffu, item, 0);
                    if (item >= nitems) break;
                    const int seg = item / nu, ul = item - seg * nu;
                    if (!((ready >> seg) & 1u)) {
                        if (!mbar_wait(&s_mbar[seg], parity, A.wait_ns, A.err)) s_terr = 1;
                        ready |= 1u << seg;
                    }
                    const int unit = s_units[cu + ul];
                    const int a = unit / A.nchunk;
                    const int k = (unit - a * A.nchunk) * RAYS + lane;
                    const AngleRec& r = A.rec[a];
                    ff part = {0.f, 0.f};
                    if (k < r.width) part = ray_segment(r, k, seg, seg_len, M, Mm, img + kPad, ld);
                    const int slot = (ul * FSEG + seg) * 32 + lane;
                    red_s[slot] = part.hi;
                    red_c[slot] = part.lo;
                }
                __syncthreads();
                if (tid == 0) s_next = 0;
                if (warp < nu) {  // finish ray (unit cu + warp, lane)
                    const int ul = warp;
                    cp_async_wait_all();
                    const int unit = s_units[cu + ul];
                    const int a = unit / A.nchunk;
                    const int k = (unit - a * A.nchunk) * RAYS + lane;
                    const AngleRec& r = A.rec[a];
                    if (k < r.width) {
                        ff tot = {red_s[(ul * FSEG) * 32 + lane], red_c[(ul * FSEG) * 32 + lane]};
                        for (int s = 1; s < FSEG; ++s) {
                            const ff o = {red_s[(ul * FSEG + s) * 32 + lane], red_c[(ul * FSEG + s) * 32 + lane]};
                            tot = ff_add(tot, o);
                        }
                        tot = ff_mul_f(r.inv_w, tot);
                        const float acc = tot.hi + tot.lo;
                        const size_t o = (size_t)a * A.stride + k;
                        const float* f = fin + ul * 96 + lane;
                        if (A.mode == 0) {
                            float res = f[32] - acc;
                            if (A.R) res *= f[64];
                            A.u[o] = res;
                        } else {
                            const float sig = A.R ? f[64] : A.sig_scalar;
                            A.u[o] = (f[0] + sig * (acc - f[32])) / (1.f + 0.5f * sig);
                        }
                    }
                }
                __syncthreads();
                if (cu + CHUNK_UNITS < nunits)
                    prefetch_finish(A, s_units, cu + CHUNK_UNITS, min(CHUNK_UNITS, nunits - cu - CHUNK_UNITS), warp,
                                    lane, fin);
            }
            if (nunits > 0) parity ^= 1u;
        }
        if (s_terr) return;  // a copy timed out (flag set); read after a block barrier
        if (!grid_sync(A, &s_flag, nbar)) return;

        // ------------------------------------------------------------ phase B
        for (int t = t0; t < t1; ++t) {
            const int tile_x0 = (t % tiles_x) * BT, tile_y0 = (t / tiles_x) * BT;
            const PhaseBConst* tbc = bc;
            const int* tkb = kb;
            const int* twd = wdt;
            __syncthreads();
            if (tid < BPIX) {
                // operands of this pixel's update (x, step, the four v terms of div v, zero
                // outside the box), copied while the window is gathered (the thread that
                // updates pixel `tid` below is the one that waits for them)
                const int prun = tid % RUNS, pp = tid / RUNS;  // partial layout [group][p][run]
                const int gi = tile_y0 + (prun >> 1), gj = tile_x0 + (prun & 1) * RUN + pp;
                if (gi < ny && gj < nx) {
                    const int o = gi * nx + gj;
                    if (A.mode == 0) {
                        cp_async4(fin + tid, xa + gi * A.lda + gj);
                    } else {
                        cp_async4(fin + tid, A.x + o);
                        cp_async4(fin + 2 * BPIX + tid, A.vx + o, gj < nx - 1);
                        cp_async4(fin + 3 * BPIX + tid, A.vx + o - (gj > 0), gj > 0);
                        cp_async4(fin + 4 * BPIX + tid, A.vy + o, gi < ny - 1);
                        cp_async4(fin + 5 * BPIX + tid, A.vy + o - (gi > 0 ? nx : 0), gi > 0);
                    }
                    if (A.C) cp_async4(fin + BPIX + tid, A.C + o);
                }
            }
            if (pre) {
                tbc = pbc + (t - t0) * A.na;
                tkb = pkb + (t - t0) * A.na;
                twd = pwd + (t - t0) * A.na;
            } else {
                for (int a = tid; a < A.na; a += PT) tile_consts(A, t, tiles_x, a, bc + a, kb + a, wdt + a);
                __syncthreads();
            }
            {
                // thread = (run of 8 pixels along a tile row, group of angles); a warp is one
                // angle group and stages that group's bins itself (no block-wide wait)
                const int run = tid % RUNS, grp = tid / RUNS;
                const int li = run >> 1, lj0 = (run & 1) * RUN;
                const int a_lo = (int)((long long)A.na * grp / BGROUPS);
                const int a_hi = (int)((long long)A.na * (grp + 1) / BGROUPS);
                {
                    const int e_lo = a_lo * BSB, e_hi = a_hi * BSB;
                    constexpr int BATCH = 8;
                    // bins are staged times 1/w of their angle (the hat weights below are then
                    // max(0, 1 - d/w), one saturating FMA each)
                    for (int e0 = e_lo + lane; e0 < e_hi; e0 += 32 * BATCH) {
                        float v[BATCH], iw[BATCH];
#pragma unroll
                        for (int q = 0; q < BATCH; ++q) {
                            const int e = e0 + q * 32;
                            v[q] = 0.f;
                            iw[q] = 0.f;
                            if (e < e_hi) {
                                const int a = e / BSB, kk = tkb[a] + (e - a * BSB);
                                iw[q] = tbc[a].iw;
                                if (kk >= 0 && kk < twd[a]) v[q] = __ldcg(A.u + (size_t)a * A.stride + kk);
                            }
                        }
#pragma unroll
                        for (int q = 0; q < BATCH; ++q)
                            if (e0 + q * 32 < e_hi) stage[e0 + q * 32] = v[q] * iw[q];
                    }
                    __syncwarp();
                }
                // two pixels of the run per packed (f32x2) operation: the same fused
                // multiply-adds as one pixel at a time, half the instructions
                float2 acc[RUN / 2];
#pragma unroll
                for (int p = 0; p < RUN / 2; ++p) acc[p] = make_float2(0.f, 0.f);
                for (int a = a_lo; a < a_hi; ++a) {
                    const PhaseBConst q = tbc[a];
                    // weights max(0, 1 - d/w) of the two bins at distances f and 1 - f,
                    // f = mf 2^-23 (the staged bins carry the 1/w)
                    const float iws = q.iw * 1.1920928955078125e-07f, niws = -iws, omiw = 1.f - q.iw;
                    int K = q.base + lj0 * q.c - li * q.s;
                    const float* srow = stage + a * BSB;
#pragma unroll
                    for (int p = 0; p < RUN / 2; ++p) {
                        const int K1 = K + q.c;
                        const int kl0 = chk(K >> 23, 0, BSB - 1, CHK_PERSIST_GATHER);
                        const int kl1 = chk(K1 >> 23, 0, BSB - 1, CHK_PERSIST_GATHER);
                        const float2 bits = make_float2(__uint_as_float(0x4B000000u | ((unsigned)K & 0x7FFFFFu)),
                                                        __uint_as_float(0x4B000000u | ((unsigned)K1 & 0x7FFFFFu)));
                        const float2 mf = __fadd2_rn(bits, make_float2(-8388608.0f, -8388608.0f));
                        const float2 w0 = make_float2(fma_sat(mf.x, niws, 1.f), fma_sat(mf.y, niws, 1.f));
                        const float2 w1 = make_float2(fma_sat(mf.x, iws, omiw), fma_sat(mf.y, iws, omiw));
                        const float2 s0 = make_float2(srow[kl0], srow[kl1]);
                        const float2 s1 = make_float2(srow[kl0 + 1], srow[kl1 + 1]);
                        acc[p] = __ffma2_rn(w0, s0, __ffma2_rn(w1, s1, acc[p]));
                        K = K1 + q.c;
                    }
                }
                // partials as [group][p][run]: consecutive lanes store consecutive words
#pragma unroll
                for (int p = 0; p < RUN / 2; ++p) {
                    bpart[grp * BPIX + (2 * p) * RUNS + run] = acc[p].x;
                    bpart[grp * BPIX + (2 * p + 1) * RUNS + run] = acc[p].y;
                }
            }
            // the 32 angle-group partials of each pixel: four quarters of 8 groups summed by
            // all threads, then the quarters by one thread per pixel, which applies the update
            const int slot = tid & (BPIX - 1), quarter = tid >> 8;
            const int prun = slot % RUNS, pp = slot / RUNS;  // partial layout [group][p][run]
            const int li = prun >> 1, lj = (prun & 1) * RUN + pp;
            const int gi = tile_y0 + li, gj = tile_x0 + lj;
            const bool upd = quarter == 0 && gi < ny && gj < nx;
            const int o = gi * nx + gj;
            __syncthreads();
            {
                const float* src = bpart + (quarter * (BGROUPS / 4)) * BPIX + slot;
                float s = src[0], c = 0.f;
#pragma unroll
                for (int g = 1; g < BGROUPS / 4; ++g) neu_add(s, c, src[g * BPIX]);
                red_s[quarter * BPIX + slot] = s;
                red_c[quarter * BPIX + slot] = c;
            }
            __syncthreads();
            if (upd) {
                float s = red_s[slot], c = red_c[slot];
#pragma unroll
                for (int q = 1; q < 4; ++q) {
                    neu_add(s, c, red_s[q * BPIX + slot]);
                    c += red_c[q * BPIX + slot];
                }
                const float acc = s + c;
                cp_async_wait_all();
                const float xo = fin[slot];
                const float cw = A.C ? fin[BPIX + slot] : A.step_scalar;
                if (A.mode == 0) {
                    float xn = fmaf(cw, acc, xo);
                    if (A.nonneg) xn = fmaxf(xn, 0.f);
                    xa[gi * A.lda + gj] = xn;
                    xaT[gj * A.ldaT + gi] = xn;
                } else {
                    // div v with the terms outside the box zero (copies zero-filled)
                    const float dv = fin[2 * BPIX + slot] - fin[3 * BPIX + slot] + fin[4 * BPIX + slot] -
                                     fin[5 * BPIX + slot];
                    const float xn = xo - cw * (acc - dv);
                    A.x[o] = xn;
                    const float xb = 2.f * xn - xo;
                    xa[gi * A.lda + gj] = xb;
                    xaT[gj * A.ldaT + gi] = xb;
                }
            }
        }
        if (!grid_sync(A, &s_flag, nbar)) return;
    }
}

size_t region_floats(int na, int nx, int ny) {
    const size_t img = std::max((size_t)ny * padded_ld(nx), (size_t)nx * padded_ld(ny));
    const size_t stageB = (size_t)((na * BSB + 3) & ~3) + 4 * (size_t)na + 2 * (size_t)na + (size_t)BGROUPS * BPIX;
    return (std::max(img, stageB) + 3) & ~(size_t)3;
}

}  // namespace

// Tiles per block of phase B and whether their constants fit the precomputed area.
static int tiles_per_block(int nx, int ny, int blocks) {
    const int tiles = ((nx + BT - 1) / BT) * ((ny + BT - 1) / BT);
    return (tiles + blocks - 1) / std::max(blocks, 1);
}

static int pre_tiles(int nx, int ny, int blocks) {
    const int tpb = tiles_per_block(nx, ny, blocks);
    return tpb <= MAXPRE ? tpb : 0;
}

size_t persist_smem_bytes(int na, int nx, int ny, int blocks) {
    const size_t pre = (size_t)pre_tiles(nx, ny, blocks) * na * (sizeof(PhaseBConst) + 2 * sizeof(int));
    return sizeof(float) * (region_floats(na, nx, ny) + 2 * CHUNK_UNITS * FSEG * 32 + FIN) + pre;
}

// Phase A units per block: each branch group gets at least one block per
// units / (total units / blocks), rounded; bound it generously.
static bool units_fit(int na, int stride, int blocks, int nx, int ny) {
    const long units = (long)na * ((stride + RAYS - 1) / RAYS);
    // the balancing sort's scratch (angle list, costs, order, buckets) lives in the region
    const bool scratch = na + 2 * units + NBUCKET <= (long)region_floats(na, nx, ny);
    return scratch && (units + blocks - 1) / blocks * 2 + 2 <= MAXUNITS;
}

cudaError_t launch_persist(const PersistLaunch& L, cudaStream_t st) {
    if (!units_fit(L.na, L.stride, L.blocks, L.nx, L.ny)) return cudaErrorInvalidConfiguration;
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
    A.region_floats = (int)region_floats(L.na, L.nx, L.ny);
    A.pre_tiles = pre_tiles(L.nx, L.ny, L.blocks);
    const size_t smem = persist_smem_bytes(L.na, L.nx, L.ny, L.blocks);
    cudaError_t e = cudaFuncSetAttribute(k_persist, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(L.bar, 0, 2 * sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    void* args[] = {&A};
    count_launches(1);
    return cudaLaunchCooperativeKernel((const void*)k_persist, dim3(L.blocks), dim3(PT), args, smem, st);
}

ROI_CHECK_TU(persist)

int persist_max_blocks(int na, int nx, int ny, int stride, int device) {
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 0;
    int optin = 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess) return 0;
    const size_t smem = persist_smem_bytes(na, nx, ny, sms);
    if (smem > (size_t)optin) return 0;
    if (cudaFuncSetAttribute(k_persist, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_persist, PT, smem) != cudaSuccess) return 0;
    const int blocks = std::min(per_sm, 1) * sms;
    return units_fit(na, stride, blocks, nx, ny) ? blocks : 0;
}

}  // namespace roi
