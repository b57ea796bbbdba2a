// filterconv_tc.cu -- the filtered sinograms C_{u_k} p_d of the paper's own method on the
// tensor cores (tcgen05.mma, kind::tf32, accumulators in tensor memory).
//
// Alg. method uses, in iteration k, the disc-subtracted sinogram filtered by u_k (Sec. 3.1,
// Eq. sirtapp; Sec. 3.3 computes these rows once per sinogram).  Per angle a the n filtered
// rows are one contraction over the 2 N_d - 1 taps t:
//     Cp[k][a][d] = sum_t u[k][a][t] p[a][d + N_d - 1 - t],
// i.e. the matrix product D[d][k] = sum_t P[d][t] U[k][t] with P the Toeplitz matrix of the
// sinogram row (M = 128 output bins per tile, one TMEM lane each) and U the filter bank
// (N = up to 256 filters, one TMEM column each).  The taps are taken 8 at a time, the K of
// one tf32 MMA.  Both operands are read from shared memory through descriptors of the
// K-major layout without swizzle: core matrices of 8 rows x 16 bytes, rows 16 bytes apart,
// 8-row groups 128 bytes apart (SBO), the two 4-tap halves of a row LBO bytes apart.
//  * The sinogram row is expanded per work item into Y[s][t2] = p[s - t2] (t2 < 8).  The P
//    tile of tap group t1 is then Y's 128 rows from s = d0 + N_d - 1 - 8 t1: the next tap
//    group is the same descriptor moved back by 8 rows, nothing is copied.
//  * The filter bank is packed once per filter set (launch_filter_pack_tc) into the same
//    core-matrix order, 16 bytes per (filter, 4 taps), and streamed through a ring of stages
//    by bulk copies (one thread), consumed by the MMAs (another thread).
// Float32 accuracy from tf32 products (the split-operand scheme of Markidis et al. 2018 in
// its tf32 form): each operand x is stored as its tf32 head hi (low 13 mantissa bits
// cleared) and the tf32 head lo of the remainder x - hi; hi*hi + hi*lo + lo*hi are
// accumulated in fp32 in tensor memory (the omitted lo*lo and the truncation of lo are
// about 2^-20 of a term).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "check.cuh"
#include "dev_common.cuh"
#include "roi_internal.h"

namespace roi {

namespace {

constexpr int TC_THREADS = 192;  // warps 0-3: epilogue (TMEM lanes 0-127); 4: bulk copies; 5: MMA issue
constexpr int TC_M = 128;        // output bins per tile
constexpr int TC_TILES = 2;      // tiles per work item, at TMEM columns 0 and 256
constexpr int TC_COLS = 512;     // TMEM columns allocated
constexpr int TC_YPAD = 128;     // zero rows of Y below s = 0
constexpr int TC_MAX_STAGES = 6;
constexpr int TC_NB_MAX = 256;   // filters per block (N of one MMA)
constexpr size_t TC_SMEM_MAX = 227 * 1024 - 1024;  // dynamic part; the static barriers stay below 1 KB
constexpr size_t TC_SMEM_RESERVE = 1024;  // alignment slack of the dynamic area

struct TcGeom {
    int kb_count;  // filter blocks
    int nb;        // filters per block (multiple of 16, <= 256), zero rows past n
    int t1n;       // tap groups of 8 (the last one zero-padded past 2 N_d - 1)
    int yr;        // rows of Y
    int passes;    // work items per (angle, filter block): 256 output bins each
    int S;         // tap groups per stage: 4 where two such stages fit, else 2
    int stages;
    size_t smem;
};

__host__ __device__ inline int round_up(int v, int m) { return (v + m - 1) / m * m; }

TcGeom tc_geom(int n, int nd) {
    TcGeom g{};
    g.kb_count = (n + TC_NB_MAX - 1) / TC_NB_MAX;
    g.nb = round_up((n + g.kb_count - 1) / g.kb_count, 16);
    g.t1n = (2 * nd - 1 + 7) / 8;
    g.yr = round_up(nd + 262, 8);
    g.passes = (nd + TC_TILES * TC_M - 1) / (TC_TILES * TC_M);
    const size_t ybytes = (size_t)64 * g.yr;
    const size_t room = TC_SMEM_MAX > ybytes + TC_SMEM_RESERVE ? TC_SMEM_MAX - ybytes - TC_SMEM_RESERVE : 0;
    for (const int S : {4, 2}) {  // fewer, longer stages cost fewer barrier round trips
        const size_t stage = (size_t)4 * S * g.nb * 16;
        g.S = S;
        g.stages = (int)std::min<size_t>(TC_MAX_STAGES, room / stage);
        g.smem = ybytes + (size_t)g.stages * stage + TC_SMEM_RESERVE;
        if (g.stages >= 2) break;
    }
    return g;
}

struct TcArgs {
    const float* ug;  // packed filter bank [a][kb][plane][t1][nb][4]
    const float* pd;  // [na][nd]
    float* cp;        // [n][na][nd]
    int n, na, nd;
    TcGeom g;
    int* err;
    unsigned long long wait_ns;
    unsigned test_extra_tx;  // testing only: bytes each stage waits for beyond those copied
};

__device__ __forceinline__ float tf32_head(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

// Shared-memory matrix descriptor: K-major, no swizzle, 8-row groups 128 bytes apart.
__device__ __forceinline__ uint64_t kmajor_desc(unsigned addr, unsigned lbo) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)(128u >> 4) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::tf32: fp32 accumulator, tf32 A and B, both K-major.
__device__ __forceinline__ uint32_t tf32_idesc(int m, int n) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(unsigned d, uint64_t a, uint64_t b, uint32_t idesc, int accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

// The barrier's next phase completes when every MMA issued so far by this thread has.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(unsigned taddr, float (&v)[16]) {
    unsigned r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// Arms the barrier for `bytes` in this phase (one arrival).
__device__ __forceinline__ void mbar_expect(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

// Bulk copy global -> shared counted against an armed barrier.
__device__ __forceinline__ void bulk_copy_tx(unsigned dst, const void* src, unsigned bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst), "l"(src),
        "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// The tap-group range [lo, hi] of output tile [d0, d0 + 128): tap t meets the tile when
// d0 <= t <= d0 + 127 + N_d - 1.
__device__ __forceinline__ void tile_taps(int d0, int nd, int t1n, int& lo, int& hi) {
    lo = d0 / 8;
    hi = min(t1n - 1, (d0 + TC_M - 1 + nd - 1) / 8);
}

__global__ void __launch_bounds__(TC_THREADS, 1) k_filter_conv_tc(TcArgs A) {
    extern __shared__ __align__(16) unsigned char tc_smem_raw[];
    __shared__ __align__(8) uint64_t full[TC_MAX_STAGES], empty[TC_MAX_STAGES], accb, drain;
    __shared__ unsigned s_tmem;
    __shared__ int s_abort, s_issued, s_consumed;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const TcGeom& g = A.g;
    const int nd = A.nd, NS = g.stages;
    // 1024-aligned dynamic area: Y (4 planes of yr rows x 16 B), then the stages
    unsigned char* base = tc_smem_raw + ((1024 - (smem_addr(tc_smem_raw) & 1023)) & 1023);
    float* Y = reinterpret_cast<float*>(base);
    const unsigned y_addr = smem_addr(base);
    const unsigned y_plane = (unsigned)g.yr * 16;
    const int S = g.S;
    const unsigned stage_bytes = 4u * S * g.nb * 16;
    const unsigned stage_plane = (unsigned)S * g.nb * 16;
    const unsigned st_addr = y_addr + 4 * y_plane;
    if (tid == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&accb, 1);
        mbar_init(&drain, 1);
        s_abort = 0;
        s_issued = 0;
        s_consumed = 0;
    }
    if (warp == 5) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&s_tmem)),
                     "r"(TC_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = s_tmem;
    const uint32_t idesc = tf32_idesc(TC_M, g.nb);
    const int items = A.na * g.kb_count * g.passes;
    int gc = 0;  // chunks issued (warp 4) or consumed (warp 5) so far, over all items
    int ic = 0;  // items done by this block
    for (int item = blockIdx.x; item < items; item += gridDim.x, ++ic) {
        const int pass = item % g.passes;
        const int kb = (item / g.passes) % g.kb_count;
        const int a = item / (g.passes * g.kb_count);
        const int d0 = pass * TC_TILES * TC_M;
        int lo[TC_TILES], hi[TC_TILES];
        bool on[TC_TILES];
        int t1a = 0x7fffffff, t1b = -1;
#pragma unroll
        for (int q = 0; q < TC_TILES; ++q) {
            on[q] = d0 + q * TC_M < nd;
            tile_taps(d0 + q * TC_M, nd, g.t1n, lo[q], hi[q]);
            if (on[q]) {
                t1a = min(t1a, lo[q]);
                t1b = max(t1b, hi[q]);
            }
        }
        const int nchunks = (t1b - t1a + S) / S;
        // ---- Y[plane = 2 hl + h][y][c] = head (hl = 0) / remainder (hl = 1) of p[y - 128 - 4h - c]
        const float* prow = A.pd + (size_t)a * nd;
        for (int idx = tid; idx < 2 * g.yr; idx += TC_THREADS) {
            const int h = idx >= g.yr ? 1 : 0;
            const int y = idx - h * g.yr;
            const int e0 = y - TC_YPAD - 4 * h;
            float vh[4], vl[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int e = e0 - c;
                const float v = (e >= 0 && e < nd) ? __ldg(prow + e) : 0.f;
                vh[c] = tf32_head(v);
                vl[c] = tf32_head(v - vh[c]);
            }
            reinterpret_cast<float4*>(Y)[(size_t)h * g.yr + y] = make_float4(vh[0], vh[1], vh[2], vh[3]);
            reinterpret_cast<float4*>(Y)[(size_t)(2 + h) * g.yr + y] = make_float4(vl[0], vl[1], vl[2], vl[3]);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // Y is read by the tensor cores
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (warp == 4) {
            if (lane == 0) {  // ---- bulk copies of the filter bank, tap groups t1a.., S per stage
                const float* ub = A.ug + (size_t)(a * g.kb_count + kb) * 4 * g.t1n * g.nb * 4;
                for (int c = 0; c < nchunks; ++c, ++gc) {
                    const int s = gc % NS;
                    if (gc >= NS && !mbar_wait(&empty[s], ((gc / NS) + 1) & 1, A.wait_ns, A.err)) {
                        s_abort = 1;
                        break;
                    }
                    const int t1c = t1a + c * S;
                    const int steps = min(S, t1b + 1 - t1c);
                    const unsigned piece = (unsigned)steps * g.nb * 16;
                    mbar_expect(&full[s], 4 * piece + A.test_extra_tx);
                    for (int pl = 0; pl < 4; ++pl)
                        bulk_copy_tx(st_addr + s * stage_bytes + pl * stage_plane,
                                     ub + ((size_t)pl * g.t1n + t1c) * g.nb * 4, piece, &full[s]);
                }
                s_issued = gc;
            }
        } else if (warp == 5) {
            if (lane == 0) {  // ---- MMAs: per tap group and tile, hi*hi + hi*lo + lo*hi
                bool ok = true;
                for (int c = 0; c < nchunks; ++c, ++gc) {
                    const int s = gc % NS;
                    if (!mbar_wait(&full[s], (gc / NS) & 1, A.wait_ns, A.err)) {
                        s_abort = 1;
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const unsigned sb = st_addr + s * stage_bytes;
                    for (int j = 0; j < S; ++j) {
                        const int t1 = t1a + c * S + j;
                        if (t1 > t1b) break;
                        const unsigned b_hi = sb + j * g.nb * 16, b_lo = b_hi + 2 * stage_plane;
                        const uint64_t dbh = kmajor_desc(b_hi, stage_plane), dbl = kmajor_desc(b_lo, stage_plane);
#pragma unroll
                        for (int q = 0; q < TC_TILES; ++q) {
                            if (!on[q] || t1 < lo[q] || t1 > hi[q]) continue;
                            // rows of Y from s = d0q + nd - 1 - 8 t1, i.e. y = s + 128
                            const int yrow = chk(d0 + q * TC_M + nd - 1 + TC_YPAD - 8 * t1, 0, g.yr - TC_M + 1,
                                                 CHK_FILTER_TC);
                            const unsigned a_hi = y_addr + (unsigned)yrow * 16, a_lo = a_hi + 2 * y_plane;
                            const uint64_t dah = kmajor_desc(a_hi, y_plane), dal = kmajor_desc(a_lo, y_plane);
                            const unsigned d = tmem + (unsigned)(q * 256);
                            mma_tf32(d, dah, dbh, idesc, t1 != lo[q]);
                            mma_tf32(d, dah, dbl, idesc, 1);
                            mma_tf32(d, dal, dbh, idesc, 1);
                        }
                    }
                    mma_commit(&empty[s]);  // the stage is free once these MMAs have read it
                }
                s_consumed = gc;
                if (ok) mma_commit(&accb);
            }
        } else {  // ---- epilogue: TMEM lane 32 warp + lane = output bin d0q + 32 warp + lane
            const bool got = mbar_wait(&accb, ic & 1, A.wait_ns, A.err);
            if (__all_sync(0xffffffffu, got)) {
                tc_fence_after();
#pragma unroll
                for (int q = 0; q < TC_TILES; ++q) {
                    if (!on[q]) continue;
                    const int d = d0 + q * TC_M + 32 * warp + lane;
                    for (int c0 = 0; c0 < g.nb; c0 += 16) {
                        float v[16];
                        tmem_ld16(tmem + ((unsigned)(32 * warp) << 16) + (unsigned)(q * 256 + c0), v);
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            const int k = kb * g.nb + c0 + j;
                            if (k < A.n && d < nd) A.cp[((size_t)k * A.na + a) * nd + d] = v[j];
                        }
                    }
                }
            } else if (lane == 0) {
                s_abort = 1;
            }
        }
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (s_abort) break;
    }
    // ---- after a time-out: no copy left writing shared memory, no MMA left running
    __syncthreads();
    if (warp == 4 && lane == 0) {
        for (int c = s_consumed; c < s_issued; ++c) mbar_wait(&full[c % NS], (c / NS) & 1, A.wait_ns, A.err);
    }
    if (warp == 5 && lane == 0) {
        mma_commit(&drain);
        mbar_wait(&drain, 0, A.wait_ns, A.err);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 5)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_COLS) : "memory");
}

// ug[a][kb][plane = 2 hl + h][t1][r][c] = head (hl = 0) / remainder (hl = 1) of
// u[kb nb + r][a][8 t1 + 4h + c]; zero past the n filters and the 2 N_d - 1 taps.
__global__ void k_filter_pack_tc(const float* __restrict__ u, float* __restrict__ ug, int n, int na, int nd,
                                 TcGeom g) {
    const int nd2 = 2 * nd - 1;
    const size_t per_ab = (size_t)2 * g.t1n * g.nb;  // (h, t1, r) units of one (a, kb)
    const size_t total = (size_t)na * g.kb_count * per_ab;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(i % g.nb);
        const int t1 = (int)((i / g.nb) % g.t1n);
        const int h = (int)((i / ((size_t)g.nb * g.t1n)) % 2);
        const size_t ab = i / per_ab;
        const int kb = (int)(ab % g.kb_count);
        const int a = (int)(ab / g.kb_count);
        const int k = kb * g.nb + r;
        float vh[4], vl[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int t = 8 * t1 + 4 * h + c;
            const float v = (k < n && t < nd2) ? u[((size_t)k * na + a) * nd2 + t] : 0.f;
            vh[c] = tf32_head(v);
            vl[c] = tf32_head(v - vh[c]);
        }
        const size_t row = (size_t)t1 * g.nb + r;
        float4* o = reinterpret_cast<float4*>(ug) + ab * 4 * (size_t)g.t1n * g.nb;
        o[(size_t)h * g.t1n * g.nb + row] = make_float4(vh[0], vh[1], vh[2], vh[3]);
        o[(size_t)(2 + h) * g.t1n * g.nb + row] = make_float4(vl[0], vl[1], vl[2], vl[3]);
    }
}

}  // namespace

bool filter_conv_tc_fits(int n, int nd) {
    if (n <= 0 || nd <= 0) return false;
    const TcGeom g = tc_geom(n, nd);
    return g.stages >= 2 && g.yr < 16384 && g.smem <= TC_SMEM_MAX;
}

size_t filter_pack_tc_floats(int n, int na, int nd) {
    const TcGeom g = tc_geom(n, nd);
    return (size_t)na * g.kb_count * 4 * g.t1n * g.nb * 4;
}

void launch_filter_pack_tc(const float* u, float* ug, int n, int na, int nd, cudaStream_t st) {
    const TcGeom g = tc_geom(n, nd);
    const size_t units = (size_t)na * g.kb_count * 2 * g.t1n * g.nb;
    count_launches(1);
    const int blocks = (int)std::min<size_t>((units + 255) / 256, 152 * 16);
    k_filter_pack_tc<<<blocks, 256, 0, st>>>(u, ug, n, na, nd, g);
}

cudaError_t launch_filter_conv_tc(const float* ug, const float* pd, float* Cp, int n, int na, int nd, int sms,
                                  int* err, unsigned long long wait_ns, unsigned test_extra_tx, cudaStream_t st) {
    TcArgs A{};
    A.ug = ug;
    A.pd = pd;
    A.cp = Cp;
    A.n = n;
    A.na = na;
    A.nd = nd;
    A.g = tc_geom(n, nd);
    A.err = err;
    A.wait_ns = wait_ns;
    A.test_extra_tx = test_extra_tx;
    if (A.g.stages < 2) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k_filter_conv_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)A.g.smem);
    if (e != cudaSuccess) return e;
    const int items = na * A.g.kb_count * A.g.passes;
    count_launches(1);
    k_filter_conv_tc<<<std::max(1, std::min(items, sms)), TC_THREADS, A.g.smem, st>>>(A);
    return cudaGetLastError();
}

ROI_CHECK_TU(filterconv_tc)

}  // namespace roi
