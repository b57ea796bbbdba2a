// batch.cu -- many local solves of uneven size in one persistent launch.
//
// One block per SM pulls regions from a device queue (largest first) and solves each
// one completely, exterior step included (region_solver.cuh: Sec. 1 scheme with the
// operators W_L, W_L^T of Sec. 2.1; SIRT, Eq. sirtit + Eq. sirtbox, or TV by
// Chambolle-Pock, Eq. priorsys).  Only block barriers separate the phases; blocks never
// wait on one another, and a region's result does not depend on the other regions of
// the batch nor on which block solved it.
//
// Batches with fewer regions than half the SMs run instead as teams of blocks (k_batch_team
// in batch_team.cu, cooperative launch): team t solves the regions t, t + teams, ...
// (largest first), its blocks sharing rays and tiles and meeting at bounded team barriers;
// results are the same bits as with one block per region.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "dev_common.cuh"
#include "region_solver.cuh"
#include "roi_internal.h"

namespace roi {

namespace {

using rs::BPT;

__global__ void __launch_bounds__(BPT, 1) k_batch(BatchArgs B) {
    extern __shared__ float4 smem4[];
    float* smem = reinterpret_cast<float*>(smem4);
    __shared__ int s_roi, s_cnt;
    __shared__ __align__(8) uint64_t s_mbar[2];
    const int tid = threadIdx.x;
    const size_t slot = blockIdx.x;
    if (tid == 0) {
        mbar_init(&s_mbar[0], 1);
        mbar_init(&s_mbar[1], 1);
    }
    unsigned parity = 0;
    rs::Team T{0, 1, nullptr, 0u, B.err, B.wait_ns};
    rs::RegionBufs bufs;
    bufs.pp = B.slot_pp + slot * B.win_cap;
    bufs.u = B.slot_u + slot * B.win_cap;
    bufs.sig = B.slot_sig + slot * B.win_cap;
    bufs.x = B.slot_x + slot * B.img_cap;
    bufs.vx = B.slot_vx + slot * B.img_cap;
    bufs.vy = B.slot_vy + slot * B.img_cap;
    bufs.tau = B.slot_tau + slot * B.img_cap;
    bufs.xa_base = B.slot_xa + slot * B.pad_cap;
    bufs.xaT_base = B.slot_xaT + slot * B.pad_cap;
    bufs.fgp = B.slot_fgp ? B.slot_fgp + slot * 5 * B.img_cap : nullptr;
    bufs.part = nullptr;
    for (;;) {
        __syncthreads();
        if (tid == 0) s_roi = atomicAdd(B.queue, 1);
        __syncthreads();
        const int qi = s_roi;
        if (qi >= B.nroi) break;
        if (!rs::solve_region_dt<true>(B.rois[B.order[qi]], bufs, T, smem, s_mbar, parity, &s_cnt)) return;
    }
}

}  // namespace

size_t batch_smem_bytes(size_t max_stage_bytes, int na, bool banded) {
    // the per-warp phase-B areas and one tile's chunk partials (cooperative phase B); with a
    // band-streamed region, the partial sums of a pass over more units than warps
    const size_t chunks = (size_t)(na + rs::ACH - 1) / rs::ACH;
    const size_t phase_b = sizeof(float) * ((size_t)rs::BNW * rs::WARP_STAGE + chunks * rs::TB * rs::TB);
    const size_t s = std::min(std::max(max_stage_bytes, phase_b), std::max(max_stage_bytes, (size_t)kStageMaxBytes));
    return banded ? s + kBandStateBytes : s;
}

cudaError_t launch_batch(const BatchArgs& B, int blocks, size_t smem, cudaStream_t st) {
    if (B.team > 1) return launch_batch_team(B, blocks, smem, st);  // batch_team.cu
    cudaError_t e = cudaFuncSetAttribute(k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(B.queue, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    count_launches(1);
    k_batch<<<blocks, BPT, smem, st>>>(B);
    return cudaGetLastError();
}

ROI_CHECK_TU(batch)

}  // namespace roi
