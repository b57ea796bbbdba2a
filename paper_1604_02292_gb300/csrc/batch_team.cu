// batch_team.cu -- batched local solves by teams of blocks (few regions, or one large box
// of roi_recon_solve_local): one cooperative launch, team t solving the regions t,
// t + teams, ... (largest first) with the whole-region solver of region_solver.cuh (Sec. 1
// scheme, operators of Sec. 2.1); its blocks share rays and tiles and meet at bounded team
// barriers.  Kept apart from batch.cu so the two kernels compile in parallel.
#include <cuda_runtime.h>
#include <stdint.h>

#include "dev_common.cuh"
#include "region_solver.cuh"
#include "roi_internal.h"

namespace roi {

namespace {

using rs::BPT;

// Teams of B.team consecutive blocks; team t owns slot t and solves regions t + i * teams.
__global__ void __launch_bounds__(BPT, 1) k_batch_team(BatchArgs B) {
    extern __shared__ float4 smem4[];
    float* smem = reinterpret_cast<float*>(smem4);
    __shared__ int s_cnt;
    __shared__ __align__(8) uint64_t s_mbar[2];
    __shared__ rs::Team s_team;
    __shared__ rs::RegionBufs s_bufs;
    const int tid = threadIdx.x;
    const int team_id = blockIdx.x / B.team, teams = gridDim.x / B.team;
    if (tid == 0) {
        mbar_init(&s_mbar[0], 1);
        mbar_init(&s_mbar[1], 1);
        s_team = rs::Team{(int)(blockIdx.x % B.team), B.team, B.bars + team_id, 0u, B.err, B.wait_ns,
                          B.absent > 0 ? (unsigned)(B.team + B.absent) : 0u};
        const size_t slot = team_id;
        s_bufs.pp = B.slot_pp + slot * B.win_cap;
        s_bufs.u = B.slot_u + slot * B.win_cap;
        s_bufs.sig = B.slot_sig + slot * B.win_cap;
        s_bufs.x = B.slot_x + slot * B.img_cap;
        s_bufs.vx = B.slot_vx + slot * B.img_cap;
        s_bufs.vy = B.slot_vy + slot * B.img_cap;
        s_bufs.tau = B.slot_tau + slot * B.img_cap;
        s_bufs.xa_base = B.slot_xa + slot * B.pad_cap;
        s_bufs.xaT_base = B.slot_xaT + slot * B.pad_cap;
        s_bufs.fgp = B.slot_fgp ? B.slot_fgp + slot * 5 * B.img_cap : nullptr;
        s_bufs.part = B.slot_part ? B.slot_part + slot * B.part_cap : nullptr;
    }
    __syncthreads();
    unsigned parity = 0;
    for (int qi = team_id; qi < B.nroi; qi += teams) {
        if (!rs::solve_region_dt<false>(B.rois[B.order[qi]], s_bufs, s_team, smem, s_mbar, parity, &s_cnt)) return;
        if (!rs::team_sync<false>(s_team)) return;  // the slot is reused by the next region
    }
}

}  // namespace

cudaError_t launch_batch_team(const BatchArgs& B, int blocks, size_t smem, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(k_batch_team, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int teams = blocks / B.team;
    e = cudaMemsetAsync(B.bars, 0, sizeof(unsigned) * teams, st);
    if (e != cudaSuccess) return e;
    BatchArgs a = B;
    void* args[] = {&a};
    count_launches(1);
    return cudaLaunchCooperativeKernel((const void*)k_batch_team, dim3(teams * B.team), dim3(BPT), args, smem, st);
}

ROI_CHECK_TU(batch_team)

}  // namespace roi
