// serve.cu -- the serving kernel: one cooperative launch whose blocks take ROI solve
// requests while the host keeps publishing them (continuous batching).
//
// The blocks form two pools: single blocks for small boxes and teams of several
// blocks for large ones (a team shortens a large request's latency; region_solver.cuh
// keeps the result identical whichever pool solves it).  Each pool reads a ring of
// request slots in page-locked host memory mapped into the device: the host writes a
// slot (descriptor + box-frame table) and then publishes it by a release store of the
// ring's tail; a free unit (single block, or the leader block of a team) claims the
// next ticket with a compare-and-swap on the pool's head counter, tells its members
// through a mailbox, solves the region (exterior step, set-up, iterations, crop into
// page-locked host memory) and marks the slot done with a release store at system
// scope, which the host polls.
//
// Every wait is bounded: a unit leaves when the host sets the close flag, when nothing
// was claimed or finished for idle_ns while no request is being solved, or after
// cap_ns of polling; team barriers and mailbox waits give up after wait_ns (plus the
// leader's longest poll) and set the error flag.  The host relaunches the kernel when
// work arrives after it has left.
#include <cuda_runtime.h>
#include <stdint.h>

#include "dev_common.cuh"
#include "region_solver.cuh"
#include "roi_internal.h"

namespace roi {

namespace {

using rs::BPT;

__device__ __forceinline__ unsigned long long ld_acquire_sys_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long ld_relaxed_gpu_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned ld_relaxed_sys_u32(const void* p) {
    unsigned v;
    asm volatile("ld.relaxed.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_relaxed_gpu_s32(const int* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Claim the next published ticket of pool P (thread 0 of a unit's leader block);
// -1: leave the kernel.
__device__ long long claim_ticket(const ServePool& P, const ServeArgs& A) {
    const unsigned long long t0 = global_ns();
    unsigned nap = 128;  // back-off of idle polls (page-locked words are read over the C2C link)
    for (;;) {
        if (ld_relaxed_sys_u32(A.close)) return -1;
        const unsigned long long tail = ld_acquire_sys_u64(P.tail);
        const unsigned long long h = ld_relaxed_gpu_u64(P.head);
        if (h < tail) {
            if (atomicCAS(P.head, h, h + 1) == h) {
                atomicAdd(A.busy, 1);
                atomicMax(A.last_ns, global_ns());
                return (long long)h;
            }
            continue;
        }
        if (ld_relaxed_gpu_s32(A.err)) return -1;
        const unsigned long long now = global_ns();
        if (now - t0 > A.cap_ns) return -1;
        if (now - t0 > A.idle_ns && ld_relaxed_gpu_s32(A.busy) == 0) {
            const unsigned long long last = ld_relaxed_gpu_u64(A.last_ns);
            if (last < now && now - last > A.idle_ns) return -1;
        }
        __nanosleep(nap);
        if (nap < 4096) nap *= 2;
    }
}

// Member blocks of a team: wait (bounded) for the leader's k-th claim.
__device__ long long wait_mail(const ServeArgs& A, int gteam, unsigned k) {
    const unsigned long long t0 = global_ns();
    const unsigned long long limit = A.cap_ns + A.wait_ns;
    for (;;) {
        unsigned v;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(A.mail_seq + gteam) : "memory");
        if (v == k) {
            long long c;
            asm volatile("ld.relaxed.gpu.global.s64 %0, [%1];" : "=l"(c) : "l"(A.mail_val + gteam) : "memory");
            return c;
        }
        if (ld_relaxed_gpu_s32(A.err)) return -1;
        if (global_ns() - t0 > limit) {
            atomicExch(A.err, 1);
            return -1;
        }
        __nanosleep(1024);
    }
}

__global__ void __launch_bounds__(BPT, 1) k_serve(const ServeArgs A) {
    extern __shared__ float4 smem4[];
    float* smem = reinterpret_cast<float*>(smem4);
    __shared__ int s_cnt;
    __shared__ long long s_claim;
    __shared__ __align__(8) uint64_t s_mbar[2];
    __shared__ __align__(16) ServeSlot s_slot;
    __shared__ rs::Team s_team;      // per-block state kept out of registers
    __shared__ int s_pool;
    __shared__ unsigned s_mail;
    const int tid = threadIdx.x;
    if (tid == 0) {
        const int b = blockIdx.x;
        const int pi = (A.pool[1].nteams > 0 && b >= A.pool[1].first_block) ? 1 : 0;
        const ServePool& P = A.pool[pi];
        const int rel = b - P.first_block;
        const int team_id = rel / P.team;
        s_pool = (rel < 0 || team_id >= P.nteams) ? -1 : pi;  // -1: not part of a unit
        s_team = rs::Team{rel - team_id * P.team, P.team, A.bars + P.team_base + team_id, 0u, A.err, A.wait_ns,
                          (A.absent > 0 && P.team > 1) ? (unsigned)(P.team + A.absent) : 0u};
        if (A.absent < 0 && P.team > 1 && s_team.member == 0) s_pool = -1;  // testing: an absent leader
        s_mail = 0;
        mbar_init(&s_mbar[0], 1);
        mbar_init(&s_mbar[1], 1);
    }
    __syncthreads();
    if (s_pool < 0) return;
    unsigned parity = 0;
    constexpr int kHeadWords = (int)(sizeof(ServeSlot) / 4);
    for (;;) {
        __syncthreads();
        if (tid == 0) {
            const ServePool& P = A.pool[s_pool];
            const int gteam = (int)(s_team.bar - A.bars);
            long long c;
            if (s_team.member == 0) {
                c = claim_ticket(P, A);
                if (P.team > 1) {
                    asm volatile("st.relaxed.gpu.global.s64 [%0], %1;" ::"l"(A.mail_val + gteam), "l"(c) : "memory");
                    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(A.mail_seq + gteam), "r"(s_mail + 1)
                                 : "memory");
                }
            } else {
                c = wait_mail(A, gteam, s_mail + 1);
            }
            ++s_mail;
            s_claim = c;
        }
        __syncthreads();
        const long long c = s_claim;
        if (c < 0) return;
        const ServePool& P = A.pool[s_pool];
        const size_t slot = (size_t)(c % P.slots);
        const unsigned char* sp = P.ring + slot * P.slot_bytes;
        AngleRec* myrec = A.rec_slots + (size_t)blockIdx.x * A.max_na;
        // descriptor and table out of the page-locked ring (system-scope loads)
        for (int w = tid; w < kHeadWords; w += BPT)
            reinterpret_cast<unsigned*>(&s_slot)[w] = ld_relaxed_sys_u32(sp + 4 * (size_t)w);
        __syncthreads();
        const int rec_words = s_slot.roi.na * (int)(sizeof(AngleRec) / 4);
        const unsigned char* rp = sp + serve_slot_header_bytes;
        for (int w = tid; w < rec_words; w += BPT)
            reinterpret_cast<unsigned*>(myrec)[w] = ld_relaxed_sys_u32(rp + 4 * (size_t)w);
        if (tid == 0) {
            s_slot.roi.rec = myrec;
            // a solo launch (one team of every block): the row-band phase A of a band-streamed
            // box uses the solo partial-sum buffer when the box's partials fit (same bits)
            s_slot.bufs.part = nullptr;
            const BatchRoi& R = s_slot.roi;
            const int es = dt_size(R.dt);
            if (A.solo_part && s_team.size > 1 && s_team.size == (int)gridDim.x && stage_mode(R.nx, R.ny, es) == 1) {
                const int br = band_rows(R.nx, R.ny, es);
                const size_t need = ((size_t)((R.ny + br - 1) / br) * R.nrow + (size_t)((R.nx + br - 1) / br) *
                                     (R.na - R.nrow)) * ((R.stride + 31) / 32) * 32;
                if (need <= A.solo_part_cap) s_slot.bufs.part = A.solo_part;
            }
        }
        __syncthreads();
        // one code path for both pools (a single block is a team of one at run time)
        const bool ok = rs::solve_region_dt<false>(s_slot.roi, s_slot.bufs, s_team, smem, s_mbar, parity, &s_cnt);
        if (!ok) return;
        __threadfence_system();  // this thread's output stores, before the completion word
        if (!rs::team_sync<false>(s_team)) return;
        if (s_team.member == 0 && tid == 0) {
            asm volatile("st.release.sys.global.u64 [%0], %1;" ::"l"(A.pool[s_pool].done + slot), "l"(s_slot.seq)
                         : "memory");
            atomicMax(A.last_ns, global_ns());
            atomicSub(A.busy, 1);
        }
    }
}

}  // namespace

size_t serve_smem_bytes() {
    // any request's staging (at most kStageMaxBytes) and the per-warp phase-B areas, then
    // the per-ray partial sums of band-streamed phase A passes
    const size_t phase_b = sizeof(float) * (size_t)rs::BNW * rs::WARP_STAGE;
    return (kStageMaxBytes > phase_b ? kStageMaxBytes : phase_b) + kBandStateBytes;
}

int serve_max_blocks(int device) {
    const size_t smem = serve_smem_bytes();
    if (cudaFuncSetAttribute(k_serve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
    int per_sm = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_serve, BPT, smem) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 0;
    return per_sm * sms;
}

cudaError_t launch_serve(const ServeArgs& A, int blocks, cudaStream_t st) {
    const size_t smem = serve_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(k_serve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    ServeArgs a = A;
    void* args[] = {&a};
    count_launches(1);
    return cudaLaunchCooperativeKernel((const void*)k_serve, dim3(blocks), dim3(BPT), args, smem, st);
}

ROI_CHECK_TU(serve)

}  // namespace roi
