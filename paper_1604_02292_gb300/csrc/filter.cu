// filter.cu -- Ram-Lak row convolution C_h (paper Eq. fbp), the first step of FBP.
//
// q[a][d] = s * ( h0 p[a][d] + sum_{odd m} h_m (p[a][d-m] + p[a][d+m]) ),  s = pi/N_theta,
// with the spatial Ram-Lak taps h0 = 1/4, h_m = -1/(pi m)^2 (odd m), 0 for even m != 0,
// applied as a linear (zero-padded) convolution of length 2 N_d - 1.
//
// One block per angle.  The row is staged in shared memory between N_d + 8 zeros
// on each side; each thread produces 8 consecutive outputs and keeps a sliding
// register window of the left (d - m) and right (d + m) samples, so each step
// m -> m + 2 costs 4 shared loads for 8 outputs.
//
// Precision: the filtered value is a small difference of large terms (h0 p[d] is
// ~0.25 p while q is ~1e-3 p for smooth data), and float taps no longer sum to the
// filter's exact total.  The kernel therefore evaluates the same linear convolution
// rearranged as
//     q[d] = s ( sum_{odd m < N_d} h_m ((p[d-m] - p[d]) + (p[d+m] - p[d])) + c p[d] ),
//     c = h0 + 2 sum_{odd m < N_d} h_m   (formed in double on the host, ~1/(pi^2 N_d)),
// which is exact algebra: every output sums the same offsets m.  For smooth data the
// differences are exact in float (Sterbenz) and small, so tap rounding no longer
// leaves a bias; the sum is accumulated with Neumaier's compensation.
#include <cuda_runtime.h>

#include "dev_common.cuh"
#include "roi_internal.h"

namespace roi {

namespace {

constexpr int OUT_PER_THREAD = 8;

template <int DT>
__global__ void k_ramp(const void* __restrict__ pv, const float* __restrict__ hodd, float* __restrict__ q, int nd,
                       float ctail) {
    using T = typename Stor<DT>::T;  // sinogram storage; the filter works in float
    extern __shared__ float sm[];
    const int pad = nd + 8;
    float* P = sm + pad;  // P[-pad .. nd + pad)
    const int a = blockIdx.x;
    const T* prow = static_cast<const T*>(pv) + (size_t)a * nd;
    for (int i = threadIdx.x; i < nd + 2 * pad; i += blockDim.x) {
        const int d = i - pad;
        sm[i] = (d >= 0 && d < nd) ? to_f32<DT>(prow[d]) : 0.f;
    }
    __syncthreads();
    const int d0 = threadIdx.x * OUT_PER_THREAD;
    if (d0 >= nd) return;
    float acc[OUT_PER_THREAD], cmp[OUT_PER_THREAD], C[OUT_PER_THREAD], L[OUT_PER_THREAD], R[OUT_PER_THREAD];
#pragma unroll
    for (int j = 0; j < OUT_PER_THREAD; ++j) {
        C[j] = P[d0 + j];
        acc[j] = ctail * C[j];
        cmp[j] = 0.f;
        L[j] = P[d0 + j - 1];
        R[j] = P[d0 + j + 1];
    }
    // m = 2t + 1; the last odd offset that can reach inside the row is < nd
    for (int m = 1; m < nd; m += 2) {
        const float h = hodd[m >> 1];
#pragma unroll
        for (int j = 0; j < OUT_PER_THREAD; ++j) {
            const float v = h * ((L[j] - C[j]) + (R[j] - C[j]));
            const float t = acc[j] + v;
            cmp[j] += fabsf(acc[j]) >= fabsf(v) ? (acc[j] - t) + v : (v - t) + acc[j];
            acc[j] = t;
        }
        // slide to m + 2: L_j <- P[d0 + j - m - 2] = L_{j-2}, R_j <- P[d0 + j + m + 2] = R_{j+2}
#pragma unroll
        for (int j = OUT_PER_THREAD - 1; j >= 2; --j) L[j] = L[j - 2];
        L[0] = P[d0 - m - 2];
        L[1] = P[d0 - m - 1];
#pragma unroll
        for (int j = 0; j < OUT_PER_THREAD - 2; ++j) R[j] = R[j + 2];
        R[OUT_PER_THREAD - 2] = P[d0 + OUT_PER_THREAD - 2 + m + 2];
        R[OUT_PER_THREAD - 1] = P[d0 + OUT_PER_THREAD - 1 + m + 2];
    }
    float* qrow = q + (size_t)a * nd;
#pragma unroll
    for (int j = 0; j < OUT_PER_THREAD; ++j)
        if (d0 + j < nd) qrow[d0 + j] = acc[j] + cmp[j];
}

}  // namespace

// Index bounds (P spans [-(nd + 8), 2 nd + 8)): with d0 <= nd - 1 and odd m <= nd - 1
// the loads reach down to P[d0 - m - 2] >= P[-(nd + 1)] and up to
// P[d0 + 7 + m + 2] <= P[2 nd + 7].  hodd needs nd / 2 + 1 entries (index m >> 1).
void launch_ramp(const void* p, int dt, const float* hodd, float* q, int na, int nd, float ctail, cudaStream_t st) {
    if (na <= 0 || nd <= 0) return;
    int threads = (nd + OUT_PER_THREAD - 1) / OUT_PER_THREAD;
    threads = (threads + 31) / 32 * 32;
    if (threads > 1024) threads = 1024;  // nd <= 8192 is checked by the caller
    const size_t smem = sizeof(float) * (size_t)(nd + 2 * (nd + 8));
    count_launches(1);
    if (dt == 1) {
        if (smem > 48 * 1024) cudaFuncSetAttribute(k_ramp<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_ramp<1><<<na, threads, smem, st>>>(p, hodd, q, nd, ctail);
    } else if (dt == 2) {
        if (smem > 48 * 1024) cudaFuncSetAttribute(k_ramp<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_ramp<2><<<na, threads, smem, st>>>(p, hodd, q, nd, ctail);
    } else {
        if (smem > 48 * 1024) cudaFuncSetAttribute(k_ramp<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_ramp<0><<<na, threads, smem, st>>>(p, hodd, q, nd, ctail);
    }
}

}  // namespace roi
