// noalloc.cu -- a forward projector entry point that allocates no device memory.
//
// roi_recon_forward_local_noalloc computes the same y = W_L x as roi_recon_forward_local
// but without a handle: its scratch (the per-angle ray table and the two zero-padded
// copies of the box image the projector reads, by rows and by columns) lives in one file-scope
// __device__ array of fixed size, so the call makes no cudaMalloc / cudaFree and
// calls nothing that allocates.  It exists for callers that cannot allocate device
// memory themselves: code whose device memory is owned by someone else's fixed
// budget (a framework's caching allocator, a serving process that reserves HBM up
// front), and loops that cannot take the implicit device synchronisation of
// cudaMalloc / cudaFree.
//
// The ray table is the host plan itself (plan_angles, the function roi_recon_plan uses),
// so the windows the kernel projects into are the windows the caller sized y with.  It
// reaches the device as kernel parameters (up to kRecsPerLaunch records per launch of
// k_put_recs): no host staging buffer, no copy from pageable memory, nothing allocated.
//
// Facts a caller must know:
//   * Every GPU that loads this library holds the array (kNoallocScratchBytes) until
//     the process exits.  With lazy module loading (the default since CUDA 12.2) the
//     module, and so the array, is loaded by the first call on each device: that call
//     may allocate the module's memory and synchronise; later calls do neither.  Make
//     the first call before any stream capture.
//   * Host code cannot use the array's name as a device address; every call looks the
//     address up with cudaGetSymbolAddress (which allocates nothing) with the caller's
//     device current, so the address stays right after a device reset.
//   * All calls share the array and it keeps the last call's contents.  Each call
//     clears and rewrites every scratch byte it reads before reading it (the zero
//     borders of the padded image copies included), so nothing carries over; but
//     calls whose work overlaps on the GPU (other streams, other host threads) race
//     on the array and must be serialised by the caller.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>

#include "roi_recon.h"
#include "roi_internal.h"

namespace {

constexpr size_t kNoallocScratchBytes = size_t(16) << 20;  // 16 MiB per device
constexpr double kPi = 3.14159265358979323846;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

// A run of host-planned ray records passed by value (kernel parameters, at most 32764
// bytes on this architecture) and stored at rec[a0 .. a0 + n).
constexpr int kRecsPerLaunch = 320;
struct RecChunk {
    int a0, n;
    roi::AngleRec r[kRecsPerLaunch];
};
static_assert(sizeof(RecChunk) <= 32000, "ray records must fit the kernel parameter space");

__global__ void k_put_recs(roi::AngleRec* rec, const RecChunk c) {
    for (int i = threadIdx.x; i < c.n; i += blockDim.x) rec[c.a0 + i] = c.r[i];
}

void put_err(char* err, int err_len, const char* msg) {
    if (err && err_len > 0) std::snprintf(err, (size_t)err_len, "%s", msg);
}

}  // namespace

extern "C" roi_status roi_recon_forward_local_noalloc(const roi_geometry* geom, const roi_region* region,
                                                      const float* x, float* y, void* cuda_stream, char* err,
                                                      int err_len) {
    put_err(err, err_len, "");
    if (!geom || !region || !x || !y) {
        put_err(err, err_len, "forward_local_noalloc: null argument");
        return ROI_EINVAL;
    }
    if (geom->n_pix < 1 || geom->n_angles < 1 || geom->n_det < 1 || geom->n_pix > 65536 ||
        geom->n_angles > 65536 || geom->n_det > 8192 || geom->storage != ROI_F32 || geom->image_storage != ROI_F32 ||
        geom->angles != nullptr) {
        put_err(err, err_len, "forward_local_noalloc: geometry must be valid, float32, with default angles");
        return ROI_EINVAL;
    }
    if (!(std::isfinite(region->cx) && std::isfinite(region->cy) && std::isfinite(region->radius) &&
          std::isfinite(region->margin) && region->radius > 0 && region->margin >= 0 &&
          region->radius + region->margin < 1e7)) {
        put_err(err, err_len, "forward_local_noalloc: region radius must be > 0, margin >= 0, all finite");
        return ROI_EINVAL;
    }
    roi::Rect box;
    if (!roi::plan_box(geom->n_pix, region->cx, region->cy, region->radius, region->margin, &box)) {
        put_err(err, err_len, "forward_local_noalloc: extended box does not intersect the grid");
        return ROI_EINVAL;
    }
    const int na = geom->n_angles;
    const size_t table_bytes = ((sizeof(roi::AngleRec) * (size_t)na + 255) / 256) * 256;
    // the two padded copies of the box image the projector reads (rows and columns)
    const size_t rows_bytes = ((sizeof(float) * (size_t)box.h * roi::padded_ld(box.w) + 255) / 256) * 256;
    const size_t cols_bytes = sizeof(float) * (size_t)box.w * roi::padded_ld(box.h);
    const size_t image_bytes = rows_bytes + cols_bytes;
    if (table_bytes + image_bytes > kNoallocScratchBytes) {
        char msg[256];
        std::snprintf(msg, sizeof msg,
                      "forward_local_noalloc: needs %zu bytes of scratch (%d angles, %d x %d box), limit is %zu",
                      table_bytes + image_bytes, na, box.w, box.h, kNoallocScratchBytes);
        put_err(err, err_len, msg);
        return ROI_EINVAL;
    }
    void* base = nullptr;
    {
        cudaError_t e = cudaGetSymbolAddress(&base, g_noalloc_scratch);
        if (e != cudaSuccess || !base) {
            char msg[256];
            std::snprintf(msg, sizeof msg, "forward_local_noalloc: cudaGetSymbolAddress failed: %s",
                          cudaGetErrorString(e));
            put_err(err, err_len, msg);
            return ROI_ECUDA;
        }
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    roi::AngleRec* rec = (roi::AngleRec*)base;
    float* xr = (float*)((unsigned char*)base + table_bytes);               // [h][w + 4]
    float* xc = (float*)((unsigned char*)base + table_bytes + rows_bytes);  // [w][h + 4]
    if (cudaMemsetAsync(xr, 0, image_bytes, st) != cudaSuccess) {
        put_err(err, err_len, "forward_local_noalloc: clearing the scratch failed");
        return ROI_ECUDA;
    }
    // The ray table: the host plan of roi_recon_plan (default angles a pi / N_theta), made
    // and sent a chunk of angles at a time; its widest window gives the stride of y.
    int wmax = 0;
    {
        RecChunk chunk;
        double ang[kRecsPerLaunch];
        for (int a0 = 0; a0 < na; a0 += kRecsPerLaunch) {
            const int n = na - a0 < kRecsPerLaunch ? na - a0 : kRecsPerLaunch;
            for (int i = 0; i < n; ++i) ang[i] = (a0 + i) * kPi / na;
            const int w = roi::plan_angles(geom->n_pix, n, geom->n_det, ang, box, box, false, chunk.r);
            wmax = w > wmax ? w : wmax;
            for (int i = 0; i < n; ++i) chunk.r[i].aidx = a0 + i;
            chunk.a0 = a0;
            chunk.n = n;
            roi::count_launches(1);
            k_put_recs<<<1, 128, 0, st>>>(rec, chunk);
        }
    }
    roi::launch_copy_pad(x, box.w, xr + roi::kPad, roi::padded_ld(box.w), box.h, box.w, st);
    roi::launch_transpose(x, box.w, xc + roi::kPad, roi::padded_ld(box.h), box.h, box.w, st);
    roi::FwdArgs a{};
    a.rec = rec;
    a.na = na;
    a.stride = roi::round_stride(wmax);  // = roi_recon_plan's window_stride
    a.nx = box.w;
    a.ny = box.h;
    a.img = xr + roi::kPad;
    a.imgT = xc + roi::kPad;
    a.img_ld = roi::padded_ld(box.w);
    a.imgT_ld = roi::padded_ld(box.h);
    a.out = y;
    a.nd = geom->n_det;
    roi::launch_forward(roi::FWD_PLAIN, a, st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        char msg[256];
        std::snprintf(msg, sizeof msg, "forward_local_noalloc: launch failed: %s", cudaGetErrorString(e));
        put_err(err, err_len, msg);
        return ROI_ECUDA;
    }
    return ROI_OK;
}
