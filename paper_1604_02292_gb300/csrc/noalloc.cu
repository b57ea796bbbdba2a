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
// Facts a caller must know:
//   * Every GPU that loads this library holds the array (kNoallocScratchBytes) until
//     the process exits.
//   * Host code cannot use the array's name as a device address; the address is
//     obtained once per device with cudaGetSymbolAddress on the first call made
//     with that device current.  That first call should come before any stream
//     capture.
//   * All calls share the array and it keeps the last call's contents.  Each call
//     clears and rewrites every scratch byte it reads before reading it (the zero
//     borders of the padded image copies included), so nothing carries over; but
//     calls whose work overlaps on the GPU (other streams, other host threads) race
//     on the array and must be serialised by the caller.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>

#include "roi_recon.h"
#include "roi_internal.h"

namespace {

constexpr size_t kNoallocScratchBytes = size_t(16) << 20;  // 16 MiB per device
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

std::mutex g_addr_mu;
void* g_addr[kMaxDevices] = {};

// Device-side copy of the host ROI plan for one angle (frame = target = box; see
// plan.cpp for the derivation of the window of bins whose Joseph rays reach the box).
__global__ void k_plan_box(roi::AngleRec* rec, int N, int na, int nd, roi::Rect box, int stride) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= na) return;
    const double kPi = 3.14159265358979323846;
    const double th = a * kPi / na;
    const double c = cos(th), s = sin(th);
    const double half = 0.5 * (N - 1), dhalf = 0.5 * (nd - 1);
    const double Xb = box.x0 + 0.5 * (box.w - 1) - half;
    const double Yb = half - (box.y0 + 0.5 * (box.h - 1));
    const int row = fabs(c) >= fabs(s) - 1e-12;
    const double wd = row ? fabs(c) : fabs(s);
    const double Tb = Xb * c + Yb * s;
    const double H = 0.5 * (fabs(c) * (box.w - 1) + fabs(s) * (box.h - 1));
    long dlo = (long)floor(Tb - H - wd + dhalf - 1e-6) + 1;
    long dhi = (long)ceil(Tb + H + wd + dhalf + 1e-6) - 1;
    dlo = dlo < 0 ? 0 : dlo;
    dhi = dhi > nd - 1 ? nd - 1 : dhi;
    int d0 = 0, width = 0;
    if (dhi >= dlo) {
        d0 = (int)dlo;
        width = (int)(dhi - dlo + 1);
    }
    if (width > stride) width = stride;  // the output row holds `stride` bins
    roi::AngleRec r;
    roi::angle_fill(r, a, c, s, row, wd, d0, width, d0 - dhalf - Tb, row ? box.w : box.h);
    rec[a] = r;
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
        geom->n_angles > 65536 || geom->n_det > 8192 || geom->storage != ROI_F32 || geom->angles != nullptr) {
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
    // The caller sizes y with the host plan's window stride; recompute it here.
    roi_solve_info info;
    if (roi_recon_plan(geom, region, &info, nullptr, nullptr) != ROI_OK) {
        put_err(err, err_len, "forward_local_noalloc: planning failed");
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
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        put_err(err, err_len, "forward_local_noalloc: no usable current CUDA device");
        return ROI_ECUDA;
    }
    void* base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_addr_mu);
        if (!g_addr[dev]) {
            void* p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                char msg[256];
                std::snprintf(msg, sizeof msg, "forward_local_noalloc: cudaGetSymbolAddress failed: %s",
                              cudaGetErrorString(e));
                put_err(err, err_len, msg);
                return ROI_ECUDA;
            }
            g_addr[dev] = p;
        }
        base = g_addr[dev];
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    roi::AngleRec* rec = (roi::AngleRec*)base;
    float* xr = (float*)((unsigned char*)base + table_bytes);               // [h][w + 4]
    float* xc = (float*)((unsigned char*)base + table_bytes + rows_bytes);  // [w][h + 4]
    if (cudaMemsetAsync(xr, 0, image_bytes, st) != cudaSuccess) {
        put_err(err, err_len, "forward_local_noalloc: clearing the scratch failed");
        return ROI_ECUDA;
    }
    roi::count_launches(1);
    k_plan_box<<<(na + 127) / 128, 128, 0, st>>>(rec, geom->n_pix, na, geom->n_det, box, info.window_stride);
    roi::launch_copy_pad(x, box.w, xr + roi::kPad, roi::padded_ld(box.w), box.h, box.w, st);
    roi::launch_transpose(x, box.w, xc + roi::kPad, roi::padded_ld(box.h), box.h, box.w, st);
    roi::FwdArgs a{};
    a.rec = rec;
    a.na = na;
    a.stride = info.window_stride;
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
