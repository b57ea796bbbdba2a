// check.cuh -- index checks of the check build (compiled with -DROI_CHECK).  An index found
// outside its range [lo, hi) is counted in this translation unit's report (with the first
// site, index and bound) and replaced by lo, so the access stays inside its buffer.  The
// product build compiles the checks away (chk returns its index).
#pragma once

#include <cuda_runtime.h>

#include "roi_internal.h"

namespace roi {

#ifdef ROI_CHECK
static __device__ CheckReport g_check_report;  // one per translation unit

__device__ __forceinline__ int chk(int i, int lo, int hi, int site) {
    if (i < lo || i >= hi) {
        if (atomicAdd(&g_check_report.count, 1) == 0) {
            g_check_report.site = site;
            g_check_report.index = i;
            g_check_report.lo = lo;
            g_check_report.hi = hi;
        }
        return lo;
    }
    return i;
}

// Reads and clears this translation unit's report.
#define ROI_CHECK_TU(name)                                                   \
    void check_take_##name(CheckReport* out) {                               \
        cudaMemcpyFromSymbol(out, g_check_report, sizeof(CheckReport));      \
        const CheckReport zero{};                                            \
        cudaMemcpyToSymbol(g_check_report, &zero, sizeof zero);              \
    }
#else
__device__ __forceinline__ int chk(int i, int, int, int) { return i; }

#define ROI_CHECK_TU(name) \
    void check_take_##name(CheckReport* out) { *out = CheckReport{}; }
#endif

// Sites of the checks (CheckReport::site).
enum CheckSite {
    CHK_PERSIST_RAY = 1,     // k_persist: image column of a ray sample (shared memory)
    CHK_PERSIST_GATHER = 2,  // k_persist: staged bin of a gathered pixel
    CHK_REGION_RAY = 3,      // whole-region solver: image column of a whole-ray sample
    CHK_REGION_BAND = 4,     // whole-region solver: image column of a banded sample
    CHK_REGION_GATHER = 5,   // whole-region solver: staged bin of a gathered pixel
    CHK_FORWARD = 6,         // k_forward: image column of a ray sample (global memory)
    CHK_BACK = 7,            // k_back: staged bin of a gathered pixel
    CHK_FILTER_TC = 8        // k_filter_conv_tc: first row of a sinogram tile's descriptor
};

}  // namespace roi
