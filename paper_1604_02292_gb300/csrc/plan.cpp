// plan.cpp -- host-side ROI planning (double precision): extended box and the
// per-angle detector windows of the rays that reach it.
//
// Sec. 2.1: many rows of W_L are zero; only the rays that reach the local part
// L carry data for the local solve.  Joseph's ray (theta, t) reaches pixel (i, j)
// exactly when |t - t_ij| < w with t_ij = x_j cos + y_i sin and w = max(|cos|, |sin|)
// of the branch taken (the hat of the linear interpolation).  Over a rectangle the
// pixel projections t_ij are spaced less than 2w apart, so the union of these open
// intervals is the single interval (T_c - H - w, T_c + H + w) around the
// rectangle's centre projection T_c, H = (|c| (w_px - 1) + |s| (h_px - 1)) / 2.
// The window holds the bins whose centres fall inside it (widened by 1e-6 so that
// a ray whose weight rounds to zero on the GPU is still kept).
#include <algorithm>
#include <cmath>
#include <vector>

#include "roi_internal.h"

namespace roi {

bool plan_box(int N, double cx, double cy, double radius, double margin, Rect* box) {
    int R = (int)std::ceil(radius + margin);
    int x0 = (int)std::floor(cx - R + 0.5);
    int y0 = (int)std::floor(cy - R + 0.5);
    int x1 = x0 + 2 * R, y1 = y0 + 2 * R;
    x0 = std::max(x0, 0);
    y0 = std::max(y0, 0);
    x1 = std::min(x1, N);
    y1 = std::min(y1, N);
    box->x0 = x0;
    box->y0 = y0;
    box->w = std::max(x1 - x0, 0);
    box->h = std::max(y1 - y0, 0);
    return box->w > 0 && box->h > 0;
}

int round_stride(int wmax) { return std::max(4, (wmax + 3) / 4 * 4); }

int plan_angles(int N, int na, int nd, const double* angles, Rect frame, Rect target, bool full_detector,
                AngleRec* rec) {
    const double half = 0.5 * (N - 1), dhalf = 0.5 * (nd - 1);
    // frame centre in world coordinates
    const double Xf = frame.x0 + 0.5 * (frame.w - 1) - half;
    const double Yf = half - (frame.y0 + 0.5 * (frame.h - 1));
    const double Xt = target.x0 + 0.5 * (target.w - 1) - half;
    const double Yt = half - (target.y0 + 0.5 * (target.h - 1));
    int wmax = 0;
    for (int a = 0; a < na; ++a) {
        const double c = std::cos(angles[a]), s = std::sin(angles[a]);
        const int row = std::fabs(c) >= std::fabs(s) - 1e-12;  // ties go to the per-row branch
        const double wd = row ? std::fabs(c) : std::fabs(s);
        int d0 = 0, width = nd;
        if (!full_detector) {
            const double Tt = Xt * c + Yt * s;
            const double H = 0.5 * (std::fabs(c) * (target.w - 1) + std::fabs(s) * (target.h - 1));
            const double lo = Tt - H - wd + dhalf, hi = Tt + H + wd + dhalf;
            long dlo = (long)std::floor(lo - 1e-6) + 1;
            long dhi = (long)std::ceil(hi + 1e-6) - 1;
            dlo = std::max(dlo, 0L);
            dhi = std::min(dhi, (long)nd - 1);
            if (dhi >= dlo) {
                d0 = (int)dlo;
                width = (int)(dhi - dlo + 1);
            } else {
                d0 = 0;
                width = 0;
            }
        }
        const double Tf = Xf * c + Yf * s;
        const int Mm = row ? frame.w : frame.h;  // minor extent
        angle_fill(rec[a], a, c, s, row, wd, d0, width, d0 - dhalf - Tf, Mm);
        wmax = std::max(wmax, width);
    }
    return wmax;
}

// Box-frame table of a region for the whole-region solvers: the angles sampled per row
// first, then the others (stable); AngleRec::aidx keeps each angle's index in the
// sinogram.  Returns the largest window width.
int plan_region_table(int N, int na, int nd, const double* angles, Rect box, AngleRec* out, int* nrow) {
    std::vector<AngleRec> loc(na);
    const int wl = plan_angles(N, na, nd, angles, box, box, false, loc.data());
    int k = 0;
    for (int a = 0; a < na; ++a)
        if (loc[a].row) out[k++] = loc[a];
    *nrow = k;
    for (int a = 0; a < na; ++a)
        if (!loc[a].row) out[k++] = loc[a];
    return wl;
}

}  // namespace roi
