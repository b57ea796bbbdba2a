// roi_internal.h -- internal types and launchers of the CUDA library (not installed).
//
// Geometry (Sec. 2.1 of the paper): a "frame" is a rectangle of the N x N grid on
// which an image lives (the whole grid for FBP and the exterior step, the extended
// ROI box for the local operators W_L, W_L^T).  A "ray set" is, per angle, a window
// of consecutive detector bins [d0, d0 + width).  For each (frame, ray set) pair the
// host builds one AngleRec per angle (in double precision) that both projector
// kernels read.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace roi {

// Per-angle record of a ray set over a frame.  Frame-centre coordinates:
//   pixel (li, lj) of the frame (row, column) sits at xi = lj - (nx-1)/2,
//   eta = (ny-1)/2 - li relative to the frame centre; bin k of the window has
//   offset t_{d0+k} - T_frame = k + phi with T_frame = Xf c + Yf s.
// Forward (ray-driven): along ray k the sample at major index m (row when `row`,
// column otherwise) has minor coordinate  A0 + k a_scale + (m - (M-1)/2) slope.
// Back (pixel-driven): pixel (li, lj) sits at window coordinate
//   kappa = xi c + eta s - phi.
struct AngleRec {
    double c, s;       // cos(theta), sin(theta)
    double phi;        // d0 - (N_d-1)/2 - T_frame
    double A0;         // (Mm-1)/2 + a_scale * phi
    double a_scale;    // 1/c (row branch) or -1/s (column branch)
    double slope;      // s/c (row branch) or c/s (column branch)
    float inv_w;       // 1 / |c| or 1 / |s|
    int row;           // 1: sample per row (|c| >= |s|), 0: per column
    int d0;            // first bin of the window
    int width;         // bins in the window (0 if no ray reaches the frame)
};

struct Rect {
    int x0, y0, w, h;
};

// Host-side plan of one region (double precision throughout).
struct Plan {
    Rect box;
    int window_max;
    int stride;        // multiple of 4, >= window_max (>= 4)
};

// -------------------------------------------------------------------- planning
// Extended box of a region; returns false when it misses the grid.
bool plan_box(int N, double cx, double cy, double radius, double margin, Rect* box);
// Fills rec[na] for `frame` with ray windows of the bins that reach `target`
// (target == frame for the local operators; the box for the exterior step with
// frame = whole grid); returns the max width.  full_detector: window = all bins.
int plan_angles(int N, int na, int nd, const double* angles, Rect frame, Rect target, bool full_detector,
                AngleRec* rec);
int round_stride(int wmax);

// ----------------------------------------------------------------- launchers
// Process-wide count of kernels launched by the library.
void count_launches(unsigned n);
unsigned long long launches_total();

enum FwdMode { FWD_PLAIN = 0, FWD_EXTERIOR = 1, FWD_SIRT = 2, FWD_CP = 3 };
enum BackMode { BACK_PLAIN = 0, BACK_SIRT = 1, BACK_CP = 2 };

struct FwdArgs {
    const AngleRec* rec;   // [na]
    int na, stride;        // window rows and their stride
    int nx, ny;            // frame size
    const float* img;      // frame image [ny][nx]
    const float* imgT;     // its transpose [nx][ny]
    Rect hole;             // FWD_EXTERIOR: frame pixels treated as zero (w = 0: none)
    float* out;            // [na][stride]
    // FWD_EXTERIOR: out = p[a][d0 + k] - W_F x
    const float* p;        // [na][nd]
    int nd;
    // FWD_SIRT: out = (pp - W x) * (R ? R[a][k] : 1)
    // FWD_CP:   out = (out + sig (W x - pp)) / (1 + sig / 2), sig = R ? R[a][k] : sig_scalar
    const float* pp;       // [na][stride]
    const float* R;        // [na][stride] or null
    float sig_scalar;
};

struct BackArgs {
    const AngleRec* rec;   // [na]
    int na, stride;
    int nx, ny;            // frame size
    const float* win;      // [na][stride] window values
    float* out;            // BACK_PLAIN: [ny][nx]; else x (in/out)
    float* outT;           // optional transpose of the written image ([nx][ny]) or null
    // BACK_SIRT: x = max(0, x + step * acc) (nonneg) with step = C ? C[pix] : step_scalar
    // BACK_CP:   x+ = x - tau (acc - div v); xbar = 2 x+ - x  (tau = C ? C[pix] : step_scalar)
    const float* C;
    float step_scalar;
    int nonneg;
    const float* vx;       // BACK_CP: [ny][nx]
    const float* vy;
    float* xbar;           // BACK_CP: [ny][nx] (its transpose goes to outT)
};

void launch_forward(FwdMode mode, const FwdArgs& a, cudaStream_t st);
void launch_back(BackMode mode, const BackArgs& a, cudaStream_t st);
// hodd[t] = s h_{2t+1}; ctail = s (h0 + 2 sum_{odd m < nd} h_m), s = pi / N_theta
void launch_ramp(const float* p, const float* hodd, float* q, int na, int nd, float ctail, cudaStream_t st);
void launch_transpose(const float* in, float* out, int rows, int cols, cudaStream_t st);
void launch_fill(float* p, float v, size_t n, cudaStream_t st);
void launch_window_ones(float* win, const AngleRec* rec, int na, int stride, cudaStream_t st);
// CP gradient dual: v = proj_{|v| <= lambda}(v + sigma_v grad xbar)
void launch_cp_dual_grad(const float* xbar, float* vx, float* vy, int nx, int ny, float sigma_v, float lambda,
                         cudaStream_t st);
void launch_cp_dual_grad_dev(const float* xbar, float* vx, float* vy, int nx, int ny, const float* sigma_dev,
                             float lambda, cudaStream_t st);
// power iteration helpers for ||K||, K = [W_L; grad]
void launch_power_ktk_grad(float* y, const float* x, int nx, int ny, cudaStream_t st);
void launch_sumsq(const float* v, int n, double* scratch, int nscratch, double* out2, cudaStream_t st);
void launch_normalize(const float* y, float* x, float* xT, int nx, int ny, const double* n2, cudaStream_t st);
void launch_fill_step(float* dst, size_t n, const double* n2, double* L_out, cudaStream_t st);
// Preconditioners from row sums (window) and column sums (box):
//   mode 0 (SIRT weights): R = s > 1e-3 ? 1/s : 0, C likewise
//   mode 1 (CP diag):      sigma_u = s > 1e-6 ? 1/s : 0; tau = 1/(colsum + |grad| column count)
void launch_precond(float* rows, int nrows_total, float* cols, int nx, int ny, int mode, cudaStream_t st);
// out = x (box) with pixels outside the disk (cx, cy, r) in box-local coordinates set to 0 if crop
void launch_crop(const float* x, float* out, int nx, int ny, double cxl, double cyl, double r, int crop,
                 cudaStream_t st);
// objective terms: part[0] = sum over rows with rowsum > 1e-6 of (wx - pp)^2, part[1] = sum |grad x|
void launch_objective(const float* wx, const float* pp, const float* rowsum, int nwin, const float* x, int nx,
                      int ny, double* scratch, int nscratch, double* out2, cudaStream_t st);

}  // namespace roi
