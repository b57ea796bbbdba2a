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

#include <cmath>
#include <string>

struct roi_recon;  // the C ABI handle (capi.cu)

namespace roi {

// Float-float numbers (hi + lo, ~44 significant bits) built from error-free float
// transformations, used where GB300's FP64 rate (1/64 of FP32) would dominate a kernel.
struct ff {
    float hi, lo;
};
#if defined(__CUDACC__)
#define ROI_HD __host__ __device__ __forceinline__
#else
#define ROI_HD inline
#endif
ROI_HD ff ff_split(double v) {
    ff r;
    r.hi = (float)v;
    r.lo = (float)(v - (double)r.hi);
    return r;
}
// a + b exactly as hi + lo (Knuth's two-sum)
ROI_HD ff two_sum(float a, float b) {
    ff r;
    r.hi = a + b;
    const float bb = r.hi - a;
    r.lo = (a - (r.hi - bb)) + (b - bb);
    return r;
}
ROI_HD ff ff_add(ff a, ff b) {
    ff s = two_sum(a.hi, b.hi);
    s.lo += a.lo + b.lo;
    return two_sum(s.hi, s.lo);
}
// a * b for float a (exact product via fma) times float-float b
ROI_HD ff ff_mul_f(float a, ff b) {
    ff p;
    p.hi = a * b.hi;
    p.lo = fmaf(a, b.hi, -p.hi) + a * b.lo;
    return two_sum(p.hi, p.lo);
}
// Neumaier-compensated accumulation of v into (s, c)
ROI_HD void neu_add(float& s, float& c, float v) {
    const float t = s + v;
    c += fabsf(s) >= fabsf(v) ? (s - t) + v : (v - t) + s;
    s = t;
}

// Per-angle record of a ray set over a frame.  Frame-centre coordinates:
//   pixel (li, lj) of the frame (row, column) sits at xi = lj - (nx-1)/2,
//   eta = (ny-1)/2 - li relative to the frame centre; bin k of the window has
//   offset t_{d0+k} - T_frame = k + phi with T_frame = Xf c + Yf s.
// Forward (ray-driven): along ray k the sample at major index m (row when `row`,
// column otherwise) has minor coordinate  A0 + k a_scale + (m - (M-1)/2) slope.
// Back (pixel-driven): pixel (li, lj) sits at window coordinate
//   kappa = xi c + eta s - phi.
// The host computes every value in double and stores it as float-float.
struct AngleRec {
    ff c, s;           // cos(theta), sin(theta)
    ff phi;            // d0 - (N_d-1)/2 - T_frame
    ff A0;             // (Mm-1)/2 + a_scale * phi
    ff a_scale;        // 1/c (row branch) or -1/s (column branch)
    ff slope;          // s/c (row branch) or c/s (column branch)
    float inv_slope;   // 1/slope (unused when flat)
    float inv_w;       // 1 / |c| or 1 / |s|
    int row;           // 1: sample per row (|c| >= |s|), 0: per column
    int flat;          // 1: |slope| < 1e-12 (rays parallel to the sampling axis)
    int d0;            // first bin of the window
    int width;         // bins in the window (0 if no ray reaches the frame)
    int aidx;          // index of the angle in the sinogram (tables may be reordered)
    int slope_q22;     // round(slope 2^22): per-sample step of the fixed-point ray coordinate
    int c_q23, s_q23;  // round(c 2^23), round(s 2^23): per-pixel steps of the gather coordinate
};

// Fills the derived fields of `r` from doubles (host and device).
ROI_HD void angle_fill(AngleRec& r, int aidx, double c, double s, int row, double wd, int d0, int width, double phi,
                       int Mm) {
    r.aidx = aidx;
    r.c = ff_split(c);
    r.s = ff_split(s);
    r.row = row;
    r.inv_w = (float)(1.0 / wd);
    r.d0 = d0;
    r.width = width;
    r.phi = ff_split(phi);
    const double as = row ? 1.0 / c : -1.0 / s;
    const double sl = row ? s / c : c / s;
    r.a_scale = ff_split(as);
    r.slope = ff_split(sl);
    r.flat = fabs(sl) < 1e-12;
    r.inv_slope = r.flat ? 0.f : (float)(1.0 / sl);
    r.A0 = ff_split(0.5 * (Mm - 1) + as * phi);
    r.slope_q22 = (int)llrint(sl * 4194304.0);
    r.c_q23 = (int)llrint(c * 8388608.0);
    r.s_q23 = (int)llrint(s * 8388608.0);
}

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
// Box-frame table for the whole-region solvers: per-row-branch angles first (stable),
// aidx = sinogram index; *nrow = their count; returns the largest window width.
int plan_region_table(int N, int na, int nd, const double* angles, Rect box, AngleRec* out, int* nrow);

// ---------------------------------------------------------------- allocation
// Every device and page-locked host allocation of the library goes through these two, so
// that a test can make the n-th one fail as if memory had run out (roi_recon_test_fail_alloc).
cudaError_t dev_malloc(void** p, size_t bytes);
cudaError_t pinned_alloc(void** p, size_t bytes, unsigned flags);

// ----------------------------------------------------------------- launchers
// Process-wide count of kernels launched by the library.
void count_launches(unsigned n);
unsigned long long launches_total();

enum FwdMode { FWD_PLAIN = 0, FWD_EXTERIOR = 1, FWD_SIRT = 2, FWD_CP = 3 };
enum BackMode { BACK_PLAIN = 0, BACK_SIRT = 1, BACK_CP = 2 };

// Images read by the forward projector are "padded": element (0, 0) sits at `img`,
// rows have stride `img_ld` = extent + 4 rounded up to a multiple of 4 (16-byte rows,
// so whole images can be staged with 16-byte copies), and the columns left and right
// of each row (indices -2, -1 and extent .. ld - 3) hold zeros.
constexpr int kPad = 2;
ROI_HD int padded_ld(int extent) { return (extent + 2 * kPad + 3) / 4 * 4; }
// The same for elements of esz bytes (rows stay multiples of 16 bytes).
ROI_HD int padded_ld_e(int extent, int esz) {
    const int unit = 16 / esz;
    return (extent + 2 * kPad + unit - 1) / unit * unit;
}
// Bytes of a storage type: 0 float, 1 bfloat16, 2 half.
ROI_HD int dt_size(int dt) { return dt == 0 ? 4 : 2; }

struct FwdArgs {
    const AngleRec* rec;   // [na]
    int na, stride;        // window rows and their stride
    int nx, ny;            // frame size
    const void* img;       // frame image [ny][img_ld], padded (float, or dt for FWD_EXTERIOR)
    const void* imgT;      // its transpose [nx][imgT_ld], padded
    int img_ld, imgT_ld;
    int dt;                // FWD_EXTERIOR: storage of img and imgT (0 float, 1 bfloat16, 2 half)
    int pdt;               // FWD_EXTERIOR: storage of p
    int seg_len;           // set by launch_forward
    Rect hole;             // FWD_EXTERIOR: frame pixels treated as zero (w = 0: none)
    float* out;            // [na][stride]
    // FWD_EXTERIOR: out = p[a][d0 + k] - W_F x
    const void* p;         // [na][nd], storage pdt
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
    float* out;            // BACK_PLAIN: result; else x (in/out); row stride out_ld
    int out_ld;
    float* outT;           // optional transpose of the written image, row stride outT_ld, or null
    int outT_ld;
    float* part;           // angle-group partials [G][ny][nx] (G = back_groups) or null (G = 1)
    // BACK_SIRT: x = max(0, x + step * acc) (nonneg) with step = C ? C[pix] : step_scalar
    // BACK_CP:   x+ = x - tau (acc - div v); xbar = 2 x+ - x  (tau = C ? C[pix] : step_scalar)
    const float* C;        // [ny][nx]
    float step_scalar;
    int nonneg;
    const float* vx;       // BACK_CP: [ny][nx]
    const float* vy;
    float* xbar;           // BACK_CP: row stride xbar_ld (its transpose goes to outT)
    int xbar_ld;
    // BACK_PLAIN on the whole grid (frame = grid): > 0 restricts the result to the field of
    // view, the pixels whose centre lies within fov_d / 2 of the rotation axis (others 0)
    int fov_d;
};

// Work splits chosen from the sizes alone (results never depend on other work).
int forward_segments(int na, int stride, int nx, int ny, int* seg_len);
int back_groups(int na, int nx, int ny);

void launch_forward(FwdMode mode, const FwdArgs& a, cudaStream_t st);
void launch_back(BackMode mode, const BackArgs& a, cudaStream_t st);
// hodd[t] = s h_{2t+1}; ctail = s (h0 + 2 sum_{odd m < nd} h_m), s = pi / N_theta
void launch_ramp(const void* p, int dt, const float* hodd, float* q, int na, int nd, float ctail, cudaStream_t st);
// Storage conversions (dt: 0 float, 1 bfloat16, 2 half; round to nearest even):
// dst[i] = src[i] for n elements
void launch_convert(const void* src, int src_dt, void* dst, int dst_dt, size_t n, cudaStream_t st);
// dst [na][nd] (storage dst_dt) = src [na][nm] (src_dt) placed at bins [off, off + nm), the
// bins outside filled with the row's first / last measured value
void launch_pad_truncated(const void* src, int src_dt, int nm, void* dst, int dst_dt, int na, int nd, int off,
                          cudaStream_t st);
// dst (storage dt, padded rows of dst_ld, pads untouched) = src [rows][cols] float (row stride
// src_ld); transpose: dst[c][r] = src[r][c]
void launch_store_padded(const float* src, int src_ld, void* dst, int dst_dt, int dst_ld, int rows, int cols,
                         int transpose, cudaStream_t st);
// dst [rows][cols] float (row stride dst_ld) = src (storage dt, row stride src_ld)
void launch_load_padded(const void* src, int src_dt, int src_ld, float* dst, int dst_ld, int rows, int cols,
                        cudaStream_t st);
// out[c][r] = in[r][c] (row strides in_ld, out_ld)
void launch_transpose(const float* in, int in_ld, float* out, int out_ld, int rows, int cols, cudaStream_t st);
// out[r][c] = in[r][c] with row strides in_ld, out_ld (pads untouched)
void launch_copy_pad(const float* in, int in_ld, float* out, int out_ld, int rows, int cols, cudaStream_t st);
void launch_fill(float* p, float v, size_t n, cudaStream_t st);
void launch_window_ones(float* win, const AngleRec* rec, int na, int stride, cudaStream_t st);
// CP gradient dual: v = proj_{|v| <= lambda}(v + sigma_v grad xbar)
void launch_cp_dual_grad(const float* xbar, int xbar_ld, float* vx, float* vy, int nx, int ny, float sigma_v,
                         float lambda, cudaStream_t st);
void launch_cp_dual_grad_dev(const float* xbar, int xbar_ld, float* vx, float* vy, int nx, int ny,
                             const float* sigma_dev, float lambda, cudaStream_t st);
// power iteration helpers for ||K||, K = [W_L; grad]
void launch_power_ktk_grad(float* y, const float* x, int x_ld, int nx, int ny, cudaStream_t st);
void launch_sumsq(const float* v, int n, double* scratch, int nscratch, double* out2, cudaStream_t st);
void launch_normalize(const float* y, float* x, int x_ld, float* xT, int xT_ld, int nx, int ny, const double* n2,
                      cudaStream_t st);
void launch_fill_step(float* dst, size_t n, const double* n2, double* L_out, cudaStream_t st);
// Preconditioners from row sums (window) and column sums (box):
//   mode 0 (SIRT weights): R = s > 1e-3 ? 1/s : 0, C likewise
//   mode 1 (CP diag):      sigma_u = s > 1e-6 ? 1/s : 0; tau = 1/(colsum + |grad| column count)
void launch_precond(float* rows, int nrows_total, float* cols, int nx, int ny, int mode, cudaStream_t st);
// out = x (box) with pixels outside the disk (cx, cy, r) in box-local coordinates set to 0 if crop
void launch_crop(const float* x, int x_ld, float* out, int nx, int ny, double cxl, double cyl, double r, int crop,
                 cudaStream_t st);
// objective terms: part[0] = sum over rows with rowsum > 1e-6 of (wx - pp)^2, part[1] = sum |grad x|
void launch_objective(const float* wx, const float* pp, const float* rowsum, int nwin, const float* x, int x_ld,
                      int nx, int ny, double* scratch, int nscratch, double* out2, cudaStream_t st);

// ---- the paper's own local method (Sec. 3), filtermethod.cu
void launch_disc_image(float* img, float* imgT, int ld, int N, cudaStream_t st);  // interior only
void launch_impulse(float* img, float* imgT, int ld, int N, cudaStream_t st);     // whole padded rows
void launch_row_sums(const float* s, int rows, int cols, double* out, cudaStream_t st);
void launch_disc_subtract(const void* p, int dt, const float* wd, float g, float* pd, size_t n, cudaStream_t st);
void launch_filter_accum(const float* hc, double* hq, float* uk, int na, int nd, int ndp, double alpha,
                         cudaStream_t st);
void launch_axpy_padded(float* c, float* cT, int ld, const float* g, float alpha, int N, cudaStream_t st);
void launch_filter_conv(const float* u, const float* pd, float* Cp, int n, int na, int nd, cudaStream_t st);
// The same on the tensor cores (filterconv_tc.cu): the filter bank packed once into its
// tf32 head/remainder core-matrix layout (filter_pack_tc_floats floats), then one launch of
// at most `sms` blocks.  filter_conv_tc_fits: the sinogram row's expansion and two stages
// fit in shared memory (N_d up to about 2500 with 200 filters).  A device wait that runs out sets *err;
// test_extra_tx > 0 (testing only) makes every stage wait for that many bytes more than
// are copied, so the waits run out.
bool filter_conv_tc_fits(int n, int nd);
size_t filter_pack_tc_floats(int n, int na, int nd);
void launch_filter_pack_tc(const float* u, float* ug, int n, int na, int nd, cudaStream_t st);
cudaError_t launch_filter_conv_tc(const float* ug, const float* pd, float* Cp, int n, int na, int nd, int sms,
                                  int* err, unsigned long long wait_ns, unsigned test_extra_tx, cudaStream_t st);
void launch_window_gather(const float* Cp_k, int nd, const AngleRec* rec, int na, int stride, float* win,
                          cudaStream_t st);
void launch_filter_update(const float* xs, const float* g, float* y, float* x, const float* shift, float lo, float hi,
                          float alpha, float* ya, int lda, float* yaT, int ldaT, int nx, int ny, cudaStream_t st);
void launch_disc_box(float* shift, int x0, int y0, int nx, int ny, int N, float g, cudaStream_t st);
void launch_add(const float* x, const float* shift, float* out, size_t n, cudaStream_t st);
// Tiling: a host-filled table of tiles (tile_src_fill into tile_src_bytes() * n bytes, copied
// to the device) pasted into out [N][N].
size_t tile_src_bytes();
void tile_src_fill(void* dst, int k, const float* box, int bw, int tx, int ty, int gx, int gy);
void launch_paste_tiles(const void* tiles_dev, int ntiles, int T, float* out, int N, cudaStream_t st);

// ---- single-launch (cooperative) solver for boxes whose padded image fits in shared memory
struct PersistLaunch {
    const AngleRec* rec;
    int na, stride, nx, ny;
    int mode;                 // 0 SIRT (nonneg, x in xa), 1 CP (x in x, xbar in xa)
    int iters;
    float* xa_base;           // padded row image buffer (row 0, column -2)
    float* xaT_base;          // padded column image buffer
    float* u;
    const float* pp;
    const float* R;
    float sig_scalar;
    float* x;
    float* vx;
    float* vy;
    const float* C;
    float step_scalar;
    const float* sigma_v_dev;
    float sigma_v;
    float lambda;
    int nonneg;
    unsigned* bar;            // 2 unsigned, zeroed by the launcher
    int* err;                 // set to 1 when a barrier wait gives up
    unsigned long long wait_ns;
    int blocks;               // <= persist_max_blocks
    int phantoms;             // extra barrier participants that never arrive (testing only)
};
size_t persist_smem_bytes(int na, int nx, int ny, int blocks);
int persist_max_blocks(int na, int nx, int ny, int stride, int device);
cudaError_t launch_persist(const PersistLaunch& L, cudaStream_t st);

// ---- how the whole-region solvers read a box image in the forward projection
// (a function of the box size alone, so a region's result never depends on where it
// is solved): 0 = the whole padded image staged in shared memory by one bulk copy
// (by every block of a team); 1 = streamed
// through shared memory in bands of band_rows() rows (as many as two buffers in
// kStageMaxBytes hold, a multiple of 8, from kBandRowsMin to kBandRowsMax),
// double-buffered; 2 = read from global memory.
constexpr size_t kStageMaxBytes = 200 * 1024;
// Shared memory past the band buffers for the per-ray partial sums of band-streamed phase A
// when a block has more ray units than warps (up to kBandStateBytes / 256 units per pass).
constexpr size_t kBandStateBytes = 24 * 1024;
constexpr int kBandRowsMin = 24;
constexpr int kBandRowsMax = 96;
ROI_HD int band_rows(int nx, int ny, int esz) {
    const size_t lr = (size_t)padded_ld_e(nx, esz), lc = (size_t)padded_ld_e(ny, esz);
    size_t rows = kStageMaxBytes / ((size_t)esz * 2 * (lr > lc ? lr : lc)) / 8 * 8;
    return (int)(rows > (size_t)kBandRowsMax ? (size_t)kBandRowsMax : rows);
}
ROI_HD int stage_mode(int nx, int ny, int esz) {
    const size_t lr = (size_t)padded_ld_e(nx, esz), lc = (size_t)padded_ld_e(ny, esz);
    const size_t full = (size_t)esz * (ny * lr > nx * lc ? ny * lr : nx * lc);
    if (full <= kStageMaxBytes) return 0;
    return band_rows(nx, ny, esz) >= kBandRowsMin ? 1 : 2;
}
// Dynamic shared memory the staging of a box of nx x ny (elements of esz bytes) needs.
ROI_HD size_t stage_bytes(int nx, int ny, int esz) {
    const size_t lr = (size_t)padded_ld_e(nx, esz), lc = (size_t)padded_ld_e(ny, esz);
    const int m = stage_mode(nx, ny, esz);
    if (m == 0) return (size_t)esz * (ny * lr > nx * lc ? ny * lr : nx * lc);
    if (m == 1) return (size_t)esz * 2 * band_rows(nx, ny, esz) * (lr > lc ? lr : lc);
    return 0;
}

// ---- phase B tile shapes of the whole-region solvers, chosen per box-size class: boxes
// of side <= 96, <= 216 (padded image staged whole), and larger (band-streamed)
constexpr int kTileShapes = 3;
constexpr int kShapeClasses = 3;
ROI_HD int shape_class(int side) { return side <= 96 ? 0 : (side <= 216 ? 1 : 2); }

// ---- whole-region solves by one block (batched) or a team of blocks (serving)
struct BatchRoi {
    const AngleRec* rec;   // box-frame table, per-row-branch angles first
    float* out;            // result [ny][nx] (device, or page-locked host memory mapped)
    int na, nrow;          // angles; the first nrow sample per row
    int nx, ny, stride;
    int reg, iters, weighting;
    float lambda, sigma_v;
    float alpha;           // SIRT scalar step 1/(N_theta N_d)
    int crop;
    float cxl, cyl, r2;    // disk crop in box coordinates
    // exterior inputs: p' = resid + W_L (box of x_fbp)
    const float* resid;    // p - W x_fbp over every ray [N_theta][resid_ld] (original angle order)
    int resid_ld;
    const void* xfbp;      // padded grid image (storage dt), element (0,0), row stride xfbp_ld
    const void* xfbpT;     // its padded transpose, same stride
    int xfbp_ld;
    int box_x0, box_y0;
    int dt;                // storage of x_fbp and of the solver's projector images xa / xaT
    // reg = 2, the paper's own method (Sec. 3): filtered sinograms C_{u_k} p_d of the whole
    // detector, [iters][N_theta][fcp_nd], and the disc added back (grey value, grid size)
    const float* fcp;
    int fcp_nd;
    float disc_g;
    int grid_n;
    // reg = 3, Alg. methodfista: FGP iterations and weight (lam_f = alpha lambda / 2)
    int n_fgp;
    float lam_f;
    int shape;             // phase B tile shape (0: 16 x 16, 1: 8 x 8, 2: 16 x 8)
};

struct BatchArgs {
    const BatchRoi* rois;
    const int* order;      // solve order (largest first)
    int nroi;
    int* queue;            // zeroed by the launcher
    float* slot_pp;        // per-block windows and box buffers
    float* slot_u;
    float* slot_sig;
    size_t win_cap;
    float* slot_x;
    float* slot_vx;
    float* slot_vy;
    float* slot_tau;
    size_t img_cap;
    float* slot_xa;        // padded images (row / column), from row 0 column -2
    float* slot_xaT;
    size_t pad_cap;
    float* slot_fgp;       // 5 img_cap per slot when a region uses reg = 3, else null
    float* slot_part;      // per-band ray partial sums of a lone box's team (row-band phase A), else null
    size_t part_cap;
    int* err;
    unsigned long long wait_ns;
    int team;              // blocks per region: 1, or > 1 for a cooperative launch of teams
    unsigned* bars;        // team > 1: one barrier counter per team (zeroed by the launcher)
    int absent;            // testing only: barrier participants per team that never arrive
};
// Device buffers of one whole-region solve: windows [na][stride]; box arrays [ny][nx];
// padded images from row 0 column -kPad, row strides padded_ld(nx) / padded_ld(ny).
struct RegionBufs {
    float* pp;
    float* u;
    float* sig;
    float* x;
    float* vx;
    float* vy;
    float* tau;
    void* xa_base;         // storage dt of the region (float, bfloat16 or half)
    void* xaT_base;
    float* fgp;            // reg = 3: FGP state, 5 box arrays (v_x, v_y, r_x, r_y, x)
    float* part;           // a band-streamed box on a large team: [band][unit][32] partial ray sums
                           // per branch (rows first), else null (see phase_a_rowband)
};

// ---- serving: one cooperative launch whose blocks take requests from rings in
// page-locked host memory (mapped), published by the host while the kernel runs.
// A ring slot holds a ServeSlot followed (at serve_slot_header_bytes) by the request's
// box-frame table of `na` AngleRec.
struct ServeSlot {
    BatchRoi roi;                  // rec is replaced on the device by the block's copy
    RegionBufs bufs;
    unsigned long long seq;        // ticket + 1, written to done[slot] on completion
};
constexpr size_t serve_slot_header_bytes = (sizeof(ServeSlot) + 255) / 256 * 256;

struct ServePool {
    const unsigned char* ring;     // device view of the ring
    unsigned long long slot_bytes;
    int slots;
    int first_block, team, nteams, team_base;
    unsigned long long* head;      // device memory: next ticket to claim
    const unsigned long long* tail;  // device view of the host-written count of published tickets
    unsigned long long* done;      // device view of the per-slot completion words
};

struct ServeArgs {
    ServePool pool[2];             // 0: requests solved by one block, 1: by a team of blocks
    const int* close;              // device view of the host's close flag
    int* busy;                     // requests being solved (device memory)
    unsigned long long* last_ns;   // time of the last claim or completion
    unsigned* bars;                // team barriers, one per team (both pools), zeroed at launch
    unsigned* mail_seq;            // leader -> members claim mailboxes, zeroed at launch
    long long* mail_val;
    AngleRec* rec_slots;           // per-block private copies of the request table [grid][max_na]
    int max_na;
    unsigned long long idle_ns;    // leave when nothing was claimed or finished for this long and nothing runs
    unsigned long long cap_ns;     // longest poll of one block
    int* err;
    unsigned long long wait_ns;
    // testing only: > 0 barrier participants per team that never arrive; < 0 the team
    // leaders stay away (members' mailbox waits run out)
    int absent;
    // solo launches (one team of every block): per-band ray partial sums for the row-band
    // phase A of band-streamed boxes, when the request's fit in solo_part_cap floats
    float* solo_part;
    size_t solo_part_cap;
};
size_t serve_smem_bytes();
int serve_max_blocks(int device);  // co-resident blocks of the serving kernel
cudaError_t launch_serve(const ServeArgs& A, int blocks, cudaStream_t st);

// A resident sinogram as seen by the server (pointers into a roi_recon handle).
struct SinoView {
    int N, na, nd;
    const double* angles;
    bool have_fbp;         // exterior-step solvers available
    const float* fcp;      // filtered sinograms of the paper's own method, fcp_n iterations
    int fcp_n;
    float disc_g;
    const void* xfbp;
    const void* xfbpT;
    int xfbp_ld;
    int dt;
    const float* resid;
    int resid_ld;
    int shape[kShapeClasses];  // tile shape per box-size class (the handle's table)
};

int sino_view(::roi_recon* h, SinoView* v, std::string* msg);

size_t batch_smem_bytes(size_t max_stage_bytes, int na, bool banded);
cudaError_t launch_batch(const BatchArgs& B, int blocks, size_t smem, cudaStream_t st);
cudaError_t launch_batch_team(const BatchArgs& B, int blocks, size_t smem, cudaStream_t st);

// ---- check build (-DROI_CHECK): index checks of the hot kernels, one report per
// translation unit; the product build's reports are always empty.
struct CheckReport {
    int count;          // indices found out of range
    int site, index;    // the first one: its site (CheckSite) and value
    int lo, hi;         // and its range
};
void check_take_persist(CheckReport* out);
void check_take_batch(CheckReport* out);
void check_take_batch_team(CheckReport* out);
void check_take_serve(CheckReport* out);
void check_take_project(CheckReport* out);
void check_take_filterconv_tc(CheckReport* out);

}  // namespace roi
