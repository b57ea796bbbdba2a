// capi.cu -- the roi_recon C ABI: handle, resident data, ROI workspace and the local
// pipeline (global FBP -> exterior subtraction -> local SIRT / Chambolle-Pock TV).
//
// Paper: Sec. 1 (exterior-subtraction ROI scheme), Sec. 2.1 (W, W_L, W_F, Eq. locouter),
// Sec. 2.2 (Eq. fbp, Eq. sirtit), Sec. 2.3 (Eq. priorsys, Eq. sirtbox), Sec. 3.1 (alpha).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <array>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "roi_recon.h"
#include "roi_internal.h"

using roi::AngleRec;
using roi::Rect;

namespace roi {
static std::atomic<unsigned long long> g_launches{0};
void count_launches(unsigned n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
unsigned long long launches_total() { return g_launches.load(std::memory_order_relaxed); }

// Allocation failure injection (testing): > 0 counts down the allocations still to succeed
// plus one; the allocation that brings it to zero fails without allocating.
static std::atomic<long long> g_fail_alloc{0};
static bool injected_failure() {
    long long v = g_fail_alloc.load(std::memory_order_relaxed);
    while (v > 0) {
        if (g_fail_alloc.compare_exchange_weak(v, v - 1, std::memory_order_relaxed)) return v == 1;
    }
    return false;
}
cudaError_t dev_malloc(void** p, size_t bytes) {
    *p = nullptr;
    if (injected_failure()) return cudaErrorMemoryAllocation;
    return cudaMalloc(p, bytes);
}
cudaError_t pinned_alloc(void** p, size_t bytes, unsigned flags) {
    *p = nullptr;
    if (injected_failure()) return cudaErrorMemoryAllocation;
    return cudaHostAlloc(p, bytes, flags);
}
}  // namespace roi

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr int kRedScratch = 2 * 152;   // doubles of reduction scratch (152 block partials x 2)

template <class T>
cudaError_t dev_alloc(T** p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    return roi::dev_malloc((void**)p, sizeof(T) * count);
}

// Grow-only device buffer.
template <class T>
struct DevBufT {  // grow-only device array of T, freed when it goes out of scope
    T* p = nullptr;
    size_t cap = 0;
    DevBufT() = default;
    DevBufT(const DevBufT&) = delete;
    DevBufT& operator=(const DevBufT&) = delete;
    ~DevBufT() { release(); }
    cudaError_t ensure(size_t n) {
        if (n <= cap) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
        cudaError_t e = dev_alloc(&p, n);
        if (e == cudaSuccess) cap = n;
        return e;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
    }
};
using DevBuf = DevBufT<float>;

// Device buffers of a batched launch: per-region angle tables, descriptors and order, the
// launch's queue and team barriers, one slot of solver state per block (or per team).  The
// handle has one set; a batch plan owns another, so that its captured launch never sees the
// buffers of a later batch.
struct BatchBufs {
    DevBufT<AngleRec> tab;
    DevBuf out;
    DevBufT<roi::BatchRoi> rois;
    DevBufT<int> order;
    DevBufT<int> queue;
    DevBufT<unsigned> bars;
    DevBuf pp, u, sig, x, vx, vy, tau, xa, xaT, fgp;
    DevBuf part;  // per-band ray partial sums of a band-streamed box on a team of every block
};

}  // namespace

namespace {
// Tile tables found by roi_recon_autotune, per geometry (grid, angles, detector, image
// storage), for the handles created afterwards.
struct TuneKey {
    int N, na, nd, dt;
    unsigned long long angles;  // FNV-1a of the angle array
    bool operator<(const TuneKey& o) const {
        return std::tie(N, na, nd, dt, angles) < std::tie(o.N, o.na, o.nd, o.dt, o.angles);
    }
};
struct TuneVal {
    std::array<int, roi::kShapeClasses> shape;  // phase B tile shape per box-size class
    std::array<int, roi::kShapeClasses> team;   // largest team of a few-region batch, per class
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneVal> g_tune;

unsigned long long fnv_doubles(const std::vector<double>& v) {
    unsigned long long h = 1469598103934665603ull;
    const unsigned char* b = reinterpret_cast<const unsigned char*>(v.data());
    for (size_t i = 0; i < v.size() * sizeof(double); ++i) h = (h ^ b[i]) * 1099511628211ull;
    return h;
}
}  // namespace

struct roi_recon {
    int N = 0, na = 0, nd = 0;
    std::vector<double> angles;
    cudaStream_t st = nullptr;
    std::string err;
    // resident data: the sinogram stored as pdt, the FBP image and the projector images of
    // whole-region solves as dt (0 float, 1 bfloat16, 2 half; pesz / esz bytes an element)
    int dt = 0, esz = 4;
    int pdt = 0, pesz = 4;
    void* p = nullptr;       // [na][nd], storage pdt
    float* q = nullptr;      // [na][nd] filtered sinogram (float)
    void* xfbp = nullptr;    // [N][N] padded (row stride xld), element (0,0)
    void* xfbpT = nullptr;   // its transpose, padded
    unsigned char* xfbp_base = nullptr;
    unsigned char* xfbpT_base = nullptr;
    int xld = 0;             // padded_ld_e(N, esz)
    DevBuf fbp32;            // 16-bit image storage: the float FBP image before narrowing [N][N]
    DevBufT<unsigned char> in_tmp;  // set_sinogram input awaiting conversion
    float* hodd = nullptr;   // Ram-Lak odd taps scaled by pi/na, [nd/2 + 1]
    float ctail = 0.f;       // (pi/na) (h0 + 2 sum_{odd m < nd} h_m)
    AngleRec* rec_fbp = nullptr;  // frame = grid, window = whole detector
    bool have_sino = false, have_fbp = false;
    // ROI plan cache
    bool plan_valid = false;
    roi_region plan_region{};
    Rect box{};
    int wmax = 0, stride = 0;
    std::vector<AngleRec> h_loc, h_ext;
    AngleRec* rec_loc = nullptr;  // frame = box
    AngleRec* rec_ext = nullptr;  // frame = grid, window of the box
    // ROI workspace: window buffers [na][stride]; box buffers [h][w]; the two images
    // the forward projector reads (xa: row layout, xaT: transposed) are padded
    DevBuf pp, u, sig, wtmp, wrow;
    DevBuf xc, vx, vy, tau, itmp;
    DevBuf xa, xaT;
    DevBuf part;             // angle-group partials of the gather
    double* red = nullptr;   // kRedScratch partials + 4 results
    int exterior_ready = 0;  // p' in `pp` matches the cached plan and FBP
    // iterate state of the last solve_local (checkpoint / resume)
    bool state_valid = false;
    bool state_region_path = false;  // the last solve_local ran in the whole-region solver
    int state_reg = 0, state_flag = 0;
    double state_lambda = 0.0;
    long long state_iters = 0;
    const unsigned char* resume = nullptr;  // state being resumed from, during solve_local_resume
    int resume_on_device = 0;
    long long resume_iters = 0;
    // optional kernel timing: event pairs per kernel class (0 forward, 1 back, 2 single-launch solve)
    bool timing = false;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> spans[4];
    // single-launch solver: barrier words, device error flag, options
    unsigned* d_bar = nullptr;
    int* d_err = nullptr;
    int device = 0;
    int opt_persistent = 1;
    int opt_tile_shape = -1;              // >= 0: phase B tile shape for every region
    int tile_shape[roi::kShapeClasses] = {0, 0, 0};  // per box-size class (roi_recon_autotune)
    int team_cap[roi::kShapeClasses] = {16, 16, 16};  // largest team per region of a few-region batch
    double team_ms[roi::kShapeClasses][4] = {};       // the autotuner's timings of the team candidates
    unsigned long long opt_wait_ns = 1000000000ull;
    int opt_phantoms = 0;
    int opt_filter_fma = 0;               // 1: filtered sinograms on the FMA pipe (not the tensor cores)
    size_t max_smem_optin = 0;
    int sms = 0;
    // batched solves: per-region tables / windows / descriptors, per-block slots, pinned staging
    BatchBufs bb;
    std::vector<roi_batch_plan*> plans;  // live batch plans (destroyed with the handle)
    // residual p - W x_fbp over every ray, [na][resid_ld] (exterior step of the
    // whole-region solvers, Eq. locouter); valid while resid_ready
    DevBuf resid;
    int resid_ld = 0;
    int resid_ready = 0;
    // the paper's own local method (Sec. 3): filters (geometry), disc subtraction and
    // filtered sinograms (current sinogram)
    int filt_n = 0;                 // filters u_1..u_filt_n in filt_u
    DevBuf filt_u;                  // [filt_n][na][2 nd - 1]
    AngleRec* rec_filt = nullptr;   // frame = grid, full detector of the filter bins
    int fcp_n = 0;                  // filtered sinograms C_{u_k} p_d, k = 1..fcp_n, in filt_cp
    DevBuf filt_cp;                 // [fcp_n][na][nd]
    DevBuf filt_pd;                 // disc-subtracted sinogram [na][nd]
    DevBuf filt_ug;                 // filt_u packed for the tensor cores (filt_ug_n filters)
    int filt_ug_n = 0;
    DevBuf op_ug;                   // scratch of roi_recon_filter_conv
    double disc_g = 0.0;
    unsigned char* pin = nullptr;  // page-locked staging of the uploads
    size_t pin_cap = 0;
    cudaEvent_t pin_free = nullptr;  // recorded after the last upload from `pin`
};

namespace {

roi_status fail(roi_recon* h, roi_status s, const char* fmt, ...) __attribute__((format(printf, 3, 4)));
roi_status fail(roi_recon* h, roi_status s, const char* fmt, ...) {
    if (h) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        h->err = buf;
    }
    return s;
}

roi_status cuda_fail(roi_recon* h, cudaError_t e, const char* where) {
    const roi_status s = (e == cudaErrorMemoryAllocation) ? ROI_ENOMEM : ROI_ECUDA;
    return fail(h, s, "%s: %s", where, cudaGetErrorString(e));
}

#define CU(h, call)                                        \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, #call); \
    } while (0)

#define LAUNCHED(h, what)                                         \
    do {                                                          \
        cudaError_t e_ = cudaGetLastError();                      \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, what);     \
    } while (0)

cudaEvent_t take_event(roi_recon* h) {
    if (h->ev_used == h->ev_pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        h->ev_pool.push_back(e);
    }
    return h->ev_pool[h->ev_used++];
}

// RAII span: records an event pair around one kernel launch when timing is on
struct Span {
    roi_recon* h;
    int cls;
    cudaEvent_t a = nullptr;
    Span(roi_recon* h_, int cls_) : h(h_), cls(cls_) {
        if (h->timing && (a = take_event(h))) cudaEventRecord(a, h->st);
    }
    ~Span() {
        if (a) {
            cudaEvent_t b = take_event(h);
            if (b) {
                cudaEventRecord(b, h->st);
                h->spans[cls].push_back({a, b});
            }
        }
    }
};

bool finite_region(const roi_region* r) {
    return std::isfinite(r->cx) && std::isfinite(r->cy) && std::isfinite(r->radius) && std::isfinite(r->margin) &&
           r->radius > 0 && r->margin >= 0 && r->radius + r->margin < 1e7;
}

bool same_region(const roi_region& a, const roi_region& b) {
    return a.cx == b.cx && a.cy == b.cy && a.radius == b.radius && a.margin == b.margin;
}

roi_status check_geometry(const roi_geometry* g) {
    if (!g) return ROI_EINVAL;
    if (g->n_pix < 1 || g->n_angles < 1 || g->n_det < 1) return ROI_EINVAL;
    if (g->n_pix > 65536 || g->n_angles > 65536 || g->n_det > 8192) return ROI_EINVAL;
    if (g->storage != ROI_F32 && g->storage != ROI_BF16 && g->storage != ROI_F16) return ROI_EINVAL;
    if (g->image_storage != ROI_F32 && g->image_storage != ROI_BF16 && g->image_storage != ROI_F16)
        return ROI_EINVAL;
    if (g->angles)
        for (int a = 0; a < g->n_angles; ++a)
            if (!std::isfinite(g->angles[a])) return ROI_EINVAL;
    return ROI_OK;
}

std::vector<double> make_angles(const roi_geometry* g) {
    std::vector<double> a(g->n_angles);
    for (int i = 0; i < g->n_angles; ++i) a[i] = g->angles ? g->angles[i] : i * kPi / g->n_angles;
    return a;
}

// Plan `region` (box, windows) and upload the per-angle tables; grows the workspace.
roi_status ensure_plan(roi_recon* h, const roi_region* region) {
    if (!finite_region(region)) return fail(h, ROI_EINVAL, "region: radius must be > 0, margin >= 0, all finite");
    if (h->plan_valid && same_region(h->plan_region, *region)) return ROI_OK;
    Rect box;
    if (!roi::plan_box(h->N, region->cx, region->cy, region->radius, region->margin, &box))
        return fail(h, ROI_EINVAL, "region: extended box does not intersect the %d x %d grid", h->N, h->N);
    h->plan_valid = false;
    h->exterior_ready = 0;
    h->state_valid = false;  // the solver buffers belong to another box now
    h->state_region_path = false;
    h->h_loc.resize(h->na);
    h->h_ext.resize(h->na);
    const Rect grid{0, 0, h->N, h->N};
    const int wl = roi::plan_angles(h->N, h->na, h->nd, h->angles.data(), box, box, false, h->h_loc.data());
    roi::plan_angles(h->N, h->na, h->nd, h->angles.data(), grid, box, false, h->h_ext.data());
    const int stride = roi::round_stride(wl);
    const size_t nwin = (size_t)h->na * stride, nimg = (size_t)box.w * box.h;
    DevBuf* wins[] = {&h->pp, &h->u, &h->sig, &h->wtmp, &h->wrow};
    for (DevBuf* b : wins) CU(h, b->ensure(nwin));
    DevBuf* imgs[] = {&h->xc, &h->vx, &h->vy, &h->tau, &h->itmp};
    for (DevBuf* b : imgs) CU(h, b->ensure(nimg));
    const size_t npad = std::max((size_t)box.h * roi::padded_ld(box.w), (size_t)box.w * roi::padded_ld(box.h));
    CU(h, h->xa.ensure(npad));
    CU(h, h->xaT.ensure(npad));
    CU(h, h->part.ensure((size_t)roi::back_groups(h->na, box.w, box.h) * nimg));
    CU(h, cudaMemcpyAsync(h->rec_loc, h->h_loc.data(), sizeof(AngleRec) * h->na, cudaMemcpyHostToDevice, h->st));
    CU(h, cudaMemcpyAsync(h->rec_ext, h->h_ext.data(), sizeof(AngleRec) * h->na, cudaMemcpyHostToDevice, h->st));
    h->box = box;
    h->wmax = wl;
    h->stride = stride;
    h->plan_region = *region;
    h->plan_valid = true;
    return ROI_OK;
}

// Padded box images: element (0,0) of xa ([h][w + 4]) and xaT ([w][h + 4]).
int lda(const roi_recon* h) { return roi::padded_ld(h->box.w); }
int ldaT(const roi_recon* h) { return roi::padded_ld(h->box.h); }
float* xa0(roi_recon* h) { return h->xa.p + roi::kPad; }
float* xaT0(roi_recon* h) { return h->xaT.p + roi::kPad; }

// Zero both padded images (pads and interior).
roi_status clear_padded(roi_recon* h) {
    const size_t n1 = (size_t)h->box.h * lda(h), n2 = (size_t)h->box.w * ldaT(h);
    CU(h, cudaMemsetAsync(h->xa.p, 0, sizeof(float) * n1, h->st));
    CU(h, cudaMemsetAsync(h->xaT.p, 0, sizeof(float) * n2, h->st));
    return ROI_OK;
}

// Load an unpadded [h][w] image (device) into xa / xaT.
roi_status load_padded(roi_recon* h, const float* x) {
    roi_status s = clear_padded(h);
    if (s != ROI_OK) return s;
    roi::launch_copy_pad(x, h->box.w, xa0(h), lda(h), h->box.h, h->box.w, h->st);
    roi::launch_transpose(x, h->box.w, xaT0(h), ldaT(h), h->box.h, h->box.w, h->st);
    return ROI_OK;
}

void fill_info(const roi_recon* h, roi_solve_info* info) {
    info->box_x0 = h->box.x0;
    info->box_y0 = h->box.y0;
    info->box_w = h->box.w;
    info->box_h = h->box.h;
    info->window_max = h->wmax;
    info->window_stride = h->stride;
}

// Forward over the box reading the padded images xa / xaT.
roi::FwdArgs fwd_local(roi_recon* h, float* out) {
    roi::FwdArgs a{};
    a.rec = h->rec_loc;
    a.na = h->na;
    a.stride = h->stride;
    a.nx = h->box.w;
    a.ny = h->box.h;
    a.img = xa0(h);
    a.imgT = xaT0(h);
    a.img_ld = lda(h);
    a.imgT_ld = ldaT(h);
    a.out = out;
    a.nd = h->nd;
    return a;
}

// Gather over the box into `out` (row stride out_ld), optionally its transpose.
roi::BackArgs back_local(roi_recon* h, const float* win, float* out, int out_ld, float* outT, int outT_ld) {
    roi::BackArgs b{};
    b.rec = h->rec_loc;
    b.na = h->na;
    b.stride = h->stride;
    b.nx = h->box.w;
    b.ny = h->box.h;
    b.win = win;
    b.out = out;
    b.out_ld = out_ld;
    b.outT = outT;
    b.outT_ld = outT_ld;
    b.part = h->part.p;
    return b;
}

// Row sums W_L 1 into h->wrow and column sums W_L^T 1 into `cols` (uses xa / xaT).
roi_status rowcol_sums(roi_recon* h, float* cols) {
    const size_t nimg = (size_t)h->box.w * h->box.h;
    roi::launch_fill(h->itmp.p, 1.f, nimg, h->st);
    roi_status s = load_padded(h, h->itmp.p);
    if (s != ROI_OK) return s;
    roi::launch_forward(roi::FWD_PLAIN, fwd_local(h, h->wrow.p), h->st);
    roi::launch_window_ones(h->wtmp.p, h->rec_loc, h->na, h->stride, h->st);
    roi::launch_back(roi::BACK_PLAIN, back_local(h, h->wtmp.p, cols, h->box.w, nullptr, 0), h->st);
    LAUNCHED(h, "row/column sums");
    return ROI_OK;
}

// Residual p - W x_fbp of every ray (full detector, no hole), computed once per FBP.
roi_status ensure_residual(roi_recon* h) {
    if (h->resid_ready) return ROI_OK;
    h->resid_ld = roi::round_stride(h->nd);
    CU(h, h->resid.ensure((size_t)h->na * h->resid_ld));
    roi::FwdArgs a{};
    a.rec = h->rec_fbp;
    a.na = h->na;
    a.stride = h->resid_ld;
    a.nx = h->N;
    a.ny = h->N;
    a.img = h->xfbp;
    a.imgT = h->xfbpT;
    a.img_ld = h->xld;
    a.imgT_ld = h->xld;
    a.dt = h->dt;
    a.pdt = h->pdt;
    a.hole = Rect{0, 0, 0, 0};
    a.out = h->resid.p;
    a.p = h->p;
    a.nd = h->nd;
    roi::launch_forward(roi::FWD_EXTERIOR, a, h->st);
    LAUNCHED(h, "residual reprojection");
    h->resid_ready = 1;
    return ROI_OK;
}

// The exterior inputs of a whole-region solve (pointers into the handle).
void exterior_inputs(const roi_recon* h, roi::BatchRoi& R, Rect box) {
    R.resid = h->resid.p;
    R.resid_ld = h->resid_ld;
    R.xfbp = h->xfbp;
    R.xfbpT = h->xfbpT;
    R.xfbp_ld = h->xld;
    R.dt = h->dt;
    R.box_x0 = box.x0;
    R.box_y0 = box.y0;
    R.alpha = (float)(1.0 / ((double)h->na * h->nd));
}

// The inputs of the paper's own method (reg 2) for a whole-region solve.
void filter_inputs(const roi_recon* h, roi::BatchRoi& R) {
    R.fcp = h->filt_cp.p;
    R.fcp_nd = h->nd;
    R.disc_g = (float)h->disc_g;
    R.grid_n = h->N;
}

roi_status run_exterior(roi_recon* h) {
    roi::FwdArgs a{};
    a.rec = h->rec_ext;
    a.na = h->na;
    a.stride = h->stride;
    a.nx = h->N;
    a.ny = h->N;
    a.img = h->xfbp;
    a.imgT = h->xfbpT;
    a.img_ld = h->xld;
    a.imgT_ld = h->xld;
    a.dt = h->dt;
    a.pdt = h->pdt;
    a.hole = h->box;
    a.out = h->pp.p;
    a.p = h->p;
    a.nd = h->nd;
    roi::launch_forward(roi::FWD_EXTERIOR, a, h->st);
    LAUNCHED(h, "exterior reprojection");
    h->exterior_ready = 1;
    return ROI_OK;
}

// SIRT iterates x in the padded image xa (and its transpose xaT) that the forward reads.
// Whether the single-launch solver can run this box; fills blocks.
bool persist_ok(roi_recon* h, int* blocks) {
    if (!h->opt_persistent) return false;
    *blocks = roi::persist_max_blocks(h->na, h->box.w, h->box.h, h->stride, h->device);
    return *blocks > 0;
}

roi::PersistLaunch persist_base(roi_recon* h, int mode, int iters, int blocks) {
    roi::PersistLaunch L{};
    L.rec = h->rec_loc;
    L.na = h->na;
    L.stride = h->stride;
    L.nx = h->box.w;
    L.ny = h->box.h;
    L.mode = mode;
    L.iters = iters;
    L.xa_base = h->xa.p;
    L.xaT_base = h->xaT.p;
    L.u = h->u.p;
    L.pp = h->pp.p;
    L.bar = h->d_bar;
    L.err = h->d_err;
    L.wait_ns = h->opt_wait_ns;
    L.blocks = blocks;
    L.phantoms = h->opt_phantoms;
    return L;
}

// Checkpoint layout: this header, then float32 arrays -- SIRT: x; CP: x, xbar, vx, vy
// ([box_h][box_w] each) and the data dual u ([n_angles][window_stride]).
struct StateHeader {
    char magic[8];
    int reg, flag;  // regularizer; SIRT weighting / CP precond
    int box_x0, box_y0, box_w, box_h;
    int na, stride;
    long long iters_done;
    double lambda;
    int reserved[2];
};
static_assert(sizeof(StateHeader) == 64, "the state header is 64 bytes");
constexpr char kStateMagic[8] = {'R', 'O', 'I', 'S', 'T', 'A', 'T', '1'};

size_t state_bytes_for(int reg, int nx, int ny, int na, int stride) {
    const size_t nimg = (size_t)nx * ny, nwin = (size_t)na * stride;
    return sizeof(StateHeader) + sizeof(float) * (reg == ROI_SIRT_NONNEG ? nimg : 4 * nimg + nwin);
}

// The iterate state being resumed from into the solver buffers (SIRT: x into the padded
// images; CP: x, vx, vy, u, and xbar into the padded images).
roi_status resume_load(roi_recon* h, bool cp) {
    const size_t nimg = (size_t)h->box.w * h->box.h, nwin = (size_t)h->na * h->stride;
    const cudaMemcpyKind k = h->resume_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const unsigned char* src = h->resume + sizeof(StateHeader);
    if (cp) {
        CU(h, cudaMemcpyAsync(h->xc.p, src, sizeof(float) * nimg, k, h->st));
        src += sizeof(float) * nimg;
    }
    CU(h, cudaMemcpyAsync(h->itmp.p, src, sizeof(float) * nimg, k, h->st));  // x (SIRT) or xbar (CP)
    src += sizeof(float) * nimg;
    if (cp) {
        CU(h, cudaMemcpyAsync(h->vx.p, src, sizeof(float) * nimg, k, h->st));
        src += sizeof(float) * nimg;
        CU(h, cudaMemcpyAsync(h->vy.p, src, sizeof(float) * nimg, k, h->st));
        src += sizeof(float) * nimg;
        CU(h, cudaMemcpyAsync(h->u.p, src, sizeof(float) * nwin, k, h->st));
    }
    return load_padded(h, h->itmp.p);
}

roi_status solve_sirt(roi_recon* h, const roi_solve_params* prm) {
    const int nx = h->box.w, ny = h->box.h;
    const size_t nwin = (size_t)h->na * h->stride;
    const float* R = nullptr;
    const float* C = nullptr;
    if (prm->weighting) {
        roi_status s = rowcol_sums(h, h->tau.p);
        if (s != ROI_OK) return s;
        CU(h, cudaMemcpyAsync(h->sig.p, h->wrow.p, sizeof(float) * nwin, cudaMemcpyDeviceToDevice, h->st));
        roi::launch_precond(h->sig.p, (int)nwin, h->tau.p, nx, ny, 0, h->st);
        R = h->sig.p;
        C = h->tau.p;
    }
    roi_status s = h->resume ? resume_load(h, false) : clear_padded(h);  // x^0 = 0, or the state's x
    if (s != ROI_OK) return s;
    const float alpha = (float)(1.0 / ((double)h->na * h->nd));
    roi::FwdArgs fa = fwd_local(h, h->u.p);
    fa.pp = h->pp.p;
    fa.R = R;
    int blocks = 0;
    if (prm->iters > 0 && persist_ok(h, &blocks)) {
        roi::PersistLaunch L = persist_base(h, 0, prm->iters, blocks);
        L.R = R;
        L.C = C;
        L.step_scalar = alpha;
        L.nonneg = 1;
        cudaError_t e;
        {
            Span sp(h, 2);
            e = roi::launch_persist(L, h->st);
        }
        if (e != cudaSuccess) return cuda_fail(h, e, "single-launch SIRT solve");
        return ROI_OK;
    }
    roi::BackArgs ba = back_local(h, h->u.p, xa0(h), lda(h), xaT0(h), ldaT(h));
    ba.C = C;
    ba.step_scalar = alpha;
    ba.nonneg = 1;
    for (int it = 0; it < prm->iters; ++it) {
        {
            Span sp(h, 0);
            roi::launch_forward(roi::FWD_SIRT, fa, h->st);
        }
        {
            Span sp(h, 1);
            roi::launch_back(roi::BACK_SIRT, ba, h->st);
        }
    }
    LAUNCHED(h, "SIRT iterations");
    return ROI_OK;
}

roi_status power_norm(roi_recon* h, int iters) {
    // ||K||, K = [W_L; grad], by power iteration on K^T K from the normalised all-ones image;
    // the iterate lives in xa / xaT, K^T K x in itmp
    const int nx = h->box.w, ny = h->box.h;
    const size_t nimg = (size_t)nx * ny;
    const float v0 = (float)(1.0 / std::sqrt((double)nimg));
    roi::launch_fill(h->itmp.p, v0, nimg, h->st);
    roi_status s = load_padded(h, h->itmp.p);
    if (s != ROI_OK) return s;
    double* n2 = h->red + kRedScratch;
    for (int it = 0; it < iters; ++it) {
        roi::launch_forward(roi::FWD_PLAIN, fwd_local(h, h->wtmp.p), h->st);
        roi::launch_back(roi::BACK_PLAIN, back_local(h, h->wtmp.p, h->itmp.p, nx, nullptr, 0), h->st);
        roi::launch_power_ktk_grad(h->itmp.p, xa0(h), lda(h), nx, ny, h->st);
        roi::launch_sumsq(h->itmp.p, (int)nimg, h->red, kRedScratch, n2, h->st);
        roi::launch_normalize(h->itmp.p, xa0(h), lda(h), xaT0(h), ldaT(h), nx, ny, n2, h->st);
    }
    LAUNCHED(h, "power iteration");
    return ROI_OK;
}

roi_status solve_cp(roi_recon* h, const roi_solve_params* prm, double* L_out) {
    const int nx = h->box.w, ny = h->box.h;
    const size_t nimg = (size_t)nx * ny, nwin = (size_t)h->na * h->stride;
    const float* sigma_v_dev = nullptr;
    float sigma_v = 0.5f;
    if (prm->precond) {
        roi_status s = rowcol_sums(h, h->tau.p);
        if (s != ROI_OK) return s;
        CU(h, cudaMemcpyAsync(h->sig.p, h->wrow.p, sizeof(float) * nwin, cudaMemcpyDeviceToDevice, h->st));
        roi::launch_precond(h->sig.p, (int)nwin, h->tau.p, nx, ny, 1, h->st);
    } else {
        roi_status s = power_norm(h, 100);
        if (s != ROI_OK) return s;
        double* n2 = h->red + kRedScratch;
        roi::launch_fill_step(h->sig.p, nwin, n2, h->red + kRedScratch + 1, h->st);
        roi::launch_fill_step(h->tau.p, nimg, n2, nullptr, h->st);
        sigma_v_dev = h->sig.p;  // same scalar step
        *L_out = 1.0;            // marker: read back later
    }
    // x in xc; xbar in the padded xa (+ transpose xaT) that the forward reads
    roi_status s0;
    if (h->resume) {
        s0 = resume_load(h, true);
    } else {
        for (DevBuf* b : {&h->xc, &h->vx, &h->vy}) roi::launch_fill(b->p, 0.f, nimg, h->st);
        roi::launch_fill(h->u.p, 0.f, nwin, h->st);
        s0 = clear_padded(h);
    }
    if (s0 != ROI_OK) return s0;
    const float lam = (float)prm->lambda;
    int blocks = 0;
    if (prm->iters > 0 && persist_ok(h, &blocks)) {
        roi::PersistLaunch L = persist_base(h, 1, prm->iters, blocks);
        L.R = h->sig.p;
        L.C = h->tau.p;
        L.x = h->xc.p;
        L.vx = h->vx.p;
        L.vy = h->vy.p;
        L.sigma_v_dev = sigma_v_dev;
        L.sigma_v = sigma_v;
        L.lambda = lam;
        cudaError_t e;
        {
            Span sp(h, 2);
            e = roi::launch_persist(L, h->st);
        }
        if (e != cudaSuccess) return cuda_fail(h, e, "single-launch Chambolle-Pock solve");
        return ROI_OK;
    }
    roi::FwdArgs fa = fwd_local(h, h->u.p);
    fa.pp = h->pp.p;
    fa.R = h->sig.p;
    roi::BackArgs ba = back_local(h, h->u.p, h->xc.p, nx, xaT0(h), ldaT(h));
    ba.C = h->tau.p;
    ba.vx = h->vx.p;
    ba.vy = h->vy.p;
    ba.xbar = xa0(h);
    ba.xbar_ld = lda(h);
    for (int it = 0; it < prm->iters; ++it) {
        {
            Span sp(h, 0);
            roi::launch_forward(roi::FWD_CP, fa, h->st);
        }
        if (sigma_v_dev)
            roi::launch_cp_dual_grad_dev(xa0(h), lda(h), h->vx.p, h->vy.p, nx, ny, sigma_v_dev, lam, h->st);
        else
            roi::launch_cp_dual_grad(xa0(h), lda(h), h->vx.p, h->vy.p, nx, ny, sigma_v, lam, h->st);
        {
            Span sp(h, 1);
            roi::launch_back(roi::BACK_CP, ba, h->st);
        }
    }
    LAUNCHED(h, "Chambolle-Pock iterations");
    return ROI_OK;
}

}  // namespace

namespace {

// Alg. filtcalc on the whole grid (Sec. 3.1): filters u_1..u_n into filt_u.
roi_status filter_compute(roi_recon* h, int n) {
    const int N = h->N, na = h->na, nd = h->nd, nd2 = 2 * nd - 1, ndp = (nd % 2) ? nd2 : 2 * nd;
    const int ld = roi::padded_ld(N);
    const Rect grid{0, 0, N, N};
    std::vector<AngleRec> rf(na);
    roi::plan_angles(N, na, ndp, h->angles.data(), grid, grid, true, rf.data());
    if (!h->rec_filt) CU(h, dev_alloc(&h->rec_filt, (size_t)na));
    CU(h, cudaMemcpyAsync(h->rec_filt, rf.data(), sizeof(AngleRec) * na, cudaMemcpyHostToDevice, h->st));
    CU(h, h->filt_u.ensure((size_t)n * na * nd2));
    DevBuf c, cT, hc, wc, g;
    DevBufT<double> hq;
    const size_t npad = (size_t)N * ld;
    CU(h, c.ensure(npad));
    CU(h, cT.ensure(npad));
    CU(h, hc.ensure((size_t)na * ndp));
    CU(h, wc.ensure((size_t)na * nd));
    CU(h, g.ensure((size_t)N * N));
    CU(h, hq.ensure((size_t)na * ndp));
    CU(h, cudaMemsetAsync(hq.p, 0, sizeof(double) * na * ndp, h->st));
    float* c0 = c.p + roi::kPad;
    float* cT0 = cT.p + roi::kPad;
    roi::launch_impulse(c0, cT0, ld, N, h->st);
    const double alpha = 1.0 / ((double)na * nd);
    roi::FwdArgs ff{};  // W_f c onto the filter detector
    ff.rec = h->rec_filt;
    ff.na = na;
    ff.stride = ndp;
    ff.nx = N;
    ff.ny = N;
    ff.img = c0;
    ff.imgT = cT0;
    ff.img_ld = ld;
    ff.imgT_ld = ld;
    ff.out = hc.p;
    roi::FwdArgs fw = ff;  // W c onto the acquisition detector
    fw.rec = h->rec_fbp;
    fw.stride = nd;
    fw.out = wc.p;
    roi::BackArgs bw{};
    bw.rec = h->rec_fbp;
    bw.na = na;
    bw.stride = nd;
    bw.nx = N;
    bw.ny = N;
    bw.win = wc.p;
    bw.out = g.p;
    bw.out_ld = N;
    bw.part = nullptr;
    for (int k = 1; k <= n; ++k) {
        roi::launch_forward(roi::FWD_PLAIN, ff, h->st);  // hq = W_f q_k once accumulated
        roi::launch_filter_accum(hc.p, hq.p, h->filt_u.p + (size_t)(k - 1) * na * nd2, na, nd, ndp, alpha, h->st);
        roi::launch_forward(roi::FWD_PLAIN, fw, h->st);
        roi::launch_back(roi::BACK_PLAIN, bw, h->st);
        roi::launch_axpy_padded(c0, cT0, ld, g.p, (float)alpha, N, h->st);
    }
    LAUNCHED(h, "filter computation");
    CU(h, cudaStreamSynchronize(h->st));  // the local buffers are freed on return
    for (DevBuf* b : {&c, &cT, &hc, &wc, &g}) b->release();
    hq.release();
    h->filt_n = n;
    h->filt_ug_n = 0;  // the packed bank is of the previous filters
    return ROI_OK;
}

// C_{u_k} p for k < n (u: [>= n][na][2 nd - 1], p: [na][nd], out: [n][na][nd]): on the
// tensor cores when the detector row fits in shared memory (the bank packed first unless
// `packed` already holds these n filters), else on the FMA pipe.  Synchronizes and reports
// a device wait that ran out.
roi_status filter_conv(roi_recon* h, int n, const float* u, const float* p, float* out, DevBuf* packed,
                       int* packed_n) {
    const int na = h->na, nd = h->nd;
    if (!h->opt_filter_fma && roi::filter_conv_tc_fits(n, nd)) {
        if (*packed_n != n) {
            *packed_n = 0;
            CU(h, packed->ensure(roi::filter_pack_tc_floats(n, na, nd)));
            roi::launch_filter_pack_tc(u, packed->p, n, na, nd, h->st);
            LAUNCHED(h, "filter bank packing");
            *packed_n = n;
        }
        Span sp(h, 3);
        CU(h, roi::launch_filter_conv_tc(packed->p, p, out, n, na, nd, std::max(1, h->sms), h->d_err, h->opt_wait_ns,
                                         h->opt_phantoms > 0 ? 16u : 0u, h->st));
    } else {
        Span sp(h, 3);
        roi::launch_filter_conv(u, p, out, n, na, nd, h->st);
    }
    LAUNCHED(h, "filtered sinograms");
    CU(h, cudaStreamSynchronize(h->st));
    int flag = 0;
    CU(h, cudaMemcpy(&flag, h->d_err, sizeof flag, cudaMemcpyDeviceToHost));
    if (flag) {
        CU(h, cudaMemset(h->d_err, 0, sizeof(int)));
        return fail(h, ROI_ETIMEOUT, "filtered sinograms: a device-side wait gave up; the result is invalid");
    }
    return ROI_OK;
}

// Disc subtraction (Sec. 3.3) and the filtered sinograms C_{u_k} p_d, k = 1..n.
roi_status filter_sinogram(roi_recon* h, int n) {
    const int N = h->N, na = h->na, nd = h->nd;
    const int ld = roi::padded_ld(N);
    const size_t ns = (size_t)na * nd;
    DevBuf D, DT, wd;
    DevBufT<double> sums;
    CU(h, D.ensure((size_t)N * ld));
    CU(h, DT.ensure((size_t)N * ld));
    CU(h, wd.ensure(ns));
    CU(h, sums.ensure(2 * (size_t)na));
    CU(h, h->filt_pd.ensure(ns));
    CU(h, cudaMemsetAsync(D.p, 0, sizeof(float) * N * ld, h->st));
    CU(h, cudaMemsetAsync(DT.p, 0, sizeof(float) * N * ld, h->st));
    roi::launch_disc_image(D.p + roi::kPad, DT.p + roi::kPad, ld, N, h->st);
    roi::FwdArgs fw{};
    fw.rec = h->rec_fbp;
    fw.na = na;
    fw.stride = nd;
    fw.nx = N;
    fw.ny = N;
    fw.img = D.p + roi::kPad;
    fw.imgT = DT.p + roi::kPad;
    fw.img_ld = ld;
    fw.imgT_ld = ld;
    fw.out = wd.p;
    roi::launch_forward(roi::FWD_PLAIN, fw, h->st);
    roi::launch_disc_subtract(h->p, h->pdt, wd.p, 0.f, h->filt_pd.p, ns, h->st);  // p as float
    roi::launch_row_sums(h->filt_pd.p, na, nd, sums.p, h->st);
    roi::launch_row_sums(wd.p, na, nd, sums.p + na, h->st);
    LAUNCHED(h, "disc projection");
    std::vector<double> hs(2 * (size_t)na);
    CU(h, cudaMemcpyAsync(hs.data(), sums.p, sizeof(double) * 2 * na, cudaMemcpyDeviceToHost, h->st));
    CU(h, cudaStreamSynchronize(h->st));
    double num = 0.0, den = 0.0;
    for (int a = 0; a < na; ++a) {
        num += hs[a] * hs[na + a];
        den += hs[na + a] * hs[na + a];
    }
    h->disc_g = den > 0.0 ? num / den : 0.0;
    roi::launch_disc_subtract(h->p, h->pdt, wd.p, (float)h->disc_g, h->filt_pd.p, ns, h->st);
    CU(h, h->filt_cp.ensure((size_t)n * ns));
    const roi_status s = filter_conv(h, n, h->filt_u.p, h->filt_pd.p, h->filt_cp.p, &h->filt_ug, &h->filt_ug_n);
    if (s != ROI_OK) return s;
    D.release();
    DT.release();
    wd.release();
    sums.release();
    h->fcp_n = n;
    return ROI_OK;
}

// Alg. method on the planned box with x >= 0 (Sec. 3.2); result (disc added back) in xc.
roi_status solve_filter(roi_recon* h, const roi_solve_params* prm) {
    const int nx = h->box.w, ny = h->box.h, na = h->na, nd = h->nd;
    const size_t nimg = (size_t)nx * ny, ns = (size_t)na * nd;
    const float alpha = (float)(1.0 / ((double)na * nd));
    float* shift = h->tau.p;
    float* y = h->vx.p;
    float* xs = h->vy.p;
    float* g = h->itmp.p;
    float* x = h->xc.p;
    roi::launch_disc_box(shift, h->box.x0, h->box.y0, nx, ny, h->N, (float)h->disc_g, h->st);
    roi::launch_fill(y, 0.f, nimg, h->st);
    roi::launch_fill(x, 0.f, nimg, h->st);
    roi_status s = clear_padded(h);
    if (s != ROI_OK) return s;
    for (int k = 1; k <= prm->iters; ++k) {
        roi::launch_window_gather(h->filt_cp.p + (size_t)(k - 1) * ns, nd, h->rec_loc, na, h->stride, h->wtmp.p,
                                  h->st);
        roi::launch_back(roi::BACK_PLAIN, back_local(h, h->wtmp.p, xs, nx, nullptr, 0), h->st);  // x_s^k
        roi::launch_forward(roi::FWD_PLAIN, fwd_local(h, h->wrow.p), h->st);                   // W_L y
        roi::launch_back(roi::BACK_PLAIN, back_local(h, h->wrow.p, g, nx, nullptr, 0), h->st);  // W_L^T W_L y
        roi::launch_filter_update(xs, g, y, x, shift, 0.f, INFINITY, alpha, xa0(h), lda(h), xaT0(h), ldaT(h), nx, ny,
                                  h->st);
    }
    roi::launch_add(x, shift, x, nimg, h->st);
    LAUNCHED(h, "filter method");
    return ROI_OK;
}

}  // namespace

namespace roi {
// The server's view of a handle's resident data; computes the residual and waits for
// it (the server works on its own stream).  Returns a roi_status.
int sino_view(roi_recon* h, SinoView* v, std::string* msg) {
    if (!h->have_fbp && h->fcp_n < 1) {
        *msg = "no FBP image and no prepared filters (call fbp or filter_prepare first)";
        return ROI_ESTATE;
    }
    roi_status s = h->have_fbp ? ensure_residual(h) : ROI_OK;
    if (s == ROI_OK) {
        cudaError_t e = cudaStreamSynchronize(h->st);
        if (e != cudaSuccess) s = cuda_fail(h, e, "residual reprojection");
    }
    if (s != ROI_OK) {
        *msg = h->err;
        return s;
    }
    v->N = h->N;
    v->na = h->na;
    v->nd = h->nd;
    v->angles = h->angles.data();
    v->have_fbp = h->have_fbp;
    v->xfbp = h->xfbp;
    v->xfbpT = h->xfbpT;
    v->xfbp_ld = h->xld;
    v->dt = h->dt;
    v->resid = h->resid.p;
    v->resid_ld = h->resid_ld;
    v->fcp = h->filt_cp.p;
    v->fcp_n = h->fcp_n;
    v->disc_g = (float)h->disc_g;
    for (int c = 0; c < kShapeClasses; ++c) v->shape[c] = h->opt_tile_shape >= 0 ? h->opt_tile_shape : h->tile_shape[c];
    return ROI_OK;
}
}  // namespace roi

extern "C" {

roi_status roi_recon_create(const roi_geometry* geom, void* cuda_stream, roi_recon_t* out) {
    if (!out) return ROI_EINVAL;
    *out = nullptr;
    if (check_geometry(geom) != ROI_OK) return ROI_EINVAL;
    roi_recon* h = new (std::nothrow) roi_recon;
    if (!h) return ROI_ENOMEM;
    h->N = geom->n_pix;
    h->na = geom->n_angles;
    h->nd = geom->n_det;
    h->angles = make_angles(geom);
    h->st = (cudaStream_t)cuda_stream;
    h->pdt = (int)geom->storage;
    h->pesz = roi::dt_size(h->pdt);
    h->dt = (int)geom->image_storage;
    h->esz = roi::dt_size(h->dt);
    h->xld = roi::padded_ld_e(h->N, h->esz);
    const size_t ns = (size_t)h->na * h->nd;
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = roi::dev_malloc(&h->p, (size_t)h->pesz * ns);
    if (e == cudaSuccess) e = dev_alloc(&h->q, ns);
    const size_t npad_bytes = (size_t)h->esz * h->N * h->xld;
    if (e == cudaSuccess) e = dev_alloc(&h->xfbp_base, npad_bytes);
    if (e == cudaSuccess) e = dev_alloc(&h->xfbpT_base, npad_bytes);
    if (e == cudaSuccess) e = cudaMemset(h->xfbp_base, 0, npad_bytes);
    if (e == cudaSuccess) e = cudaMemset(h->xfbpT_base, 0, npad_bytes);
    if (e == cudaSuccess) {
        h->xfbp = h->xfbp_base + (size_t)roi::kPad * h->esz;
        h->xfbpT = h->xfbpT_base + (size_t)roi::kPad * h->esz;
    }
    if (e == cudaSuccess) e = dev_alloc(&h->hodd, (size_t)h->nd / 2 + 1);
    if (e == cudaSuccess) e = dev_alloc(&h->rec_fbp, (size_t)h->na);
    if (e == cudaSuccess) e = dev_alloc(&h->rec_loc, (size_t)h->na);
    if (e == cudaSuccess) e = dev_alloc(&h->rec_ext, (size_t)h->na);
    if (e == cudaSuccess) e = dev_alloc(&h->red, (size_t)kRedScratch + 4);
    if (e == cudaSuccess) e = dev_alloc(&h->d_bar, 2);
    if (e == cudaSuccess) e = dev_alloc(&h->d_err, 1);
    if (e == cudaSuccess) e = cudaMemset(h->d_err, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaGetDevice(&h->device);
    if (e == cudaSuccess) {
        int v = 0;
        e = cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
        h->max_smem_optin = (size_t)v;
    }
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->pin_free, cudaEventDisableTiming);
    if (e == cudaSuccess) {
        // Ram-Lak odd taps h_m = -1/(pi m)^2, m = 2t + 1, scaled by pi / N_theta (Eq. fbp)
        std::vector<float> ho((size_t)h->nd / 2 + 1);
        const double scale = kPi / h->na;
        double tail = 0.25;  // h0 + 2 sum over the odd offsets the convolution reaches (m < nd)
        for (size_t t = 0; t < ho.size(); ++t) {
            const double m = 2.0 * t + 1.0;
            const double hm = -1.0 / (kPi * kPi * m * m);
            ho[t] = (float)(scale * hm);
            if (m < h->nd) tail += 2.0 * hm;
        }
        h->ctail = (float)(scale * tail);
        std::vector<AngleRec> rf(h->na);
        const Rect grid{0, 0, h->N, h->N};
        roi::plan_angles(h->N, h->na, h->nd, h->angles.data(), grid, grid, true, rf.data());
        e = cudaMemcpy(h->hodd, ho.data(), sizeof(float) * ho.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(h->rec_fbp, rf.data(), sizeof(AngleRec) * h->na, cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        roi_recon_destroy(h);
        return e == cudaErrorMemoryAllocation ? ROI_ENOMEM : ROI_ECUDA;
    }
    {
        std::lock_guard<std::mutex> g(g_tune_mu);
        auto it = g_tune.find(TuneKey{h->N, h->na, h->nd, h->dt, fnv_doubles(h->angles)});
        if (it != g_tune.end())
            for (int c = 0; c < roi::kShapeClasses; ++c) {
                h->tile_shape[c] = it->second.shape[c];
                h->team_cap[c] = it->second.team[c];
            }
    }
    *out = h;
    return ROI_OK;
}

void roi_recon_destroy(roi_recon_t h) {
    if (!h) return;
    cudaStreamSynchronize(h->st);
    while (!h->plans.empty()) roi_recon_batch_plan_destroy(h, h->plans.back());
    for (void* b : {h->p, (void*)h->q, (void*)h->xfbp_base, (void*)h->xfbpT_base, (void*)h->hodd})
        if (b) cudaFree(b);
    h->fbp32.release();
    h->in_tmp.release();
    for (DevBuf* b : {&h->filt_u, &h->filt_cp, &h->filt_pd, &h->filt_ug, &h->op_ug}) b->release();
    if (h->rec_filt) cudaFree(h->rec_filt);
    for (AngleRec* b : {h->rec_fbp, h->rec_loc, h->rec_ext})
        if (b) cudaFree(b);
    if (h->red) cudaFree(h->red);
    if (h->d_bar) cudaFree(h->d_bar);
    if (h->d_err) cudaFree(h->d_err);
    h->resid.release();  // the batch buffers (h->bb) are freed with the handle
    if (h->pin) cudaFreeHost(h->pin);
    if (h->pin_free) cudaEventDestroy(h->pin_free);
    for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
    for (DevBuf* b : {&h->pp, &h->u, &h->sig, &h->wtmp, &h->wrow, &h->xc, &h->vx, &h->vy, &h->tau, &h->itmp, &h->xa,
                      &h->xaT})
        b->release();
    h->part.release();
    delete h;
}

const char* roi_recon_last_error(roi_recon_t h) { return h ? h->err.c_str() : "null handle"; }

roi_status roi_recon_set_sinogram(roi_recon_t h, const void* p, roi_dtype dt, int on_device) {
    if (!h) return ROI_EINVAL;
    h->err.clear();
    if (!p) return fail(h, ROI_EINVAL, "set_sinogram: null pointer");
    if (dt != ROI_F32 && dt != ROI_BF16 && dt != ROI_F16) return fail(h, ROI_EINVAL, "set_sinogram: unknown dtype");
    const size_t n = (size_t)h->na * h->nd;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if ((int)dt == h->pdt) {
        CU(h, cudaMemcpyAsync(h->p, p, (size_t)h->pesz * n, kind, h->st));
    } else {  // narrow (or widen) to the storage type on the device
        const size_t in_bytes = (size_t)roi::dt_size((int)dt) * n;
        CU(h, h->in_tmp.ensure(in_bytes));
        CU(h, cudaMemcpyAsync(h->in_tmp.p, p, in_bytes, kind, h->st));
        roi::launch_convert(h->in_tmp.p, (int)dt, h->p, h->pdt, n, h->st);
        LAUNCHED(h, "set_sinogram conversion");
    }
    h->have_sino = true;
    h->have_fbp = false;
    h->exterior_ready = 0;
    h->resid_ready = 0;
    h->fcp_n = 0;
    return ROI_OK;
}

roi_status roi_recon_set_sinogram_truncated(roi_recon_t h, const void* p, roi_dtype dt, int on_device,
                                           int n_measured) {
    if (!h) return ROI_EINVAL;
    h->err.clear();
    if (!p) return fail(h, ROI_EINVAL, "set_sinogram_truncated: null pointer");
    if (dt != ROI_F32 && dt != ROI_BF16 && dt != ROI_F16)
        return fail(h, ROI_EINVAL, "set_sinogram_truncated: unknown dtype");
    if (n_measured < 1 || n_measured > h->nd || (h->nd - n_measured) % 2)
        return fail(h, ROI_EINVAL, "set_sinogram_truncated: n_measured must be in [1, n_det] with n_det - n_measured even");
    const size_t in_bytes = (size_t)roi::dt_size((int)dt) * h->na * n_measured;
    CU(h, h->in_tmp.ensure(in_bytes));
    CU(h, cudaMemcpyAsync(h->in_tmp.p, p, in_bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                          h->st));
    roi::launch_pad_truncated(h->in_tmp.p, (int)dt, n_measured, h->p, h->pdt, h->na, h->nd,
                              (h->nd - n_measured) / 2, h->st);
    LAUNCHED(h, "set_sinogram_truncated padding");
    h->have_sino = true;
    h->have_fbp = false;
    h->exterior_ready = 0;
    h->resid_ready = 0;
    h->fcp_n = 0;
    return ROI_OK;
}

roi_status roi_recon_ramp_filter(roi_recon_t h, float* q) {
    if (!h) return ROI_EINVAL;
    h->err.clear();
    if (!q) return fail(h, ROI_EINVAL, "ramp_filter: null output");
    if (!h->have_sino) return fail(h, ROI_ESTATE, "ramp_filter: no sinogram (call set_sinogram first)");
    roi::launch_ramp(h->p, h->pdt, h->hodd, q, h->na, h->nd, h->ctail, h->st);
    LAUNCHED(h, "ramp filter");
    return ROI_OK;
}

roi_status roi_recon_fbp(roi_recon_t h, float* out_or_null) {
    if (!h) return ROI_EINVAL;
    h->err.clear();
    if (!h->have_sino) return fail(h, ROI_ESTATE, "fbp: no sinogram (call set_sinogram first)");
    roi::launch_ramp(h->p, h->pdt, h->hodd, h->q, h->na, h->nd, h->ctail, h->st);
    roi::BackArgs b{};
    b.rec = h->rec_fbp;
    b.na = h->na;
    b.stride = h->nd;
    b.nx = h->N;
    b.ny = h->N;
    b.win = h->q;
    b.part = nullptr;  // the whole grid has enough tiles for one angle group
    // the cached global reconstruction is kept inside its field of view only: outside the
    // disc of diameter min(N, N_d) some angles miss the pixel, its FBP value is not set by
    // the data, and reprojecting it in the exterior step would make p' inconsistent
    b.fov_d = std::min(h->N, h->nd);
    if (h->dt == 0) {  // straight into the padded image and its transpose
        b.out = static_cast<float*>(h->xfbp);
        b.out_ld = h->xld;
        b.outT = static_cast<float*>(h->xfbpT);
        b.outT_ld = h->xld;
        roi::launch_back(roi::BACK_PLAIN, b, h->st);
    } else {  // float image, then narrowed into the padded image and its transpose
        CU(h, h->fbp32.ensure((size_t)h->N * h->N));
        b.out = h->fbp32.p;
        b.out_ld = h->N;
        roi::launch_back(roi::BACK_PLAIN, b, h->st);
        roi::launch_store_padded(h->fbp32.p, h->N, h->xfbp, h->dt, h->xld, h->N, h->N, 0, h->st);
        roi::launch_store_padded(h->fbp32.p, h->N, h->xfbpT, h->dt, h->xld, h->N, h->N, 1, h->st);
    }
    LAUNCHED(h, "fbp");
    if (out_or_null) {
        if (h->dt == 0)
            CU(h, cudaMemcpy2DAsync(out_or_null, sizeof(float) * h->N, h->xfbp, sizeof(float) * h->xld,
                                    sizeof(float) * h->N, h->N, cudaMemcpyDeviceToDevice, h->st));
        else  // the resident (narrowed) image, widened
            roi::launch_load_padded(h->xfbp, h->dt, h->xld, out_or_null, h->N, h->N, h->N, h->st);
    }
    h->have_fbp = true;
    h->exterior_ready = 0;
    h->resid_ready = 0;
    return ROI_OK;
}

roi_status roi_recon_plan(const roi_geometry* geom, const roi_region* region, roi_solve_info* info, int* d0,
                          int* width) {
    if (check_geometry(geom) != ROI_OK || !region || !info) return ROI_EINVAL;
    if (!finite_region(region)) return ROI_EINVAL;
    Rect box;
    if (!roi::plan_box(geom->n_pix, region->cx, region->cy, region->radius, region->margin, &box)) return ROI_EINVAL;
    std::vector<double> ang = make_angles(geom);
    std::vector<AngleRec> rec(geom->n_angles);
    const int wl = roi::plan_angles(geom->n_pix, geom->n_angles, geom->n_det, ang.data(), box, box, false, rec.data());
    std::memset(info, 0, sizeof *info);
    info->box_x0 = box.x0;
    info->box_y0 = box.y0;
    info->box_w = box.w;
    info->box_h = box.h;
    info->window_max = wl;
    info->window_stride = roi::round_stride(wl);
    for (int a = 0; a < geom->n_angles; ++a) {
        if (d0) d0[a] = rec[a].d0;
        if (width) width[a] = rec[a].width;
    }
    return ROI_OK;
}

roi_status roi_recon_reproject_exterior(roi_recon_t h, const roi_region* region, float* window_out_or_null,
                                        int* d0_out_or_null) {
    if (!h || !region) return ROI_EINVAL;
    h->err.clear();
    if (!h->have_fbp) return fail(h, ROI_ESTATE, "reproject_exterior: no FBP image (call fbp first)");
    roi_status s = ensure_plan(h, region);
    if (s != ROI_OK) return s;
    s = run_exterior(h);
    if (s != ROI_OK) return s;
    if (window_out_or_null)
        CU(h, cudaMemcpyAsync(window_out_or_null, h->pp.p, sizeof(float) * (size_t)h->na * h->stride,
                              cudaMemcpyDeviceToDevice, h->st));
    if (d0_out_or_null) {
        for (int a = 0; a < h->na; ++a) d0_out_or_null[a] = h->h_loc[a].d0;
        CU(h, cudaStreamSynchronize(h->st));
    }
    return ROI_OK;
}

roi_status roi_recon_forward_local(roi_recon_t h, const roi_region* region, const float* x, float* y) {
    if (!h || !region) return ROI_EINVAL;
    h->err.clear();
    h->state_valid = false;
    h->state_region_path = false;
    if (!x || !y) return fail(h, ROI_EINVAL, "forward_local: null pointer");
    roi_status s = ensure_plan(h, region);
    if (s != ROI_OK) return s;
    s = load_padded(h, x);
    if (s != ROI_OK) return s;
    roi::launch_forward(roi::FWD_PLAIN, fwd_local(h, y), h->st);
    LAUNCHED(h, "forward_local");
    return ROI_OK;
}

roi_status roi_recon_back_local(roi_recon_t h, const roi_region* region, const float* y, float* x) {
    if (!h || !region) return ROI_EINVAL;
    h->err.clear();
    h->state_valid = false;
    h->state_region_path = false;
    if (!x || !y) return fail(h, ROI_EINVAL, "back_local: null pointer");
    roi_status s = ensure_plan(h, region);
    if (s != ROI_OK) return s;
    roi::launch_back(roi::BACK_PLAIN, back_local(h, y, x, h->box.w, nullptr, 0), h->st);
    LAUNCHED(h, "back_local");
    return ROI_OK;
}

namespace {

roi_status solve_batch_impl(roi_recon* h, int n, const roi_region* regions, const roi_solve_params* params,
                            float* const* outs, int out_on_device, roi_solve_info* infos, int team_req,
                            BatchBufs* own = nullptr, cudaGraphExec_t* capture = nullptr);

roi_status solve_local_impl(roi_recon* h, const roi_region* region, const roi_solve_params* params, float* out,
                            int out_on_device, roi_solve_info* info) {
    h->state_valid = false;  // the solver buffers are about to change
    h->state_region_path = false;
    if (!out) return fail(h, ROI_EINVAL, "solve_local: null output");
    if (params->reg == ROI_FILTER_TV || params->reg == ROI_FILTER_ISTA) {  // run in the whole-region solver
        if (params->eval_objective) return fail(h, ROI_EINVAL, "solve_local: no objective for this regularizer");
        float* outs[1] = {out};
        return roi_recon_solve_batch(h, 1, region, params, outs, out_on_device, info);
    }
    if (params->reg != ROI_SIRT_NONNEG && params->reg != ROI_TV_CP && params->reg != ROI_FILTER_SIRT)
        return fail(h, ROI_EINVAL, "solve_local: unknown regularizer %d", (int)params->reg);
    if (params->iters < 0 || params->iters > 1000000) return fail(h, ROI_EINVAL, "solve_local: iters out of range");
    if (!std::isfinite(params->lambda) || params->lambda < 0)
        return fail(h, ROI_EINVAL, "solve_local: lambda must be finite and >= 0");
    const bool filt = params->reg == ROI_FILTER_SIRT;
    if (filt) {
        if (params->eval_objective) return fail(h, ROI_EINVAL, "solve_local: no objective for ROI_FILTER_SIRT");
        if (h->fcp_n < params->iters)
            return fail(h, ROI_ESTATE, "solve_local: filters for %d iterations not prepared (filter_prepare)",
                        params->iters);
    } else if (!h->have_fbp) {
        return fail(h, ROI_ESTATE, "solve_local: no FBP image (call fbp first)");
    }
    roi_status s = ensure_plan(h, region);
    if (s != ROI_OK) return s;
    int pblocks = 0;
    if (!filt && h->opt_persistent && params->iters > 0 && !persist_ok(h, &pblocks) && !h->resume &&
        !params->eval_objective && (params->reg == ROI_SIRT_NONNEG || params->precond)) {
        // a box too large for the single-launch solver: the whole-region solver, one
        // cooperative team of every co-resident block, exterior step p' = r + W_L x_fbp
        // (Eq. locouter with the residual r = p - W x_fbp of the FBP)
        float* outs[1] = {out};
        s = solve_batch_impl(h, 1, region, params, outs, out_on_device, info, -1);
        if (s == ROI_OK) h->state_region_path = true;
        return s;
    }
    double L_flag = 0.0;
    if (filt) {
        s = solve_filter(h, params);
    } else {
        s = run_exterior(h);
        if (s != ROI_OK) return s;
        if (params->reg == ROI_SIRT_NONNEG)
            s = solve_sirt(h, params);
        else
            s = solve_cp(h, params, &L_flag);
    }
    if (s != ROI_OK) return s;
    const int nx = h->box.w, ny = h->box.h;
    const size_t nimg = (size_t)nx * ny;
    const double cxl = region->cx - h->box.x0, cyl = region->cy - h->box.y0;
    // the solution: SIRT keeps x in the padded xa, CP and the filter method in xc
    const bool sirt = params->reg == ROI_SIRT_NONNEG;
    const float* xs = sirt ? xa0(h) : h->xc.p;
    const int xs_ld = sirt ? lda(h) : nx;
    float* dst = out_on_device ? out : h->itmp.p;
    roi::launch_crop(xs, xs_ld, dst, nx, ny, cxl, cyl, region->radius, params->crop_disk, h->st);
    LAUNCHED(h, "crop");
    double objective = 0.0, L = 0.0;
    if (params->eval_objective) {
        // ||W_L x - p'||^2 over rays that reach the box + lambda TV(x)
        if (sirt || !params->precond) {
            // row sums were not computed by the solver: W_L 1 into wrow (vx, vy, xc are free now)
            float* xkeep = sirt ? h->xc.p : h->vy.p;
            roi::launch_copy_pad(xs, xs_ld, xkeep, nx, ny, nx, h->st);  // unpadded copy of x
            roi::launch_fill(h->vx.p, 1.f, nimg, h->st);
            s = load_padded(h, h->vx.p);
            if (s != ROI_OK) return s;
            roi::launch_forward(roi::FWD_PLAIN, fwd_local(h, h->wrow.p), h->st);
            s = load_padded(h, xkeep);
            if (s != ROI_OK) return s;
            roi::launch_forward(roi::FWD_PLAIN, fwd_local(h, h->wtmp.p), h->st);
            roi::launch_objective(h->wtmp.p, h->pp.p, h->wrow.p, h->na * h->stride, xkeep, nx, nx, ny, h->red,
                                  kRedScratch, h->red + kRedScratch + 2, h->st);
        } else {
            s = load_padded(h, h->xc.p);
            if (s != ROI_OK) return s;
            roi::launch_forward(roi::FWD_PLAIN, fwd_local(h, h->wtmp.p), h->st);
            roi::launch_objective(h->wtmp.p, h->pp.p, h->wrow.p, h->na * h->stride, h->xc.p, nx, nx, ny, h->red,
                                  kRedScratch, h->red + kRedScratch + 2, h->st);
        }
        LAUNCHED(h, "objective");
        double r2[2];
        CU(h, cudaMemcpyAsync(r2, h->red + kRedScratch + 2, sizeof r2, cudaMemcpyDeviceToHost, h->st));
        CU(h, cudaStreamSynchronize(h->st));
        objective = r2[0] + params->lambda * r2[1];
    }
    if (L_flag != 0.0 && info) {
        CU(h, cudaMemcpyAsync(&L, h->red + kRedScratch + 1, sizeof L, cudaMemcpyDeviceToHost, h->st));
        CU(h, cudaStreamSynchronize(h->st));
    }
    if (!out_on_device) {
        CU(h, cudaMemcpyAsync(out, h->itmp.p, sizeof(float) * nimg, cudaMemcpyDeviceToHost, h->st));
        s = roi_recon_sync(h);
        if (s != ROI_OK) return s;
    }
    if (!filt && !params->eval_objective) {  // the buffers hold this solve's iterate state
        h->state_valid = true;
        h->state_reg = (int)params->reg;
        h->state_flag = sirt ? params->weighting : params->precond;
        h->state_lambda = sirt ? 0.0 : params->lambda;
        h->state_iters = h->resume_iters + params->iters;
    }
    if (info) {
        fill_info(h, info);
        info->iters_done = (int)(h->resume_iters + params->iters);
        info->step_L = L;
        info->objective = objective;
    }
    return ROI_OK;
}

}  // namespace

roi_status roi_recon_solve_local(roi_recon_t h, const roi_region* region, const roi_solve_params* params, float* out,
                                 int out_on_device, roi_solve_info* info) {
    if (!h || !region || !params) return ROI_EINVAL;
    h->err.clear();
    return solve_local_impl(h, region, params, out, out_on_device, info);
}

roi_status roi_recon_state_size(roi_recon_t h, size_t* bytes) {
    if (!h || !bytes) return ROI_EINVAL;
    h->err.clear();
    if (!h->state_valid && h->state_region_path)
        return fail(h, ROI_ESTATE,
                    "state_size: the last solve ran in the whole-region solver, which keeps no resumable state "
                    "(ROI_OPT_SINGLE_LAUNCH = 0 keeps one for large boxes)");
    if (!h->state_valid) return fail(h, ROI_ESTATE, "state_size: no solver state (run solve_local first)");
    *bytes = state_bytes_for(h->state_reg, h->box.w, h->box.h, h->na, h->stride);
    return ROI_OK;
}

roi_status roi_recon_state_export(roi_recon_t h, void* dst, size_t bytes, int on_device) {
    if (!h) return ROI_EINVAL;
    h->err.clear();
    if (!dst) return fail(h, ROI_EINVAL, "state_export: null destination");
    if (!h->state_valid && h->state_region_path)
        return fail(h, ROI_ESTATE,
                    "state_export: the last solve ran in the whole-region solver, which keeps no resumable state "
                    "(ROI_OPT_SINGLE_LAUNCH = 0 keeps one for large boxes)");
    if (!h->state_valid) return fail(h, ROI_ESTATE, "state_export: no solver state (run solve_local first)");
    const int nx = h->box.w, ny = h->box.h;
    const size_t need = state_bytes_for(h->state_reg, nx, ny, h->na, h->stride);
    if (bytes < need) return fail(h, ROI_EINVAL, "state_export: %zu bytes given, %zu needed", bytes, need);
    StateHeader hd{};
    std::memcpy(hd.magic, kStateMagic, sizeof hd.magic);
    hd.reg = h->state_reg;
    hd.flag = h->state_flag;
    hd.box_x0 = h->box.x0;
    hd.box_y0 = h->box.y0;
    hd.box_w = nx;
    hd.box_h = ny;
    hd.na = h->na;
    hd.stride = h->stride;
    hd.iters_done = h->state_iters;
    hd.lambda = h->state_lambda;
    unsigned char* d = static_cast<unsigned char*>(dst);
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (on_device)
        CU(h, cudaMemcpyAsync(d, &hd, sizeof hd, cudaMemcpyHostToDevice, h->st));
    else
        std::memcpy(d, &hd, sizeof hd);
    d += sizeof hd;
    const size_t row = sizeof(float) * nx, img = row * ny;
    if (h->state_reg == ROI_SIRT_NONNEG) {
        CU(h, cudaMemcpy2DAsync(d, row, xa0(h), sizeof(float) * lda(h), row, ny, k, h->st));  // x
    } else {
        CU(h, cudaMemcpyAsync(d, h->xc.p, img, k, h->st));  // x
        d += img;
        CU(h, cudaMemcpy2DAsync(d, row, xa0(h), sizeof(float) * lda(h), row, ny, k, h->st));  // xbar
        d += img;
        CU(h, cudaMemcpyAsync(d, h->vx.p, img, k, h->st));
        d += img;
        CU(h, cudaMemcpyAsync(d, h->vy.p, img, k, h->st));
        d += img;
        CU(h, cudaMemcpyAsync(d, h->u.p, sizeof(float) * (size_t)h->na * h->stride, k, h->st));
    }
    CU(h, cudaStreamSynchronize(h->st));
    return ROI_OK;
}

roi_status roi_recon_solve_local_resume(roi_recon_t h, const roi_region* region, const roi_solve_params* params,
                                        const void* state, size_t bytes, int state_on_device, float* out,
                                        int out_on_device, roi_solve_info* info) {
    if (!h || !region || !params) return ROI_EINVAL;
    h->err.clear();
    if (!state) return fail(h, ROI_EINVAL, "solve_local_resume: null state");
    if (params->reg != ROI_SIRT_NONNEG && params->reg != ROI_TV_CP)
        return fail(h, ROI_EINVAL, "solve_local_resume: only SIRT and CP-TV solves resume");
    if (bytes < sizeof(StateHeader)) return fail(h, ROI_EINVAL, "solve_local_resume: state too short");
    StateHeader hd{};
    if (state_on_device) {
        CU(h, cudaMemcpyAsync(&hd, state, sizeof hd, cudaMemcpyDeviceToHost, h->st));
        CU(h, cudaStreamSynchronize(h->st));
    } else {
        std::memcpy(&hd, state, sizeof hd);
    }
    if (std::memcmp(hd.magic, kStateMagic, sizeof hd.magic) != 0)
        return fail(h, ROI_EINVAL, "solve_local_resume: not a solver state");
    roi_status s = ensure_plan(h, region);
    if (s != ROI_OK) return s;
    const bool sirt = params->reg == ROI_SIRT_NONNEG;
    if (hd.reg != (int)params->reg || hd.flag != (sirt ? params->weighting : params->precond) ||
        (!sirt && hd.lambda != params->lambda))
        return fail(h, ROI_EINVAL, "solve_local_resume: regularizer, weighting / precond or lambda differ from the state's");
    if (hd.box_x0 != h->box.x0 || hd.box_y0 != h->box.y0 || hd.box_w != h->box.w || hd.box_h != h->box.h ||
        hd.na != h->na || hd.stride != h->stride || hd.iters_done < 0)
        return fail(h, ROI_EINVAL, "solve_local_resume: the state's box or window layout differs from the region's");
    if (bytes < state_bytes_for(hd.reg, hd.box_w, hd.box_h, hd.na, hd.stride))
        return fail(h, ROI_EINVAL, "solve_local_resume: state too short for its box");
    h->resume = static_cast<const unsigned char*>(state);
    h->resume_on_device = state_on_device;
    h->resume_iters = hd.iters_done;
    s = solve_local_impl(h, region, params, out, out_on_device, info);
    h->resume = nullptr;
    h->resume_iters = 0;
    return s;
}

roi_status roi_recon_filter_prepare(roi_recon_t h, int n_iters) {
    if (!h) return ROI_EINVAL;
    h->err.clear();
    h->state_valid = false;
    h->state_region_path = false;
    if (n_iters < 1 || n_iters > 100000) return fail(h, ROI_EINVAL, "filter_prepare: n_iters out of range");
    if (!h->have_sino) return fail(h, ROI_ESTATE, "filter_prepare: no sinogram (call set_sinogram first)");
    if (h->filt_n < n_iters) {
        h->fcp_n = 0;
        roi_status s = filter_compute(h, n_iters);
        if (s != ROI_OK) return s;
    }
    if (h->fcp_n < n_iters) return filter_sinogram(h, n_iters);
    return ROI_OK;
}

roi_status roi_recon_filter_conv(roi_recon_t h, int n, const float* u, const float* p, float* out) {
    if (!h) return ROI_EINVAL;
    h->err.clear();
    if (n < 1 || n > 100000 || !u || !p || !out) return fail(h, ROI_EINVAL, "filter_conv: bad arguments");
    int packed = -1;  // the caller's filters: always packed afresh
    return filter_conv(h, n, u, p, out, &h->op_ug, &packed);
}

roi_status roi_recon_filter_get(roi_recon_t h, int n_filters, float* u_out, double* disc_grey) {
    if (!h) return ROI_EINVAL;
    h->err.clear();
    if (h->fcp_n < 1) return fail(h, ROI_ESTATE, "filter_get: call filter_prepare first");
    if (n_filters < 0) return fail(h, ROI_EINVAL, "filter_get: n_filters < 0");
    const int k = std::min(n_filters, h->filt_n);
    if (u_out && k > 0)
        CU(h, cudaMemcpyAsync(u_out, h->filt_u.p, sizeof(float) * (size_t)k * h->na * (2 * h->nd - 1),
                              cudaMemcpyDeviceToDevice, h->st));
    if (disc_grey) *disc_grey = h->disc_g;
    return ROI_OK;
}

namespace {

// roi_recon_solve_batch with a choice of launch: team_req = 0 picks it from the number of
// regions (one block per region, or teams of up to 16 blocks for few regions); team_req < 0
// makes one team of every co-resident block (a lone large region).
roi_status solve_batch_impl(roi_recon* h, int n, const roi_region* regions, const roi_solve_params* params,
                            float* const* outs, int out_on_device, roi_solve_info* infos, int team_req,
                            BatchBufs* own, cudaGraphExec_t* capture) {
    BatchBufs& bb = own ? *own : h->bb;
    if (n < 0 || (n > 0 && (!regions || !params || !outs))) return fail(h, ROI_EINVAL, "solve_batch: bad arguments");
    if (n == 0) return ROI_OK;
    bool need_fbp = false;
    bool need_fgp = false;
    for (int i = 0; i < n; ++i) {
        const bool filt = params[i].reg == ROI_FILTER_SIRT || params[i].reg == ROI_FILTER_TV ||
                          params[i].reg == ROI_FILTER_ISTA;
        need_fbp = need_fbp || !filt;
        need_fgp = need_fgp || params[i].reg == ROI_FILTER_TV || params[i].reg == ROI_FILTER_ISTA;
    }
    if (need_fbp && !h->have_fbp) return fail(h, ROI_ESTATE, "solve_batch: no FBP image (call fbp first)");
    const int na = h->na;
    // ---- host plan of every region
    std::vector<Rect> boxes(n);
    std::vector<int> strides(n);
    size_t out_total = 0, win_cap = 0, img_cap = 0, pad_cap = 0, max_stage = 0;
    size_t max_banded_units = 0;  // ray units of the largest band-streamed region
    int max_side = 0;             // the largest box side (its class sets the team size of few regions)
    std::vector<double> cost(n);
    std::vector<AngleRec> loc(na);
    for (int i = 0; i < n; ++i) {
        const roi_solve_params& P = params[i];
        if (!finite_region(&regions[i]))
            return fail(h, ROI_EINVAL, "solve_batch: region %d: radius must be > 0, margin >= 0, all finite", i);
        if (P.reg < ROI_SIRT_NONNEG || P.reg > ROI_FILTER_ISTA)
            return fail(h, ROI_EINVAL, "solve_batch: region %d: unknown regularizer", i);
        if (P.reg >= ROI_FILTER_SIRT && h->fcp_n < P.iters)
            return fail(h, ROI_ESTATE, "solve_batch: region %d: filters for %d iterations not prepared", i, P.iters);
        if (P.inner_iters < 0 || P.inner_iters > 100000)
            return fail(h, ROI_EINVAL, "solve_batch: region %d: inner_iters out of range", i);
        if (P.iters < 0 || P.iters > 1000000) return fail(h, ROI_EINVAL, "solve_batch: region %d: iters out of range", i);
        if (!std::isfinite(P.lambda) || P.lambda < 0) return fail(h, ROI_EINVAL, "solve_batch: region %d: bad lambda", i);
        if (P.reg == ROI_TV_CP && !P.precond)
            return fail(h, ROI_EINVAL, "solve_batch: region %d: batched CP uses the diagonal steps (precond = 1)", i);
        if (!outs[i]) return fail(h, ROI_EINVAL, "solve_batch: region %d: null output", i);
        Rect box;
        if (!roi::plan_box(h->N, regions[i].cx, regions[i].cy, regions[i].radius, regions[i].margin, &box))
            return fail(h, ROI_EINVAL, "solve_batch: region %d: extended box misses the grid", i);
        const int wl = roi::plan_angles(h->N, na, h->nd, h->angles.data(), box, box, false, loc.data());
        boxes[i] = box;
        strides[i] = roi::round_stride(wl);
        out_total += (size_t)box.w * box.h;
        win_cap = std::max(win_cap, (size_t)na * strides[i]);
        img_cap = std::max(img_cap, (size_t)box.w * box.h);
        // padded images in the storage type, counted in floats (whole 16-byte units)
        const size_t pr = (size_t)box.h * roi::padded_ld_e(box.w, h->esz) * h->esz;
        const size_t pc = (size_t)box.w * roi::padded_ld_e(box.h, h->esz) * h->esz;
        pad_cap = std::max(pad_cap, (std::max(pr, pc) + 15) / 16 * 4);
        max_stage = std::max(max_stage, roi::stage_bytes(box.w, box.h, h->esz));
        if (roi::stage_mode(box.w, box.h, h->esz) == 1)
            max_banded_units = std::max(max_banded_units, (size_t)na * ((strides[i] + 31) / 32));
        cost[i] = (double)box.w * box.h * na * (double)std::max(P.iters, 1);
        max_side = std::max(max_side, std::max(box.w, box.h));
    }
    if (need_fbp) {
        roi_status s0 = ensure_residual(h);
        if (s0 != ROI_OK) return s0;
    }
    // ---- device storage
    CU(h, bb.tab.ensure((size_t)n * na));
    CU(h, bb.rois.ensure(n));
    CU(h, bb.order.ensure(n));
    CU(h, bb.queue.ensure(1));
    if (!out_on_device) CU(h, bb.out.ensure(out_total));
    // few regions: teams of blocks per region (co-resident: at most one block per SM)
    int blocks = std::max(1, h->sms);
    int team = std::min(h->team_cap[roi::shape_class(max_side)], blocks / n);
    if (team_req < 0) team = std::min(blocks, roi::serve_max_blocks(h->device));
    if (team > 1) {
        blocks = std::min(blocks, roi::serve_max_blocks(h->device));
        team = std::min(team, blocks);
        blocks = (blocks / team) * team;
        CU(h, bb.bars.ensure((size_t)blocks / team));
    }
    // one slot of buffers per block, or per team of blocks
    const size_t slots = team > 1 ? (size_t)blocks / team : (size_t)blocks;
    for (DevBuf* b : {&bb.pp, &bb.u, &bb.sig}) CU(h, b->ensure(win_cap * slots));
    for (DevBuf* b : {&bb.x, &bb.vx, &bb.vy, &bb.tau}) CU(h, b->ensure(img_cap * slots));
    for (DevBuf* b : {&bb.xa, &bb.xaT}) CU(h, b->ensure(pad_cap * slots));
    if (need_fgp) CU(h, bb.fgp.ensure(5 * img_cap * slots));
    // ---- page-locked staging: tables, descriptors, order
    const size_t tab_bytes = sizeof(AngleRec) * (size_t)n * na;
    const size_t roi_bytes = sizeof(roi::BatchRoi) * (size_t)n;
    const size_t ord_bytes = sizeof(int) * (size_t)n;
    const size_t pin_need = tab_bytes + roi_bytes + ord_bytes;
    CU(h, cudaEventSynchronize(h->pin_free));  // the previous uploads have left the staging area
    if (pin_need > h->pin_cap) {
        if (h->pin) cudaFreeHost(h->pin);
        h->pin = nullptr;
        h->pin_cap = 0;
        CU(h, roi::pinned_alloc((void**)&h->pin, pin_need, cudaHostAllocDefault));
        h->pin_cap = pin_need;
    }
    AngleRec* ptab = reinterpret_cast<AngleRec*>(h->pin);
    roi::BatchRoi* prois = reinterpret_cast<roi::BatchRoi*>(h->pin + tab_bytes);
    int* pord = reinterpret_cast<int*>(h->pin + tab_bytes + roi_bytes);
    size_t ooff = 0;
    size_t part_cap = 0;  // a team of every block: phase A of band-streamed boxes by row band
    for (int i = 0; i < n; ++i) {
        const Rect box = boxes[i];
        int nr = 0;
        const int wl = roi::plan_region_table(h->N, na, h->nd, h->angles.data(), box, ptab + (size_t)i * na, &nr);
        if (team_req < 0 && team > 1 && roi::stage_mode(box.w, box.h, h->esz) == 1 &&
            (size_t)na * ((strides[i] + 31) / 32) > (size_t)32 * team) {  // as the solver's test
            const int br = roi::band_rows(box.w, box.h, h->esz), nch = (strides[i] + 31) / 32;
            part_cap = std::max(part_cap, ((size_t)(box.h + br - 1) / br * nr + (size_t)(box.w + br - 1) / br * (na - nr)) *
                                              nch * 32);
        }
        const roi_solve_params& P = params[i];
        roi::BatchRoi& R = prois[i];
        R = roi::BatchRoi{};
        R.rec = bb.tab.p + (size_t)i * na;
        R.out = out_on_device ? outs[i] : bb.out.p + ooff;
        R.na = na;
        R.nrow = nr;
        R.nx = box.w;
        R.ny = box.h;
        R.stride = strides[i];
        R.reg = (int)P.reg;  // 0 SIRT, 1 CP-TV, 2 filter SIRT, 3 filter FISTA-TV, 4 filter Haar-ISTA
        R.iters = P.iters;
        R.weighting = P.reg == ROI_SIRT_NONNEG && P.weighting ? 1 : 0;
        R.lambda = (float)P.lambda;
        R.sigma_v = 0.5f;
        R.crop = P.crop_disk ? 1 : 0;
        R.cxl = (float)(regions[i].cx - box.x0);
        R.cyl = (float)(regions[i].cy - box.y0);
        R.r2 = (float)(regions[i].radius * regions[i].radius);
        exterior_inputs(h, R, box);
        filter_inputs(h, R);
        R.n_fgp = P.inner_iters ? P.inner_iters : 100;
        R.lam_f = (float)(0.5 * P.lambda / ((double)na * h->nd));
        R.shape = h->opt_tile_shape >= 0 ? h->opt_tile_shape : h->tile_shape[roi::shape_class(std::max(box.w, box.h))];
        ooff += (size_t)box.w * box.h;
        pord[i] = i;
        if (infos) {
            infos[i].box_x0 = box.x0;
            infos[i].box_y0 = box.y0;
            infos[i].box_w = box.w;
            infos[i].box_h = box.h;
            infos[i].window_max = wl;
            infos[i].window_stride = strides[i];
            infos[i].iters_done = P.iters;
            infos[i].step_L = 0.0;
            infos[i].objective = 0.0;
        }
    }
    std::stable_sort(pord, pord + n, [&](int a, int b) { return cost[a] > cost[b]; });
    CU(h, cudaMemcpyAsync(bb.tab.p, ptab, tab_bytes, cudaMemcpyHostToDevice, h->st));
    CU(h, cudaMemcpyAsync(bb.rois.p, prois, roi_bytes, cudaMemcpyHostToDevice, h->st));
    CU(h, cudaMemcpyAsync(bb.order.p, pord, ord_bytes, cudaMemcpyHostToDevice, h->st));
    CU(h, cudaEventRecord(h->pin_free, h->st));
    if (part_cap) CU(h, bb.part.ensure(part_cap * slots));
    // ---- all solves, exterior steps included, in one persistent launch
    roi::BatchArgs B{};
    B.rois = bb.rois.p;
    B.order = bb.order.p;
    B.nroi = n;
    B.queue = bb.queue.p;
    B.slot_pp = bb.pp.p;
    B.slot_u = bb.u.p;
    B.slot_sig = bb.sig.p;
    B.win_cap = win_cap;
    B.slot_x = bb.x.p;
    B.slot_vx = bb.vx.p;
    B.slot_vy = bb.vy.p;
    B.slot_tau = bb.tau.p;
    B.img_cap = img_cap;
    B.slot_xa = bb.xa.p;
    B.slot_xaT = bb.xaT.p;
    B.pad_cap = pad_cap;
    B.slot_fgp = need_fgp ? bb.fgp.p : nullptr;
    B.slot_part = part_cap ? bb.part.p : nullptr;
    B.part_cap = part_cap;
    B.err = h->d_err;
    B.wait_ns = h->opt_wait_ns;
    B.team = team > 1 ? team : 1;
    B.bars = team > 1 ? bb.bars.p : nullptr;
    B.absent = h->opt_phantoms;
    // partial-sum room for band-streamed passes when a block gets 128 or more units of a region
    const size_t per_block = (max_banded_units + (team > 1 ? team : 1) - 1) / (team > 1 ? team : 1);
    const size_t smem = roi::batch_smem_bytes(max_stage, h->na, per_block >= 128);
    cudaError_t e;
    if (capture) {  // a batch plan: the uploads done, the launch alone captured into a graph
        // (on a private stream: the handle's stream may be the legacy default stream, which
        // cannot be captured; the graph is replayed on the handle's stream)
        CU(h, cudaStreamSynchronize(h->st));
        cudaStream_t cs = nullptr;
        CU(h, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
        if (e == cudaSuccess) {
            e = roi::launch_batch(B, blocks, smem, cs);
            cudaGraph_t graph = nullptr;
            const cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
            if (e == cudaSuccess) e = e2;
            if (e == cudaSuccess) e = cudaGraphInstantiate(capture, graph, 0);
            if (graph) cudaGraphDestroy(graph);
        }
        cudaStreamDestroy(cs);
        if (e != cudaSuccess) return cuda_fail(h, e, "batch plan capture");
        return ROI_OK;
    }
    {
        Span sp(h, 2);
        e = roi::launch_batch(B, blocks, smem, h->st);
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "batched solve launch");
    if (!out_on_device) {
        std::vector<float> all(out_total);
        CU(h, cudaMemcpyAsync(all.data(), bb.out.p, sizeof(float) * out_total, cudaMemcpyDeviceToHost, h->st));
        roi_status s = roi_recon_sync(h);
        if (s != ROI_OK) return s;
        size_t o = 0;
        for (int i = 0; i < n; ++i) {
            const size_t m = (size_t)boxes[i].w * boxes[i].h;
            std::memcpy(outs[i], all.data() + o, sizeof(float) * m);
            o += m;
        }
    }
    return ROI_OK;
}

}  // namespace

roi_status roi_recon_solve_batch(roi_recon_t h, int n, const roi_region* regions, const roi_solve_params* params,
                                 float* const* outs, int out_on_device, roi_solve_info* infos) {
    if (!h) return ROI_EINVAL;
    h->err.clear();
    return solve_batch_impl(h, n, regions, params, outs, out_on_device, infos, 0);
}

// A batch planned once and launched as one captured CUDA graph (config 3's persistent launch):
// its own copy of the batch buffers, the graph of the launch (the queue or team-barrier reset
// and the kernel).
struct roi_batch_plan {
    roi_recon* h = nullptr;
    BatchBufs bb;
    cudaGraphExec_t exec = nullptr;
};

roi_status roi_recon_batch_plan_create(roi_recon_t h, int n, const roi_region* regions,
                                       const roi_solve_params* params, float* const* outs, roi_solve_info* infos,
                                       roi_batch_plan_t* out) {
    if (!h || !out) return ROI_EINVAL;
    h->err.clear();
    *out = nullptr;
    if (n < 1 || !regions || !params || !outs) return fail(h, ROI_EINVAL, "batch_plan_create: bad arguments");
    for (int i = 0; i < n; ++i)
        if (params[i].reg != ROI_SIRT_NONNEG && params[i].reg != ROI_TV_CP)
            return fail(h, ROI_EINVAL, "batch_plan_create: region %d: plans take SIRT and CP-TV regions", i);
    roi_batch_plan* P = new (std::nothrow) roi_batch_plan;
    if (!P) return fail(h, ROI_ENOMEM, "batch_plan_create: host memory");
    P->h = h;
    const roi_status s = solve_batch_impl(h, n, regions, params, outs, 1, infos, 0, &P->bb, &P->exec);
    if (s != ROI_OK) {
        cudaStreamSynchronize(h->st);
        if (P->exec) cudaGraphExecDestroy(P->exec);
        delete P;
        return s;
    }
    h->plans.push_back(P);
    *out = P;
    return ROI_OK;
}

roi_status roi_recon_batch_plan_launch(roi_recon_t h, roi_batch_plan_t plan) {
    if (!h || !plan || plan->h != h) return ROI_EINVAL;
    h->err.clear();
    if (!h->have_fbp) return fail(h, ROI_ESTATE, "batch_plan_launch: no FBP image (call fbp first)");
    const roi_status s = ensure_residual(h);  // this sinogram's residual, on the handle's stream
    if (s != ROI_OK) return s;
    Span sp(h, 2);
    CU(h, cudaGraphLaunch(plan->exec, h->st));
    h->state_valid = false;
    h->state_region_path = false;
    return ROI_OK;
}

roi_status roi_recon_batch_plan_destroy(roi_recon_t h, roi_batch_plan_t plan) {
    if (!h || !plan) return ROI_EINVAL;
    auto it = std::find(h->plans.begin(), h->plans.end(), plan);
    if (it == h->plans.end()) return ROI_EINVAL;
    cudaStreamSynchronize(h->st);  // no launch of the plan in flight when its buffers go
    if (plan->exec) cudaGraphExecDestroy(plan->exec);
    h->plans.erase(it);
    delete plan;
    return ROI_OK;
}

roi_status roi_recon_solve_tiled(roi_recon_t h, int tile, int margin, const roi_solve_params* params, float* out) {
    if (!h) return ROI_EINVAL;
    h->err.clear();
    if (!params || !out) return fail(h, ROI_EINVAL, "solve_tiled: null argument");
    if (tile < 2 || tile % 2 || h->N % tile) return fail(h, ROI_EINVAL, "solve_tiled: tile must be even and divide N");
    if (margin < 0 || margin > h->N) return fail(h, ROI_EINVAL, "solve_tiled: margin out of range");
    if (params->crop_disk) return fail(h, ROI_EINVAL, "solve_tiled: tiles are squares (crop_disk = 0)");
    const int nt = h->N / tile, n = nt * nt;
    std::vector<roi_region> regions(n);
    std::vector<roi_solve_params> prms(n, *params);
    std::vector<Rect> boxes(n);
    size_t total = 0;
    for (int ti = 0; ti < nt; ++ti)
        for (int tj = 0; tj < nt; ++tj) {
            roi_region& r = regions[ti * nt + tj];
            r.cx = tj * tile + 0.5 * (tile - 1);
            r.cy = ti * tile + 0.5 * (tile - 1);
            r.radius = 0.5 * tile;
            r.margin = margin;
            Rect box;
            roi::plan_box(h->N, r.cx, r.cy, r.radius, r.margin, &box);
            boxes[ti * nt + tj] = box;
            total += (size_t)box.w * box.h;
        }
    DevBuf boxes_out;
    CU(h, boxes_out.ensure(total));
    std::vector<float*> outs(n);
    size_t off = 0;
    for (int k = 0; k < n; ++k) {
        outs[k] = boxes_out.p + off;
        off += (size_t)boxes[k].w * boxes[k].h;
    }
    roi_status s = roi_recon_solve_batch(h, n, regions.data(), prms.data(), outs.data(), 1, nullptr);
    if (s != ROI_OK) return s;
    std::vector<unsigned char> tab(roi::tile_src_bytes() * n);
    for (int ti = 0; ti < nt; ++ti)
        for (int tj = 0; tj < nt; ++tj) {
            const int k = ti * nt + tj;
            roi::tile_src_fill(tab.data(), k, outs[k], boxes[k].w, tj * tile - boxes[k].x0, ti * tile - boxes[k].y0,
                               tj * tile, ti * tile);
        }
    DevBufT<unsigned char> tab_dev;
    CU(h, tab_dev.ensure(tab.size()));
    CU(h, cudaMemcpyAsync(tab_dev.p, tab.data(), tab.size(), cudaMemcpyHostToDevice, h->st));
    roi::launch_paste_tiles(tab_dev.p, n, tile, out, h->N, h->st);
    LAUNCHED(h, "tile paste");
    CU(h, cudaStreamSynchronize(h->st));  // the scratch buffers are freed on return
    return ROI_OK;
}

roi_status roi_recon_autotune(roi_recon_t h, int regions_per_class, int iters, int* shapes_out, double* ms_out) {
    if (!h) return ROI_EINVAL;
    h->err.clear();
    if (!h->have_fbp) return fail(h, ROI_ESTATE, "autotune: no FBP image (call fbp first)");
    if (regions_per_class < 0 || regions_per_class > 100000 || iters < 0 || iters > 100000)
        return fail(h, ROI_EINVAL, "autotune: regions_per_class or iters out of range");
    const int n = regions_per_class ? regions_per_class : 2 * std::max(h->sms, 1);
    const int it = iters ? iters : 20;
    // box sides of the classes (side = 2 ceil(1.5 r) with margin r / 2)
    const int side_lo[roi::kShapeClasses] = {48, 97, 217}, side_hi[roi::kShapeClasses] = {96, 216, 384};
    unsigned long long rng = 0x9E3779B97F4A7C15ull;  // splitmix64, seeded the same every call
    auto uni = [&rng]() {
        unsigned long long z = (rng += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return (double)((z ^ (z >> 31)) >> 11) * (1.0 / 9007199254740992.0);
    };
    const int keep = h->opt_tile_shape;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CU(h, cudaEventCreate(&e0));
    cudaError_t ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(h, ce, "autotune events");
    }
    roi_status st = ROI_OK;
    DevBuf outb;
    for (int c = 0; c < roi::kShapeClasses && st == ROI_OK; ++c) {
        const int hi = std::min(side_hi[c], h->N);
        if (hi < side_lo[c]) {  // the grid has no box of this class
            for (int sh = 0; sh < roi::kTileShapes; ++sh)
                if (ms_out) ms_out[c * roi::kTileShapes + sh] = 0.0;
            for (int k = 0; k < 4; ++k) h->team_ms[c][k] = 0.0;
            continue;
        }
        std::vector<roi_region> regs(n);
        std::vector<roi_solve_params> prms(n);
        std::vector<float*> outs(n);
        size_t total = 0;
        std::vector<size_t> off(n);
        for (int i = 0; i < n; ++i) {
            const int side = side_lo[c] + (int)(uni() * (hi - side_lo[c] + 1));
            const double r = std::max(1.0, (side / 2 - 0.5) / 1.5);  // box 2 ceil(1.5 r) = side (even)
            const double ext = std::ceil(1.5 * r);
            const double span = std::max(0.0, h->N - 2.0 * ext);
            regs[i] = roi_region{ext + uni() * span, ext + uni() * span, r, 0.5 * r};
            prms[i] = roi_solve_params{};
            prms[i].reg = (i & 1) ? ROI_TV_CP : ROI_SIRT_NONNEG;
            prms[i].lambda = (i & 1) ? 0.01 : 0.0;
            prms[i].iters = it;
            prms[i].precond = 1;
            Rect box;
            roi::plan_box(h->N, regs[i].cx, regs[i].cy, regs[i].radius, regs[i].margin, &box);
            off[i] = total;
            total += (size_t)box.w * box.h;
        }
        st = outb.ensure(total) == cudaSuccess ? ROI_OK : fail(h, ROI_ENOMEM, "autotune: output buffer");
        if (st != ROI_OK) break;
        for (int i = 0; i < n; ++i) outs[i] = outb.p + off[i];
        double best = 0.0;
        int best_sh = 0;
        for (int sh = 0; sh < roi::kTileShapes && st == ROI_OK; ++sh) {
            h->opt_tile_shape = sh;
            double ms = 0.0;
            for (int rep = 0; rep < 3 && st == ROI_OK; ++rep) {  // a warm-up, then the best of two
                cudaEventRecord(e0, h->st);
                st = solve_batch_impl(h, n, regs.data(), prms.data(), outs.data(), 1, nullptr, 0);
                cudaEventRecord(e1, h->st);
                if (st == ROI_OK) st = roi_recon_sync(h);
                float t = 0.f;
                if (st == ROI_OK && cudaEventElapsedTime(&t, e0, e1) == cudaSuccess && rep > 0)
                    ms = rep == 1 ? t : std::min(ms, (double)t);
            }
            if (ms_out) ms_out[c * roi::kTileShapes + sh] = ms;
            if (st == ROI_OK && (sh == 0 || ms < best)) {
                best = ms;
                best_sh = sh;
            }
        }
        if (st == ROI_OK) h->tile_shape[c] = best_sh;
        // the team size of a few-region batch (8 regions of the class, the chosen shape):
        // results are the same bits for every team size, only the time differs
        h->opt_tile_shape = -1;
        const int nf = std::min(n, 8);
        static const int caps[4] = {4, 8, 16, 32};
        double best_t = 0.0;
        int best_cap = h->team_cap[c];
        const int keep_cap = h->team_cap[c];
        for (int k = 0; k < 4 && st == ROI_OK; ++k) {
            h->team_cap[c] = caps[k];
            double ms = 0.0;
            for (int rep = 0; rep < 3 && st == ROI_OK; ++rep) {
                cudaEventRecord(e0, h->st);
                st = solve_batch_impl(h, nf, regs.data(), prms.data(), outs.data(), 1, nullptr, 0);
                cudaEventRecord(e1, h->st);
                if (st == ROI_OK) st = roi_recon_sync(h);
                float t = 0.f;
                if (st == ROI_OK && cudaEventElapsedTime(&t, e0, e1) == cudaSuccess && rep > 0)
                    ms = rep == 1 ? t : std::min(ms, (double)t);
            }
            h->team_ms[c][k] = ms;
            if (st == ROI_OK && (k == 0 || ms < best_t)) {
                best_t = ms;
                best_cap = caps[k];
            }
        }
        h->team_cap[c] = st == ROI_OK ? best_cap : keep_cap;
    }
    outb.release();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->opt_tile_shape = keep;
    h->state_valid = false;
    h->state_region_path = false;
    if (st != ROI_OK) return st;
    if (shapes_out)
        for (int c = 0; c < roi::kShapeClasses; ++c) shapes_out[c] = h->tile_shape[c];
    std::lock_guard<std::mutex> g(g_tune_mu);
    auto& t = g_tune[TuneKey{h->N, h->na, h->nd, h->dt, fnv_doubles(h->angles)}];
    for (int c = 0; c < roi::kShapeClasses; ++c) {
        t.shape[c] = h->tile_shape[c];
        t.team[c] = h->team_cap[c];
    }
    return ROI_OK;
}

roi_status roi_recon_set_tile_shapes(roi_recon_t h, const int* shapes) {
    if (!h) return ROI_EINVAL;
    h->err.clear();
    if (!shapes) return fail(h, ROI_EINVAL, "set_tile_shapes: null argument");
    for (int c = 0; c < roi::kShapeClasses; ++c)
        if (shapes[c] < 0 || shapes[c] >= roi::kTileShapes)
            return fail(h, ROI_EINVAL, "set_tile_shapes: unknown shape %d", shapes[c]);
    for (int c = 0; c < roi::kShapeClasses; ++c) h->tile_shape[c] = shapes[c];
    return ROI_OK;
}

roi_status roi_recon_get_tile_shapes(roi_recon_t h, int* shapes) {
    if (!h || !shapes) return ROI_EINVAL;
    for (int c = 0; c < roi::kShapeClasses; ++c) shapes[c] = h->tile_shape[c];
    return ROI_OK;
}

roi_status roi_recon_set_team_caps(roi_recon_t h, const int* caps) {
    if (!h) return ROI_EINVAL;
    h->err.clear();
    if (!caps) return fail(h, ROI_EINVAL, "set_team_caps: null argument");
    for (int c = 0; c < roi::kShapeClasses; ++c)
        if (caps[c] < 1 || caps[c] > 1024) return fail(h, ROI_EINVAL, "set_team_caps: team size %d out of range", caps[c]);
    for (int c = 0; c < roi::kShapeClasses; ++c) h->team_cap[c] = caps[c];
    return ROI_OK;
}

roi_status roi_recon_get_team_caps(roi_recon_t h, int* caps, double* ms_out) {
    if (!h || !caps) return ROI_EINVAL;
    for (int c = 0; c < roi::kShapeClasses; ++c) {
        caps[c] = h->team_cap[c];
        if (ms_out)
            for (int k = 0; k < 4; ++k) ms_out[c * 4 + k] = h->team_ms[c][k];
    }
    return ROI_OK;
}

roi_status roi_recon_set_timing(roi_recon_t h, int enable) {
    if (!h) return ROI_EINVAL;
    h->err.clear();
    CU(h, cudaStreamSynchronize(h->st));
    h->timing = enable != 0;
    for (auto& s : h->spans) s.clear();
    h->ev_used = 0;
    return ROI_OK;
}

roi_status roi_recon_set_option(roi_recon_t h, roi_option opt, long long value) {
    if (!h) return ROI_EINVAL;
    h->err.clear();
    switch (opt) {
        case ROI_OPT_SINGLE_LAUNCH:
            h->opt_persistent = value != 0;
            return ROI_OK;
        case ROI_OPT_WAIT_LIMIT_US:
            if (value < 1 || value > 600000000LL) return fail(h, ROI_EINVAL, "set_option: wait limit out of range");
            h->opt_wait_ns = (unsigned long long)value * 1000ull;
            return ROI_OK;
        case ROI_OPT_TEST_ABSENT_BLOCKS:
            if (value < 0 || value > 1024) return fail(h, ROI_EINVAL, "set_option: absent blocks out of range");
            h->opt_phantoms = (int)value;
            return ROI_OK;
        case ROI_OPT_TILE_SHAPE:
            if (value < -1 || value >= roi::kTileShapes) return fail(h, ROI_EINVAL, "set_option: unknown tile shape");
            h->opt_tile_shape = (int)value;
            return ROI_OK;
        case ROI_OPT_FILTER_CONV:
            if (value < 0 || value > 1) return fail(h, ROI_EINVAL, "set_option: filter convolution path is 0 or 1");
            h->opt_filter_fma = (int)value;
            return ROI_OK;
    }
    return fail(h, ROI_EINVAL, "set_option: unknown option %d", (int)opt);
}

int roi_recon_check_report(int* site, int* index) {
    cudaDeviceSynchronize();
    roi::CheckReport reps[6];
    roi::check_take_persist(&reps[0]);
    roi::check_take_batch(&reps[1]);
    roi::check_take_batch_team(&reps[2]);
    roi::check_take_serve(&reps[3]);
    roi::check_take_project(&reps[4]);
    roi::check_take_filterconv_tc(&reps[5]);
    int total = 0, first = -1;
    for (int i = 0; i < 6; ++i) {
        if (reps[i].count > 0 && first < 0) first = i;
        total += reps[i].count;
    }
    if (site) *site = first >= 0 ? reps[first].site : 0;
    if (index) *index = first >= 0 ? reps[first].index : 0;
    return total;
}

roi_status roi_recon_sync(roi_recon_t h) {
    if (!h) return ROI_EINVAL;
    h->err.clear();
    CU(h, cudaStreamSynchronize(h->st));
    int flag = 0;
    CU(h, cudaMemcpy(&flag, h->d_err, sizeof flag, cudaMemcpyDeviceToHost));
    if (flag) {
        CU(h, cudaMemset(h->d_err, 0, sizeof(int)));
        return fail(h, ROI_ETIMEOUT, "a device-side wait of a single-launch solve gave up; its result is invalid");
    }
    return ROI_OK;
}

roi_status roi_recon_kernel_times(roi_recon_t h, int kernel, int* launches, double* total_ms) {
    if (!h || kernel < 0 || kernel > 3 || !launches || !total_ms) return ROI_EINVAL;
    h->err.clear();
    CU(h, cudaStreamSynchronize(h->st));
    double ms = 0.0;
    for (auto& pr : h->spans[kernel]) {
        float t = 0.f;
        CU(h, cudaEventElapsedTime(&t, pr.first, pr.second));
        ms += t;
    }
    *launches = (int)h->spans[kernel].size();
    *total_ms = ms;
    return ROI_OK;
}

unsigned long long roi_recon_launch_count(void) { return roi::launches_total(); }

roi_status roi_recon_test_fail_alloc(int nth) {
    if (nth < 0) return ROI_EINVAL;
    roi::g_fail_alloc.store(nth, std::memory_order_relaxed);
    return ROI_OK;
}

}  // extern "C"
