// server.cu -- host side of the ROI server (roi_server_* in roi_recon.h): admission by
// memory budget, publication into the rings read by the serving kernel (serve.cu),
// completion polling, memory recycling and kernel relaunch.
//
// Sec. 5.5 of the paper: local reconstructions are independent, so many of them can be
// in flight at once.  Requests are planned on the host at submission (box, per-angle
// windows), queued per unit pool in arrival order and admitted in that order while the
// state of the admitted requests fits the device budget and their results fit the
// page-locked result area.  Admission writes the ring slot (descriptor + table) and
// then publishes it with a release store of the ring's tail; the kernel's units claim
// tickets while it runs.  Completion words written by the kernel (release, system
// scope) are polled with acquire loads; a completed request frees its ring slot and
// device state, its result stays in the page-locked area until roi_server_take.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "roi_internal.h"
#include "roi_recon.h"

using roi::AngleRec;
using roi::Rect;

namespace {

constexpr size_t kAlign = 256;
size_t round_up(size_t n) { return (n + kAlign - 1) / kAlign * kAlign; }

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

// First-fit allocator of offsets in [0, size) with coalescing of free ranges.
struct Arena {
    size_t size = 0, used = 0, peak = 0;
    std::map<size_t, size_t> free_;  // offset -> length
    void init(size_t n) {
        size = n;
        used = peak = 0;
        free_.clear();
        if (n) free_[0] = n;
    }
    bool alloc(size_t n, size_t* off) {
        n = round_up(n);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < n) continue;
            *off = it->first;
            const size_t rest = it->second - n, o2 = it->first + n;
            free_.erase(it);
            if (rest) free_[o2] = rest;
            used += n;
            peak = std::max(peak, used);
            return true;
        }
        return false;
    }
    void release(size_t off, size_t n) {
        n = round_up(n);
        used -= n;
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

// Byte layout of a request's device state (one block of the device arena).
struct StateLayout {
    size_t pp, u, sig, x, vx, vy, tau, xa, xaT, fgp, total;
};
StateLayout state_layout(int na, int stride, int nx, int ny, int esz, bool fgp = false) {
    StateLayout L{};
    const size_t win = round_up(sizeof(float) * (size_t)na * stride);
    const size_t img = round_up(sizeof(float) * (size_t)nx * ny);
    const size_t pr = round_up((size_t)esz * ny * roi::padded_ld_e(nx, esz));  // projector images: storage type
    const size_t pc = round_up((size_t)esz * nx * roi::padded_ld_e(ny, esz));
    size_t o = 0;
    L.pp = o, o += win;
    L.u = o, o += win;
    L.sig = o, o += win;
    L.x = o, o += img;
    L.vx = o, o += img;
    L.vy = o, o += img;
    L.tau = o, o += img;
    L.xa = o, o += pr;
    L.xaT = o, o += pc;
    L.fgp = o;
    if (fgp) o += 5 * img;
    L.total = o;
    return L;
}

struct Req {
    long long id = 0;
    int sino = 0, pool = 0;
    roi_region region{};
    roi_solve_params prm{};
    Rect box{};
    int stride = 0, nrow = 0;
    std::vector<AngleRec> rec;
    StateLayout lay{};
    size_t dev_off = 0, host_off = 0, host_bytes = 0;
    bool has_dev = false, has_host = false;
    long long ticket = -1;
    double t_submit = 0, t_publish = 0, t_done = 0;
    double est_ms = 0;  // estimated time of a solve on every block (the solo launch)
    roi_status status = ROI_OK;
    int state = 0;  // 0 pending, 1 published, 2 done
};

struct Pool {
    int team = 1, nteams = 0, first_block = 0, team_base = 0;
    int slots = 0;
    size_t slot_bytes = 0;
    unsigned char* ring_h = nullptr;  // page-locked
    unsigned char* ring_d = nullptr;  // its device view
    unsigned long long* head_d = nullptr;
    std::vector<Req*> occupant;
    int live = 0;  // published and not yet completed
    long long next_ticket = 0;
    std::deque<Req*> pending;
};

// page-locked control words
struct Ctl {
    unsigned long long tail[2];
    int close;
    int pad;
};

}  // namespace

struct roi_server {
    roi_server_config cfg{};
    int device = 0;
    cudaStream_t st = nullptr;
    std::string err;
    std::vector<roi::SinoView> sinos;
    Pool pools[2];
    int blocks = 0, max_na = 0;
    bool rings_ready = false;
    // device memory
    unsigned char* arena_d = nullptr;
    Arena darena;
    unsigned char* dctl = nullptr;  // busy, last_ns, err, heads, bars, mail_seq, mail_val
    int* busy_d = nullptr;
    unsigned long long* last_d = nullptr;
    int* err_d = nullptr;
    unsigned* bars_d = nullptr;
    unsigned* mseq_d = nullptr;
    long long* mval_d = nullptr;
    AngleRec* rec_slots_d = nullptr;
    float* solo_part_d = nullptr;  // row-band partial sums of solo launches (see ensure_rings)
    size_t solo_part_cap = 0;      // floats
    size_t ctl_reset_bytes = 0;  // bars + mail words, zeroed at each launch
    unsigned* ctl_reset_d = nullptr;
    // page-locked memory
    unsigned char* out_h = nullptr;
    unsigned char* out_d = nullptr;
    Arena harena;
    Ctl* ctl_h = nullptr;
    Ctl* ctl_d = nullptr;
    unsigned long long* done_h[2] = {nullptr, nullptr};
    unsigned long long* done_d[2] = {nullptr, nullptr};
    unsigned char* ring_alloc = nullptr;
    // kernel state
    bool running = false;
    int mode = 0;          // of the running (or next) kernel: 0 the configured pools, 1 solo
    bool leaving = false;  // the close flag was set to end a solo launch
    cudaEvent_t ev_end = nullptr;
    long long launches = 0;
    // options (roi_server_set_option), read at each launch
    unsigned long long opt_wait_ns = 2000000000ull;  // team barrier / mailbox wait limit
    int opt_absent = 0;                               // testing only: absent participants / leaders
    // requests
    std::mutex mu;
    std::thread worker;
    std::atomic<bool> stop{false};
    bool started = false;
    long long next_id = 1;
    std::unordered_map<long long, Req*> reqs;
    std::deque<roi_server_completion> completed;
    long long n_submitted = 0, n_completed = 0, n_failed = 0, n_outstanding = 0, n_cancelled = 0;
};

namespace {

roi_status sfail(roi_server* s, roi_status st, const char* fmt, ...) __attribute__((format(printf, 3, 4)));
roi_status sfail(roi_server* s, roi_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    s->err = buf;
    return st;
}

roi_status scuda(roi_server* s, cudaError_t e, const char* where) {
    return sfail(s, e == cudaErrorMemoryAllocation ? ROI_ENOMEM : ROI_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define SCU(s, call)                                        \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return scuda(s, e_, #call);  \
    } while (0)

bool finite_region(const roi_region* r) {
    return r && std::isfinite(r->cx) && std::isfinite(r->cy) && std::isfinite(r->radius) &&
           std::isfinite(r->margin) && r->radius > 0 && r->margin >= 0 && r->radius + r->margin < 1e7;
}

// Plan of one request on a sinogram of N, na, nd; false when the box misses the grid.
bool plan_request(int N, int na, int nd, const double* angles, const roi_region& region, Rect* box, int* stride,
                  int* nrow, std::vector<AngleRec>* rec) {
    if (!roi::plan_box(N, region.cx, region.cy, region.radius, region.margin, box)) return false;
    if (rec) {
        rec->resize(na);
        const int wl = roi::plan_region_table(N, na, nd, angles, *box, rec->data(), nrow);
        *stride = roi::round_stride(wl);
    } else {
        std::vector<AngleRec> tmp(na);
        const int wl = roi::plan_angles(N, na, nd, angles, *box, *box, false, tmp.data());
        *stride = roi::round_stride(wl);
    }
    return true;
}

// Allocates the rings, per-block tables and control words (at the first submit, once
// the largest angle count is known).
roi_status ensure_rings(roi_server* s) {
    if (s->rings_ready) return ROI_OK;
    if (s->sinos.empty()) return sfail(s, ROI_ESTATE, "submit: no sinogram registered");
    s->max_na = 0;
    for (auto& v : s->sinos) s->max_na = std::max(s->max_na, v.na);
    const size_t slot_bytes = roi::serve_slot_header_bytes + round_up(sizeof(AngleRec) * (size_t)s->max_na);
    size_t ring_total = 0;
    for (Pool& P : s->pools) {
        P.slot_bytes = slot_bytes;
        P.occupant.assign(P.slots, nullptr);
        ring_total += P.nteams > 0 ? slot_bytes * P.slots : 0;
    }
    if (!s->ring_alloc)  // (kept when a later allocation here failed and submit is retried)
        SCU(s, roi::pinned_alloc((void**)&s->ring_alloc, std::max<size_t>(ring_total, kAlign),
                                 cudaHostAllocMapped | cudaHostAllocPortable));
    size_t off = 0;
    for (Pool& P : s->pools) {
        if (P.nteams == 0) continue;
        P.ring_h = s->ring_alloc + off;
        off += slot_bytes * P.slots;
        void* d = nullptr;
        SCU(s, cudaHostGetDevicePointer(&d, P.ring_h, 0));
        P.ring_d = (unsigned char*)d;
    }
    if (!s->rec_slots_d)
        SCU(s, roi::dev_malloc((void**)&s->rec_slots_d, sizeof(AngleRec) * (size_t)s->max_na * s->blocks));
    if (!s->solo_part_d) {
        // the largest square box of each geometry whose images are band-streamed, its row-band
        // partials (a box's window is below 1.5 side + 8 bins), at most 64 MB: larger boxes
        // keep the per-32-unit phase A (the kernel checks each request's own size)
        size_t need = 0;
        for (const roi::SinoView& v : s->sinos) {
            const int es = roi::dt_size(v.dt);
            for (int side = std::min(v.N, 4096); side >= 1; --side)
                if (roi::stage_mode(side, side, es) == 1) {
                    const int br = roi::band_rows(side, side, es);
                    need = std::max(need, (size_t)((side + br - 1) / br) * v.na * ((side * 3 / 2 + 8 + 31) / 32) * 32);
                    break;
                }
        }
        need = std::min<size_t>(need, (size_t)16 << 20);
        if (need) {
            SCU(s, roi::dev_malloc((void**)&s->solo_part_d, sizeof(float) * need));
            s->solo_part_cap = need;
        }
    }
    s->rings_ready = true;
    return ROI_OK;
}

void push_completion(roi_server* s, Req* r) {
    roi_server_completion c{};
    c.id = r->id;
    c.status = r->status;
    c.sino = r->sino;
    c.box_x0 = r->box.x0;
    c.box_y0 = r->box.y0;
    c.box_w = r->box.w;
    c.box_h = r->box.h;
    c.pool = r->pool;
    c.t_submit_ms = r->t_submit;
    c.t_publish_ms = r->t_publish;
    c.t_done_ms = r->t_done;
    s->completed.push_back(c);
}

void complete(roi_server* s, Pool& P, size_t slot, Req* r, roi_status status) {
    r->t_done = now_ms();
    r->status = status;
    r->state = 2;
    P.occupant[slot] = nullptr;
    --P.live;
    if (r->has_dev) {
        s->darena.release(r->dev_off, r->lay.total);
        r->has_dev = false;
    }
    if (status != ROI_OK && r->has_host) {
        s->harena.release(r->host_off, r->host_bytes);
        r->has_host = false;
    }
    --s->n_outstanding;
    if (status == ROI_OK)
        ++s->n_completed;
    else
        ++s->n_failed;
    push_completion(s, r);
}

void poll_done(roi_server* s) {
    for (int pi = 0; pi < 2; ++pi) {
        Pool& P = s->pools[pi];
        if (P.nteams == 0 || !s->rings_ready) continue;
        for (int k = 0; k < P.slots; ++k) {
            Req* r = P.occupant[k];
            if (!r) continue;
            const unsigned long long v = __atomic_load_n(s->done_h[pi] + k, __ATOMIC_ACQUIRE);
            if (v == (unsigned long long)r->ticket + 1ull) complete(s, P, k, r, ROI_OK);
        }
    }
}

// Writes slot `slot` of pool P for request r and publishes ticket r->ticket.
void publish(roi_server* s, int pi, Req* r, size_t slot) {
    Pool& P = s->pools[pi];
    const roi::SinoView& v = s->sinos[r->sino];
    unsigned char* sp = P.ring_h + slot * P.slot_bytes;
    roi::ServeSlot hdr{};
    roi::BatchRoi& R = hdr.roi;
    R.rec = nullptr;
    R.out = reinterpret_cast<float*>(s->out_d + r->host_off);
    R.na = v.na;
    R.nrow = r->nrow;
    R.nx = r->box.w;
    R.ny = r->box.h;
    R.stride = r->stride;
    R.reg = (int)r->prm.reg;  // 0 SIRT, 1 CP-TV, 2 filter SIRT, 3 filter FISTA-TV, 4 filter Haar-ISTA
    R.n_fgp = r->prm.inner_iters ? r->prm.inner_iters : 100;
    R.lam_f = (float)(0.5 * r->prm.lambda / ((double)v.na * v.nd));
    R.iters = r->prm.iters;
    R.weighting = r->prm.reg == ROI_SIRT_NONNEG && r->prm.weighting ? 1 : 0;
    R.lambda = (float)r->prm.lambda;
    R.sigma_v = 0.5f;
    R.alpha = (float)(1.0 / ((double)v.na * v.nd));
    R.crop = r->prm.crop_disk ? 1 : 0;
    R.cxl = (float)(r->region.cx - r->box.x0);
    R.cyl = (float)(r->region.cy - r->box.y0);
    R.r2 = (float)(r->region.radius * r->region.radius);
    R.resid = v.resid;
    R.resid_ld = v.resid_ld;
    R.xfbp = v.xfbp;
    R.xfbpT = v.xfbpT;
    R.xfbp_ld = v.xfbp_ld;
    R.box_x0 = r->box.x0;
    R.box_y0 = r->box.y0;
    R.dt = v.dt;
    R.fcp = v.fcp;
    R.fcp_nd = v.nd;
    R.disc_g = v.disc_g;
    R.grid_n = v.N;
    R.shape = v.shape[roi::shape_class(std::max(r->box.w, r->box.h))];
    unsigned char* base = s->arena_d + r->dev_off;
    roi::RegionBufs& B = hdr.bufs;
    B.pp = reinterpret_cast<float*>(base + r->lay.pp);
    B.u = reinterpret_cast<float*>(base + r->lay.u);
    B.sig = reinterpret_cast<float*>(base + r->lay.sig);
    B.x = reinterpret_cast<float*>(base + r->lay.x);
    B.vx = reinterpret_cast<float*>(base + r->lay.vx);
    B.vy = reinterpret_cast<float*>(base + r->lay.vy);
    B.tau = reinterpret_cast<float*>(base + r->lay.tau);
    B.xa_base = base + r->lay.xa;
    B.xaT_base = base + r->lay.xaT;
    B.fgp = r->prm.reg >= ROI_FILTER_TV ? reinterpret_cast<float*>(base + r->lay.fgp) : nullptr;
    B.part = nullptr;
    hdr.seq = (unsigned long long)r->ticket + 1ull;
    std::memcpy(sp, &hdr, sizeof hdr);
    std::memcpy(sp + roi::serve_slot_header_bytes, r->rec.data(), sizeof(AngleRec) * r->rec.size());
    r->t_publish = now_ms();
    r->state = 1;
    P.occupant[slot] = r;
    ++P.live;
    // the slot's contents before the new tail (release, read by the kernel with acquire)
    __atomic_store_n(&s->ctl_h->tail[pi], (unsigned long long)(r->ticket + 1), __ATOMIC_RELEASE);
}

// Single-block units left by the default pool split (the rest of the blocks form teams).
constexpr int kSingleUnits = 24;

// A solo launch serves the queue one request at a time on every block (the latency of a
// whole-GPU solve, the plain one-at-a-time throughput).  It is asked to leave when the work
// queued behind it, estimated in solo milliseconds, exceeds cfg.solo_queue_ms (or more than
// kSoloQueue requests wait): the pools' throughput is then worth more than the solo latency.
constexpr int kSoloQueue = 64;
// Estimated solo time of a request: its projector work at a whole-GPU rate, but no less than
// a fixed cost per iteration (a small box is latency-bound on a team of every block).
constexpr double kSoloLerpsPerMs = 1.1e9;
constexpr double kSoloIterMs = 0.012;

double solo_ms_live(const roi_server* s) {
    double w = 0.0;
    for (const Req* r : s->pools[1].occupant)
        if (r && r->state == 1) w += r->est_ms;
    return w;
}

// Admits pending requests in arrival order per pool while their state fits the budgets.
// A small-box request goes to the team pool instead when a team is idle there and no
// large request waits for one (unless no_spill): at light load a request then runs on a
// team of blocks rather than one block, at heavy load the teams are busy and it stays in
// its pool.  While a solo launch runs (and is not leaving), every request goes to the team
// ring.  The result is the same bits either way.
void admit(roi_server* s) {
    for (int pi = 0; pi < 2; ++pi) {
        std::deque<Req*>& pend = s->pools[pi].pending;
        while (!pend.empty()) {
            Req* r = pend.front();
            Pool& T = s->pools[1];
            const int to = ((s->mode == 1 && !s->leaving) ||
                            (pi == 0 && !s->cfg.no_spill && T.nteams > 0 && T.pending.empty() && T.live < T.nteams &&
                             !T.occupant[(size_t)(T.next_ticket % T.slots)]))
                               ? 1
                               : pi;
            Pool& P = s->pools[to];
            const size_t slot = (size_t)(P.next_ticket % P.slots);
            if (P.occupant[slot]) break;  // ring full at this position
            size_t doff = 0, hoff = 0;
            if (!s->darena.alloc(r->lay.total, &doff)) break;
            if (!s->harena.alloc(r->host_bytes, &hoff)) {
                s->darena.release(doff, r->lay.total);
                break;
            }
            r->dev_off = doff;
            r->host_off = hoff;
            r->has_dev = r->has_host = true;
            r->ticket = P.next_ticket++;
            r->pool = to;
            pend.pop_front();
            publish(s, to, r, slot);
        }
    }
}

bool any_published(const roi_server* s) {
    for (const Pool& P : s->pools)
        for (const Req* r : P.occupant)
            if (r) return true;
    return false;
}

roi_status launch(roi_server* s) {
    SCU(s, cudaMemsetAsync(s->ctl_reset_d, 0, s->ctl_reset_bytes, s->st));
    __atomic_store_n(&s->ctl_h->close, 0, __ATOMIC_RELEASE);  // no kernel runs here
    s->leaving = false;
    SCU(s, cudaMemsetAsync(s->busy_d, 0, sizeof(int), s->st));
    SCU(s, cudaMemsetAsync(s->last_d, 0, sizeof(unsigned long long), s->st));
    roi::ServeArgs A{};
    for (int pi = 0; pi < 2; ++pi) {
        const Pool& P = s->pools[pi];
        roi::ServePool& D = A.pool[pi];
        D.ring = P.ring_d;
        D.slot_bytes = P.slot_bytes;
        D.slots = P.slots;
        D.first_block = P.first_block;
        D.team = P.team;
        D.nteams = P.nteams;
        D.team_base = P.team_base;
        D.head = P.head_d;
        D.tail = &s->ctl_d->tail[pi];
        D.done = s->done_d[pi];
    }
    if (s->mode == 1) {  // solo: no single-block units, one team of every block
        A.pool[0].nteams = 0;
        A.pool[1].first_block = 0;
        A.pool[1].team = s->blocks;
        A.pool[1].nteams = 1;
        A.pool[1].team_base = 0;
    }
    A.close = &s->ctl_d->close;
    A.busy = s->busy_d;
    A.last_ns = s->last_d;
    A.bars = s->bars_d;
    A.mail_seq = s->mseq_d;
    A.mail_val = s->mval_d;
    A.rec_slots = s->rec_slots_d;
    A.max_na = s->max_na;
    A.idle_ns = (unsigned long long)s->cfg.idle_us * 1000ull;
    // a unit polls for work at most 60 s; with absent leaders (testing) their members'
    // mailbox waits, bounded by this plus the wait limit, run out soon
    A.cap_ns = s->opt_absent < 0 ? s->opt_wait_ns : 60ull * 1000000000ull;
    A.err = s->err_d;
    A.wait_ns = s->opt_wait_ns;
    A.absent = s->opt_absent;
    A.solo_part = s->mode == 1 ? s->solo_part_d : nullptr;
    A.solo_part_cap = s->solo_part_cap;
    cudaError_t e = roi::launch_serve(A, s->blocks, s->st);
    if (e != cudaSuccess) return scuda(s, e, "serving kernel launch");
    SCU(s, cudaEventRecord(s->ev_end, s->st));
    s->running = true;
    ++s->launches;
    return ROI_OK;
}

// The kernel has left: requests it claimed but did not finish have failed.
roi_status kernel_ended(roi_server* s) {
    s->running = false;
    poll_done(s);
    int flag = 0;
    unsigned long long heads[2] = {0, 0};
    SCU(s, cudaMemcpyAsync(&flag, s->err_d, sizeof flag, cudaMemcpyDeviceToHost, s->st));
    for (int pi = 0; pi < 2; ++pi)
        SCU(s, cudaMemcpyAsync(&heads[pi], s->pools[pi].head_d, sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                               s->st));
    SCU(s, cudaStreamSynchronize(s->st));
    for (int pi = 0; pi < 2; ++pi) {
        Pool& P = s->pools[pi];
        for (int k = 0; k < P.slots; ++k) {
            Req* r = P.occupant[k];
            if (r && (unsigned long long)r->ticket < heads[pi]) complete(s, P, k, r, flag ? ROI_ETIMEOUT : ROI_ECUDA);
        }
    }
    if (flag) {
        SCU(s, cudaMemsetAsync(s->err_d, 0, sizeof(int), s->st));
        return sfail(s, ROI_ETIMEOUT, "a device-side wait of the serving kernel gave up; its requests failed");
    }
    return ROI_OK;
}

roi_status progress_locked(roi_server* s) {
    roi_status st = ROI_OK;
    if (s->running) {
        const cudaError_t q = cudaEventQuery(s->ev_end);
        if (q == cudaSuccess) {
            st = kernel_ended(s);
        } else if (q != cudaErrorNotReady) {
            return scuda(s, q, "serving kernel");
        }
    }
    if (!s->rings_ready) return st;
    poll_done(s);
    // Mode of the next launch: a lone request on an idle server runs on one team of every
    // block (solo: the latency of a whole-GPU solve); otherwise the configured pools.
    if (!s->running) {
        size_t pend = 0;
        double work = 0.0;
        for (const Pool& P : s->pools) {
            pend += P.pending.size();
            for (const Req* r : P.pending) work += r->est_ms;
        }
        s->mode = (!s->cfg.no_spill && s->pools[1].nteams > 0 && s->pools[0].live + s->pools[1].live == 0 &&
                   (pend == 1 || (pend > 1 && pend <= (size_t)kSoloQueue && work <= s->cfg.solo_queue_ms)))
                      ? 1
                      : 0;
    }
    admit(s);
    // A queue behind a solo launch (more queued work than solo_queue_ms, or more than
    // kSoloQueue requests): let it finish the request it holds and leave, so the next launch
    // serves the queue with the configured pools, whose throughput is higher.
    if (s->running && s->mode == 1 && !s->leaving &&
        (solo_ms_live(s) > s->cfg.solo_queue_ms || s->pools[1].live > kSoloQueue)) {
        __atomic_store_n(&s->ctl_h->close, 1, __ATOMIC_RELEASE);
        s->leaving = true;
    }
    if (!s->running && any_published(s)) {
        roi_status l = launch(s);
        if (l != ROI_OK) return l;
    }
    return st;
}

void worker_loop(roi_server* s) {
    cudaSetDevice(s->device);
    while (!s->stop.load(std::memory_order_relaxed)) {
        bool idle;
        {
            std::lock_guard<std::mutex> g(s->mu);
            progress_locked(s);
            idle = s->n_outstanding == 0;
        }
        std::this_thread::sleep_for(std::chrono::microseconds(idle ? 200 : 20));
    }
}

void free_all(roi_server* s) {
    if (s->arena_d) cudaFree(s->arena_d);
    if (s->dctl) cudaFree(s->dctl);
    if (s->rec_slots_d) cudaFree(s->rec_slots_d);
    if (s->solo_part_d) cudaFree(s->solo_part_d);
    if (s->out_h) cudaFreeHost(s->out_h);
    if (s->ctl_h) cudaFreeHost(s->ctl_h);
    if (s->ring_alloc) cudaFreeHost(s->ring_alloc);
    if (s->ev_end) cudaEventDestroy(s->ev_end);
    if (s->st) cudaStreamDestroy(s->st);
    for (auto& kv : s->reqs) delete kv.second;
    s->reqs.clear();
}

}  // namespace

extern "C" {

roi_status roi_server_create(const roi_server_config* cfg_in, roi_server_t* out) {
    if (!out) return ROI_EINVAL;
    *out = nullptr;
    roi_server_config cfg{};
    if (cfg_in) cfg = *cfg_in;
    if (cfg.device_bytes == 0) cfg.device_bytes = (size_t)4 << 30;
    if (cfg.host_bytes == 0) cfg.host_bytes = (size_t)512 << 20;
    if (cfg.ring_slots == 0) cfg.ring_slots = 1024;
    if (cfg.team_blocks == 0) cfg.team_blocks = 16;
    if (cfg.large_side == 0) cfg.large_side = 256;
    if (cfg.idle_us == 0) cfg.idle_us = 2000;
    if (cfg.solo_queue_ms == 0) cfg.solo_queue_ms = 250;
    if (cfg.ring_slots < 1 || cfg.ring_slots > (1 << 20) || cfg.team_blocks < 1 || cfg.team_blocks > 1024 ||
        cfg.teams < -1 || cfg.large_side < 1 || cfg.idle_us < 1 || cfg.idle_us > 10000000 || cfg.no_spill < 0 ||
        cfg.no_spill > 1 || cfg.solo_queue_ms < 0 || cfg.solo_queue_ms > 3600000)
        return ROI_EINVAL;
    roi_server* s = new (std::nothrow) roi_server;
    if (!s) return ROI_ENOMEM;
    s->cfg = cfg;
    cudaError_t e = cudaGetDevice(&s->device);
    if (e == cudaSuccess) {
        s->blocks = roi::serve_max_blocks(s->device);
        if (s->blocks < 1) e = cudaErrorInvalidConfiguration;
    }
    if (e == cudaSuccess) {
        int coop = 0;
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, s->device);
        if (!coop) e = cudaErrorNotSupported;
    }
    if (e == cudaSuccess) {
        // pool split: teams of team_blocks from the top, single blocks below
        // default: every block but kSingleUnits in teams (boxes of side >= large_side carry
        // most of the work of a log-uniform radius mix)
        int teams = cfg.teams < 0 ? std::max(s->blocks - kSingleUnits, 0) / cfg.team_blocks : cfg.teams;
        teams = std::min(teams, (s->blocks - 1) / cfg.team_blocks);  // keep at least one single block
        teams = std::max(teams, 0);
        Pool& P0 = s->pools[0];
        Pool& P1 = s->pools[1];
        P0.team = 1;
        P0.nteams = s->blocks - teams * cfg.team_blocks;
        P0.first_block = 0;
        P0.team_base = 0;
        P1.team = cfg.team_blocks;
        P1.nteams = teams;
        P1.first_block = P0.nteams;
        P1.team_base = P0.nteams;
        for (Pool& P : s->pools) P.slots = cfg.ring_slots;
        s->cfg.teams = teams;
    }
    const int nteam_total = s->pools[0].nteams + s->pools[1].nteams;
    // device control block: [busy int][err int][last u64][head u64 x2] | bars | mail_seq | mail_val
    const size_t fixed = 64;
    const size_t bars_b = sizeof(unsigned) * (size_t)nteam_total, mseq_b = bars_b;
    const size_t mval_off = round_up(fixed + bars_b + mseq_b);
    const size_t ctl_bytes = mval_off + sizeof(long long) * (size_t)nteam_total;
    if (e == cudaSuccess) e = roi::dev_malloc((void**)&s->dctl, ctl_bytes);
    if (e == cudaSuccess) e = cudaMemset(s->dctl, 0, ctl_bytes);
    if (e == cudaSuccess) {
        s->busy_d = reinterpret_cast<int*>(s->dctl);
        s->err_d = reinterpret_cast<int*>(s->dctl + 4);
        s->last_d = reinterpret_cast<unsigned long long*>(s->dctl + 8);
        s->pools[0].head_d = reinterpret_cast<unsigned long long*>(s->dctl + 16);
        s->pools[1].head_d = reinterpret_cast<unsigned long long*>(s->dctl + 24);
        s->bars_d = reinterpret_cast<unsigned*>(s->dctl + fixed);
        s->mseq_d = reinterpret_cast<unsigned*>(s->dctl + fixed + bars_b);
        s->mval_d = reinterpret_cast<long long*>(s->dctl + mval_off);
        s->ctl_reset_d = s->bars_d;
        s->ctl_reset_bytes = bars_b + mseq_b;
        if (s->ctl_reset_bytes == 0) s->ctl_reset_bytes = 4;
    }
    if (e == cudaSuccess) e = roi::dev_malloc((void**)&s->arena_d, cfg.device_bytes);
    if (e == cudaSuccess) s->darena.init(cfg.device_bytes);
    if (e == cudaSuccess)
        e = roi::pinned_alloc((void**)&s->out_h, cfg.host_bytes, cudaHostAllocMapped | cudaHostAllocPortable);
    if (e == cudaSuccess) {
        void* d = nullptr;
        e = cudaHostGetDevicePointer(&d, s->out_h, 0);
        s->out_d = (unsigned char*)d;
        s->harena.init(cfg.host_bytes);
    }
    // control words and completion words, page-locked
    const size_t done_b = sizeof(unsigned long long) * (size_t)cfg.ring_slots;
    if (e == cudaSuccess)
        e = roi::pinned_alloc((void**)&s->ctl_h, round_up(sizeof(Ctl)) + 2 * round_up(done_b),
                              cudaHostAllocMapped | cudaHostAllocPortable);
    if (e == cudaSuccess) {
        std::memset(s->ctl_h, 0, round_up(sizeof(Ctl)) + 2 * round_up(done_b));
        void* d = nullptr;
        e = cudaHostGetDevicePointer(&d, s->ctl_h, 0);
        s->ctl_d = (Ctl*)d;
        for (int pi = 0; pi < 2; ++pi) {
            s->done_h[pi] = reinterpret_cast<unsigned long long*>(reinterpret_cast<unsigned char*>(s->ctl_h) +
                                                                  round_up(sizeof(Ctl)) + pi * round_up(done_b));
            s->done_d[pi] = reinterpret_cast<unsigned long long*>(reinterpret_cast<unsigned char*>(s->ctl_d) +
                                                                  round_up(sizeof(Ctl)) + pi * round_up(done_b));
        }
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_end, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        free_all(s);
        delete s;
        return e == cudaErrorMemoryAllocation ? ROI_ENOMEM : ROI_ECUDA;
    }
    *out = s;
    return ROI_OK;
}

roi_status roi_server_add_sinogram(roi_server_t s, roi_recon_t h, int* sino_id) {
    if (!s) return ROI_EINVAL;
    std::lock_guard<std::mutex> g(s->mu);
    if (!h || !sino_id) return sfail(s, ROI_EINVAL, "add_sinogram: null argument");
    if (s->rings_ready) return sfail(s, ROI_ESTATE, "add_sinogram: sinograms must be added before the first submit");
    roi::SinoView v{};
    std::string msg;
    const int st = roi::sino_view(h, &v, &msg);
    if (st != ROI_OK) return sfail(s, (roi_status)st, "add_sinogram: %s", msg.c_str());
    s->sinos.push_back(v);
    *sino_id = (int)s->sinos.size() - 1;
    return ROI_OK;
}

roi_status roi_server_submit(roi_server_t s, int sino_id, const roi_region* region, const roi_solve_params* params,
                             long long* id) {
    if (!s) return ROI_EINVAL;
    std::lock_guard<std::mutex> g(s->mu);
    if (!region || !params || !id) return sfail(s, ROI_EINVAL, "submit: null argument");
    if (sino_id < 0 || sino_id >= (int)s->sinos.size()) return sfail(s, ROI_EINVAL, "submit: unknown sinogram %d", sino_id);
    const roi_solve_params& P = *params;
    if (!finite_region(region)) return sfail(s, ROI_EINVAL, "submit: radius must be > 0, margin >= 0, all finite");
    if (P.reg < ROI_SIRT_NONNEG || P.reg > ROI_FILTER_ISTA) return sfail(s, ROI_EINVAL, "submit: unknown regularizer");
    if (P.inner_iters < 0 || P.inner_iters > 100000) return sfail(s, ROI_EINVAL, "submit: inner_iters out of range");
    if (P.iters < 0 || P.iters > 1000000) return sfail(s, ROI_EINVAL, "submit: iters out of range");
    if (!std::isfinite(P.lambda) || P.lambda < 0) return sfail(s, ROI_EINVAL, "submit: bad lambda");
    if (P.reg == ROI_TV_CP && !P.precond) return sfail(s, ROI_EINVAL, "submit: served CP uses the diagonal steps (precond = 1)");
    roi_status rs = ensure_rings(s);
    if (rs != ROI_OK) return rs;
    const roi::SinoView& v = s->sinos[sino_id];
    const bool filt = P.reg >= ROI_FILTER_SIRT;
    if (filt && v.fcp_n < P.iters)
        return sfail(s, ROI_ESTATE, "submit: sinogram %d has filters for %d iterations, %d asked", sino_id, v.fcp_n,
                     P.iters);
    if (!filt && !v.have_fbp)
        return sfail(s, ROI_ESTATE, "submit: sinogram %d has no FBP image", sino_id);
    Req* r = new (std::nothrow) Req;
    if (!r) return sfail(s, ROI_ENOMEM, "submit: out of host memory");
    if (!plan_request(v.N, v.na, v.nd, v.angles, *region, &r->box, &r->stride, &r->nrow, &r->rec)) {
        delete r;
        return sfail(s, ROI_EINVAL, "submit: extended box misses the %d x %d grid", v.N, v.N);
    }
    r->lay = state_layout(v.na, r->stride, r->box.w, r->box.h, roi::dt_size(v.dt), P.reg >= ROI_FILTER_TV);
    r->host_bytes = sizeof(float) * (size_t)r->box.w * r->box.h;
    {
        double lerps = 0.0;  // per iteration: window rays x box side, then pixels x angles
        for (const AngleRec& a : r->rec) lerps += (double)a.width * std::max(r->box.w, r->box.h);
        lerps += (double)r->box.w * r->box.h * v.na;
        const double it = std::max(P.iters, 1);
        r->est_ms = std::max(it * lerps / kSoloLerpsPerMs, it * kSoloIterMs);
    }
    if (round_up(r->lay.total) > s->darena.size || round_up(r->host_bytes) > s->harena.size) {
        const size_t need = r->lay.total;
        delete r;
        return sfail(s, ROI_ENOMEM, "submit: request needs %zu device bytes, more than the budget", need);
    }
    r->id = s->next_id++;
    r->sino = sino_id;
    r->region = *region;
    r->prm = P;
    const int side = std::max(r->box.w, r->box.h);
    r->pool = (s->pools[1].nteams > 0 && side >= s->cfg.large_side) ? 1 : 0;
    r->t_submit = now_ms();
    s->reqs[r->id] = r;
    s->pools[r->pool].pending.push_back(r);
    ++s->n_submitted;
    ++s->n_outstanding;
    *id = r->id;
    return ROI_OK;
}

roi_status roi_server_start(roi_server_t s) {
    if (!s) return ROI_EINVAL;
    std::lock_guard<std::mutex> g(s->mu);
    if (s->started) return ROI_OK;
    s->stop = false;
    s->worker = std::thread(worker_loop, s);
    s->started = true;
    return ROI_OK;
}

roi_status roi_server_stop(roi_server_t s) {
    if (!s) return ROI_EINVAL;
    {
        std::lock_guard<std::mutex> g(s->mu);
        if (!s->started) return ROI_OK;
        s->stop = true;
    }
    s->worker.join();
    std::lock_guard<std::mutex> g(s->mu);
    s->started = false;
    return ROI_OK;
}

roi_status roi_server_progress(roi_server_t s) {
    if (!s) return ROI_EINVAL;
    std::lock_guard<std::mutex> g(s->mu);
    return progress_locked(s);
}

int roi_server_poll(roi_server_t s, roi_server_completion* out, int max) {
    if (!s || max < 0 || (max > 0 && !out)) return -1;
    std::lock_guard<std::mutex> g(s->mu);
    int n = 0;
    while (n < max && !s->completed.empty()) {
        out[n++] = s->completed.front();
        s->completed.pop_front();
    }
    return n;
}

roi_status roi_server_take(roi_server_t s, long long id, float* dst) {
    if (!s) return ROI_EINVAL;
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return sfail(s, ROI_EINVAL, "take: unknown request %lld", id);
    Req* r = it->second;
    if (r->state != 2) return sfail(s, ROI_EBUSY, "take: request %lld not complete", id);
    const roi_status st = r->status;
    if (st == ROI_OK && dst) std::memcpy(dst, s->out_h + r->host_off, r->host_bytes);
    if (r->has_host) s->harena.release(r->host_off, r->host_bytes);
    s->reqs.erase(it);
    delete r;
    if (st != ROI_OK) return sfail(s, st, "take: request %lld failed", id);
    return ROI_OK;
}

roi_status roi_server_drain(roi_server_t s, double timeout_ms) {
    if (!s) return ROI_EINVAL;
    const double t0 = now_ms();
    for (;;) {
        {
            std::lock_guard<std::mutex> g(s->mu);
            if (!s->started) {
                roi_status st = progress_locked(s);
                if (st != ROI_OK && st != ROI_ETIMEOUT) return st;
            }
            if (s->n_outstanding == 0) return ROI_OK;
        }
        if (now_ms() - t0 > timeout_ms) return sfail(s, ROI_EBUSY, "drain: requests still outstanding");
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

roi_status roi_server_stats_get(roi_server_t s, roi_server_stats* out) {
    if (!s || !out) return ROI_EINVAL;
    std::lock_guard<std::mutex> g(s->mu);
    out->submitted = s->n_submitted;
    out->completed = s->n_completed;
    out->failed = s->n_failed;
    long long pend = 0, infl = 0;
    for (const Pool& P : s->pools) {
        pend += (long long)P.pending.size();
        for (const Req* r : P.occupant) infl += r != nullptr;
    }
    out->pending = pend;
    out->in_flight = infl;
    out->kernel_launches = s->launches;
    out->device_in_use = s->darena.used;
    out->device_peak = s->darena.peak;
    out->host_in_use = s->harena.used;
    out->host_peak = s->harena.peak;
    out->blocks = s->blocks;
    out->single_units = s->pools[0].nteams;
    out->teams = s->pools[1].nteams;
    out->team_blocks = s->pools[1].team;
    out->cancelled = s->n_cancelled;
    return ROI_OK;
}

roi_status roi_server_cancel(roi_server_t s, long long id) {
    if (!s) return ROI_EINVAL;
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return sfail(s, ROI_EINVAL, "cancel: unknown request %lld", id);
    Req* r = it->second;
    if (r->state == 1) return sfail(s, ROI_EBUSY, "cancel: request %lld is already on the device", id);
    if (r->state == 2) return sfail(s, ROI_EINVAL, "cancel: request %lld has completed", id);
    std::deque<Req*>& pend = s->pools[r->pool].pending;
    auto q = std::find(pend.begin(), pend.end(), r);
    if (q == pend.end()) return sfail(s, ROI_EINVAL, "cancel: request %lld is not queued", id);
    pend.erase(q);
    r->t_done = now_ms();
    r->status = ROI_ECANCELED;
    r->state = 2;
    --s->n_outstanding;
    ++s->n_cancelled;
    push_completion(s, r);
    return ROI_OK;
}

roi_status roi_server_set_option(roi_server_t s, roi_option opt, long long value) {
    if (!s) return ROI_EINVAL;
    std::lock_guard<std::mutex> g(s->mu);
    switch (opt) {
        case ROI_OPT_WAIT_LIMIT_US:
            if (value < 1 || value > 600000000LL) return sfail(s, ROI_EINVAL, "set_option: wait limit out of range");
            s->opt_wait_ns = (unsigned long long)value * 1000ull;
            return ROI_OK;
        case ROI_OPT_TEST_ABSENT_BLOCKS:
            if (value < -1 || value > 1024) return sfail(s, ROI_EINVAL, "set_option: absent blocks out of range");
            s->opt_absent = (int)value;
            return ROI_OK;
        default:
            break;
    }
    return sfail(s, ROI_EINVAL, "set_option: option %d does not apply to a server", (int)opt);
}

const char* roi_server_last_error(roi_server_t s) { return s ? s->err.c_str() : "null server"; }

void roi_server_destroy(roi_server_t s) {
    if (!s) return;
    roi_server_stop(s);
    {
        std::lock_guard<std::mutex> g(s->mu);
        // drop requests that were never published, then let the kernel leave
        for (Pool& P : s->pools) P.pending.clear();
        if (s->ctl_h) __atomic_store_n(&s->ctl_h->close, 1, __ATOMIC_RELEASE);
        if (s->running) {
            cudaEventSynchronize(s->ev_end);
            s->running = false;
        }
    }
    free_all(s);
    delete s;
}

roi_status roi_server_footprint(int n_pix, int n_angles, int n_det, roi_dtype storage, const roi_region* region,
                                size_t* device_bytes, size_t* host_bytes, int* box_side) {
    if (n_pix < 1 || n_angles < 1 || n_det < 1 || n_pix > 65536 || n_angles > 65536 || n_det > 8192 ||
        !finite_region(region) || (storage != ROI_F32 && storage != ROI_BF16 && storage != ROI_F16))
        return ROI_EINVAL;
    std::vector<double> ang(n_angles);
    for (int a = 0; a < n_angles; ++a) ang[a] = a * 3.14159265358979323846 / n_angles;
    Rect box{};
    int stride = 0, nrow = 0;
    if (!plan_request(n_pix, n_angles, n_det, ang.data(), *region, &box, &stride, &nrow, nullptr)) return ROI_EINVAL;
    const StateLayout L = state_layout(n_angles, stride, box.w, box.h, roi::dt_size((int)storage));
    if (device_bytes) *device_bytes = round_up(L.total);
    if (host_bytes) *host_bytes = round_up(sizeof(float) * (size_t)box.w * box.h);
    if (box_side) *box_side = std::max(box.w, box.h);
    return ROI_OK;
}

}  // extern "C"
