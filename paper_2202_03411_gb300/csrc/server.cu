// server.cu -- native request scheduler for many concurrent shape fits on one
// GPU (continuous admission under a device-memory budget).
//
// Threads: one scheduler thread owns admission; each slot owns a host thread
// and a CUDA stream and runs its requests one after another.  A request is
// admitted when a slot is idle and the bytes that slot must hold for it fit
// under the budget.  Slots keep the handle (and fit buffers) of their last
// geometry; idle slots' handles are evicted when the budget needs room.
// Requests therefore overlap on the device as far as slots and memory allow,
// and new arrivals are taken in as soon as either frees up.
//
// Accounting: `reserved` is the sum over slots of `held`, the bytes a slot
// holds or has been promised for its current geometry.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <tuple>

#include "internal.cuh"

namespace scm {

using Clock = std::chrono::steady_clock;

struct GeomKey {
    int nx = 0, ny = 0, nz = 0, det_nx = 0, det_ny = 0;
    double voxel = 0, wavelength = 0, theta = 0;
    bool operator<(const GeomKey &o) const {
        return std::tie(nx, ny, nz, det_nx, det_ny, voxel, wavelength, theta) <
               std::tie(o.nx, o.ny, o.nz, o.det_nx, o.det_ny, o.voxel, o.wavelength, o.theta);
    }
    bool operator==(const GeomKey &o) const { return !(*this < o) && !(o < *this); }
};

struct Req {
    long long ticket = 0;
    scatman_config cfg;
    scatman_shape shape;
    std::vector<double> alm;
    std::vector<float> target;
    int want_gradient = 0;
    float *I_out = nullptr;
    double *grad_out = nullptr;
    double *loss_out = nullptr;
    GeomKey key;
    long long need = 0;
    Clock::time_point t_submit, t_done;
    bool done = false;
    int status = SCATMAN_OK;
};

struct Slot {
    int id = 0;
    cudaStream_t stream = nullptr;
    std::thread thr;
    std::shared_ptr<Req> job;       // set by the scheduler, cleared by the slot
    long long held = 0;             // bytes accounted to this slot
    bool has_cache = false;         // a handle for `key` exists
    GeomKey key{};
    scatman_handle *h = nullptr;
    float *d_target = nullptr;
    void *d_w = nullptr;
    double *d_loss = nullptr;
};

static long long round_2mib(long long b) {
    const long long g = 2ll << 20;
    return b <= 0 ? 0 : (b + g - 1) / g * g;
}

}  // namespace scm

struct scatman_server {
    scatman_server_config cfg;
    int device = 0;
    std::mutex mu;
    std::condition_variable cv;         // any state change
    std::deque<std::shared_ptr<scm::Req>> queue;
    std::map<long long, std::shared_ptr<scm::Req>> reqs;
    std::vector<std::unique_ptr<scm::Slot>> slots;
    std::thread sched;
    bool stopping = false;
    bool sched_done = false;
    long long next_ticket = 1;
    long long reserved = 0;
    scatman_server_stats stats{};
};

namespace scm {

// Device bytes a slot holds for a geometry: the handle plus the fit buffers
// (target, residual, loss partials).
static long long slot_bytes(const scatman_config &c, int precision, double width) {
    scatman_config cc = c;
    cc.precision = precision;
    cc.soft = 1;
    cc.soft_width = width;
    const long long fp = scatman_footprint_bytes(&cc);
    if (fp < 0) return fp;
    const long long npix = (long long)c.det_nx * c.det_ny;
    const int elem = precision == SCATMAN_FP64 ? 8 : 4;
    return fp + round_2mib(npix * 4) + round_2mib(npix * elem) + round_2mib(256 * 8);
}

static void free_cache(Slot &s) {
    if (s.h) scatman_destroy(s.h);
    if (s.d_target) cudaFree(s.d_target);
    if (s.d_w) cudaFree(s.d_w);
    if (s.d_loss) cudaFree(s.d_loss);
    s.h = nullptr;
    s.d_target = nullptr;
    s.d_w = nullptr;
    s.d_loss = nullptr;
    s.has_cache = false;
}

// Runs one request on the slot's stream; returns the request's status.
static int run_request(const scatman_server_config &scfg, Slot &s, Req &r) {
    const int prec = scfg.precision;
    const bool f64 = prec == SCATMAN_FP64;
    if (!s.has_cache || !(s.key == r.key)) {
        free_cache(s);
        scatman_config c = r.cfg;
        c.precision = prec;
        c.soft = 1;
        c.soft_width = scfg.soft_width;
        c.q_list = nullptr;
        c.n_q = 0;
        int rc = scatman_create(&c, s.stream, &s.h);
        if (rc) {
            s.h = nullptr;
            return rc;
        }
        const long long n = s.h->n_pix;
        if (cudaMalloc((void **)&s.d_target, n * sizeof(float)) != cudaSuccess ||
            cudaMalloc(&s.d_w, n * (f64 ? 8 : 4)) != cudaSuccess ||
            cudaMalloc((void **)&s.d_loss, 256 * sizeof(double)) != cudaSuccess) {
            free_cache(s);
            return SCATMAN_ERR_OOM;
        }
        s.has_cache = true;
        s.key = r.key;
    }
    scatman_handle *h = s.h;
    const long long n = h->n_pix;
    r.shape.alm = r.alm.empty() ? nullptr : r.alm.data();
    int rc = scatman_voxelise(h, &r.shape);
    if (rc) return rc;
    rc = scatman_forward(h, h->d_I, nullptr);
    if (rc) return rc;
    if (cudaMemcpyAsync(s.d_target, r.target.data(), n * sizeof(float), cudaMemcpyHostToDevice, s.stream) !=
        cudaSuccess)
        return SCATMAN_ERR_CUDA;
    const int nb = l2_residual_blocks(n);
    if (launch_l2_residual(f64, h->d_I, s.d_target, n, s.d_w, s.d_loss, nb, s.stream) != cudaSuccess)
        return SCATMAN_ERR_CUDA;
    std::vector<double> grad;
    if (r.want_gradient) {
        grad.resize(scatman_param_count(h));
        rc = scatman_backward(h, s.d_w, grad.data());
        if (rc) return rc;
    }
    std::vector<double> loss_part(nb);
    if (cudaMemcpyAsync(loss_part.data(), s.d_loss, nb * sizeof(double), cudaMemcpyDeviceToHost, s.stream) !=
        cudaSuccess)
        return SCATMAN_ERR_CUDA;
    std::vector<double> Id;
    if (r.I_out) {
        cudaError_t e;
        if (f64) {
            Id.resize(n);
            e = cudaMemcpyAsync(Id.data(), h->d_I, n * 8, cudaMemcpyDeviceToHost, s.stream);
        } else {
            e = cudaMemcpyAsync(r.I_out, h->d_I, n * 4, cudaMemcpyDeviceToHost, s.stream);
        }
        if (e != cudaSuccess) return SCATMAN_ERR_CUDA;
    }
    rc = scatman_sync(h);
    if (rc) return rc;
    if (f64 && r.I_out)
        for (long long i = 0; i < n; ++i) r.I_out[i] = (float)Id[i];
    double loss = 0.0;
    for (int b = 0; b < nb; ++b) loss += loss_part[b];
    if (r.loss_out) *r.loss_out = loss;
    if (r.want_gradient) std::memcpy(r.grad_out, grad.data(), grad.size() * sizeof(double));
    return SCATMAN_OK;
}

static void slot_main(scatman_server *srv, Slot *s) {
    cudaSetDevice(srv->device);
    std::unique_lock<std::mutex> lk(srv->mu);
    while (true) {
        srv->cv.wait(lk, [&] { return s->job != nullptr || srv->sched_done; });
        if (!s->job) break;
        std::shared_ptr<Req> r = s->job;
        lk.unlock();
        const int st = run_request(srv->cfg, *s, *r);
        if (st != SCATMAN_OK) free_cache(*s);          // never keep a handle in an unknown state
        lk.lock();
        if (!s->has_cache) {
            srv->reserved -= s->held;
            s->held = 0;
        }
        r->status = st;
        r->t_done = Clock::now();
        r->done = true;
        if (st == SCATMAN_OK) ++srv->stats.completed;
        else ++srv->stats.failed;
        --srv->stats.inflight;
        s->job = nullptr;
        srv->stats.bytes_reserved = srv->reserved;
        srv->cv.notify_all();
    }
}

static void sched_main(scatman_server *srv) {
    cudaSetDevice(srv->device);
    std::unique_lock<std::mutex> lk(srv->mu);
    const long long budget = srv->cfg.hbm_budget_bytes;
    while (true) {
        srv->cv.wait(lk, [&] {
            if (srv->stopping && srv->queue.empty()) return true;
            if (srv->queue.empty()) return false;
            for (auto &s : srv->slots)
                if (!s->job) return true;
            return false;
        });
        if (srv->queue.empty()) break;                   // stopping and drained
        std::shared_ptr<Req> r = srv->queue.front();
        Slot *pick = nullptr;
        for (auto &s : srv->slots)                       // an idle slot that already holds this geometry
            if (!s->job && s->has_cache && s->key == r->key) { pick = s.get(); break; }
        long long delta = 0;
        if (!pick) {
            for (auto &s : srv->slots)                   // else an empty idle slot
                if (!s->job && s->held == 0) { pick = s.get(); break; }
            if (!pick)
                for (auto &s : srv->slots)               // else the idle slot holding the most bytes
                    if (!s->job && (!pick || s->held > pick->held)) pick = s.get();
            delta = r->need - pick->held;
            if (srv->reserved + delta > budget) {
                // make room: release other idle slots' handles, largest first
                std::vector<Slot *> idle;
                for (auto &s : srv->slots)
                    if (!s->job && s.get() != pick && s->held > 0) idle.push_back(s.get());
                std::sort(idle.begin(), idle.end(), [](Slot *a, Slot *b) { return a->held > b->held; });
                for (Slot *s : idle) {
                    if (srv->reserved + delta <= budget) break;
                    free_cache(*s);
                    srv->reserved -= s->held;
                    s->held = 0;
                }
            }
            if (srv->reserved + delta > budget) {
                bool any_busy = false;
                for (auto &s : srv->slots) any_busy |= (s->job != nullptr);
                if (!any_busy) {                          // cannot fit even alone
                    srv->queue.pop_front();
                    r->status = SCATMAN_ERR_ADMISSION;
                    r->t_done = Clock::now();
                    r->done = true;
                    ++srv->stats.failed;
                    srv->cv.notify_all();
                    continue;
                }
                srv->cv.wait(lk);                        // wait for a completion and retry
                continue;
            }
            srv->reserved += delta;
            pick->held = r->need;
        }
        srv->queue.pop_front();
        pick->job = r;
        ++srv->stats.inflight;
        srv->stats.inflight_peak = std::max(srv->stats.inflight_peak, srv->stats.inflight);
        srv->stats.bytes_reserved = srv->reserved;
        srv->stats.bytes_reserved_peak = std::max(srv->stats.bytes_reserved_peak, srv->reserved);
        srv->cv.notify_all();
    }
    srv->sched_done = true;
    srv->cv.notify_all();
}

}  // namespace scm

using namespace scm;

extern "C" {

long long scatman_footprint_bytes(const scatman_config *c) {
    if (!c || c->nx < 1 || c->ny < 1 || c->nz < 1) return -1;
    const long long nvox = (long long)c->nx * c->ny * c->nz;
    const long long npix = c->q_list ? c->n_q : (long long)c->det_nx * c->det_ny;
    if (npix < 1) return -1;
    const bool f64 = c->precision == SCATMAN_FP64;
    const bool uniform = !c->q_list && c->detector == SCATMAN_DETECTOR_UNIFORM_Q;
    const bool tc = c->precision >= SCATMAN_TC_F16_SPLIT;
    const long long cx = f64 ? 16 : 8;
    long long s_bytes;
    if (tc) {
        const long long Nxp = (c->nx + 15) / 16 * 16, Nyp = (c->ny + 15) / 16 * 16;
        s_bytes = (long long)c->nz * 3 * Nxp * Nyp * 2;   // planes -Im, Re, Im
    } else {
        s_bytes = nvox * cx;
    }
    long long b = 0;
    b += round_2mib(npix * 24);                 // q
    if (tc) b += round_2mib(24LL * c->nz + 8);  // slice bounds and occupied-slice list
    b += round_2mib(nvox * 4);                  // occupancy
    b += round_2mib(s_bytes);                   // slices
    b += round_2mib(npix * cx);                 // field cache
    b += round_2mib(npix * (f64 ? 8 : 4));      // intensity scratch
    if (uniform && c->precision >= SCATMAN_TC_F16_SPLIT) {
        b += round_2mib((long long)scm::uq_tc_h_bytes(c->nx, c->nz, c->det_ny));   // y-contracted 16-bit planes
        b += round_2mib(npix * 8);                                                 // q_z table
        b += round_2mib(24LL * c->det_ny);                                         // detector row q
    } else if (uniform) {
        b += round_2mib((long long)c->det_ny * c->nx * c->nz * cx);   // y-contracted slices
        b += round_2mib(npix * 8);                                    // q_z table
    } else if (!tc) {
        b += round_2mib(64 * npix * cx);        // partial fields (upper bound on splits)
    } else {
        b += round_2mib(256LL * 128 * 4 * 8);   // last wave's partial fields (< 256 SMs, <= 4 parts)
    }
    b += round_2mib(nvox * cx);                 // adjoint field (backward)
    if (tc) {
        // adjoint partial fields (<= 8), scale, pixel table, y-phase operand tiles
        const long long Nyp16 = ((c->ny + 7) / 8 * 8 + 15) / 16 * 16;
        b += round_2mib(8 * nvox * 8) + round_2mib(4) + round_2mib(48 * npix) +
             round_2mib((npix + 31) / 32 * 2 * Nyp16 * 128);
    }
    b += round_2mib((608LL * ((SCATMAN_MAX_LMAX + 1) * (SCATMAN_MAX_LMAX + 1) + 2) + 256) * 8);
    return b;
}

int scatman_server_create(const scatman_server_config *cfg, scatman_server **out) {
    if (!out) return SCATMAN_ERR_ARG;
    *out = nullptr;
    if (!cfg || cfg->hbm_budget_bytes <= 0 || cfg->slots < 1 || cfg->slots > 64 || !(cfg->soft_width > 0) ||
        cfg->precision < SCATMAN_FP64 || cfg->precision > SCATMAN_TC_BF16)
        return SCATMAN_ERR_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SCATMAN_ERR_UNSUPPORTED;
    int major = 0, minor = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    if (!(major == 10 && minor == 3)) return SCATMAN_ERR_UNSUPPORTED;
    scatman_server *srv = new scatman_server();
    srv->cfg = *cfg;
    srv->device = dev;
    for (int i = 0; i < cfg->slots; ++i) {
        auto s = std::make_unique<Slot>();
        s->id = i;
        if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
            for (auto &t : srv->slots) cudaStreamDestroy(t->stream);
            delete srv;
            return SCATMAN_ERR_CUDA;
        }
        srv->slots.push_back(std::move(s));
    }
    for (auto &s : srv->slots) s->thr = std::thread(slot_main, srv, s.get());
    srv->sched = std::thread(sched_main, srv);
    *out = srv;
    return SCATMAN_OK;
}

int scatman_server_submit(scatman_server *srv, const scatman_request *req, long long *ticket) {
    if (!srv || !req || !ticket || !req->target) return SCATMAN_ERR_ARG;
    const scatman_config &g = req->geometry;
    if (g.nx < 1 || g.ny < 1 || g.nz < 1 || g.det_nx < 1 || g.det_ny < 1 || g.q_list)
        return SCATMAN_ERR_ARG;
    if (req->want_gradient && !req->grad_out) return SCATMAN_ERR_ARG;
    const scatman_shape &sh = req->shape;
    // fit requests take parametric shapes (sphere, ellipsoid, harmonics): map
    // shapes have no gradient, and their arrays are only borrowed for a call
    if (sh.kind < SCATMAN_SPHERE || sh.kind > SCATMAN_SPHHARM) return SCATMAN_ERR_ARG;
    if (sh.kind == SCATMAN_SPHHARM && (sh.lmax < 0 || sh.lmax > SCATMAN_MAX_LMAX || (sh.lmax > 0 && !sh.alm)))
        return SCATMAN_ERR_ARG;
    auto r = std::make_shared<Req>();
    r->cfg = g;
    r->shape = sh;
    if (sh.kind == SCATMAN_SPHHARM && sh.lmax > 0) r->alm.assign(sh.alm, sh.alm + (sh.lmax + 1) * (sh.lmax + 1));
    const long long npix = (long long)g.det_nx * g.det_ny;
    r->target.assign(req->target, req->target + npix);
    r->want_gradient = req->want_gradient;
    r->I_out = req->I_out;
    r->grad_out = req->grad_out;
    r->loss_out = req->loss_out;
    r->key = GeomKey{g.nx, g.ny, g.nz, g.det_nx, g.det_ny, g.voxel, g.wavelength, g.theta_max_deg};
    r->need = slot_bytes(g, srv->cfg.precision, srv->cfg.soft_width);
    if (r->need < 0) return SCATMAN_ERR_ARG;
    if (r->need > srv->cfg.hbm_budget_bytes) return SCATMAN_ERR_ADMISSION;
    r->t_submit = Clock::now();
    std::lock_guard<std::mutex> lk(srv->mu);
    if (srv->stopping) return SCATMAN_ERR_STATE;
    r->ticket = srv->next_ticket++;
    srv->reqs[r->ticket] = r;
    srv->queue.push_back(r);
    ++srv->stats.submitted;
    *ticket = r->ticket;
    srv->cv.notify_all();
    return SCATMAN_OK;
}

int scatman_server_wait(scatman_server *srv, long long ticket, double timeout_s, int *status, double *latency_s) {
    if (!srv) return SCATMAN_ERR_ARG;
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(ticket);
    if (it == srv->reqs.end()) return SCATMAN_ERR_ARG;
    std::shared_ptr<Req> r = it->second;
    auto pred = [&] { return r->done; };
    if (timeout_s < 0) {
        srv->cv.wait(lk, pred);
    } else if (!srv->cv.wait_for(lk, std::chrono::duration<double>(timeout_s), pred)) {
        return SCATMAN_ERR_TIMEOUT;
    }
    if (status) *status = r->status;
    if (latency_s) *latency_s = std::chrono::duration<double>(r->t_done - r->t_submit).count();
    srv->reqs.erase(it);
    return SCATMAN_OK;
}

int scatman_server_stats_get(scatman_server *srv, scatman_server_stats *out) {
    if (!srv || !out) return SCATMAN_ERR_ARG;
    std::lock_guard<std::mutex> lk(srv->mu);
    *out = srv->stats;
    out->bytes_reserved = srv->reserved;
    return SCATMAN_OK;
}

void scatman_server_destroy(scatman_server *srv) {
    if (!srv) return;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stopping = true;
        srv->cv.notify_all();
    }
    if (srv->sched.joinable()) srv->sched.join();
    for (auto &s : srv->slots)
        if (s->thr.joinable()) s->thr.join();
    for (auto &s : srv->slots) {
        free_cache(*s);
        cudaStreamDestroy(s->stream);
    }
    delete srv;
}

}  // extern "C"
