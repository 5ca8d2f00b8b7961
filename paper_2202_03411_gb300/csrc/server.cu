// server.cu -- native request scheduler for many concurrent shape fits on one
// GPU (continuous admission under a device-memory budget).
//
// Threads: one scheduler thread owns admission; each slot owns a host thread
// and a CUDA stream and runs its requests one after another.  Handles (with a
// fit's buffers) live in a server-wide cache keyed by geometry: a request
// takes an idle handle of its geometry when there is one, else the slot
// creates one, and after the request the handle goes back to the cache, so
// a steady mix of geometries runs without device allocations (which stall
// every stream).  A request is admitted when a slot is idle and, if it needs
// a new handle, the handle's bytes fit under the budget after evicting idle
// handles, least recently used first.  Requests therefore overlap on the
// device as far as slots and memory allow, and new arrivals are taken in as
// soon as either frees up.
//
// Accounting: `reserved` is the sum of the bytes of every handle in existence
// (idle, in use, or promised to a slot that is creating it).
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

// A handle and its fit buffers for one geometry.
struct Cached {
    GeomKey key;
    scatman_handle *h = nullptr;
    float *d_target = nullptr;
    void *d_w = nullptr;
    double *d_loss = nullptr;
    long long bytes = 0;            // accounted bytes
    unsigned long long last_use = 0;
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
    std::unique_ptr<Cached> handle; // from the cache, or null: the slot creates one of `need` bytes
};

struct Slot {
    int id = 0;
    cudaStream_t stream = nullptr;
    std::thread thr;
    std::shared_ptr<Req> job;       // set by the scheduler, cleared by the slot
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
    std::vector<std::unique_ptr<scm::Cached>> idle;   // handles not in use
    unsigned long long use_clock = 0;
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

static void free_cached(Cached &c) {
    if (c.h) scatman_destroy(c.h);
    if (c.d_target) cudaFree(c.d_target);
    if (c.d_w) cudaFree(c.d_w);
    if (c.d_loss) cudaFree(c.d_loss);
    c.h = nullptr;
    c.d_target = nullptr;
    c.d_w = nullptr;
    c.d_loss = nullptr;
}

// A new handle and fit buffers for the request's geometry on the slot's stream.
static int create_cached(const scatman_server_config &scfg, Slot &s, const Req &r, Cached &c) {
    const bool f64 = scfg.precision == SCATMAN_FP64;
    scatman_config cfg = r.cfg;
    cfg.precision = scfg.precision;
    cfg.soft = 1;
    cfg.soft_width = scfg.soft_width;
    cfg.q_list = nullptr;
    cfg.n_q = 0;
    c.key = r.key;
    int rc = scatman_create(&cfg, s.stream, &c.h);
    if (rc) {
        c.h = nullptr;
        return rc;
    }
    const long long n = c.h->n_pix;
    if (device_malloc((void **)&c.d_target, n * sizeof(float)) != cudaSuccess ||
        device_malloc(&c.d_w, n * (f64 ? 8 : 4)) != cudaSuccess ||
        device_malloc((void **)&c.d_loss, 256 * sizeof(double)) != cudaSuccess) {
        free_cached(c);
        return SCATMAN_ERR_OOM;
    }
    return SCATMAN_OK;
}

// Runs one request on the slot's stream with handle `c`; returns the status.
static int run_request(const scatman_server_config &scfg, Slot &s, Req &r, Cached &c) {
    const StageRange nvtx_range("server request");
    const bool f64 = scfg.precision == SCATMAN_FP64;
    scatman_handle *h = c.h;
    // a cached handle may come from another slot: its work is finished, and
    // the handle was created on a caller-owned stream, so it can move
    h->stream = s.stream;
    const long long n = h->n_pix;
    r.shape.alm = r.alm.empty() ? nullptr : r.alm.data();
    int rc = scatman_voxelise(h, &r.shape);
    if (rc) return rc;
    rc = scatman_forward(h, h->d_I, nullptr);
    if (rc) return rc;
    if (cudaMemcpyAsync(c.d_target, r.target.data(), n * sizeof(float), cudaMemcpyHostToDevice, s.stream) !=
        cudaSuccess)
        return SCATMAN_ERR_CUDA;
    const int nb = l2_residual_blocks(n);
    if (launch_l2_residual(f64, h->d_I, c.d_target, n, c.d_w, c.d_loss, nb, s.stream) != cudaSuccess)
        return SCATMAN_ERR_CUDA;
    std::vector<double> grad;
    if (r.want_gradient) {
        grad.resize(scatman_param_count(h));
        rc = scatman_backward(h, c.d_w, grad.data());
        if (rc) return rc;
    }
    std::vector<double> loss_part(nb);
    if (cudaMemcpyAsync(loss_part.data(), c.d_loss, nb * sizeof(double), cudaMemcpyDeviceToHost, s.stream) !=
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
        std::unique_ptr<Cached> c = std::move(r->handle);
        const long long promised = r->need;
        lk.unlock();
        int st = SCATMAN_OK;
        if (!c) {
            c = std::make_unique<Cached>();
            c->bytes = promised;
            st = create_cached(srv->cfg, *s, *r, *c);
        }
        if (st == SCATMAN_OK) st = run_request(srv->cfg, *s, *r, *c);
        if (st != SCATMAN_OK) free_cached(*c);          // never keep a handle in an unknown state
        lk.lock();
        if (st == SCATMAN_OK) {
            c->last_use = ++srv->use_clock;
            srv->idle.push_back(std::move(c));
        } else {
            srv->reserved -= c->bytes;
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
        for (auto &s : srv->slots)
            if (!s->job) { pick = s.get(); break; }
        // an idle handle of this geometry, most recently used first
        int best = -1;
        for (int i = 0; i < (int)srv->idle.size(); ++i)
            if (srv->idle[i]->key == r->key && (best < 0 || srv->idle[i]->last_use > srv->idle[best]->last_use))
                best = i;
        if (best >= 0) {
            r->handle = std::move(srv->idle[best]);
            srv->idle.erase(srv->idle.begin() + best);
        } else {
            if (srv->reserved + r->need > budget) {
                // make room: release idle handles, least recently used first
                std::sort(srv->idle.begin(), srv->idle.end(),
                          [](const std::unique_ptr<Cached> &a, const std::unique_ptr<Cached> &b) {
                              return a->last_use > b->last_use;
                          });
                while (!srv->idle.empty() && srv->reserved + r->need > budget) {
                    free_cached(*srv->idle.back());
                    srv->reserved -= srv->idle.back()->bytes;
                    srv->idle.pop_back();
                }
            }
            if (srv->reserved + r->need > budget) {
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
            srv->reserved += r->need;                    // the slot creates the handle
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
    b += round_2mib(4LL * (long long)scm::slice_geom_ints(c->nz));   // slice geometry and the unit list
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
        // Jacobi-Anger order fields (at most 64 orders) and their coefficients
        b += round_2mib(64LL * c->nx * c->ny * 8) + round_2mib(64LL * c->nz * 8);
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

int scatman_server_cancel(scatman_server *srv, long long ticket) {
    if (!srv) return SCATMAN_ERR_ARG;
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(ticket);
    if (it == srv->reqs.end()) return SCATMAN_ERR_ARG;
    std::shared_ptr<Req> r = it->second;
    auto q = std::find(srv->queue.begin(), srv->queue.end(), r);
    if (q == srv->queue.end()) return SCATMAN_ERR_STATE;     // admitted, running or finished
    srv->queue.erase(q);
    r->status = SCATMAN_ERR_CANCELLED;
    r->t_done = Clock::now();
    r->done = true;
    ++srv->stats.cancelled;
    srv->cv.notify_all();
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
    for (auto &c : srv->idle) free_cached(*c);
    srv->idle.clear();
    for (auto &s : srv->slots) cudaStreamDestroy(s->stream);
    delete srv;
}

}  // extern "C"
