// Serving engine: continuous batching of independent slice solves on one
// capacity-sized handle (declared in include/recon.h).
#include <chrono>
#include <cstring>
#include <deque>
#include <map>
#include <new>
#include <vector>

#include "ctx.h"

namespace recon {
int check_params(const recon_params& p);       // csrc/api.cu
int check_geometry(const recon_geometry& g);   // csrc/api.cu

namespace {

double now_ms() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Request {
    uint64_t ticket;
    recon_geometry geom;
    recon_params params;
    std::vector<float> lo, hi;
    double t_submit;
    double t_admit;
    long long footprint;
};

struct Done {
    std::vector<float> Z, rho;
    recon_result res;
};

bool seven_smooth(int n) {
    if (n < 1) return false;
    for (int p : {2, 3, 5, 7})
        while (n % p == 0) n /= p;
    return n == 1;
}

}  // namespace
}  // namespace recon

using namespace recon;

struct recon_server {
    Ctx c;
    recon_server_config cfg;
    std::deque<Request> queue;
    std::vector<int> slot_busy;
    std::vector<Request> in_slot;
    std::map<uint64_t, Done> done;
    uint64_t next_ticket = 1;
    long long in_use = 0;
    long long cap_px = 0, cap_sino = 0;
};

namespace {

long long footprint(const recon_server& s, int nx, int ny) {
    const long long elem = s.cfg.precision == 1 ? 4 : 8;
    const long long pitch = (nx + 31) / 32 * 32, cp = (nx / 2 + 1 + 15) / 16 * 16;
    return elem * ((long long)kNumFields * ny * pitch + 2LL * kNumSpectra * ny * cp);
}

std::vector<int> active_slots(const recon_server& s) {
    std::vector<int> a;
    for (int i = 0; i < (int)s.slot_busy.size(); ++i)
        if (s.slot_busy[i]) a.push_back(i);
    return a;
}

}  // namespace

extern "C" {

int recon_server_create(const recon_server_config* cfg, void* stream, recon_server** out) {
    if (!cfg || !out || cfg->max_slots < 1 || cfg->max_nx < 1 || cfg->max_ny < 1 || cfg->max_nx > RECON_MAX_SIDE ||
        cfg->max_ny > RECON_MAX_SIDE || (cfg->precision != 0 && cfg->precision != 1) || cfg->max_views < 0 ||
        cfg->max_bins < 0) {
        set_error("recon_server_create: bad configuration");
        return RECON_EINVAL;
    }
    *out = nullptr;
    recon_server* s = new (std::nothrow) recon_server();
    if (!s) return RECON_ENOMEM;
    s->cfg = *cfg;
    Ctx& c = s->c;
    c.n = cfg->max_slots;
    c.precision = cfg->precision;
    c.stream = (cudaStream_t)stream;
    c.server_mode = true;
    c.cap_nx = cfg->max_nx;
    c.cap_ny = cfg->max_ny;
    recon_geometry g{};
    g.nx = cfg->max_nx;
    g.ny = cfg->max_ny;
    g.pixel_mm = 1.0;
    recon_params p;
    recon_default_params(&p);
    p.precision = cfg->precision;
    c.geo.assign(c.n, g);
    c.prm.assign(c.n, p);
    int rc = solver_setup(c);
    if (!rc) rc = solver_rebuild_lists(c, {});
    s->cap_px = (long long)cfg->max_nx * cfg->max_ny;
    s->cap_sino = (long long)cfg->max_views * cfg->max_bins;
    if (!rc && s->cap_sino > 0) {
        for (int i = 0; i < 2 && !rc; ++i) {
            cudaError_t e = cudaMalloc((void**)&c.d_sino[i], sizeof(float) * s->cap_sino * c.n);
            if (e != cudaSuccess) rc = cuda_fail(e, "cudaMalloc server sinograms");
            else c.allocations.push_back(c.d_sino[i]);
        }
        if (!rc) {
            cudaError_t e = cudaMalloc((void**)&c.d_filt, sizeof(float) * s->cap_sino);
            if (e != cudaSuccess) rc = cuda_fail(e, "cudaMalloc server filter scratch");
            else c.allocations.push_back(c.d_filt);
        }
    }
    if (rc) {
        for (void* q : c.allocations) cudaFree(q);
        if (c.h_cg_pending) cudaFreeHost(c.h_cg_pending);
        delete s;
        return rc;
    }
    s->slot_busy.assign(c.n, 0);
    s->in_slot.resize(c.n);
    *out = s;
    return RECON_OK;
}

int recon_submit(recon_server* s, const recon_request* r, uint64_t* ticket) {
    if (!s || !r || !ticket || !r->low || !r->high) {
        set_error("recon_submit: bad arguments");
        return RECON_EINVAL;
    }
    const recon_geometry& g = r->geom;
    // a request is checked in full here, so a bad one never reaches a step shared with others
    if (int rc = check_geometry(g)) return rc;
    if (int rc = check_params(r->params)) return rc;
    if (g.nx < 1 || g.ny < 1 || g.nx > s->cfg.max_nx || g.ny > s->cfg.max_ny || !seven_smooth(g.nx) ||
        !seven_smooth(g.ny) || r->params.precision != s->cfg.precision || r->params.order != 0 ||
        r->params.domain != 0) {
        set_error("recon_submit: size above the slot capacity, not 7-smooth, precision/order mismatch, or domain 1");
        return RECON_EINVAL;
    }
    if (g.n_views > 0 && ((long long)g.n_views * g.n_bins > s->cap_sino || g.n_bins < 1)) {
        set_error("recon_submit: sinogram above the slot capacity");
        return RECON_EINVAL;
    }
    Request q;
    q.ticket = s->next_ticket++;
    q.geom = g;
    q.params = r->params;
    const size_t n = g.n_views > 0 ? (size_t)g.n_views * g.n_bins : (size_t)g.nx * g.ny;
    q.lo.assign(r->low, r->low + n);
    q.hi.assign(r->high, r->high + n);
    q.t_submit = now_ms();
    q.t_admit = 0.0;
    q.footprint = footprint(*s, g.nx, g.ny);
    if (s->cfg.hbm_budget_bytes > 0 && (double)q.footprint > s->cfg.hbm_budget_bytes) {
        set_error("recon_submit: request footprint above the HBM budget");
        return RECON_EBUDGET;
    }
    *ticket = q.ticket;
    s->queue.push_back(std::move(q));
    return RECON_OK;
}

int recon_server_step(recon_server* s, int32_t n_iters, int32_t* n_active) {
    if (!s || n_iters < 0) return RECON_EINVAL;
    Ctx& c = s->c;
    int rc;
    // admission
    std::vector<int> fresh;
    while (!s->queue.empty()) {
        Request& q = s->queue.front();
        if (s->cfg.hbm_budget_bytes > 0 && (double)(s->in_use + q.footprint) > s->cfg.hbm_budget_bytes) break;
        int slot = -1;
        for (int i = 0; i < c.n; ++i)
            if (!s->slot_busy[i]) {
                slot = i;
                break;
            }
        if (slot < 0) break;
        if ((rc = solver_configure_slot(c, slot, q.geom, q.params))) return rc;
        float* lo = c.d_stage[0] + c.sg[slot].ext_off;
        float* hi = c.d_stage[1] + c.sg[slot].ext_off;
        if (q.geom.n_views > 0) {
            float* sl = c.d_sino[0] + s->cap_sino * slot;
            float* sh = c.d_sino[1] + s->cap_sino * slot;
            RECON_CUDA(cudaMemcpyAsync(sl, q.lo.data(), sizeof(float) * q.lo.size(), cudaMemcpyHostToDevice, c.stream));
            RECON_CUDA(cudaMemcpyAsync(sh, q.hi.data(), sizeof(float) * q.hi.size(), cudaMemcpyHostToDevice, c.stream));
            if ((rc = ct_fbp(q.geom, 1, sl, lo, c.d_filt, c.stream, &c.launches))) return rc;
            if ((rc = ct_fbp(q.geom, 1, sh, hi, c.d_filt, c.stream, &c.launches))) return rc;
        } else {
            RECON_CUDA(cudaMemcpyAsync(lo, q.lo.data(), sizeof(float) * q.lo.size(), cudaMemcpyHostToDevice, c.stream));
            RECON_CUDA(cudaMemcpyAsync(hi, q.hi.data(), sizeof(float) * q.hi.size(), cudaMemcpyHostToDevice, c.stream));
        }
        RECON_CUDA(cudaStreamSynchronize(c.stream));   // the request's host vectors are released below
        q.t_admit = now_ms();
        s->in_use += q.footprint;
        s->slot_busy[slot] = 1;
        s->in_slot[slot] = std::move(q);
        s->in_slot[slot].lo.clear();
        s->in_slot[slot].hi.clear();
        s->queue.pop_front();
        fresh.push_back(slot);
    }
    if (!fresh.empty()) {
        if ((rc = solver_rebuild_lists(c, active_slots(*s)))) return rc;
        if ((rc = solver_init_slots(c, fresh, c.d_stage[0], c.d_stage[1]))) return rc;
    }
    // continuous batching: one launch sequence per iteration for every slot
    if (!active_slots(*s).empty()) {
        for (int k = 0; k < n_iters; ++k)
            if ((rc = solver_iterate(c, false))) return rc;
    }
    // retirement
    std::vector<SliceState> st;
    if ((rc = solver_read_state(c, st))) return rc;
    std::vector<int> finished;
    for (int i = 0; i < c.n; ++i)
        if (s->slot_busy[i] && !st[i].active) finished.push_back(i);
    if (!finished.empty()) {
        if ((rc = solver_extract_slots(c, finished, c.d_stage[0], c.d_stage[1]))) return rc;
        for (int i : finished) {
            Request& q = s->in_slot[i];
            Done d;
            const size_t n = (size_t)q.geom.nx * q.geom.ny;
            d.Z.resize(n);
            d.rho.resize(n);
            RECON_CUDA(cudaMemcpyAsync(d.Z.data(), c.d_stage[0] + c.sg[i].ext_off, sizeof(float) * n,
                                       cudaMemcpyDeviceToHost, c.stream));
            RECON_CUDA(cudaMemcpyAsync(d.rho.data(), c.d_stage[1] + c.sg[i].ext_off, sizeof(float) * n,
                                       cudaMemcpyDeviceToHost, c.stream));
            RECON_CUDA(cudaStreamSynchronize(c.stream));
            const double t = now_ms();
            d.res.status = RECON_OK;
            d.res.iters = st[i].k;
            d.res.queue_ms = q.t_admit - q.t_submit;
            d.res.latency_ms = t - q.t_submit;
            s->done[q.ticket] = std::move(d);
            s->in_use -= q.footprint;
            s->slot_busy[i] = 0;
        }
        if ((rc = solver_rebuild_lists(c, active_slots(*s)))) return rc;
    }
    if (n_active) *n_active = (int32_t)active_slots(*s).size();
    return RECON_OK;
}

int recon_poll(recon_server* s, uint64_t ticket, float* Z, float* rhoe, recon_result* res) {
    if (!s) return RECON_EINVAL;
    auto it = s->done.find(ticket);
    if (it == s->done.end()) {
        for (const Request& q : s->queue)
            if (q.ticket == ticket) return 0;
        for (int i = 0; i < (int)s->slot_busy.size(); ++i)
            if (s->slot_busy[i] && s->in_slot[i].ticket == ticket) return 0;
        set_error("recon_poll: unknown ticket");
        return RECON_EINVAL;
    }
    if (Z) std::memcpy(Z, it->second.Z.data(), sizeof(float) * it->second.Z.size());
    if (rhoe) std::memcpy(rhoe, it->second.rho.data(), sizeof(float) * it->second.rho.size());
    if (res) *res = it->second.res;
    s->done.erase(it);
    return 1;
}

int recon_server_stats(recon_server* s, int64_t* out4) {
    if (!s || !out4) return RECON_EINVAL;
    out4[0] = (int64_t)s->queue.size();
    out4[1] = (int64_t)active_slots(*s).size();
    out4[2] = (int64_t)s->done.size();
    out4[3] = s->in_use;
    return RECON_OK;
}

void recon_server_destroy(recon_server* s) {
    if (!s) return;
    cudaStreamSynchronize(s->c.stream);
    for (void* q : s->c.allocations) cudaFree(q);
    if (s->c.h_cg_pending) cudaFreeHost(s->c.h_cg_pending);
    delete s;
}

}  // extern "C"
