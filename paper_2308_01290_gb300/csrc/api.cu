// C ABI of librecon (declared in include/recon.h).
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "ctx.h"

struct recon_ctx {
    recon::Ctx c;
};

namespace recon {

namespace {
thread_local std::string g_last_error;

bool seven_smooth(int n) {
    if (n < 1) return false;
    for (int p : {2, 3, 5, 7})
        while (n % p == 0) n /= p;
    return n == 1;
}

constexpr int kFbpGroup = 8;   // slices per FBP launch pair in recon_set_data

bool same_spectrum(const recon_spectrum& a, const recon_spectrum& b) {
    if (a.kind != b.kind || a.kev != b.kev || a.kvp != b.kvp || a.n_filters != b.n_filters) return false;
    for (int i = 0; i < a.n_filters && i < RECON_MAX_FILTERS; ++i)
        if (a.filters[i].Z != b.filters[i].Z || a.filters[i].rhoe != b.filters[i].rhoe ||
            a.filters[i].thickness_mm != b.filters[i].thickness_mm)
            return false;
    return true;
}

bool same_spectra(const recon_params& a, const recon_params& b) {
    return same_spectrum(a.low, b.low) && same_spectrum(a.high, b.high) && a.basis_z[0] == b.basis_z[0] &&
           a.basis_z[1] == b.basis_z[1] && a.basis_rhoe[0] == b.basis_rhoe[0] && a.basis_rhoe[1] == b.basis_rhoe[1];
}

bool same_geometry(const recon_geometry& a, const recon_geometry& b) {
    return a.nx == b.nx && a.ny == b.ny && a.pixel_mm == b.pixel_mm && a.n_views == b.n_views &&
           a.n_bins == b.n_bins && a.sid_mm == b.sid_mm && a.sdd_mm == b.sdd_mm && a.bin_mm == b.bin_mm &&
           a.start_rad == b.start_rad && a.arc_rad == b.arc_rad;
}

void free_ctx(Ctx& c) {
    solver_free_graph(c);
    if (c.graph_stream) cudaStreamDestroy(c.graph_stream);
    for (cudaEvent_t e : c.graph_ev)
        if (e) cudaEventDestroy(e);
    c.graph_stream = nullptr;
    if (c.side_stream) {
        cudaStreamSynchronize(c.side_stream);
        cudaStreamDestroy(c.side_stream);
    }
    for (cudaEvent_t e : c.side_ev)
        if (e) cudaEventDestroy(e);
    c.side_stream = nullptr;
    if (c.copy_stream) {
        cudaStreamSynchronize(c.copy_stream);
        cudaStreamDestroy(c.copy_stream);
    }
    for (cudaEvent_t e : c.copy_ev)
        if (e) cudaEventDestroy(e);
    c.copy_stream = nullptr;
    if (c.d2h_stream) {
        cudaStreamSynchronize(c.d2h_stream);
        cudaStreamDestroy(c.d2h_stream);
    }
    for (cudaEvent_t e : c.d2h_ev)
        if (e) cudaEventDestroy(e);
    c.d2h_stream = nullptr;
    for (void* p : c.allocations) cudaFree(p);
    c.allocations.clear();
    if (c.h_cg_pending) cudaFreeHost(c.h_cg_pending);
    c.h_cg_pending = nullptr;
}
}  // namespace

// Argument checks shared by the batch handle and the serving engine; they
// touch no device state.
int check_params(const recon_params& p) {
    if (!(p.lambda > 0) || !(p.beta0 > 0) || !(p.beta_max > 0) || !(p.tau > 0) || p.iters < 0 ||
        p.cg_max_iters < 0 || !(p.cg_tol >= 0) || (p.precision != 0 && p.precision != 1) ||
        (p.order != 0 && p.order != 1) || (p.pcg_kernel != 0 && p.pcg_kernel != 2 && p.pcg_kernel != 3) ||
        (p.domain < 0 || p.domain > 2) || (p.domain != 0 && (p.precision != 1 || p.order != 0)) || !(p.e1_kev > 0) ||
        !(p.e2_kev > 0) || p.e1_kev == p.e2_kev) {
        set_error("invalid recon_params");
        return RECON_EINVAL;
    }
    const recon_spectrum* arms[2] = {&p.low, &p.high};
    for (auto* s : arms) {
        if (s->kind == 0 && !(s->kev > 0)) { set_error("invalid mono energy"); return RECON_EINVAL; }
        if (s->kind == 1 && !(s->kvp > 11)) { set_error("invalid kVp"); return RECON_EINVAL; }
        if (s->kind != 0 && s->kind != 1) { set_error("invalid spectrum kind"); return RECON_EINVAL; }
        if (s->n_filters < 0 || s->n_filters > RECON_MAX_FILTERS) { set_error("invalid filters"); return RECON_EINVAL; }
    }
    return RECON_OK;
}

int check_geometry(const recon_geometry& g) {
    if (g.nx < 1 || g.ny < 1 || g.nx > RECON_MAX_SIDE || g.ny > RECON_MAX_SIDE) {
        set_error("image size outside [1, RECON_MAX_SIDE]");
        return RECON_EINVAL;
    }
    if (!seven_smooth(g.nx) || !seven_smooth(g.ny)) {
        set_error("image sizes must factor into 2, 3, 5, 7");
        return RECON_EINVAL;
    }
    if (g.n_views < 0 || (g.n_views > 0 && (g.n_bins < 1 || !(g.sdd_mm > g.sid_mm) || !(g.sid_mm > 0) ||
                                            !(g.bin_mm > 0) || !(g.pixel_mm > 0)))) {
        set_error("invalid fan-beam geometry");
        return RECON_EINVAL;
    }
    if (g.n_views > 0 && 0.5 * g.pixel_mm * std::sqrt((double)g.nx * g.nx + (double)g.ny * g.ny) >= g.sid_mm) {
        set_error("image reaches the source circle");
        return RECON_EINVAL;
    }
    // sinogram inputs go through the FBP: its limits are checked here too,
    // so a request that passes cannot fail later inside a shared step
    if (g.n_views > 0) return ct_fbp_check(g, 1);
    return RECON_OK;
}

void set_error(const std::string& msg) { g_last_error = msg; }

int cuda_fail(cudaError_t e, const char* what) {
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? RECON_ENOMEM : RECON_ECUDA;
}

}  // namespace recon

using namespace recon;

extern "C" {

int recon_default_params(recon_params* p) {
    if (!p) return RECON_EINVAL;
    std::memset(p, 0, sizeof(*p));
    p->low.kind = 0;
    p->low.kev = 60.0;
    p->high.kind = 0;
    p->high.kev = 90.0;
    p->e1_kev = 50.0;
    p->e2_kev = 200.0;
    p->basis_z[0] = 13.0;
    p->basis_rhoe[0] = 1.7;
    p->basis_z[1] = 7.45;
    p->basis_rhoe[1] = 1.0;
    p->lambda = 1e-2;
    p->beta0 = 2e-2;
    p->beta_max = 1e5;
    p->tau = 1.0;
    p->kappa = 0.0;
    p->iters = 50;
    p->precision = 1;
    p->order = 0;
    p->cg_max_iters = 64;
    p->cg_tol = 1e-6;
    p->z_clip_max = 30.0;
    p->rho_air = 0.1;
    p->pcg_kernel = 0;
    p->domain = 0;
    return RECON_OK;
}

int recon_init_batch(int32_t n, const recon_geometry* geoms, const recon_params* params, void* stream,
                     recon_ctx** out) {
    if (!out || n < 1 || !geoms || !params) {
        set_error("recon_init_batch: bad arguments");
        return RECON_EINVAL;
    }
    *out = nullptr;
    for (int s = 0; s < n; ++s) {
        int rc = check_geometry(geoms[s]);
        if (!rc) rc = check_params(params[s]);
        if (rc) return rc;
        if (params[s].precision != params[0].precision || params[s].order != params[0].order ||
            params[s].pcg_kernel != params[0].pcg_kernel || params[s].domain != params[0].domain) {
            set_error("all slices of a batch need the same precision, order, pcg_kernel and domain");
            return RECON_EINVAL;
        }
        if ((geoms[s].n_views > 0) != (geoms[0].n_views > 0)) {
            set_error("all slices of a batch take images, or all take sinograms");
            return RECON_EINVAL;
        }
        if (params[0].domain != 0) {
            const recon_geometry& a = geoms[s];
            const recon_geometry& b = geoms[0];
            if (a.n_views < 1 || a.nx != b.nx || a.ny != b.ny || a.n_views != b.n_views || a.n_bins != b.n_bins ||
                a.pixel_mm != b.pixel_mm || a.sid_mm != b.sid_mm || a.sdd_mm != b.sdd_mm || a.bin_mm != b.bin_mm ||
                a.start_rad != b.start_rad || a.arc_rad != b.arc_rad) {
                set_error("domains 1 and 2 need sinogram inputs and one geometry for every slice of the batch");
                return RECON_EINVAL;
            }
        }
        if (params[0].domain == 2 && !same_spectra(params[s], params[0])) {
            set_error("domain 2 needs the same spectra and basis materials for every slice of the batch");
            return RECON_EINVAL;
        }
    }
    recon_ctx* h = new (std::nothrow) recon_ctx();
    if (!h) return RECON_ENOMEM;
    Ctx& c = h->c;
    c.n = n;
    c.precision = params[0].precision;
    c.stream = (cudaStream_t)stream;
    c.geo.assign(geoms, geoms + n);
    c.prm.assign(params, params + n);
    c.sino_input = geoms[0].n_views > 0;
    int rc = solver_setup(c);
    if (!rc && c.sino_input) {
        c.sino_off.resize(n);
        long long off = 0;
        long long max_one = 0;
        for (int s = 0; s < n; ++s) {
            c.sino_off[s] = off;
            const long long one = (long long)geoms[s].n_views * geoms[s].n_bins;
            off += one;
            max_one = one > max_one ? one : max_one;
        }
        c.sino_elems = off;
        for (int i = 0; i < 2 && !rc; ++i) {
            cudaError_t e = cudaMalloc((void**)&c.d_sino[i], sizeof(float) * off);
            if (e != cudaSuccess) rc = cuda_fail(e, "cudaMalloc sinogram");
            else c.allocations.push_back(c.d_sino[i]);
        }
        if (!rc) {
            // filtered sinograms of up to kFbpGroup slices (one FBP launch pair per group)
            cudaError_t e = cudaMalloc((void**)&c.d_filt, sizeof(float) * max_one * kFbpGroup);
            if (e != cudaSuccess) rc = cuda_fail(e, "cudaMalloc filter scratch");
            else c.allocations.push_back(c.d_filt);
        }
    }
    if (!rc && params[0].domain != 0) rc = solver_setup_sino(c);
    if (rc) {
        free_ctx(c);
        delete h;
        return rc;
    }
    *out = h;
    return RECON_OK;
}

int recon_init(const recon_geometry* geom, const recon_params* params, void* stream, recon_ctx** out) {
    return recon_init_batch(1, geom, params, stream, out);
}

// The FBP of both staged sinograms of every slice into the unpadded image
// staging buffers d_stage[0], d_stage[1].  Consecutive slices of one geometry
// go through the FBP together, up to kFbpGroup at a time (their sinograms and
// images are contiguous).  With host sinograms (hlo, hhi), each group's two
// sinograms are copied on the copy stream and the group's FBP waits for that
// copy only, so every copy after the first runs beside the FBP of the groups
// before it.
static int copy_stream_ready(Ctx& c) {
    if (!c.copy_stream) {
        RECON_CUDA(cudaStreamCreateWithFlags(&c.copy_stream, cudaStreamNonBlocking));
        for (cudaEvent_t& e : c.copy_ev) RECON_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    return RECON_OK;
}

static int fbp_pair(Ctx& c, const float* hlo = nullptr, const float* hhi = nullptr) {
    if (hlo) {
        int rc;
        if ((rc = copy_stream_ready(c))) return rc;
        // the copies overwrite d_sino: after everything already queued on the stream
        RECON_CUDA(cudaEventRecord(c.copy_ev[0], c.stream));
        RECON_CUDA(cudaStreamWaitEvent(c.copy_stream, c.copy_ev[0], 0));
    }
    for (int s = 0; s < c.n;) {
        int k = 1;
        while (k < kFbpGroup && s + k < c.n && same_geometry(c.geo[s + k], c.geo[s])) ++k;
        if (hlo) {
            const long long end = s + k < c.n ? c.sino_off[s + k] : c.sino_elems;
            const size_t bytes = sizeof(float) * (size_t)(end - c.sino_off[s]);
            RECON_CUDA(cudaMemcpyAsync(c.d_sino[0] + c.sino_off[s], hlo + c.sino_off[s], bytes, cudaMemcpyHostToDevice,
                                       c.copy_stream));
            RECON_CUDA(cudaMemcpyAsync(c.d_sino[1] + c.sino_off[s], hhi + c.sino_off[s], bytes, cudaMemcpyHostToDevice,
                                       c.copy_stream));
            // a wait takes the record before it, so the one event serves every group
            RECON_CUDA(cudaEventRecord(c.copy_ev[1], c.copy_stream));
            RECON_CUDA(cudaStreamWaitEvent(c.stream, c.copy_ev[1], 0));
        }
        for (int a = 0; a < 2; ++a) {
            const int rc = ct_fbp(c.geo[s], k, c.d_sino[a] + c.sino_off[s], c.d_stage[a] + c.sg[s].ext_off, c.d_filt,
                                  c.stream, &c.launches);
            if (rc) return rc;
        }
        s += k;
    }
    return RECON_OK;
}

int recon_set_data(recon_ctx* h, const float* low, const float* high, int on_device) {
    if (!h || !low || !high) {
        set_error("recon_set_data: bad arguments");
        return RECON_EINVAL;
    }
    Ctx& c = h->c;
    const float* lo = low;
    const float* hi = high;
    int rc;
    if (c.sino_input) {
        if (on_device) {
            RECON_CUDA(cudaMemcpyAsync(c.d_sino[0], low, sizeof(float) * c.sino_elems, cudaMemcpyDeviceToDevice,
                                       c.stream));
            RECON_CUDA(cudaMemcpyAsync(c.d_sino[1], high, sizeof(float) * c.sino_elems, cudaMemcpyDeviceToDevice,
                                       c.stream));
            if ((rc = fbp_pair(c))) return rc;
        } else if ((rc = fbp_pair(c, low, high))) {
            return rc;
        }
        lo = c.d_stage[0];
        hi = c.d_stage[1];
    } else if (!on_device) {
        RECON_CUDA(cudaMemcpyAsync(c.d_stage[0], low, sizeof(float) * c.ext_elems, cudaMemcpyHostToDevice, c.stream));
        RECON_CUDA(cudaMemcpyAsync(c.d_stage[1], high, sizeof(float) * c.ext_elems, cudaMemcpyHostToDevice, c.stream));
        lo = c.d_stage[0];
        hi = c.d_stage[1];
    }
    if ((rc = solver_load_images(c, lo, hi, 1))) return rc;
    if ((rc = solver_init_maps(c))) return rc;
    if (c.domain == 1 && (rc = solver_modeb_data(c))) return rc;
    if (c.autotune && !c.tuned && (rc = solver_autotune(c))) return rc;
    c.has_data = true;
    return RECON_OK;
}

int recon_step(recon_ctx* h, int32_t n_iters, recon_stats* stats) {
    if (!h || n_iters < 0) {
        set_error("recon_step: bad arguments");
        return RECON_EINVAL;
    }
    Ctx& c = h->c;
    if (!c.has_data) {
        set_error("recon_step before recon_set_data");
        return RECON_ESTATE;
    }
    int rc;
    for (int k = 0; k < n_iters; ++k) {
        const bool want = stats && k == n_iters - 1;
        if ((rc = solver_iterate(c, want))) return rc;
    }
    if (stats) {
        std::vector<SliceState> st;
        if ((rc = solver_read_state(c, st))) return rc;
        for (int s = 0; s < c.n; ++s) {
            recon_stats& o = stats[s];
            std::memset(&o, 0, sizeof(o));
            const SliceState& x = st[s];
            o.k = x.k;
            o.cg_iters = x.cg_it;
            // the beta factor of one iteration (none for a slice of zero iterations)
            const double kap = c.prm[s].kappa > 0 ? c.prm[s].kappa
                               : c.prm[s].iters > 0
                                   ? std::pow(c.prm[s].beta_max / c.prm[s].beta0, 1.0 / c.prm[s].iters)
                                   : 1.0;
            o.beta = n_iters > 0 ? x.beta / kap : x.beta;
            o.fid_low = x.stat[0];
            o.fid_high = x.stat[1];
            o.model_e1 = x.stat[2];
            o.model_e2 = x.stat[3];
            o.relax = o.beta * x.stat[4];
            long long tot = 0;
            for (int m = 0; m < 4; ++m) {
                o.nnz[m] = x.nnz[m];
                tot += x.nnz[m];
            }
            o.l0 = c.prm[s].lambda * (double)tot;
            o.cg_rel_residual = x.bb > 0 ? std::sqrt(x.rr / x.bb) : 0.0;
        }
    }
    RECON_CUDA(cudaGetLastError());
    return RECON_OK;
}

int recon_get(recon_ctx* h, float* Z, float* rhoe, float* f1, float* f2, int on_device) {
    if (!h) return RECON_EINVAL;
    Ctx& c = h->c;
    if (!c.has_data) {
        set_error("recon_get before recon_set_data");
        return RECON_ESTATE;
    }
    int rc;
    if (on_device) return solver_extract(c, Z, rhoe, f1, f2, 1);
    if ((rc = copy_stream_ready(c))) return rc;
    float* outs[4] = {Z, rhoe, f1, f2};
    // Two outputs at a time through the two unpadded staging buffers, in
    // groups of kFbpGroup slices: a group is copied out on the copy stream
    // while the stream extracts the next one.
    for (int k = 0; k < 4; k += 2) {
        float* a = outs[k] ? c.d_stage[0] : nullptr;
        float* b = outs[k + 1] ? c.d_stage[1] : nullptr;
        if (!a && !b) continue;
        for (int s0 = 0; s0 < c.n; s0 += kFbpGroup) {
            const int s1 = s0 + kFbpGroup < c.n ? s0 + kFbpGroup : c.n;
            if (k == 0) rc = solver_extract_range(c, s0, s1, a, b, nullptr, nullptr);
            else rc = solver_extract_range(c, s0, s1, nullptr, nullptr, a, b);
            if (rc) return rc;
            RECON_CUDA(cudaEventRecord(c.copy_ev[1], c.stream));
            RECON_CUDA(cudaStreamWaitEvent(c.copy_stream, c.copy_ev[1], 0));
            const long long e0 = c.sg[s0].ext_off, e1 = s1 < c.n ? c.sg[s1].ext_off : c.ext_elems;
            const size_t bytes = sizeof(float) * (size_t)(e1 - e0);
            if (a) RECON_CUDA(cudaMemcpyAsync(outs[k] + e0, a + e0, bytes, cudaMemcpyDeviceToHost, c.copy_stream));
            if (b)
                RECON_CUDA(cudaMemcpyAsync(outs[k + 1] + e0, b + e0, bytes, cudaMemcpyDeviceToHost, c.copy_stream));
        }
        // the next pair (or the next call) reuses the staging buffers: after these copies
        RECON_CUDA(cudaEventRecord(c.copy_ev[0], c.copy_stream));
        RECON_CUDA(cudaStreamWaitEvent(c.stream, c.copy_ev[0], 0));
    }
    RECON_CUDA(cudaStreamSynchronize(c.copy_stream));
    return RECON_OK;
}

int recon_direct(recon_ctx* h, float* Z, float* rhoe, int on_device) {
    if (!h || !Z || !rhoe) return RECON_EINVAL;
    Ctx& c = h->c;
    if (!c.has_data) {
        set_error("recon_direct before recon_set_data");
        return RECON_ESTATE;
    }
    // in the sinogram domains the loaded fields hold the data images of the f
    // updates, so the FBP pair is formed again from the staged sinograms
    int rc;
    const float* lo = nullptr;
    const float* hi = nullptr;
    if (c.domain != 0) {
        if ((rc = fbp_pair(c))) return rc;
        lo = c.d_stage[0];
        hi = c.d_stage[1];
    }
    if (on_device) return solver_direct(c, lo, hi, Z, rhoe);
    if ((rc = solver_direct(c, lo, hi, c.d_stage[0], c.d_stage[1]))) return rc;
    RECON_CUDA(cudaMemcpyAsync(Z, c.d_stage[0], sizeof(float) * c.ext_elems, cudaMemcpyDeviceToHost, c.stream));
    RECON_CUDA(cudaMemcpyAsync(rhoe, c.d_stage[1], sizeof(float) * c.ext_elems, cudaMemcpyDeviceToHost, c.stream));
    RECON_CUDA(cudaStreamSynchronize(c.stream));
    return RECON_OK;
}

int recon_mono(recon_ctx* h, int32_t n_e, const double* kev, float* out, int on_device) {
    if (!h || !kev || !out || n_e < 1 || n_e > 16) {
        set_error("recon_mono: bad arguments (1 to 16 energies per call)");
        return RECON_EINVAL;
    }
    Ctx& c = h->c;
    if (!c.has_data) {
        set_error("recon_mono before recon_set_data");
        return RECON_ESTATE;
    }
    if (on_device) return solver_mono(c, n_e, kev, out);
    // host output: one energy at a time through the unpadded staging buffer
    for (int k = 0; k < n_e; ++k) {
        int rc;
        if ((rc = solver_mono(c, 1, kev + k, c.d_stage[0]))) return rc;
        RECON_CUDA(cudaMemcpyAsync(out + (size_t)k * c.ext_elems, c.d_stage[0], sizeof(float) * c.ext_elems,
                                   cudaMemcpyDeviceToHost, c.stream));
        RECON_CUDA(cudaStreamSynchronize(c.stream));
    }
    return RECON_OK;
}

int recon_get_async(recon_ctx* h, float* Z, float* rhoe, float* f1, float* f2) {
    if (!h) return RECON_EINVAL;
    Ctx& c = h->c;
    if (!c.has_data) {
        set_error("recon_get_async before recon_set_data");
        return RECON_ESTATE;
    }
    int rc;
    if (!c.d2h_stream) {
        for (int i = 0; i < 2; ++i) {
            cudaError_t e = cudaMalloc((void**)&c.d_out[i], sizeof(float) * (c.ext_elems > 0 ? c.ext_elems : 1));
            if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc output staging");
            c.allocations.push_back(c.d_out[i]);
        }
        RECON_CUDA(cudaStreamCreateWithFlags(&c.d2h_stream, cudaStreamNonBlocking));
        for (cudaEvent_t& e : c.d2h_ev) RECON_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    float* outs[4] = {Z, rhoe, f1, f2};
    for (int k = 0; k < 4; k += 2) {
        float* a = outs[k] ? c.d_out[0] : nullptr;
        float* b = outs[k + 1] ? c.d_out[1] : nullptr;
        if (!a && !b) continue;
        // the output staging is free once the copies queued before (this call's or an earlier one's) are done
        RECON_CUDA(cudaEventRecord(c.d2h_ev[0], c.d2h_stream));
        RECON_CUDA(cudaStreamWaitEvent(c.stream, c.d2h_ev[0], 0));
        for (int s0 = 0; s0 < c.n; s0 += kFbpGroup) {
            const int s1 = s0 + kFbpGroup < c.n ? s0 + kFbpGroup : c.n;
            if (k == 0) rc = solver_extract_range(c, s0, s1, a, b, nullptr, nullptr);
            else rc = solver_extract_range(c, s0, s1, nullptr, nullptr, a, b);
            if (rc) return rc;
            RECON_CUDA(cudaEventRecord(c.d2h_ev[1], c.stream));
            RECON_CUDA(cudaStreamWaitEvent(c.d2h_stream, c.d2h_ev[1], 0));
            const long long e0 = c.sg[s0].ext_off, e1 = s1 < c.n ? c.sg[s1].ext_off : c.ext_elems;
            const size_t bytes = sizeof(float) * (size_t)(e1 - e0);
            if (a) RECON_CUDA(cudaMemcpyAsync(outs[k] + e0, a + e0, bytes, cudaMemcpyDeviceToHost, c.d2h_stream));
            if (b)
                RECON_CUDA(cudaMemcpyAsync(outs[k + 1] + e0, b + e0, bytes, cudaMemcpyDeviceToHost, c.d2h_stream));
        }
    }
    return RECON_OK;
}

int recon_sync(recon_ctx* h) {
    if (!h) return RECON_EINVAL;
    RECON_CUDA(cudaStreamSynchronize(h->c.stream));
    if (h->c.copy_stream) RECON_CUDA(cudaStreamSynchronize(h->c.copy_stream));
    if (h->c.d2h_stream) RECON_CUDA(cudaStreamSynchronize(h->c.d2h_stream));
    return RECON_OK;
}

void recon_destroy(recon_ctx* h) {
    if (!h) return;
    cudaStreamSynchronize(h->c.stream);
    if (h->c.graph_stream) cudaStreamSynchronize(h->c.graph_stream);
    free_ctx(h->c);
    delete h;
}

int recon_solve(const float* lowE, const float* highE, const recon_geometry* geom, double lambda, double beta,
                int32_t iters, float* Z_out, float* rhoe_out) {
    if (!lowE || !highE || !geom || !Z_out || !rhoe_out) {
        set_error("recon_solve: bad arguments");
        return RECON_EINVAL;
    }
    recon_params p;
    recon_default_params(&p);
    p.lambda = lambda;
    p.beta0 = beta;
    p.iters = iters;
    recon_ctx* h = nullptr;
    int rc = recon_init(geom, &p, nullptr, &h);
    if (rc) return rc;
    rc = recon_set_data(h, lowE, highE, 0);
    if (!rc) rc = recon_step(h, iters, nullptr);
    if (!rc) rc = recon_get(h, Z_out, rhoe_out, nullptr, nullptr, 0);
    recon_destroy(h);
    return rc;
}

const char* recon_strerror(int code) {
    switch (code) {
        case RECON_OK: return "ok";
        case RECON_EINVAL: return "invalid argument";
        case RECON_ENOMEM: return "out of memory";
        case RECON_ECUDA: return "CUDA error";
        case RECON_ETIMEOUT: return "device wait timed out";
        case RECON_ENAN: return "non-finite values";
        case RECON_EBUDGET: return "memory budget exceeded";
        case RECON_ESTATE: return "call out of order";
        default: return "unknown error";
    }
}

const char* recon_last_error(void) { return g_last_error.c_str(); }

int recon_model_tables(const recon_params* params, double* out) {
    if (!params || !out) return RECON_EINVAL;
    const Tables t = make_tables(*params);
    const double v[18] = {t.a[0][0], t.a[0][1], t.a[1][0], t.a[1][1], t.b[0][0], t.b[0][1], t.b[1][0], t.b[1][1],
                          t.P[0],    t.P[1],    t.psi[0],  t.psi[1],  t.r,       t.c_f[0],  t.c_f[1],  t.c_rho,
                          t.a_w,     t.S};
    std::memcpy(out, v, sizeof(v));
    return 18;
}

int recon_debug_field(recon_ctx* h, int32_t field, int32_t slice, void** dev_ptr, int32_t* pitch,
                      int32_t* elem_bytes) {
    if (!h || field < 0 || field >= kNumFields || slice < 0 || slice >= h->c.n || !dev_ptr) return RECON_EINVAL;
    Ctx& c = h->c;
    *dev_ptr = static_cast<char*>(c.field[field]) + c.elem * c.sg[slice].off;
    if (pitch) *pitch = c.sg[slice].pitch;
    if (elem_bytes) *elem_bytes = (int32_t)c.elem;
    return RECON_OK;
}

int recon_debug_io(recon_ctx* h, int32_t field, int32_t slice, double* host, int32_t to_device) {
    if (!h || !host || field < 0 || field >= kNumFields || slice < 0 || slice >= h->c.n) return RECON_EINVAL;
    Ctx& c = h->c;
    const SliceGeom& g = c.sg[slice];
    const size_t rowb = c.elem * g.nx;
    std::vector<unsigned char> tmp(rowb * g.ny);
    char* dev = static_cast<char*>(c.field[field]) + c.elem * g.off;
    if (to_device) {
        for (long long i = 0; i < (long long)g.nx * g.ny; ++i) {
            if (c.elem == 4) reinterpret_cast<float*>(tmp.data())[i] = (float)host[i];
            else reinterpret_cast<double*>(tmp.data())[i] = host[i];
        }
        RECON_CUDA(cudaMemcpy2DAsync(dev, c.elem * g.pitch, tmp.data(), rowb, rowb, g.ny, cudaMemcpyHostToDevice,
                                     c.stream));
        RECON_CUDA(cudaStreamSynchronize(c.stream));
    } else {
        RECON_CUDA(cudaMemcpy2DAsync(tmp.data(), rowb, dev, c.elem * g.pitch, rowb, g.ny, cudaMemcpyDeviceToHost,
                                     c.stream));
        RECON_CUDA(cudaStreamSynchronize(c.stream));
        for (long long i = 0; i < (long long)g.nx * g.ny; ++i)
            host[i] = c.elem == 4 ? (double)reinterpret_cast<float*>(tmp.data())[i]
                                  : reinterpret_cast<double*>(tmp.data())[i];
    }
    return RECON_OK;
}

int recon_debug_op(recon_ctx* h, int32_t op) {
    if (!h) return RECON_EINVAL;
    if (!h->c.has_data && op != RECON_OP_INIT) {
        set_error("recon_debug_op before recon_set_data");
        return RECON_ESTATE;
    }
    return solver_op(h->c, op);
}

int recon_debug_scalars(recon_ctx* h, int32_t slice, double* out) {
    if (!h || !out || slice < 0 || slice >= h->c.n) return RECON_EINVAL;
    std::vector<SliceState> st;
    int rc = solver_read_state(h->c, st);
    if (rc) return rc;
    const SliceState& x = st[slice];
    out[0] = x.beta;
    out[1] = x.beta_t;
    out[2] = x.k;
    out[3] = x.abar2;
    out[4] = x.cg_it;
    out[5] = x.bb > 0 ? std::sqrt(x.rr / x.bb) : 0.0;
    return RECON_OK;
}

int64_t recon_kernel_launches(recon_ctx* h) {
    return h ? h->c.launches + solver_graph_loop_launches(h->c) : -1;
}

int recon_set_autotune(recon_ctx* h, int32_t mode) {
    if (!h || mode < 0 || mode > 2) {
        set_error("recon_set_autotune: bad arguments");
        return RECON_EINVAL;
    }
    h->c.autotune = mode;
    h->c.tuned = false;
    return RECON_OK;
}

int recon_tuning(recon_ctx* h, int32_t* out2) {
    if (!h || !out2) return RECON_EINVAL;
    out2[0] = h->c.grid_mult;
    out2[1] = h->c.row_budget;
    return RECON_OK;
}

int recon_set_graph(recon_ctx* h, int32_t on) {
    if (!h || (on != 0 && on != 1)) {
        set_error("recon_set_graph: bad arguments");
        return RECON_EINVAL;
    }
    return solver_set_graph(h->c, on == 1);
}

int recon_profile(recon_ctx* h, uint32_t mask) {
    if (!h) return RECON_EINVAL;
    h->c.prof_mask = mask;
    return RECON_OK;
}

int recon_profile_read(recon_ctx* h, double* ms, int64_t* launches, uint64_t* bytes) {
    if (!h) return RECON_EINVAL;
    long long l[KF_COUNT];
    unsigned long long b[KF_COUNT];
    int rc = solver_profile_read(h->c, ms, l, b);
    if (rc) return rc;
    for (int f = 0; f < KF_COUNT; ++f) {
        if (launches) launches[f] = l[f];
        if (bytes) bytes[f] = b[f];
    }
    return RECON_OK;
}

static_assert(KF_COUNT == RECON_KF_COUNT, "kernel families of the header and the solver");

const char* recon_profile_name(int32_t f) {
    static const char* names[KF_COUNT] = {"thr_rhs",   "fft_rows_fwd", "fft_cols", "fft_rows_inv",
                                          "synth",     "pcg_start",    "pcg_fwd",  "pcg_cols",
                                          "pcg_inv",   "fcg",          "project",
                                          "mg_fwd",    "mg_y",         "mg_pq",    "mg_levels",
                                          "mg_block",  "mg_setup",     "other"};
    return (f >= 0 && f < KF_COUNT) ? names[f] : "?";
}

int recon_abi_sizes(int64_t* out4) {
    if (!out4) return RECON_EINVAL;
    out4[0] = sizeof(recon_geometry);
    out4[1] = sizeof(recon_spectrum);
    out4[2] = sizeof(recon_params);
    out4[3] = sizeof(recon_stats);
    return RECON_OK;
}

}  // extern "C"
