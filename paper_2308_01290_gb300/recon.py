"""Thin ctypes binding of librecon (include/recon.h): argument marshalling only.

Every computation runs in the CUDA library; this module converts Python
arguments to the C structs and pointers of the ABI and raises ReconError on a
negative return code.  Device buffers are passed as integer addresses (for
example ``tensor.data_ptr()`` of a CUDA tensor), host buffers as NumPy
float32 arrays.  Importing this module loads the library and fails loudly
when it has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "librecon.so")

RECON_MAX_FILTERS = 4
FIELDS = dict(F1=0, F2=1, RHO=2, Z=3, MUL=4, MUH=5, RHS_F1=6, RHS_F2=7, DIV_RHO=8, DIV_Z=9, RHS_RHO=10, A2=11,
              RHS_Z=12, CG_R=13, CG_P0=14, CG_P1=15, CG_Q=16, CG_Y=17, CG_R2=18)
OPS = dict(INIT=0, THRESH_RHS=1, SOLVE_F=2, SYNTH=3, SOLVE_RHO=4, SOLVE_Z=5, NEXT_BETA=6, Z_MATVEC=7)


class Geometry(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("pixel_mm", C.c_double), ("n_views", C.c_int32),
                ("n_bins", C.c_int32), ("sid_mm", C.c_double), ("sdd_mm", C.c_double), ("bin_mm", C.c_double),
                ("start_rad", C.c_double), ("arc_rad", C.c_double)]


class Filter(C.Structure):
    _fields_ = [("Z", C.c_double), ("rhoe", C.c_double), ("thickness_mm", C.c_double)]


class Spectrum(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n_filters", C.c_int32), ("kev", C.c_double), ("kvp", C.c_double),
                ("filters", Filter * RECON_MAX_FILTERS)]


class Params(C.Structure):
    _fields_ = [("low", Spectrum), ("high", Spectrum), ("e1_kev", C.c_double), ("e2_kev", C.c_double),
                ("basis_z", C.c_double * 2), ("basis_rhoe", C.c_double * 2), ("lambda_", C.c_double),
                ("beta0", C.c_double), ("beta_max", C.c_double), ("tau", C.c_double), ("kappa", C.c_double),
                ("iters", C.c_int32), ("precision", C.c_int32), ("order", C.c_int32), ("cg_max_iters", C.c_int32),
                ("cg_tol", C.c_double), ("z_clip_max", C.c_double), ("rho_air", C.c_double),
                ("pcg_kernel", C.c_int32), ("domain", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("k", C.c_int32), ("cg_iters", C.c_int32), ("beta", C.c_double), ("fid_low", C.c_double),
                ("fid_high", C.c_double), ("model_e1", C.c_double), ("model_e2", C.c_double),
                ("relax", C.c_double), ("l0", C.c_double), ("nnz", C.c_int64 * 4),
                ("cg_rel_residual", C.c_double)]


class ServerConfig(C.Structure):
    _fields_ = [("max_slots", C.c_int32), ("max_nx", C.c_int32), ("max_ny", C.c_int32), ("max_views", C.c_int32),
                ("max_bins", C.c_int32), ("precision", C.c_int32), ("hbm_budget_bytes", C.c_double)]


class Request(C.Structure):
    _fields_ = [("geom", Geometry), ("params", Params), ("low", C.c_void_p), ("high", C.c_void_p)]


class Result(C.Structure):
    _fields_ = [("status", C.c_int32), ("iters", C.c_int32), ("queue_ms", C.c_double), ("latency_ms", C.c_double)]


class ReconError(RuntimeError):
    pass


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"librecon is not built ({LIB_PATH} missing); run __graft_entry__.build() "
                          "or python paper_2308_01290_gb300/build_lib.py")
    lib = C.CDLL(LIB_PATH)
    P, I, D, VP = C.POINTER, C.c_int, C.c_double, C.c_void_p
    sig = {
        "recon_default_params": (I, [P(Params)]),
        "recon_init": (I, [P(Geometry), P(Params), VP, P(VP)]),
        "recon_init_batch": (I, [C.c_int32, P(Geometry), P(Params), VP, P(VP)]),
        "recon_set_data": (I, [VP, VP, VP, I]),
        "recon_step": (I, [VP, C.c_int32, P(Stats)]),
        "recon_get": (I, [VP, VP, VP, VP, VP, I]),
        "recon_get_async": (I, [VP, VP, VP, VP, VP]),
        "recon_sync": (I, [VP]),
        "recon_direct": (I, [VP, VP, VP, I]),
        "recon_mono": (I, [VP, C.c_int32, P(D), VP, I]),
        "recon_iqa": (I, [C.c_int32, C.c_int32, C.c_int32, VP, VP, VP, P(D), VP]),
        "recon_destroy": (None, [VP]),
        "recon_solve": (I, [VP, VP, P(Geometry), D, D, C.c_int32, VP, VP]),
        "recon_strerror": (C.c_char_p, [I]),
        "recon_last_error": (C.c_char_p, []),
        "recon_project": (I, [P(Geometry), C.c_int32, VP, VP, VP]),
        "recon_backproject": (I, [P(Geometry), C.c_int32, VP, VP, VP]),
        "recon_fbp": (I, [P(Geometry), C.c_int32, VP, VP, VP]),
        "recon_fbp_noalloc": (I, [P(Geometry), C.c_int32, VP, VP, VP]),
        "recon_simulate": (I, [P(Geometry), P(Params), C.c_int32, VP, VP, VP, D, VP, VP, VP]),
        "recon_model_tables": (I, [P(Params), P(D)]),
        "recon_debug_field": (I, [VP, C.c_int32, C.c_int32, P(VP), P(C.c_int32), P(C.c_int32)]),
        "recon_debug_op": (I, [VP, C.c_int32]),
        "recon_debug_io": (I, [VP, C.c_int32, C.c_int32, P(D), C.c_int32]),
        "recon_debug_scalars": (I, [VP, C.c_int32, P(D)]),
        "recon_kernel_launches": (C.c_int64, [VP]),
        "recon_set_graph": (I, [VP, C.c_int32]),
        "recon_set_autotune": (I, [VP, C.c_int32]),
        "recon_tuning": (I, [VP, P(C.c_int32)]),
        "recon_abi_sizes": (I, [P(C.c_int64)]),
        "recon_server_create": (I, [P(ServerConfig), VP, P(VP)]),
        "recon_submit": (I, [VP, P(Request), P(C.c_uint64)]),
        "recon_server_step": (I, [VP, C.c_int32, P(C.c_int32)]),
        "recon_poll": (I, [VP, C.c_uint64, VP, VP, P(Result)]),
        "recon_server_stats": (I, [VP, P(C.c_int64)]),
        "recon_server_destroy": (None, [VP]),
        "recon_profile": (I, [VP, C.c_uint32]),
        "recon_profile_read": (I, [VP, P(D), P(C.c_int64), P(C.c_uint64)]),
        "recon_profile_name": (C.c_char_p, [C.c_int32]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()


def _check_layout():
    out = (C.c_int64 * 4)()
    lib.recon_abi_sizes(out)
    mine = (C.sizeof(Geometry), C.sizeof(Spectrum), C.sizeof(Params), C.sizeof(Stats))
    if tuple(out) != mine:
        raise ImportError(f"ctypes struct layout {mine} differs from librecon's {tuple(out)}")


_check_layout()
EXPORTS = ("recon_default_params", "recon_init", "recon_init_batch", "recon_set_data", "recon_step", "recon_get",
           "recon_get_async",
           "recon_sync", "recon_destroy", "recon_solve", "recon_strerror", "recon_last_error", "recon_project",
           "recon_backproject", "recon_fbp", "recon_fbp_noalloc", "recon_simulate", "recon_model_tables", "recon_debug_field",
           "recon_debug_op", "recon_debug_io", "recon_debug_scalars", "recon_kernel_launches", "recon_set_graph",
           "recon_set_autotune", "recon_tuning",
           "recon_abi_sizes", "recon_profile", "recon_profile_read", "recon_profile_name", "recon_server_create",
           "recon_submit", "recon_server_step", "recon_poll", "recon_server_stats", "recon_server_destroy",
           "recon_direct", "recon_mono", "recon_iqa")
KF_COUNT = 18


def _check(rc, what):
    if rc < 0:
        msg = lib.recon_last_error().decode()
        raise ReconError(f"{what}: {lib.recon_strerror(rc).decode()} ({rc}): {msg}")
    return rc


def _ptr(x):
    """Address of a device buffer (int or object with data_ptr()) or host ndarray."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        assert x.dtype == np.float32 and x.flags["C_CONTIGUOUS"], "host buffers must be C-contiguous float32"
        return x.ctypes.data
    raise TypeError(type(x))


# --------------------------------------------------------------------------
# struct builders
# --------------------------------------------------------------------------

def geometry(nx, ny, pixel_mm=1.0, n_views=0, n_bins=0, sid_mm=1000.0, sdd_mm=1500.0, bin_mm=1.0,
             start_rad=0.0, arc_rad=2 * np.pi) -> Geometry:
    return Geometry(int(nx), int(ny), float(pixel_mm), int(n_views), int(n_bins), float(sid_mm), float(sdd_mm),
                    float(bin_mm), float(start_rad), float(arc_rad))


def geometry_from_acq(acq, image_input=False) -> Geometry:
    return geometry(acq.nx, acq.ny, acq.pixel_mm, 0 if image_input else acq.n_views, acq.n_bins, acq.sid_mm,
                    acq.sdd_mm, acq.bin_mm)


def spectrum(spec) -> Spectrum:
    """From a synthetic.phantoms.Spectrum-like object."""
    s = Spectrum()
    s.kind = 0 if spec.kind == "mono" else 1
    s.kev = float(spec.kev)
    s.kvp = float(spec.kvp)
    s.n_filters = len(spec.filters)
    for i, (_, z, rho, t) in enumerate(spec.filters):
        s.filters[i] = Filter(float(z), float(rho), float(t))
    return s


def default_params(**kw) -> Params:
    p = Params()
    _check(lib.recon_default_params(C.byref(p)), "recon_default_params")
    for k, v in kw.items():
        if k in ("low", "high"):
            setattr(p, k, spectrum(v) if not isinstance(v, Spectrum) else v)
        elif k == "lam":
            p.lambda_ = float(v)
        else:
            setattr(p, k, v)
    return p


def model_tables(params: Params) -> np.ndarray:
    out = (C.c_double * 32)()
    n = _check(lib.recon_model_tables(C.byref(params), out), "recon_model_tables")
    return np.array(out[:n])


# --------------------------------------------------------------------------
# solve handle
# --------------------------------------------------------------------------

class Solver:
    """A batch of slices solved together (recon_init_batch)."""

    def __init__(self, geoms, params, stream=None):
        if isinstance(geoms, Geometry):
            geoms = [geoms]
        if isinstance(params, Params):
            params = [params] * len(geoms)
        assert len(params) == len(geoms)
        self.n = len(geoms)
        ga = (Geometry * self.n)(*geoms)
        pa = (Params * self.n)(*params)
        h = C.c_void_p()
        _check(lib.recon_init_batch(self.n, ga, pa, stream, C.byref(h)), "recon_init_batch")
        self.h = h
        self.geoms = list(geoms)

    def close(self):
        if self.h:
            lib.recon_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_data(self, low, high, on_device=None):
        if on_device is None:
            on_device = not isinstance(low, np.ndarray)
        _check(lib.recon_set_data(self.h, _ptr(low), _ptr(high), int(on_device)), "recon_set_data")

    def step(self, n_iters, stats=False):
        if stats:
            arr = (Stats * self.n)()
            _check(lib.recon_step(self.h, int(n_iters), arr), "recon_step")
            return [arr[i] for i in range(self.n)]
        _check(lib.recon_step(self.h, int(n_iters), None), "recon_step")
        return None

    def get(self, Z=None, rhoe=None, f1=None, f2=None, on_device=None):
        anyb = next((b for b in (Z, rhoe, f1, f2) if b is not None), None)
        if on_device is None:
            on_device = anyb is not None and not isinstance(anyb, np.ndarray)
        _check(lib.recon_get(self.h, _ptr(Z), _ptr(rhoe), _ptr(f1), _ptr(f2), int(on_device)), "recon_get")

    def get_host(self):
        """(Z, rho_e, f1, f2) as lists of per-slice float32 arrays."""
        tot = sum(g.nx * g.ny for g in self.geoms)
        outs = [np.empty(tot, np.float32) for _ in range(4)]
        self.get(*outs)
        res = []
        for o in outs:
            parts, off = [], 0
            for g in self.geoms:
                parts.append(o[off:off + g.nx * g.ny].reshape(g.ny, g.nx))
                off += g.nx * g.ny
            res.append(parts)
        return res

    def get_async(self, Z=None, rhoe=None, f1=None, f2=None):
        """Host maps without waiting for the copies (recon_get_async): the
        buffers (host addresses, pinned for overlap) are complete after sync()."""
        _check(lib.recon_get_async(self.h, _ptr(Z), _ptr(rhoe), _ptr(f1), _ptr(f2)), "recon_get_async")

    def sync(self):
        _check(lib.recon_sync(self.h), "recon_sync")

    def direct(self, Z=None, rhoe=None, on_device=None):
        """Z and rho_e of the two-step image-based method (recon_direct); with
        no buffers, host arrays per slice."""
        if Z is None:
            tot = sum(g.nx * g.ny for g in self.geoms)
            Z, rhoe = np.empty(tot, np.float32), np.empty(tot, np.float32)
            _check(lib.recon_direct(self.h, _ptr(Z), _ptr(rhoe), 0), "recon_direct")
            return self._split(Z), self._split(rhoe)
        if on_device is None:
            on_device = not isinstance(Z, np.ndarray)
        _check(lib.recon_direct(self.h, _ptr(Z), _ptr(rhoe), int(on_device)), "recon_direct")
        return None

    def mono(self, kev, out=None, on_device=None):
        """Monoenergetic images at the energies kev (recon_mono); with no
        buffer, a list (per energy) of per-slice host arrays."""
        e = np.ascontiguousarray(np.atleast_1d(np.asarray(kev, np.float64)))
        ep = e.ctypes.data_as(C.POINTER(C.c_double))
        if out is None:
            tot = sum(g.nx * g.ny for g in self.geoms)
            buf = np.empty(len(e) * tot, np.float32)
            _check(lib.recon_mono(self.h, len(e), ep, _ptr(buf), 0), "recon_mono")
            return [self._split(buf[k * tot:(k + 1) * tot]) for k in range(len(e))]
        if on_device is None:
            on_device = not isinstance(out, np.ndarray)
        _check(lib.recon_mono(self.h, len(e), ep, _ptr(out), int(on_device)), "recon_mono")
        return None

    def _split(self, flat):
        parts, off = [], 0
        for g in self.geoms:
            parts.append(flat[off:off + g.nx * g.ny].reshape(g.ny, g.nx))
            off += g.nx * g.ny
        return parts

    def field(self, name, slice_=0):
        p = C.c_void_p()
        pitch = C.c_int32()
        eb = C.c_int32()
        _check(lib.recon_debug_field(self.h, FIELDS[name], int(slice_), C.byref(p), C.byref(pitch), C.byref(eb)),
               "recon_debug_field")
        return p.value, pitch.value, eb.value

    def read(self, name, slice_=0):
        g = self.geoms[slice_]
        out = np.empty((g.ny, g.nx), np.float64)
        _check(lib.recon_debug_io(self.h, FIELDS[name], int(slice_), out.ctypes.data_as(C.POINTER(C.c_double)), 0),
               "recon_debug_io")
        return out

    def write(self, name, values, slice_=0):
        g = self.geoms[slice_]
        buf = np.ascontiguousarray(np.asarray(values, np.float64).reshape(g.ny, g.nx))
        _check(lib.recon_debug_io(self.h, FIELDS[name], int(slice_), buf.ctypes.data_as(C.POINTER(C.c_double)), 1),
               "recon_debug_io")

    def op(self, name):
        _check(lib.recon_debug_op(self.h, OPS[name]), "recon_debug_op")

    def scalars(self, slice_=0):
        out = (C.c_double * 8)()
        _check(lib.recon_debug_scalars(self.h, int(slice_), out), "recon_debug_scalars")
        return dict(beta=out[0], beta_t=out[1], k=int(out[2]), abar2=out[3], cg_iters=int(out[4]),
                    cg_rel_residual=out[5])

    def profile(self, mask):
        _check(lib.recon_profile(self.h, int(mask)), "recon_profile")

    def profile_read(self):
        """{family name: (ms, launches, algorithmic bytes)} since the last read."""
        ms = (C.c_double * KF_COUNT)()
        la = (C.c_int64 * KF_COUNT)()
        by = (C.c_uint64 * KF_COUNT)()
        _check(lib.recon_profile_read(self.h, ms, la, by), "recon_profile_read")
        return {lib.recon_profile_name(f).decode(): (ms[f], la[f], by[f]) for f in range(KF_COUNT)}

    def launches(self):
        return int(lib.recon_kernel_launches(self.h))

    def set_graph(self, on=True):
        """Run each following iteration as one CUDA graph launch (recon_set_graph)."""
        _check(lib.recon_set_graph(self.h, 1 if on else 0), "recon_set_graph")

    def set_autotune(self, mode=1):
        """Tune the launch shapes at the next set_data (recon_set_autotune)."""
        _check(lib.recon_set_autotune(self.h, int(mode)), "recon_set_autotune")

    def tuning(self):
        """(grid multiplier, row-item slots) in use (recon_tuning)."""
        out = (C.c_int32 * 2)()
        _check(lib.recon_tuning(self.h, out), "recon_tuning")
        return int(out[0]), int(out[1])


def solve(low, high, geom: Geometry, lam, beta, iters):
    """One-shot recon_solve on host float32 arrays; returns (Z, rho_e)."""
    low = np.ascontiguousarray(low, np.float32)
    high = np.ascontiguousarray(high, np.float32)
    Z = np.empty((geom.ny, geom.nx), np.float32)
    R = np.empty((geom.ny, geom.nx), np.float32)
    _check(lib.recon_solve(_ptr(low), _ptr(high), C.byref(geom), float(lam), float(beta), int(iters), _ptr(Z),
                           _ptr(R)), "recon_solve")
    return Z, R


def project(geom, n, img, sino, stream=None):
    _check(lib.recon_project(C.byref(geom), int(n), _ptr(img), _ptr(sino), stream), "recon_project")


def backproject(geom, n, sino, img, stream=None):
    _check(lib.recon_backproject(C.byref(geom), int(n), _ptr(sino), _ptr(img), stream), "recon_backproject")


def fbp(geom, n, sino, img, stream=None):
    _check(lib.recon_fbp(C.byref(geom), int(n), _ptr(sino), _ptr(img), stream), "recon_fbp")


FBP_NOALLOC_MAX = 2 * 1024 * 1024


def fbp_noalloc(geom, n, sino, img, stream=None):
    """recon_fbp_noalloc: FBP with the library's fixed scratch (no allocation)."""
    _check(lib.recon_fbp_noalloc(C.byref(geom), int(n), _ptr(sino), _ptr(img), stream), "recon_fbp_noalloc")


def simulate(geom, params, n, Z, rhoe, noise, i0, sino_low, sino_high, stream=None):
    _check(lib.recon_simulate(C.byref(geom), C.byref(params), int(n), _ptr(Z), _ptr(rhoe), _ptr(noise), float(i0),
                              _ptr(sino_low), _ptr(sino_high), stream), "recon_simulate")


# --------------------------------------------------------------------------
# serving engine
# --------------------------------------------------------------------------

class Server:
    """recon_server: continuous batching of independent slice solves."""

    def __init__(self, max_slots, max_nx, max_ny, max_views=0, max_bins=0, precision=1, hbm_budget_bytes=0.0,
                 stream=None):
        cfg = ServerConfig(int(max_slots), int(max_nx), int(max_ny), int(max_views), int(max_bins), int(precision),
                           float(hbm_budget_bytes))
        h = C.c_void_p()
        _check(lib.recon_server_create(C.byref(cfg), stream, C.byref(h)), "recon_server_create")
        self.h = h
        self.shapes = {}

    def close(self):
        if self.h:
            lib.recon_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, geom, params, low, high):
        low = np.ascontiguousarray(low, np.float32)
        high = np.ascontiguousarray(high, np.float32)
        req = Request(geom, params, low.ctypes.data, high.ctypes.data)
        t = C.c_uint64()
        _check(lib.recon_submit(self.h, C.byref(req), C.byref(t)), "recon_submit")
        self.shapes[t.value] = (geom.ny, geom.nx)
        return t.value

    def step(self, n_iters=1):
        n = C.c_int32()
        _check(lib.recon_server_step(self.h, int(n_iters), C.byref(n)), "recon_server_step")
        return n.value

    def poll(self, ticket):
        """None while pending, else (Z, rho_e, Result)."""
        ny, nx = self.shapes[ticket]
        Z = np.empty((ny, nx), np.float32)
        R = np.empty((ny, nx), np.float32)
        res = Result()
        rc = _check(lib.recon_poll(self.h, C.c_uint64(ticket), Z.ctypes.data, R.ctypes.data, C.byref(res)),
                    "recon_poll")
        if rc == 0:
            return None
        del self.shapes[ticket]
        return Z, R, res

    def stats(self):
        out = (C.c_int64 * 4)()
        _check(lib.recon_server_stats(self.h, out), "recon_server_stats")
        return dict(queued=out[0], active=out[1], finished=out[2], footprint=out[3])


def iqa(n, nx, ny, x, ref, mask=None, stream=None):
    """(PSNR, NMAD, SSIM) per slice of device maps x against ref (recon_iqa);
    an (n, 3) array."""
    out = np.empty(3 * int(n), np.float64)
    _check(lib.recon_iqa(int(n), int(nx), int(ny), _ptr(x), _ptr(ref), _ptr(mask) if mask is not None else None,
                         out.ctypes.data_as(C.POINTER(C.c_double)), stream), "recon_iqa")
    return out.reshape(int(n), 3)
