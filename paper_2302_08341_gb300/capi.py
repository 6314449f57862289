"""ctypes binding of libflood.so (C ABI in include/flood.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  Arrays may be numpy arrays (host memory) or torch tensors
(host or device); streams may be a torch.cuda.Stream, a raw cudaStream_t
integer, or None for torch's current stream.  There is no CPU fallback: if
the library has not been built, loading it raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libflood.so")

FLOOD_OK = 0
ERRORS = {-1: "FLOOD_ERR_ARG", -2: "FLOOD_ERR_CUDA", -3: "FLOOD_ERR_OOM",
          -4: "FLOOD_ERR_TIMEOUT", -5: "FLOOD_ERR_NAN", -6: "FLOOD_ERR_STATE"}

EXPORTED = ["flood_default_params", "flood_last_error", "flood_create_grid", "flood_destroy",
            "flood_ensemble_init", "flood_step", "flood_gauge_sample", "pf_assimilate",
            "pf_resample_systematic", "flood_get_state", "flood_set_state", "flood_get_members",
            "flood_set_members", "flood_volume_report", "flood_launch_count", "flood_sync",
            "flood_profile", "flood_set_launch", "flood_get_launch", "flood_set_engine",
            "flood_set_wait_budget",
            "flood_adjoint", "flood_adjoint_timing", "flood_batch_create", "flood_batch_destroy",
            "flood_batch_last_error", "flood_batch_init", "flood_batch_step",
            "flood_batch_set_launch", "flood_batch_get_state", "flood_batch_members",
            "flood_batch_launch_count", "flood_autotune", "flood_storage_static",
            "flood_storage_static_error", "flood_set_roughness_factor",
            "flood_get_roughness_factor", "flood_roughness_factor_grad", "flood_calibration_step",
            "flood_batch_set_engine", "flood_track_max_depth", "flood_get_max_depth",
            "flood_ensemble_products", "flood_set_land_cover", "flood_set_land_params",
            "flood_get_land_params", "flood_drained_volume", "flood_flow_sample", "flood_set_inflow",
            "flood_inflow_volume", "flood_batch_autotune", "flood_batch_set_wait_budget",
            "flood_adjoint_land_grad", "flood_batch_init_members", "flood_batch_get_member_state",
            "flood_batch_set_land_cover", "flood_batch_set_land_params", "flood_batch_drained_volume",
            "flood_set_graphs", "flood_graph_stats"]


class LandClass(C.Structure):
    """flood_land_class: Manning n, runoff coefficient, drainage and
    outside-the-domain flags of one land-cover class (Section 4.1)."""
    _fields_ = [("n", C.c_float), ("runoff", C.c_float), ("drains", C.c_int), ("outside", C.c_int)]


class Section(C.Structure):
    """flood_section: a straight line of links (axis 0: east links of cells
    (r, fixed), r in [start, end); axis 1: south links of cells (fixed, c))."""
    _fields_ = [("axis", C.c_int), ("fixed", C.c_int), ("start", C.c_int), ("end", C.c_int)]


class FloodError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class LossSpec(C.Structure):
    """flood_loss_spec (include/flood.h)."""
    _fields_ = [("n_samples", C.c_int32), ("n_gauges", C.c_int32), ("sample_dt", C.c_double),
                ("cells", C.c_void_p), ("d", C.c_void_p)]


class Params(C.Structure):
    """flood_params (include/flood.h)."""
    _fields_ = [("dx", C.c_double), ("g", C.c_double), ("alpha", C.c_double),
                ("dt_cap", C.c_double), ("dt_fixed", C.c_double), ("h_eps", C.c_double),
                ("h_floor", C.c_double), ("rain_block", C.c_double), ("edge_slope", C.c_double),
                ("limiter", C.c_int32), ("east_outflow", C.c_int32), ("south_outflow", C.c_int32),
                ("reserved", C.c_int32)]

    @staticmethod
    def default(**kw):
        p = Params()
        lib().flood_default_params(C.byref(p))
        for k, v in kw.items():
            if not hasattr(p, k):
                raise AttributeError(k)
            setattr(p, k, v)
        return p


_lib = None
_VP = C.c_void_p


def lib(path: str = LIB_PATH):
    """Load libflood.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libflood.so not found at {path}: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    L = C.CDLL(path)
    L.flood_default_params.argtypes = [C.POINTER(Params)]
    L.flood_default_params.restype = None
    L.flood_last_error.argtypes = [_VP]
    L.flood_last_error.restype = C.c_char_p
    L.flood_create_grid.argtypes = [C.POINTER(_VP), C.c_int, C.c_int, _VP, _VP, C.POINTER(Params)]
    L.flood_destroy.argtypes = [_VP]
    L.flood_ensemble_init.argtypes = [_VP, C.c_int, _VP, C.c_int, _VP, _VP, _VP, C.c_int,
                                      C.c_double, _VP]
    L.flood_step.argtypes = [_VP, C.c_int, C.c_double, _VP]
    L.flood_gauge_sample.argtypes = [_VP, C.c_int, _VP, _VP, _VP]
    L.pf_assimilate.argtypes = [_VP, C.c_int, _VP, _VP, _VP, C.c_double, C.c_double, C.c_int,
                                C.c_double, _VP, _VP, _VP, _VP, _VP, _VP]
    L.pf_resample_systematic.argtypes = [C.c_int, _VP, C.c_double, _VP, _VP]
    L.flood_get_state.argtypes = [_VP, C.c_int, _VP, _VP, _VP, _VP]
    L.flood_set_state.argtypes = [_VP, C.c_int, _VP, _VP, _VP, _VP]
    L.flood_get_members.argtypes = [_VP, _VP, _VP, _VP, _VP, _VP, _VP]
    L.flood_set_members.argtypes = [_VP, _VP, _VP, _VP]
    L.flood_volume_report.argtypes = [_VP, _VP, _VP, _VP, _VP]
    L.flood_launch_count.argtypes = [_VP]
    L.flood_launch_count.restype = C.c_int64
    L.flood_sync.argtypes = [_VP, _VP]
    L.flood_profile.argtypes = [_VP, C.c_int, _VP, _VP]
    L.flood_set_launch.argtypes = [_VP, C.c_int, C.c_int]
    L.flood_get_launch.argtypes = [_VP, _VP, _VP]
    L.flood_set_engine.argtypes = [_VP, C.c_int]
    L.flood_adjoint.argtypes = [_VP, C.POINTER(LossSpec), C.c_int, _VP, _VP, _VP, _VP, _VP, _VP]
    L.flood_adjoint_timing.argtypes = [_VP, _VP, _VP]
    L.flood_set_wait_budget.argtypes = [_VP, C.c_int64]
    L.flood_set_graphs.argtypes = [_VP, C.c_int]
    L.flood_graph_stats.argtypes = [_VP, _VP, _VP]
    L.flood_batch_autotune.argtypes = [_VP, C.c_double, _VP, _VP, _VP, _VP, _VP]
    L.flood_batch_set_wait_budget.argtypes = [_VP, C.c_int64]
    L.flood_autotune.argtypes = [_VP, C.c_int, _VP, _VP, _VP, _VP, _VP]
    L.flood_storage_static.argtypes = [_VP, C.c_int, C.c_int, C.c_int, C.c_double, _VP, _VP]
    L.flood_set_roughness_factor.argtypes = [_VP, C.c_int, C.c_int, _VP, _VP]
    L.flood_get_roughness_factor.argtypes = [_VP, _VP, _VP, _VP]
    L.flood_roughness_factor_grad.argtypes = [_VP, _VP, _VP]
    L.flood_calibration_step.argtypes = [_VP, C.c_double, C.c_double, _VP, _VP]
    L.flood_storage_static_error.argtypes = []
    L.flood_storage_static_error.restype = C.c_char_p
    L.flood_batch_create.argtypes = [C.POINTER(_VP), C.c_int, _VP, _VP, _VP, _VP,
                                     C.POINTER(Params)]
    L.flood_batch_destroy.argtypes = [_VP]
    L.flood_batch_last_error.argtypes = [_VP]
    L.flood_batch_last_error.restype = C.c_char_p
    L.flood_batch_init.argtypes = [_VP, _VP, _VP, _VP, _VP, _VP, _VP]
    L.flood_batch_step.argtypes = [_VP, C.c_double, _VP]
    L.flood_batch_set_launch.argtypes = [_VP, C.c_int, C.c_int]
    L.flood_batch_set_engine.argtypes = [_VP, C.c_int]
    L.flood_set_land_cover.argtypes = [_VP, _VP, C.c_int, C.POINTER(LandClass)]
    L.flood_set_land_params.argtypes = [_VP, _VP, _VP]
    L.flood_get_land_params.argtypes = [_VP, _VP, _VP]
    L.flood_drained_volume.argtypes = [_VP, _VP]
    L.flood_adjoint_land_grad.argtypes = [_VP, _VP, _VP, _VP]
    L.flood_flow_sample.argtypes = [_VP, C.c_int, C.POINTER(Section), _VP, _VP]
    L.flood_set_inflow.argtypes = [_VP, C.c_int, C.c_int, _VP, C.c_int]
    L.flood_inflow_volume.argtypes = [_VP, _VP]
    L.flood_track_max_depth.argtypes = [_VP, C.c_int, _VP]
    L.flood_get_max_depth.argtypes = [_VP, C.c_int, _VP, _VP]
    L.flood_ensemble_products.argtypes = [_VP, C.c_double, C.c_int, _VP, _VP, _VP, _VP]
    L.flood_batch_get_state.argtypes = [_VP, C.c_int, _VP, _VP, _VP, _VP]
    L.flood_batch_get_member_state.argtypes = [_VP, C.c_int, C.c_int, _VP, _VP, _VP, _VP]
    L.flood_batch_init_members.argtypes = [_VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP]
    L.flood_batch_members.argtypes = [_VP, _VP, _VP, _VP, _VP, _VP, _VP]
    L.flood_batch_set_land_cover.argtypes = [_VP, C.c_int, _VP, C.c_int, C.POINTER(LandClass)]
    L.flood_batch_set_land_params.argtypes = [_VP, C.c_int, _VP, _VP]
    L.flood_batch_drained_volume.argtypes = [_VP, _VP]
    L.flood_batch_launch_count.argtypes = [_VP]
    L.flood_batch_launch_count.restype = C.c_int64
    for name in EXPORTED:
        if name not in ("flood_default_params", "flood_last_error", "flood_launch_count",
                        "flood_batch_last_error", "flood_batch_launch_count",
                        "flood_storage_static_error"):
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


def ptr(a):
    """Raw pointer of a numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    raise TypeError(f"unsupported buffer type {type(a)}")


def stream_handle(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _f32(a, shape=None):
    if hasattr(a, "data_ptr"):
        return a
    a = np.ascontiguousarray(a, dtype=np.float32)
    if shape is not None and a.shape != tuple(shape):
        a = a.reshape(shape)
    return a


def _check(rc, handle=None):
    if rc != FLOOD_OK:
        msg = lib().flood_last_error(handle)
        raise FloodError(rc, msg.decode() if msg else "")


def resample_systematic(w, u, stream=None):
    """DA step (IV) on the device for given weights (FP64) and offset u."""
    w = np.ascontiguousarray(w, dtype=np.float64)
    idx = np.zeros(len(w), dtype=np.int32)
    s = stream_handle(stream)
    _check(lib().pf_resample_systematic(len(w), ptr(w), float(u), ptr(idx), s))
    _sync_stream(s)
    return idx


def _sync_stream(s):
    try:
        import torch
        if torch.cuda.is_available():
            if s is None:
                torch.cuda.synchronize()
            else:
                torch.cuda.ExternalStream(s).synchronize()
    except ImportError:
        pass


class Grid:
    """One terrain (bed z and base Manning n, shared by all members) and its
    ensemble on the GPU."""

    def __init__(self, z, n, params: Params | None = None):
        L = lib()
        self.params = params if params is not None else Params.default()
        zz = _f32(z); nn = _f32(n)
        ny, nx = (int(zz.shape[0]), int(zz.shape[1]))
        self.ny, self.nx = ny, nx
        h = _VP()
        _check(L.flood_create_grid(C.byref(h), ny, nx, ptr(zz), ptr(nn), C.byref(self.params)))
        self.h = h
        self.M = 0

    def close(self):
        if getattr(self, "h", None):
            lib().flood_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ---- ensemble -------------------------------------------------------
    def ensemble_init(self, M, rain_mult, scale, hyetograph, h0=None, t0=0.0, stream=None):
        rm = _f32(rain_mult); sc = _f32(scale); hy = _f32(hyetograph)
        per = 0
        h0a = None
        if h0 is not None:
            h0a = _f32(h0)
            per = 1 if len(h0a.shape) == 3 else 0
        _check(lib().flood_ensemble_init(self.h, int(M), ptr(h0a), per, ptr(rm), ptr(sc), ptr(hy),
                                         int(hy.shape[0]) if len(hy.shape) else 0, float(t0),
                                         stream_handle(stream)), self.h)
        self.M = int(M)

    def step(self, n_steps=0, t_end=-1.0, stream=None):
        _check(lib().flood_step(self.h, int(n_steps), float(t_end), stream_handle(stream)), self.h)

    def advance_to(self, t_end, stream=None):
        self.step(0, t_end, stream)

    def sync(self, stream=None):
        _check(lib().flood_sync(self.h, stream_handle(stream)), self.h)

    def gauge_sample(self, cells, out=None, stream=None):
        cells = np.ascontiguousarray(cells, dtype=np.int32)
        y = out if out is not None else np.zeros((self.M, len(cells)), dtype=np.float32)
        s = stream_handle(stream)
        _check(lib().flood_gauge_sample(self.h, len(cells), ptr(cells), ptr(y), s), self.h)
        if out is None:
            _sync_stream(s)
        return y

    def pf_assimilate(self, d, sigma, u, beta, y=None, sigma_rel=0.0, n_thr_frac=0.8,
                      force=False, stream=None, outputs=None):
        """DA steps (II)-(V).  Returns a dict with weights, idx, neff,
        resampled (host copies; the call synchronises the stream) unless
        `outputs` supplies the destination buffers."""
        G = int(d.shape[0]) if hasattr(d, "shape") else len(d)
        if not hasattr(d, "data_ptr"):
            d = np.ascontiguousarray(d, dtype=np.float64)
        if sigma is None or hasattr(sigma, "data_ptr"):
            sg = sigma
        else:
            sg = np.ascontiguousarray(np.broadcast_to(sigma, (G,)), dtype=np.float64)
        beta = _f32(beta)
        ya = None if y is None else _f32(y)
        if outputs is None:
            out = dict(weights=np.zeros(self.M), idx=np.zeros(self.M, dtype=np.int32),
                       neff=np.zeros(1), resampled=np.zeros(1, dtype=np.int32))
        else:
            out = outputs
        s = stream_handle(stream)
        _check(lib().pf_assimilate(self.h, G, ptr(ya), ptr(d), ptr(sg), float(sigma_rel),
                                   float(n_thr_frac), int(bool(force)), float(u), ptr(beta),
                                   ptr(out["weights"]), ptr(out["idx"]), ptr(out["neff"]),
                                   ptr(out["resampled"]), s), self.h)
        if outputs is None:
            _sync_stream(s)
            return dict(weights=out["weights"], idx=out["idx"], neff=float(out["neff"][0]),
                        resampled=bool(out["resampled"][0]))
        return out

    # ---- state access -----------------------------------------------------
    def get_state(self, member, stream=None):
        h = np.zeros((self.ny, self.nx), np.float32)
        qx = np.zeros_like(h); qy = np.zeros_like(h)
        s = stream_handle(stream)
        _check(lib().flood_get_state(self.h, int(member), ptr(h), ptr(qx), ptr(qy), s), self.h)
        _sync_stream(s)
        return h, qx, qy

    def set_state(self, member, h=None, qx=None, qy=None, stream=None):
        a = [None if v is None else _f32(v, (self.ny, self.nx)) for v in (h, qx, qy)]
        _check(lib().flood_set_state(self.h, int(member), ptr(a[0]), ptr(a[1]), ptr(a[2]),
                                     stream_handle(stream)), self.h)

    def members(self):
        M = self.M
        out = dict(t=np.zeros(M), steps=np.zeros(M, np.int64), rain_mult=np.zeros(M, np.float32),
                   scale=np.zeros(M, np.float32), weights=np.zeros(M), hmax=np.zeros(M, np.float32))
        _check(lib().flood_get_members(self.h, ptr(out["t"]), ptr(out["steps"]),
                                       ptr(out["rain_mult"]), ptr(out["scale"]),
                                       ptr(out["weights"]), ptr(out["hmax"])), self.h)
        return out

    def set_members(self, rain_mult=None, scale=None, weights=None):
        rm = None if rain_mult is None else _f32(rain_mult)
        sc = None if scale is None else _f32(scale)
        w = None if weights is None else np.ascontiguousarray(weights, np.float64)
        _check(lib().flood_set_members(self.h, ptr(rm), ptr(sc), ptr(w)), self.h)

    def volumes(self):
        M = self.M
        out = dict(storage=np.zeros(M), rain=np.zeros(M), outflow=np.zeros(M), clamp=np.zeros(M))
        _check(lib().flood_volume_report(self.h, ptr(out["storage"]), ptr(out["rain"]),
                                         ptr(out["outflow"]), ptr(out["clamp"])), self.h)
        return out

    def set_launch(self, rows_per_strip=0, members_per_cta=0):
        """Step-kernel launch shape; (0, 0) = automatic."""
        _check(lib().flood_set_launch(self.h, int(rows_per_strip), int(members_per_cta)), self.h)

    def set_engine(self, engine):
        """0: direct loads, 1: TMA-staged tiles, 2: one launch per member per
        step (the plain form, for comparison); identical results."""
        _check(lib().flood_set_engine(self.h, int(engine)), self.h)

    def set_wait_budget(self, cycles):
        """Clock-cycle limit of the TMA step kernel's row waits (< 0: the
        default); a failure-detection hook (flood_set_wait_budget)."""
        _check(lib().flood_set_wait_budget(self.h, int(cycles)), self.h)

    def set_graphs(self, on=True):
        """CUDA-graph replay of runs of 24 steps in advance_to / step
        (flood_set_graphs); identical results."""
        _check(lib().flood_set_graphs(self.h, int(bool(on))), self.h)

    def graph_stats(self):
        """(runs captured, runs replayed) so far (flood_graph_stats)."""
        c = C.c_int64(); r = C.c_int64()
        _check(lib().flood_graph_stats(self.h, C.byref(c), C.byref(r)), self.h)
        return c.value, r.value

    def get_launch(self):
        r = C.c_int(); m = C.c_int()
        _check(lib().flood_get_launch(self.h, C.byref(r), C.byref(m)), self.h)
        return r.value, m.value

    def autotune(self, steps_per_trial=6, stream=None):
        """Pick the fastest step-kernel configuration on the live ensemble
        (which is left unchanged); returns (rows, members_per_cta, engine, ms)."""
        r = C.c_int(); mp = C.c_int(); e = C.c_int(); t = C.c_double()
        _check(lib().flood_autotune(self.h, int(steps_per_trial), C.byref(r), C.byref(mp),
                                    C.byref(e), C.byref(t), stream_handle(stream)), self.h)
        return r.value, mp.value, e.value, t.value

    def profile(self, enable=True):
        """Turn per-launch step-kernel timing on/off; returns (ms, launches)
        accumulated since the previous call."""
        ms = C.c_double(); n = C.c_int64()
        _check(lib().flood_profile(self.h, int(bool(enable)), C.byref(ms), C.byref(n)), self.h)
        return ms.value, n.value

    def adjoint(self, cells, d, sample_dt, ckpt_every=0, grad_n=True, grad_h0=True, stream=None):
        """Gauge-misfit loss per member over the observation window and its
        gradients (flood_adjoint).  d: [n_samples][n_gauges] observed depths
        at t0 + s * sample_dt.  Returns a dict of host arrays."""
        cells = np.ascontiguousarray(cells, dtype=np.int32)
        d = np.ascontiguousarray(d, dtype=np.float64)
        ns, G = d.shape
        spec = LossSpec(ns, G, float(sample_dt), cells.ctypes.data, d.ctypes.data)
        M = self.M
        out = dict(loss=np.zeros(M), grad_rain=np.zeros(M), grad_scale=np.zeros(M),
                   grad_n=np.zeros((self.ny, self.nx), np.float32) if grad_n else None,
                   grad_h0=np.zeros((M, self.ny, self.nx), np.float32) if grad_h0 else None)
        _check(lib().flood_adjoint(self.h, C.byref(spec), int(ckpt_every), ptr(out["grad_n"]),
                                   ptr(out["grad_rain"]), ptr(out["grad_scale"]),
                                   ptr(out["grad_h0"]), ptr(out["loss"]), stream_handle(stream)),
               self.h)
        f = C.c_double(); r = C.c_double()
        _check(lib().flood_adjoint_timing(self.h, C.byref(f), C.byref(r)), self.h)
        out["forward_ms"], out["reverse_ms"] = f.value, r.value
        return out

    def set_land_cover(self, cls, classes):
        """cls: [ny][nx] uint8 class per cell; classes: list of (n, runoff,
        drains, outside) tuples (flood_set_land_cover)."""
        cls = np.ascontiguousarray(cls, dtype=np.uint8)
        tab = (LandClass * len(classes))(*[LandClass(float(n), float(r), int(d), int(o))
                                           for n, r, d, o in classes])
        self._lc_K = len(classes)
        _check(lib().flood_set_land_cover(self.h, cls.ctypes.data, len(classes), tab), self.h)

    def set_land_params(self, n_class=None, drain_rate=None):
        nc = None if n_class is None else np.ascontiguousarray(n_class, np.float32)
        dr = None if drain_rate is None else np.ascontiguousarray(drain_rate, np.float32)
        _check(lib().flood_set_land_params(self.h, None if nc is None else nc.ctypes.data,
                                           None if dr is None else dr.ctypes.data), self.h)

    def land_params(self):
        n = np.zeros((self.M, self._lc_K), np.float32)
        d = np.zeros(self.M, np.float32)
        _check(lib().flood_get_land_params(self.h, n.ctypes.data, d.ctypes.data), self.h)
        return n, d

    def set_inflow(self, r0, r1, series):
        """Inflow hydrograph through the west-edge links of rows [r0, r1):
        discharge per rain block (m^3/s) (flood_set_inflow)."""
        q = np.ascontiguousarray(series, np.float32)
        _check(lib().flood_set_inflow(self.h, int(r0), int(r1), q.ctypes.data if len(q) else None,
                                      len(q)), self.h)

    def inflow_volume(self):
        out = np.zeros(self.M)
        _check(lib().flood_inflow_volume(self.h, out.ctypes.data), self.h)
        return out

    def flow_sample(self, sections, stream=None):
        """Discharge (m^3/s) of every member through every section
        (flood_flow_sample); sections: (axis, fixed, start, end) tuples."""
        tab = (Section * len(sections))(*[Section(*map(int, s)) for s in sections])
        out = np.zeros((self.M, len(sections)), np.float32)
        _check(lib().flood_flow_sample(self.h, len(sections), tab, out.ctypes.data,
                                       stream_handle(stream)), self.h)
        return out

    def drained(self):
        out = np.zeros(self.M)
        _check(lib().flood_drained_volume(self.h, out.ctypes.data), self.h)
        return out

    def adjoint_land_grad(self, classes=True, stream=None):
        """Land-cover gradients of the last adjoint (flood_adjoint_land_grad):
        (dL_i/dn_k as [M][n_classes] FP64 or None, dL_i/d(drainage rate)
        as [M] FP64)."""
        gn = np.zeros((self.M, self._lc_K)) if classes else None
        gd = np.zeros(self.M)
        _check(lib().flood_adjoint_land_grad(self.h, ptr(gn), gd.ctypes.data,
                                             stream_handle(stream)), self.h)
        return gn, gd

    def track_max_depth(self, on=True, stream=None):
        """Running maximum depth of every member (flood_track_max_depth)."""
        _check(lib().flood_track_max_depth(self.h, 1 if on else 0, stream_handle(stream)), self.h)

    def max_depth(self, member, stream=None):
        out = np.zeros((self.ny, self.nx), np.float32)
        _check(lib().flood_get_max_depth(self.h, int(member), out.ctypes.data,
                                         stream_handle(stream)), self.h)
        return out

    def ensemble_products(self, threshold=0.2, levels=(0.1, 0.5, 0.9), stream=None, out=None):
        """Exceedance probability of the maximum depth and its percentile
        maps (flood_ensemble_products); host arrays, or the caller's buffers
        out = (exceed [ny][nx], pct [n_levels][ny][nx]), FP32 numpy arrays or
        torch tensors (device tensors keep the maps on the device)."""
        lv = np.ascontiguousarray(levels, dtype=np.float64)
        if out is None:
            exceed = np.zeros((self.ny, self.nx), np.float32)
            pct = np.zeros((len(lv), self.ny, self.nx), np.float32)
        else:
            exceed, pct = out
        _check(lib().flood_ensemble_products(self.h, float(threshold), len(lv),
                                             lv.ctypes.data if len(lv) else None, ptr(exceed),
                                             ptr(pct) if len(lv) else None,
                                             stream_handle(stream)), self.h)
        return exceed, pct

    def set_roughness_factor(self, f, stream=None):
        """Roughness n = n0 * f[block] over a coarse [cy][cx] factor field
        (flood_set_roughness_factor); f: numpy array or torch tensor."""
        if hasattr(f, "data_ptr"):
            cy, cx = f.shape
            _check(lib().flood_set_roughness_factor(self.h, int(cy), int(cx), C.c_void_p(f.data_ptr()),
                                                    stream_handle(stream)), self.h)
            return
        f = np.ascontiguousarray(f, dtype=np.float32)
        cy, cx = f.shape
        _check(lib().flood_set_roughness_factor(self.h, int(cy), int(cx), f.ctypes.data,
                                                stream_handle(stream)), self.h)

    def roughness_factor(self):
        cy = C.c_int(); cx = C.c_int()
        _check(lib().flood_get_roughness_factor(self.h, C.byref(cy), C.byref(cx), None), self.h)
        f = np.zeros((cy.value, cx.value), np.float32)
        _check(lib().flood_get_roughness_factor(self.h, None, None, f.ctypes.data), self.h)
        return f

    def roughness_factor_grad(self, stream=None):
        """dL/df of the last adjoint (flood_roughness_factor_grad)."""
        cy = C.c_int(); cx = C.c_int()
        _check(lib().flood_get_roughness_factor(self.h, C.byref(cy), C.byref(cx), None), self.h)
        out = np.zeros((cy.value, cx.value))
        _check(lib().flood_roughness_factor_grad(self.h, out.ctypes.data, stream_handle(stream)),
               self.h)
        return out

    def calibration_step(self, eta=1.0, delta=0.2, stream=None):
        """One clipped Polyak step from the last adjoint (flood_calibration_step);
        returns the per-member losses it used."""
        loss = np.zeros(self.M)
        _check(lib().flood_calibration_step(self.h, float(eta), float(delta), loss.ctypes.data,
                                            stream_handle(stream)), self.h)
        return loss

    @property
    def launch_count(self):
        return int(lib().flood_launch_count(self.h))


def _bcheck(rc, handle=None):
    if rc != FLOOD_OK:
        msg = lib().flood_batch_last_error(handle)
        raise FloodError(rc, msg.decode() if msg else "")


class Batch:
    """Uneven batch of independent scenarios (flood_batch_*): each with its
    own grid, bed, roughness, storm and duration, and one or more members
    (each with its own rain multiplier, Manning scale, state and clock)."""

    def __init__(self, zs, ns, params: Params | None = None):
        L = lib()
        self.params = params if params is not None else Params.default()
        self._z = [np.ascontiguousarray(z, np.float32) for z in zs]
        self._n = [np.ascontiguousarray(n, np.float32) for n in ns]
        self.S = len(self._z)
        self.shapes = [z.shape for z in self._z]
        ny = np.array([s[0] for s in self.shapes], np.int32)
        nx = np.array([s[1] for s in self.shapes], np.int32)
        zp = (C.c_void_p * self.S)(*[z.ctypes.data for z in self._z])
        np_ = (C.c_void_p * self.S)(*[n.ctypes.data for n in self._n])
        h = _VP()
        _bcheck(L.flood_batch_create(C.byref(h), self.S, ny.ctypes.data, nx.ctypes.data, zp, np_,
                                     C.byref(self.params)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().flood_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def init(self, hyetographs, rain_mult, scale, t_end, stream=None, members=None):
        """Start every scenario dry at t = 0.  members: per-scenario member
        counts (None: one each); rain_mult and scale then hold one value per
        member, scenario by scenario (flood_batch_init_members)."""
        self._hy = [np.ascontiguousarray(h, np.float32) for h in hyetographs]
        hp = (C.c_void_p * self.S)(*[h.ctypes.data for h in self._hy])
        nb = np.array([len(h) for h in self._hy], np.int32)
        rm = np.ascontiguousarray(rain_mult, np.float32)
        sc = np.ascontiguousarray(scale, np.float32)
        te = np.ascontiguousarray(t_end, np.float64)
        if members is None:
            _bcheck(lib().flood_batch_init(self.h, hp, nb.ctypes.data, rm.ctypes.data,
                                           sc.ctypes.data, te.ctypes.data, stream_handle(stream)),
                    self.h)
            self.members_per = np.ones(self.S, np.int32)
        else:
            mc = np.ascontiguousarray(members, np.int32)
            if rm.size != mc.sum() or sc.size != mc.sum():
                raise ValueError("rain_mult and scale need one value per member")
            _bcheck(lib().flood_batch_init_members(self.h, hp, nb.ctypes.data, mc.ctypes.data,
                                                   rm.ctypes.data, sc.ctypes.data, te.ctypes.data,
                                                   stream_handle(stream)), self.h)
            self.members_per = mc.copy()

    def step(self, t_stop, stream=None):
        _bcheck(lib().flood_batch_step(self.h, float(t_stop), stream_handle(stream)), self.h)

    def set_launch(self, rows_per_strip, warps_per_cta=4):
        _bcheck(lib().flood_batch_set_launch(self.h, int(rows_per_strip), int(warps_per_cta)),
                self.h)

    def set_wait_budget(self, cycles):
        """Clock-cycle limit of the persistent form's grid-barrier waits (< 0:
        the default); a failure-detection hook (flood_batch_set_wait_budget)."""
        _bcheck(lib().flood_batch_set_wait_budget(self.h, int(cycles)), self.h)

    def autotune(self, trial_s=30.0, stream=None):
        """Pick the fastest batched-step configuration on the live batch, which
        is left unchanged (flood_batch_autotune); returns (rows, warps per
        CTA, engine, trial ms)."""
        r = C.c_int(); w = C.c_int(); e = C.c_int(); t = C.c_double()
        _bcheck(lib().flood_batch_autotune(self.h, float(trial_s), C.byref(r), C.byref(w),
                                           C.byref(e), C.byref(t), stream_handle(stream)), self.h)
        return r.value, w.value, e.value, t.value

    def set_engine(self, engine):
        """0: direct loads, 1: TMA-staged rows (graph-replayed launches), 2: the
        TMA-staged march in one persistent launch per step call (identical
        results)."""
        _bcheck(lib().flood_batch_set_engine(self.h, int(engine)), self.h)

    def get_state(self, i, stream=None, member=0):
        """State of member `member` of scenario i (h, qx, qy host arrays)."""
        ny, nx = self.shapes[i]
        h = np.zeros((ny, nx), np.float32); qx = np.zeros_like(h); qy = np.zeros_like(h)
        _bcheck(lib().flood_batch_get_member_state(self.h, int(i), int(member), h.ctypes.data,
                                                   qx.ctypes.data, qy.ctypes.data,
                                                   stream_handle(stream)), self.h)
        return h, qx, qy

    def members(self):
        """Per-member clocks and volumes, scenario by scenario (per scenario
        with one member each)."""
        S = int(np.sum(getattr(self, "members_per", np.ones(self.S))))
        out = dict(t=np.zeros(S), steps=np.zeros(S, np.int64), storage=np.zeros(S),
                   rain=np.zeros(S), outflow=np.zeros(S), clamp=np.zeros(S))
        _bcheck(lib().flood_batch_members(self.h, *(out[k].ctypes.data for k in
                                                     ("t", "steps", "storage", "rain", "outflow",
                                                      "clamp"))), self.h)
        return out

    def set_land_cover(self, i, cls, classes):
        """Land cover of scenario i (flood_batch_set_land_cover): cls [ny][nx]
        uint8; classes: list of (n, runoff, drains, outside) tuples.  Before
        init, for every scenario or none."""
        cls = np.ascontiguousarray(cls, dtype=np.uint8)
        tab = (LandClass * len(classes))(*[LandClass(float(n), float(r), int(d), int(o))
                                           for n, r, d, o in classes])
        _bcheck(lib().flood_batch_set_land_cover(self.h, int(i), cls.ctypes.data, len(classes), tab),
                self.h)

    def set_land_params(self, i, n_class=None, drain_rate=None):
        """Per-member class roughness [members][n_classes] and drainage rates
        [members] of scenario i (flood_batch_set_land_params)."""
        nc = None if n_class is None else np.ascontiguousarray(n_class, np.float32)
        dr = None if drain_rate is None else np.ascontiguousarray(drain_rate, np.float32)
        _bcheck(lib().flood_batch_set_land_params(self.h, int(i), None if nc is None else nc.ctypes.data,
                                                  None if dr is None else dr.ctypes.data), self.h)

    def drained(self):
        """Drained volume per member, scenario by scenario (FP64, m^3)."""
        S = int(np.sum(getattr(self, "members_per", np.ones(self.S))))
        out = np.zeros(S)
        _bcheck(lib().flood_batch_drained_volume(self.h, out.ctypes.data), self.h)
        return out

    @property
    def launch_count(self):
        return int(lib().flood_batch_launch_count(self.h))
