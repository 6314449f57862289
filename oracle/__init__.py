"""FP64 CPU oracle (test infrastructure only).

Plain, slow, obviously correct statement of the ensemble local-inertial flood
model (Eq. 1-6) and its particle filter (Eq. 9-12, systematic resampling,
replacement and perturbation, Section 2.2 / 3.3 / 4.4) of arXiv 2302.08341.
The arithmetic lives in ``oracle.c``; this module compiles it with gcc and
wraps it with ctypes over float64 numpy arrays.

Only the tests, the smoke check and the benchmark's CPU-baseline leg use this
package.  It shares no code with the CUDA library and is never called by it.
The GPU library stores x links as ``qx[r][c]`` = link east of cell (r, c)
(``ny x nx``); the oracle stores the paper's full link arrays including both
edges (``ny x (nx+1)``), so callers compare ``oracle_qx[:, 1:]`` with the
GPU's ``qx`` (and likewise ``qy[1:, :]``).
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, -O2, no FP contraction so the
    result is the same on x86-64 and aarch64)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", "-fopenmp", "-o", _LIB + ".tmp", _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class OrcParams(C.Structure):
    _fields_ = [("ny", C.c_int), ("nx", C.c_int), ("dx", C.c_double), ("g", C.c_double),
                ("alpha", C.c_double), ("dt_cap", C.c_double), ("dt_fixed", C.c_double),
                ("h_eps", C.c_double), ("h_floor", C.c_double), ("rain_block", C.c_double),
                ("edge_slope", C.c_double), ("limiter", C.c_int), ("east_outflow", C.c_int),
                ("south_outflow", C.c_int), ("rc", C.c_void_p), ("drain", C.c_void_p),
                ("inflow", C.c_void_p), ("inflow_blocks", C.c_int), ("inflow_r0", C.c_int),
                ("inflow_r1", C.c_int), ("inflow_q", C.c_double)]


class OrcVolumes(C.Structure):
    _fields_ = [("rain", C.c_double), ("outflow", C.c_double), ("clamp", C.c_double),
                ("drained", C.c_double), ("inflow", C.c_double)]


_D = C.POINTER(C.c_double)
_I32 = C.POINTER(C.c_int32)
_I64 = C.POINTER(C.c_int64)


def load(path: str):
    """Open an oracle shared library and declare its prototypes."""
    L = C.CDLL(path)
    if True:
        L.orc_dt.restype = C.c_double
        L.orc_dt.argtypes = [C.POINTER(OrcParams), C.c_double, C.c_double, C.c_double, _D]
        L.orc_rain_rate.restype = C.c_double
        L.orc_rain_rate.argtypes = [C.POINTER(OrcParams), _D, C.c_int, C.c_double]
        L.orc_link_flux.restype = C.c_double
        L.orc_link_flux.argtypes = [C.POINTER(OrcParams)] + [C.c_double] * 7
        L.orc_step.restype = None
        L.orc_step.argtypes = [C.POINTER(OrcParams), _D, _D, C.c_double, C.c_double, C.c_double,
                               _D, _D, _D, _D, _D, C.POINTER(OrcVolumes)]
        L.orc_hmax.restype = C.c_double
        L.orc_hmax.argtypes = [C.c_int, C.c_int, _D]
        L.orc_storage.restype = C.c_double
        L.orc_storage.argtypes = [C.c_int, C.c_int, C.c_double, _D]
        L.orc_advance.restype = C.c_long
        L.orc_advance.argtypes = [C.POINTER(OrcParams), _D, _D, C.c_double, C.c_double, _D,
                                  C.c_int, _D, _D, _D, _D, C.c_double, C.c_long,
                                  C.POINTER(OrcVolumes), _D, C.c_long]
        L.orc_advance_ensemble.restype = None
        L.orc_advance_ensemble.argtypes = [C.POINTER(OrcParams), C.c_int, _D, _D, _D, _D, _D,
                                           C.c_int, _D, _D, _D, _D, C.c_double, C.c_long,
                                           C.POINTER(OrcVolumes), _I64, C.c_int]
        L.orc_gauge_sample.restype = None
        L.orc_gauge_sample.argtypes = [C.c_int, C.c_int, C.c_int, _I32, _D, _D]
        L.orc_pf_weights.restype = C.c_int
        L.orc_pf_weights.argtypes = [C.c_int, C.c_int, _D, _D, _D, C.c_double, _D, _D, _D]
        L.orc_resample_systematic.restype = None
        L.orc_resample_systematic.argtypes = [C.c_int, _D, C.c_double, _I32]
        L.orc_assign_slots.restype = None
        L.orc_assign_slots.argtypes = [C.c_int, _I32, _I32]
        L.orc_step_adjoint.restype = None
        L.orc_step_adjoint.argtypes = [C.POINTER(OrcParams), _D, _D, C.c_double, C.c_double,
                                       C.c_double, C.c_double, _D, _D, _D, _D, _D, _D, _D, _D, _D,
                                       _D]
        L.orc_loss_and_grad.restype = C.c_double
        L.orc_loss_and_grad.argtypes = [C.POINTER(OrcParams), _D, _D, C.c_double, C.c_double, _D,
                                        C.c_int, _D, C.c_double, C.c_int, C.c_int, _I32, _D, _D,
                                        _D, _D, _D, _D, C.POINTER(C.c_long)]
    return L


def lib():
    global _lib
    if _lib is None:
        _lib = load(build())
    return _lib


def compile_variant(src_text: str, out_path: str) -> str:
    """Compile a modified copy of the oracle source (used by the tests that
    plant mistakes in the oracle to show its pins catch them)."""
    c_path = out_path + ".c"
    with open(c_path, "w") as f:
        f.write(src_text)
    subprocess.run(["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
                    "-fopenmp", "-o", out_path, c_path, "-lm"], check=True)
    return out_path


def source() -> str:
    with open(_SRC) as f:
        return f.read()


def _d(a):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def _i32(a):
    assert a.dtype == np.int32 and a.flags.c_contiguous
    return a.ctypes.data_as(_I32)


@dataclasses.dataclass
class Params:
    """Scheme constants.  Defaults: g = 9.81, Courant k = 0.7 (Eq. 4),
    step cap 1 s, no flow only where the flow depth is zero (h_eps = 0),
    rain blocks of 300 s (Section 3.1), limiter on, free outflow through the
    east edge only."""
    ny: int
    nx: int
    dx: float = 3.0
    g: float = 9.81
    alpha: float = 0.7
    dt_cap: float = 1.0
    dt_fixed: float = 0.0
    h_eps: float = 0.0
    h_floor: float = 1e-6
    rain_block: float = 300.0
    edge_slope: float = 0.005
    limiter: int = 1
    east_outflow: int = 1
    south_outflow: int = 0
    # land cover (Section 4.1): per-cell runoff coefficient and drainage rate
    # (m/s), float64 [ny, nx] arrays held here, or None
    rc: np.ndarray | None = None
    drain: np.ndarray | None = None
    # inflow hydrograph: discharge per rain block (m^3/s, float64 array held
    # here, or None) through the west edge links of rows [inflow_r0, inflow_r1)
    inflow: np.ndarray | None = None
    inflow_r0: int = 0
    inflow_r1: int = 0
    inflow_q: float = 0.0

    def c(self) -> OrcParams:
        vals = []
        for f, _ in OrcParams._fields_:
            v = getattr(self, f, None)
            if f in ("rc", "drain"):
                if v is not None:
                    assert v.dtype == np.float64 and v.flags.c_contiguous and v.shape == (self.ny, self.nx)
                    v = v.ctypes.data
            elif f == "inflow":
                if v is not None:
                    assert v.dtype == np.float64 and v.flags.c_contiguous and v.ndim == 1
                    v = v.ctypes.data
            elif f == "inflow_blocks":
                v = 0 if self.inflow is None else len(self.inflow)
            vals.append(v)
        return OrcParams(*vals)


def dt(p: Params, hmax: float, t: float, t_end: float = -1.0):
    """Eq. 4 time step with the event clipping; returns (dt, t_next)."""
    tn = C.c_double()
    d = lib().orc_dt(C.byref(p.c()), hmax, t, t_end, C.byref(tn))
    return d, tn.value


def link_flux(p: Params, h1, z1, h2, z2, q, nl, dt_):
    return lib().orc_link_flux(C.byref(p.c()), h1, z1, h2, z2, q, nl, dt_)


@dataclasses.dataclass
class Member:
    """State of one member in the oracle's link layout (float64)."""
    h: np.ndarray    # [ny, nx]
    qx: np.ndarray   # [ny, nx+1]
    qy: np.ndarray   # [ny+1, nx]
    t: float = 0.0
    rain: float = 0.0
    outflow: float = 0.0
    clamp: float = 0.0
    drained: float = 0.0
    inflow: float = 0.0
    steps: int = 0

    @staticmethod
    def dry(ny, nx, h0=None):
        h = np.zeros((ny, nx)) if h0 is None else np.array(h0, dtype=np.float64)
        return Member(h=h, qx=np.zeros((ny, nx + 1)), qy=np.zeros((ny + 1, nx)))

    def copy(self):
        return dataclasses.replace(self, h=self.h.copy(), qx=self.qx.copy(), qy=self.qy.copy())


def step(p: Params, z, n, scale, rain, dt_, m: Member):
    """One iteration (Eq. 2-3 on every link, Eq. 5 and Eq. 1 on every cell)."""
    z = np.ascontiguousarray(z, np.float64); n = np.ascontiguousarray(n, np.float64)
    qxn = np.empty_like(m.qx); qyn = np.empty_like(m.qy)
    v = OrcVolumes(m.rain, m.outflow, m.clamp, m.drained, m.inflow)
    lib().orc_step(C.byref(p.c()), _d(z), _d(n), scale, rain, dt_, _d(m.h), _d(m.qx), _d(m.qy),
                   _d(qxn), _d(qyn), C.byref(v))
    m.rain, m.outflow, m.clamp, m.drained, m.inflow = v.rain, v.outflow, v.clamp, v.drained, v.inflow
    m.steps += 1


def advance(p: Params, z, n, scale, rain_mult, hyeto, m: Member, t_end=-1.0, max_steps=-1,
            log_dt=False):
    """Evolve one member (Eq. 6) to t_end (or max_steps steps).  Returns the
    list of step lengths when log_dt is set, else the number of steps."""
    z = np.ascontiguousarray(z, np.float64); n = np.ascontiguousarray(n, np.float64)
    hy = np.ascontiguousarray(hyeto, np.float64)
    t = C.c_double(m.t)
    v = OrcVolumes(m.rain, m.outflow, m.clamp, m.drained, m.inflow)
    cap = (max_steps if max_steps > 0 else 2_000_000) if log_dt else 0
    log = np.zeros(max(cap, 1))
    k = lib().orc_advance(C.byref(p.c()), _d(z), _d(n), float(scale), float(rain_mult),
                          _d(hy), len(hy), _d(m.h), _d(m.qx), _d(m.qy), C.byref(t), float(t_end),
                          int(max_steps), C.byref(v), _d(log) if log_dt else None, cap)
    m.t = t.value
    m.rain, m.outflow, m.clamp, m.drained, m.inflow = v.rain, v.outflow, v.clamp, v.drained, v.inflow
    m.steps += k
    return log[:k].copy() if log_dt else k


class Ensemble:
    """M members in member-major float64 arrays, with prior weights."""

    def __init__(self, p: Params, M: int, h0=None):
        self.p, self.M = p, M
        ny, nx = p.ny, p.nx
        self.h = np.zeros((M, ny, nx)) if h0 is None else np.array(
            np.broadcast_to(h0, (M, ny, nx)), dtype=np.float64, order="C")
        self.qx = np.zeros((M, ny, nx + 1))
        self.qy = np.zeros((M, ny + 1, nx))
        self.t = np.zeros(M)
        self.vol = (OrcVolumes * M)()
        self.steps = np.zeros(M, dtype=np.int64)
        self.w = np.full(M, 1.0 / M)

    def advance(self, z, n, scale, rain_mult, hyeto, t_end=-1.0, max_steps=-1, nthreads=1):
        z = np.ascontiguousarray(z, np.float64); n = np.ascontiguousarray(n, np.float64)
        sc = np.ascontiguousarray(scale, np.float64); rm = np.ascontiguousarray(rain_mult, np.float64)
        hy = np.ascontiguousarray(hyeto, np.float64)
        st = np.zeros(self.M, dtype=np.int64)
        lib().orc_advance_ensemble(C.byref(self.p.c()), self.M, _d(z), _d(n), _d(sc), _d(rm),
                                   _d(hy), len(hy), _d(self.h), _d(self.qx), _d(self.qy),
                                   _d(self.t), float(t_end), int(max_steps), self.vol,
                                   st.ctypes.data_as(_I64), int(nthreads))
        self.steps += st
        return st

    def volumes(self):
        return np.array([[v.rain, v.outflow, v.clamp, v.drained, v.inflow] for v in self.vol])

    def storage(self):
        dx = self.p.dx
        return np.array([storage(self.h[m], dx) for m in range(self.M)])


def hmax(h):
    h = np.ascontiguousarray(h, np.float64)
    return lib().orc_hmax(h.shape[0], h.shape[1], _d(h))


def storage(h, dx):
    h = np.ascontiguousarray(h, np.float64)
    return lib().orc_storage(h.shape[0], h.shape[1], dx, _d(h))


def gauge_sample(h, cells):
    """DA step (I): y[m][g] = depth of member m at gauge cell g."""
    h = np.ascontiguousarray(h, np.float64)
    M = h.shape[0]
    ncell = h.shape[1] * h.shape[2]
    cells = np.ascontiguousarray(cells, np.int32)
    y = np.zeros((M, len(cells)))
    lib().orc_gauge_sample(M, ncell, len(cells), _i32(cells), _d(h), _d(y))
    return y


def pf_weights(y, d, sigma, w_prior, sigma_rel=0.0):
    """Eq. 9-12: posterior weights and N_eff."""
    y = np.ascontiguousarray(y, np.float64)
    M, G = y.shape
    d = np.ascontiguousarray(d, np.float64)
    sg = np.ascontiguousarray(np.broadcast_to(sigma, (G,)), np.float64)
    wp = np.ascontiguousarray(w_prior, np.float64)
    wo = np.zeros(M)
    ne = C.c_double()
    rc = lib().orc_pf_weights(M, G, _d(y), _d(d), _d(sg), float(sigma_rel), _d(wp), _d(wo),
                              C.byref(ne))
    if rc != 0:
        raise ValueError("all posterior weights are zero")
    return wo, ne.value


def resample_systematic(w, u):
    w = np.ascontiguousarray(w, np.float64)
    idx = np.zeros(len(w), dtype=np.int32)
    lib().orc_resample_systematic(len(w), _d(w), float(u), _i32(idx))
    return idx


def assign_slots(idx):
    idx = np.ascontiguousarray(idx, np.int32)
    src = np.zeros(len(idx), dtype=np.int32)
    lib().orc_assign_slots(len(idx), _i32(idx), _i32(src))
    return src


def pf_assimilate(ens: Ensemble, y, d, sigma, rain_mult, scale, u, beta, n_thr_frac=0.8,
                  force=False, sigma_rel=0.0):
    """DA steps (I)-(V) of Section 3.3 on an oracle ensemble: weights
    (Eq. 9-12); if N_eff < n_thr_frac * M (or forced) systematic resampling,
    slot replacement, rain multiplier x beta and weights reset to 1/M.
    Returns (w_post, neff, idx or None, new rain_mult, new scale)."""
    w, neff = pf_weights(y, d, sigma, ens.w, sigma_rel)
    rain_mult = np.array(rain_mult, dtype=np.float64)
    scale = np.array(scale, dtype=np.float64)
    if not (force or neff < n_thr_frac * ens.M):
        ens.w = w
        return w, neff, None, rain_mult, scale
    idx = resample_systematic(w, u)
    src = assign_slots(idx)
    ens.h = ens.h[src].copy(); ens.qx = ens.qx[src].copy(); ens.qy = ens.qy[src].copy()
    ens.t = ens.t[src].copy()
    rain_mult = rain_mult[src] * np.asarray(beta, np.float64)
    scale = scale[src]
    ens.w = np.full(ens.M, 1.0 / ens.M)
    return w, neff, idx, rain_mult, scale


def step_adjoint(p: Params, z, n, scale, rate, rain_mult, dt_, m: Member, lh, lqx, lqy):
    """Reverse of one iteration at state m (the step's input).  lh, lqx, lqy
    (oracle layout) are the loss's sensitivities to the step's outputs; they
    are overwritten with those to its inputs.  Returns (grad_n, grad_rain,
    grad_scale) contributions of this step."""
    z = np.ascontiguousarray(z, np.float64); n = np.ascontiguousarray(n, np.float64)
    gn = np.zeros(z.shape)
    gr = C.c_double(0.0); gs = C.c_double(0.0)
    lib().orc_step_adjoint(C.byref(p.c()), _d(z), _d(n), float(scale), float(rate),
                           float(rain_mult), float(dt_), _d(m.h), _d(m.qx), _d(m.qy), _d(lh),
                           _d(lqx), _d(lqy), _d(gn), C.byref(gr), C.byref(gs), None)
    return gn, gr.value, gs.value


def loss_and_grad(p: Params, z, n, scale, rain_mult, hyeto, h0, sample_dt, d, cells):
    """Gauge-misfit loss sum_s sum_g (h(t_s)[cell_g] - d[s][g])^2 at
    t_s = s * sample_dt and its gradients with respect to the base Manning
    field, the initial depth, the rain multiplier and the Manning scale,
    and (land cover) grad_drain = dL/d(kappa) for the drainage field p.drain
    scaled by kappa, at kappa = 1."""
    z = np.ascontiguousarray(z, np.float64); n = np.ascontiguousarray(n, np.float64)
    hy = np.ascontiguousarray(hyeto, np.float64)
    h0 = np.ascontiguousarray(np.broadcast_to(h0, z.shape), np.float64)
    d = np.ascontiguousarray(d, np.float64)
    cells = np.ascontiguousarray(cells, np.int32)
    ns, G = d.shape
    gn = np.zeros(z.shape); gh = np.zeros(z.shape)
    gr = C.c_double(); gs = C.c_double(); gk = C.c_double(); nst = C.c_long()
    loss = lib().orc_loss_and_grad(C.byref(p.c()), _d(z), _d(n), float(scale), float(rain_mult),
                                   _d(hy), len(hy), _d(h0), float(sample_dt), ns, G, _i32(cells),
                                   _d(d), _d(gn), _d(gh), C.byref(gr), C.byref(gs),
                                   C.byref(gk), C.byref(nst))
    return dict(loss=loss, grad_n=gn, grad_h0=gh, grad_rain=gr.value, grad_scale=gs.value,
                grad_drain=gk.value, steps=nst.value)


def section_flow(m: Member, dx: float, axis: int, fixed: int, start: int, end: int) -> float:
    """Discharge (m^3/s) through a straight section of links, positive toward
    increasing index: axis 0 sums the links east of cells (r, fixed) for r in
    [start, end); axis 1 the links south of cells (fixed, c) for c in
    [start, end).  Q = sum of q * dx (the link discharges of Eq. 5)."""
    if axis == 0:
        q = m.qx[start:end, fixed + 1]      # oracle link c lies between cells c-1 and c
    else:
        q = m.qy[fixed + 1, start:end]
    acc = 0.0
    for v in q:
        acc += float(v) * dx
    return acc
