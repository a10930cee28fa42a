"""Test infrastructure, not product code: ctypes wrapper of the FP64 CPU oracle fitter.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this module. The oracle (kf_oracle.cpp) is a plain, slow FP64 Kalman-filter fit
(RKN propagation with Jacobian transport, Highland scattering and Bethe mean energy loss,
Joseph-form gain-matrix update with chi2, backward Rauch-Tung-Striebel smoother) written
from the methods the paper cites (paper Sec. 2, second paragraph). It shares no code with
the CUDA path.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None

MUON_MASS = 0.1056583755
# Silicon (PDG): Z/A, mean excitation energy (eV), density (g/cm3), plasma energy (eV).
SI = (0.49848, 173.0, 2.329, 31.05)

STATUS = {
    "MAX_STEPS": 1 << 0, "SURFACE_MISSED": 1 << 1, "PARTICLE_STOPPED": 1 << 2,
    "UPDATE_NOT_SPD": 1 << 3, "SMOOTHER_NOT_SPD": 1 << 4, "TOO_FEW_HITS": 1 << 5,
    "OUT_OF_FIELD": 1 << 6, "BAD_INPUT": 1 << 7, "STEP_UNDERFLOW": 1 << 8, "NON_FINITE": 1 << 9,
}


def build(force: bool = False) -> str:
    """Compiles liboracle.so: -O2, no fast-math, no FMA contraction (plain IEEE FP64)."""
    src = os.path.join(_HERE, "kf_oracle.cpp")
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math",
                               "-shared", "-fPIC", "-pthread", "-o", _SO, src])
    return _SO


class OField(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("B", ctypes.c_double * 3), ("nr", ctypes.c_int),
                ("nz", ctypes.c_int), ("r0", ctypes.c_double), ("dr", ctypes.c_double),
                ("z0", ctypes.c_double), ("dz", ctypes.c_double),
                ("Br", ctypes.c_void_p), ("Bz", ctypes.c_void_p)]


class OOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("h_max", ctypes.c_double), ("h_min", ctypes.c_double),
                ("surf_tol", ctypes.c_double), ("mass", ctypes.c_double),
                ("max_steps", ctypes.c_uint32), ("ZA", ctypes.c_double), ("I_eV", ctypes.c_double),
                ("rho", ctypes.c_double), ("hwp_eV", ctypes.c_double), ("mlp_bf16", ctypes.c_void_p),
                ("smoother", ctypes.c_int), ("inflation", ctypes.c_double)]


@dataclass
class Options:
    tol: float = 1e-4        # RKN local error tolerance, mm
    h_max: float = 1000.0    # mm
    h_min: float = 1e-4      # mm
    surf_tol: float = 1e-2   # mm
    mass: float = MUON_MASS  # GeV
    max_steps: int = 10000   # step attempts per surface
    material: tuple = SI
    mlp: object = None       # 5057 BF16 weights (uint16) of the step proposer, or None
    smoother: int = 0        # 0: RTS; 1: two-filter (backward filter + weighted mean with the seed)
    inflation: float = 1e3   # two-filter: factor on the backward filter's starting covariance

    def _c(self) -> OOpts:
        o = OOpts()
        o.tol, o.h_max, o.h_min, o.surf_tol, o.mass = self.tol, self.h_max, self.h_min, \
            self.surf_tol, self.mass
        o.max_steps = self.max_steps
        o.ZA, o.I_eV, o.rho, o.hwp_eV = self.material
        o.smoother, o.inflation = int(self.smoother), float(self.inflation)
        if self.mlp is not None:
            w = np.ascontiguousarray(self.mlp, dtype=np.uint16)
            o._keep = w
            o.mlp_bf16 = w.ctypes.data
        return o


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        vp, d, u32 = ctypes.c_void_p, ctypes.c_double, ctypes.c_uint32
        L.orc_fit.restype = ctypes.c_int
        L.orc_fit.argtypes = [vp, u32, ctypes.POINTER(OField), ctypes.POINTER(OOpts), u32, ctypes.c_uint64,
                              vp, vp, vp,
                              vp, vp, vp, vp, vp, vp, vp, vp, vp, ctypes.c_int]
        L.orc_fit_all_states.restype = ctypes.c_int
        L.orc_fit_all_states.argtypes = [vp, u32, ctypes.POINTER(OField), ctypes.POINTER(OOpts), u32, ctypes.c_uint64,
                                         vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, ctypes.c_int]
        L.orc_record_steps.restype = ctypes.c_uint64
        L.orc_record_steps.argtypes = [vp, u32, ctypes.POINTER(OField), ctypes.POINTER(OOpts), u32, ctypes.c_uint64,
                                       vp, vp, vp, vp, vp, vp, ctypes.c_uint64]
        L.orc_field_at.argtypes = [ctypes.POINTER(OField), vp, u32, vp, vp]
        L.orc_rkn_fixed.argtypes = [ctypes.POINTER(OField), vp, vp, d, d, u32, vp, vp, vp]
        L.orc_rkn_step.argtypes = [ctypes.POINTER(OField), vp, vp, d, d, vp, vp, vp]
        L.orc_transport.restype = u32
        L.orc_transport.argtypes = [vp, u32, u32, ctypes.POINTER(OField), ctypes.POINTER(OOpts), vp, vp,
                                    vp, vp]
        L.orc_material.restype = u32
        L.orc_material.argtypes = [vp, ctypes.POINTER(OOpts), vp, vp, vp, vp]
        L.orc_linear_chain.restype = u32
        L.orc_linear_chain.argtypes = [ctypes.c_int, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
        L.orc_linear_chain_two_filter.restype = u32
        L.orc_linear_chain_two_filter.argtypes = [ctypes.c_int, vp, vp, vp, vp, vp, vp, d, vp, vp]
        L.orc_fit_states.restype = u32
        L.orc_fit_states.argtypes = [vp, u32, ctypes.POINTER(OField), ctypes.POINTER(OOpts), u32, vp, vp,
                                     vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
        L.orc_mlp_forward.argtypes = [vp, vp, u32, vp]
        L.orc_propose_start.argtypes = [vp, u32, ctypes.POINTER(OField), ctypes.POINTER(OOpts), u32,
                                        ctypes.c_uint64, vp, vp, vp, vp]
        L.orc_estimate_seeds.argtypes = [vp, u32, ctypes.POINTER(OField), u32, ctypes.c_uint64, vp, vp, vp,
                                         ctypes.c_int, vp, vp, vp]
        L.orc_find_tracks.argtypes = [vp, u32, ctypes.POINTER(OField), ctypes.POINTER(OOpts), vp, u32, vp, u32,
                                      vp, vp, u32, vp, vp, vp, d, u32, u32, u32, vp, vp, vp, vp, vp, ctypes.c_int]
        L.orc_helix_seed.restype = u32
        L.orc_helix_seed.argtypes = [vp, vp, vp, d, vp]
        L.orc_update.restype = u32
        L.orc_update.argtypes = [vp, vp, vp, vp, vp]
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def make_field(kind=0, B=(0.0, 0.0, 2.0), nr=0, nz=0, r0=0.0, dr=1.0, z0=0.0, dz=1.0, Br=None,
               Bz=None):
    """Field description; ``Br``/``Bz`` are float32 [nz, nr] arrays (kept referenced)."""
    f = OField()
    f.kind = kind
    for i in range(3):
        f.B[i] = float(B[i])
    f.nr, f.nz, f.r0, f.dr, f.z0, f.dz = nr, nz, r0, dr, z0, dz
    keep = []
    if Br is not None:
        Br = np.ascontiguousarray(Br, dtype=np.float32)
        Bz = np.ascontiguousarray(Bz, dtype=np.float32)
        keep = [Br, Bz]
        f.Br, f.Bz = _p(Br), _p(Bz)
    f._keep = keep
    return f


def field_from(fld) -> OField:
    """Converts a ``synth.Field``-like object (kind, B, nr, ..., Br, Bz) to the oracle's struct."""
    return make_field(fld.kind, fld.B, fld.nr, fld.nz, fld.r0, fld.dr, fld.z0, fld.dz, fld.Br, fld.Bz)


def surfaces14(table: np.ndarray) -> np.ndarray:
    """[n, 14] = u, v, n, c, thickness, X0 from a [n, >=14] table."""
    return np.ascontiguousarray(table[:, :14], dtype=np.float64)


@dataclass
class FitResult:
    par: np.ndarray
    cov: np.ndarray
    chi2: np.ndarray
    ndf: np.ndarray
    status: np.ndarray
    steps: np.ndarray
    cov_filt0: np.ndarray
    states_par: np.ndarray | None = None       # [n_meas, 5] smoothed parameters of every entry
    states_cov: np.ndarray | None = None       # [n_meas, 15] smoothed covariances (packed)
    states_cov_filt: np.ndarray | None = None  # [n_meas, 15] filtered covariances (packed)


def fit(surfaces: np.ndarray, fld: OField, opts: Options, offsets, meas, sid, seed_par, seed_cov,
        n_threads: int = 1, states: bool = False) -> FitResult:
    """Fits every track. ``meas`` [m, 5], ``seed_par`` [n, 5], ``seed_cov`` [n, 15] (packed).
    With ``states`` the result also holds every entry's smoothed state and filtered covariance
    (NaN for tracks with a fatal status)."""
    L = lib()
    s = surfaces14(surfaces)
    offsets = np.ascontiguousarray(offsets, dtype=np.uint32)
    n = offsets.shape[0] - 1
    meas = _f64(meas)
    sid = np.ascontiguousarray(sid, dtype=np.uint32)
    seed_par, seed_cov = _f64(seed_par), _f64(seed_cov)
    par, cov = np.zeros((n, 5)), np.zeros((n, 15))
    chi2, ndf = np.zeros(n), np.zeros(n, np.int32)
    status, steps = np.zeros(n, np.uint32), np.zeros((n, 2), np.uint32)
    cf0 = np.zeros((n, 15))
    o = opts._c()
    if not states:
        L.orc_fit(_p(s), s.shape[0], ctypes.byref(fld), ctypes.byref(o), n, meas.shape[0], _p(offsets), _p(meas),
                  _p(sid), _p(seed_par), _p(seed_cov), _p(par), _p(cov), _p(chi2), _p(ndf), _p(status),
                  _p(steps), _p(cf0), int(n_threads))
        return FitResult(par, cov, chi2, ndf, status, steps, cf0)
    m = meas.shape[0]
    sp, sc, scf = np.zeros((m, 5)), np.zeros((m, 15)), np.zeros((m, 15))
    L.orc_fit_all_states(_p(s), s.shape[0], ctypes.byref(fld), ctypes.byref(o), n, m, _p(offsets), _p(meas), _p(sid),
                     _p(seed_par), _p(seed_cov), _p(par), _p(cov), _p(chi2), _p(ndf), _p(status), _p(steps), _p(cf0),
                     _p(sp), _p(sc), _p(scf), int(n_threads))
    return FitResult(par, cov, chi2, ndf, status, steps, cf0, sp, sc, scf)


def fit_tracks(workload, opts: Options | None = None, n_threads: int = 1, tracks=None) -> FitResult:
    """Fits a ``synth.Workload`` (or ``tracks`` of it)."""
    t = tracks if tracks is not None else workload.tracks
    o = opts or Options(mass=workload.mass)
    return fit(workload.geometry.table, field_from(workload.field), o, t.offsets, t.meas, t.sid,
               t.seed_par, t.seed_cov, n_threads)


def record_steps(surfaces: np.ndarray, fld: OField, opts: Options, offsets, meas, sid, seed_par, seed_cov,
                 capacity: int = 2_000_000) -> np.ndarray:
    """Training records [n, 13] of the step proposer (12 network inputs, label) from the
    oracle's plain adaptive fit: every accepted step that the step-size control limited."""
    s = surfaces14(surfaces)
    offsets = np.ascontiguousarray(offsets, dtype=np.uint32)
    meas, seed_par, seed_cov = _f64(meas), _f64(seed_par), _f64(seed_cov)
    sid = np.ascontiguousarray(sid, dtype=np.uint32)
    rec = np.zeros((capacity, 13), np.float32)
    o = opts._c()
    n = lib().orc_record_steps(_p(s), s.shape[0], ctypes.byref(fld), ctypes.byref(o), offsets.shape[0] - 1,
                               meas.shape[0], _p(offsets), _p(meas), _p(sid), _p(seed_par), _p(seed_cov), _p(rec),
                               capacity)
    return rec[:min(int(n), capacity)].copy()


def field_at(fld: OField, x: np.ndarray):
    x = _f64(x).reshape(-1, 3)
    B = np.zeros_like(x)
    oof = np.zeros(x.shape[0], np.uint8)
    lib().orc_field_at(ctypes.byref(fld), _p(x), x.shape[0], _p(B), _p(oof))
    return B, oof


def rkn_fixed(fld: OField, r, T, lam, h, n_steps):
    r, T = _f64(r), _f64(T)
    ro, To, D = np.zeros(3), np.zeros(3), np.zeros((7, 7))
    lib().orc_rkn_fixed(ctypes.byref(fld), _p(r), _p(T), lam, h, n_steps, _p(ro), _p(To), _p(D))
    return ro, To, D


def rkn_step(fld: OField, r, T, lam, h):
    r, T = _f64(r), _f64(T)
    ro, To, e = np.zeros(3), np.zeros(3), np.zeros(1)
    lib().orc_rkn_step(ctypes.byref(fld), _p(r), _p(T), lam, h, _p(ro), _p(To), _p(e))
    return ro, To, float(e[0])


def transport(surfaces, a, b, fld: OField, opts: Options, par):
    s = surfaces14(surfaces)
    par = _f64(par)
    out, J = np.zeros(5), np.zeros((5, 5))
    att = np.zeros(1, np.uint32)
    o = opts._c()
    st = lib().orc_transport(_p(s), a, b, ctypes.byref(fld), ctypes.byref(o), _p(par), _p(out), _p(J),
                             _p(att))
    return out, J, int(st), int(att[0])


def material(surface_row, opts: Options, par):
    s = surfaces14(np.atleast_2d(surface_row))
    par = _f64(par)
    th0, qop, dedx = np.zeros(1), np.zeros(1), np.zeros(1)
    o = opts._c()
    st = lib().orc_material(_p(s), ctypes.byref(o), _p(par), _p(th0), _p(qop), _p(dedx))
    return float(th0[0]), float(qop[0]), float(dedx[0]), int(st)


def linear_chain(J, Q, p0, C0, m, V):
    """Oracle update + RTS on a linear-Gaussian chain (see kf_oracle.cpp)."""
    N = m.shape[0]
    J, Q, p0, C0, m, V = map(_f64, (J, Q, p0, C0, m, V))
    ps, Cs, chi2 = np.zeros((N, 5)), np.zeros((N, 5, 5)), np.zeros(1)
    pf, Cf = np.zeros((N, 5)), np.zeros((N, 5, 5))
    st = lib().orc_linear_chain(N, _p(J), _p(Q), _p(p0), _p(C0), _p(m), _p(V), _p(ps), _p(Cs),
                                _p(chi2), _p(pf), _p(Cf))
    return ps, Cs, float(chi2[0]), int(st), pf, Cf


def linear_chain_two_filter(J, Q, p0, C0, m, V, inflation):
    """Two-filter smoother of the linear chain: the smoothed state at step 0 and its status."""
    N = m.shape[0]
    J, Q, p0, C0, m, V = (_f64(x) for x in (J, Q, p0, C0, m, V))
    ps, Cs = np.zeros(5), np.zeros((5, 5))
    st = lib().orc_linear_chain_two_filter(N, _p(J), _p(Q), _p(p0), _p(C0), _p(m), _p(V), float(inflation), _p(ps),
                                           _p(Cs))
    return ps, Cs, st


def fit_states(surfaces, fld: OField, opts: Options, meas, sid, seed_par, seed_cov):
    """One track's per-measurement predicted / filtered / smoothed states and Jacobians."""
    s = surfaces14(surfaces)
    meas, seed_par, seed_cov = _f64(meas), _f64(seed_par), _f64(seed_cov)
    sid = np.ascontiguousarray(sid, dtype=np.uint32)
    N = meas.shape[0]
    out = {k: np.zeros((N, 5)) for k in ("pp", "pf", "ps")}
    out.update({k: np.zeros((N, 5, 5)) for k in ("Cp", "Cf", "Cs", "J")})
    chi2 = np.zeros(1)
    o = opts._c()
    st = lib().orc_fit_states(_p(s), s.shape[0], ctypes.byref(fld), ctypes.byref(o), N, _p(meas),
                              _p(sid), _p(seed_par), _p(seed_cov), _p(out["pp"]), _p(out["Cp"]),
                              _p(out["pf"]), _p(out["Cf"]), _p(out["J"]), _p(out["ps"]),
                              _p(out["Cs"]), _p(chi2))
    out["chi2"] = float(chi2[0])
    out["status"] = int(st)
    return out


def mlp_forward(w_bf16, x):
    """Raw outputs of the step-proposer network (FP32 arithmetic, BF16 weights) for x [n, 12]."""
    w = np.ascontiguousarray(w_bf16, dtype=np.uint16)
    x = np.ascontiguousarray(x, dtype=np.float32).reshape(-1, 12)
    out = np.zeros(x.shape[0], np.float32)
    lib().orc_mlp_forward(_p(w), _p(x), x.shape[0], _p(out))
    return out


def propose_start(surfaces: np.ndarray, fld: OField, opts: Options, offsets, sid, seed_par, n_meas: int):
    """Learned mode: every track's proposed starting step-size control (mm), from the network of
    ``opts.mlp`` on the seed state at its first surface toward its second."""
    s = surfaces14(surfaces)
    offsets = np.ascontiguousarray(offsets, dtype=np.uint32)
    n = offsets.shape[0] - 1
    sid = np.ascontiguousarray(sid, dtype=np.uint32)
    seed_par = _f64(seed_par)
    h0 = np.zeros(n)
    o = opts._c()
    lib().orc_propose_start(_p(s), s.shape[0], ctypes.byref(fld), ctypes.byref(o), n, int(n_meas), _p(offsets),
                            _p(sid), _p(seed_par), _p(h0))
    return h0


def estimate_seeds(surfaces: np.ndarray, fld: OField, offsets, meas, sid, first_three: bool = False):
    """Seed parameters [n, 5], packed covariances [n, 15] and status [n] of every track from the
    helix through three of its measurements: the first, middle and last, or the first three
    (status 1: fewer than 3, 2: no curvature, q/p = 0, 4: bad offsets or surface ids)."""
    s = surfaces14(surfaces)
    offsets = np.ascontiguousarray(offsets, dtype=np.uint32)
    n = offsets.shape[0] - 1
    meas = _f64(meas)
    sid = np.ascontiguousarray(sid, dtype=np.uint32)
    par, cov, st = np.zeros((n, 5)), np.zeros((n, 15)), np.zeros(n, dtype=np.uint32)
    lib().orc_estimate_seeds(_p(s), s.shape[0], ctypes.byref(fld), n, int(sid.shape[0]), _p(offsets), _p(meas),
                             _p(sid), int(bool(first_three)), _p(par), _p(cov), _p(st))
    return par, cov, st


def find_tracks(surfaces: np.ndarray, fld: OField, opts: Options, layers, rings, meas_off, meas, seed_sid, seed_par,
                seed_cov, chi2_max: float = 15.0, beam: int = 3, max_holes: int = 2, max_entries: int = 24,
                n_threads: int = 8):
    """Combinatorial Kalman filter track finding (see kf_oracle.cpp): for every seed the best
    candidate's entries (surface ids, bit 31 for holes; measurement indices, -1 for holes)."""
    s = surfaces14(surfaces)
    layers, rings = _f64(layers), _f64(rings)
    meas_off = np.ascontiguousarray(meas_off, dtype=np.uint32)
    meas = _f64(meas)
    seed_sid = np.ascontiguousarray(seed_sid, dtype=np.uint32)
    seed_par, seed_cov = _f64(seed_par), _f64(seed_cov)
    n = seed_sid.shape[0]
    ne, nm, c2 = np.zeros(n, np.uint32), np.zeros(n, np.uint32), np.zeros(n)
    es, em = np.zeros((n, max_entries), np.uint32), np.zeros((n, max_entries), np.int32)
    o = opts._c()
    lib().orc_find_tracks(_p(s), s.shape[0], ctypes.byref(fld), ctypes.byref(o), _p(layers), layers.shape[0],
                          _p(rings), meas.shape[0], _p(meas_off), _p(meas), n, _p(seed_sid), _p(seed_par),
                          _p(seed_cov), float(chi2_max), int(beam), int(max_holes), int(max_entries), _p(ne), _p(nm),
                          _p(c2), _p(es), _p(em), int(n_threads))
    return {"n_entries": ne, "n_meas": nm, "chi2": c2, "sid": es, "meas": em}


def helix_seed(r1, r2, r3, bz: float):
    """(phi, theta, q/p) at r1 of the helix through three points in an axial field B_z, and the
    status (2: no curvature)."""
    out = np.zeros(3)
    st = lib().orc_helix_seed(_p(_f64(r1)), _p(_f64(r2)), _p(_f64(r3)), float(bz), _p(out))
    return out, int(st)


def update(m, V, p, C):
    m, V, p, C = _f64(m), _f64(V), _f64(p).copy(), _f64(C).copy()
    chi2 = np.zeros(1)
    st = lib().orc_update(_p(m), _p(V), _p(p), _p(C), _p(chi2))
    return p, C, float(chi2[0]), int(st)


def unpack(cov15: np.ndarray) -> np.ndarray:
    """[..., 15] packed upper triangle -> [..., 5, 5] symmetric."""
    iu = np.triu_indices(5)
    out = np.zeros(cov15.shape[:-1] + (5, 5))
    out[..., iu[0], iu[1]] = cov15
    out[..., iu[1], iu[0]] = cov15
    return out
