"""Seeded synthetic inputs: detector geometries, the solenoid field map and simulated tracks.

This module serves both the CUDA fitter and the CPU oracle. It holds none of the fitter's
arithmetic (no Runge-Kutta-Nystrom stepping, Jacobian, Kalman update or smoother): truth
trajectories are exact helix segments and the simulated world scatters and loses energy as
the fit assumes (paper Sec. 3: ODD-like barrel + endcaps, 2 T along z, muon hypothesis).

The workload recipes below are synthetic stand-ins for the paper's Geant4 ttbar samples in
the Open Data Detector, which are not available here:

* ``telescope``          9 planes normal to x at x = 0..400 mm, 0.3 mm Si, B = 2 T along z,
                         muons p ~ U(1, 10) GeV, azimuth and dip ~ U(+-0.1) rad about x.
* ``barrel_endcap``      10 barrel layers r = 32..1000 mm (log-spaced) of 70x30 mm modules,
                         7 disks per side at |z| = 600..3000 mm; pions, pT log-uniform
                         0.5-100 GeV, eta ~ U(+-3), vertex z ~ N(0, 50 mm), 6-18 hits.
* ``solenoid_map``       finite solenoid (R = 1.2 m, L = 5.8 m, 2 T central) on a 5 mm r-z grid.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "libsynth.so")
_lib = None

MUON_MASS = 0.1056583755
PION_MASS = 0.13957039
SI_THICKNESS = 0.3
SI_X0 = 93.7


def build(force: bool = False) -> str:
    """Compiles libsynth.so in-tree (portable flags: builds on x86_64 and aarch64)."""
    src = os.path.join(_HERE, "synth.cpp")
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread",
                               "-o", _SO, src])
    return _SO


class _Field(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("B", ctypes.c_double * 3), ("nr", ctypes.c_int),
                ("nz", ctypes.c_int), ("r0", ctypes.c_double), ("dr", ctypes.c_double),
                ("z0", ctypes.c_double), ("dz", ctypes.c_double),
                ("Br", ctypes.c_void_p), ("Bz", ctypes.c_void_p)]


class _Params(ctypes.Structure):
    _fields_ = [("start", ctypes.c_int), ("mom_mode", ctypes.c_int), ("pmin", ctypes.c_double),
                ("pmax", ctypes.c_double), ("dir_mode", ctypes.c_int), ("ang", ctypes.c_double),
                ("eta_max", ctypes.c_double), ("z0_sigma", ctypes.c_double),
                ("mass", ctypes.c_double), ("sigma_hit", ctypes.c_double),
                ("sigma_v", ctypes.c_double), ("ms", ctypes.c_int), ("eloss", ctypes.c_int),
                ("seed_sigma", ctypes.c_double * 5), ("seed_smear", ctypes.c_int),
                ("seed_cot", ctypes.c_int),
                ("cov_inflate", ctypes.c_double), ("min_hits", ctypes.c_int),
                ("max_hits", ctypes.c_int), ("step", ctypes.c_double),
                ("r_max", ctypes.c_double), ("z_max", ctypes.c_double), ("p_hole", ctypes.c_double)]


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        vp, d, u32, u64 = ctypes.c_void_p, ctypes.c_double, ctypes.c_uint32, ctypes.c_uint64
        L.syn_geometry_telescope.restype = vp
        L.syn_geometry_telescope.argtypes = [ctypes.c_int, d, d, d]
        L.syn_geometry_barrel_endcap.restype = vp
        L.syn_geometry_barrel_endcap.argtypes = [d, d]
        L.syn_geometry_size.restype = u32
        L.syn_geometry_size.argtypes = [vp]
        L.syn_geometry_export.argtypes = [vp, vp]
        L.syn_geometry_free.argtypes = [vp]
        L.syn_geometry_layer_sizes.argtypes = [vp, vp, vp]
        L.syn_geometry_layers.argtypes = [vp, vp, vp]
        L.syn_cel.restype = d
        L.syn_cel.argtypes = [d, d, d, d]
        L.syn_solenoid.argtypes = [d, d, d, d, ctypes.POINTER(d), ctypes.POINTER(d)]
        L.syn_solenoid_map.argtypes = [ctypes.c_int, ctypes.c_int, d, d, d, d, d, d, d, vp, vp]
        L.syn_event_counts.argtypes = [u64, u32, u32, u32, vp]
        L.syn_simulate.restype = vp
        L.syn_simulate.argtypes = [vp, ctypes.POINTER(_Field), ctypes.POINTER(_Params), u64, u32, vp,
                                   ctypes.c_int]
        L.syn_result_sizes.argtypes = [vp, ctypes.POINTER(u64), ctypes.POINTER(u64)]
        L.syn_result_export.argtypes = [vp] * 10
        L.syn_result_free.argtypes = [vp]
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


# ----------------------------------------------------------------------------- geometry
@dataclass
class Geometry:
    """Planar surfaces; ``table`` is [n, 16] = u[3] v[3] n[3] c[3] thickness X0 half_u half_v.
    ``layers`` [n_layers, 8] and ``rings`` [n_rings, 4] describe the barrel cylinders and endcap
    disks the modules tile (empty for a telescope); see syn_geometry_layers in synth.cpp."""
    table: np.ndarray
    _handle: int = 0
    layers: np.ndarray = None
    rings: np.ndarray = None

    @property
    def n(self) -> int:
        return self.table.shape[0]

    @property
    def u(self):
        return self.table[:, 0:3]

    @property
    def v(self):
        return self.table[:, 3:6]

    @property
    def normal(self):
        return self.table[:, 6:9]

    @property
    def center(self):
        return self.table[:, 9:12]

    @property
    def thickness(self):
        return self.table[:, 12]

    @property
    def x0(self):
        return self.table[:, 13]

    def rotation(self) -> np.ndarray:
        """[n, 9] row-major 3x3 matrices whose columns are u, v, n."""
        R = np.stack([self.u, self.v, self.normal], axis=2)  # [n, 3(row), 3(col)]
        return np.ascontiguousarray(R.reshape(-1, 9))

    def __del__(self):
        if self._handle and _lib is not None:
            _lib.syn_geometry_free(ctypes.c_void_p(self._handle))
            self._handle = 0


def _export_geometry(h) -> Geometry:
    L = lib()
    n = L.syn_geometry_size(h)
    t = np.zeros((n, 16), dtype=np.float64)
    L.syn_geometry_export(h, _ptr(t))
    nl, nr = ctypes.c_uint32(), ctypes.c_uint32()
    L.syn_geometry_layer_sizes(ctypes.c_void_p(h), ctypes.byref(nl), ctypes.byref(nr))
    layers, rings = np.zeros((nl.value, 8)), np.zeros((nr.value, 4))
    if nl.value:
        L.syn_geometry_layers(ctypes.c_void_p(h), _ptr(layers), _ptr(rings))
    return Geometry(t, h, layers, rings)


def telescope_geometry(n_planes: int = 9, spacing: float = 50.0, thickness: float = SI_THICKNESS,
                       x0: float = SI_X0) -> Geometry:
    return _export_geometry(lib().syn_geometry_telescope(n_planes, spacing, thickness, x0))


def barrel_endcap_geometry(thickness: float = SI_THICKNESS, x0: float = SI_X0) -> Geometry:
    return _export_geometry(lib().syn_geometry_barrel_endcap(thickness, x0))


# ----------------------------------------------------------------------------- field
@dataclass
class Field:
    """Uniform field ``B`` (T), or an r-z grid ``Br``/``Bz`` [nz, nr] float32 with node
    r = r0 + i dr, z = z0 + j dz (mm)."""
    kind: int
    B: tuple = (0.0, 0.0, 0.0)
    nr: int = 0
    nz: int = 0
    r0: float = 0.0
    dr: float = 1.0
    z0: float = 0.0
    dz: float = 1.0
    Br: np.ndarray | None = None
    Bz: np.ndarray | None = None

    def _c(self) -> _Field:
        f = _Field()
        f.kind = self.kind
        for i in range(3):
            f.B[i] = float(self.B[i])
        f.nr, f.nz, f.r0, f.dr, f.z0, f.dz = self.nr, self.nz, self.r0, self.dr, self.z0, self.dz
        f.Br = _ptr(self.Br) if self.Br is not None else None
        f.Bz = _ptr(self.Bz) if self.Bz is not None else None
        return f


def uniform_field(bz: float = 2.0) -> Field:
    return Field(kind=0, B=(0.0, 0.0, bz))


def cel(kc, p, c, s) -> float:
    return lib().syn_cel(kc, p, c, s)


def solenoid_raw(a: float, b: float, rho: float, z: float):
    """Field of an ideal solenoid (radius a, half-length b) in units of mu0 n I / pi."""
    br, bz = ctypes.c_double(), ctypes.c_double()
    lib().syn_solenoid(a, b, rho, z, ctypes.byref(br), ctypes.byref(bz))
    return br.value, bz.value


def solenoid_map(radius: float = 1200.0, length: float = 5800.0, bz_center: float = 2.0,
                 r_max: float = 1200.0, z_half: float = 3500.0, step: float = 5.0) -> Field:
    nr = int(round(r_max / step)) + 1
    nz = int(round(2 * z_half / step)) + 1
    Br = np.zeros((nz, nr), dtype=np.float32)
    Bz = np.zeros((nz, nr), dtype=np.float32)
    lib().syn_solenoid_map(nr, nz, 0.0, step, -z_half, step, radius, 0.5 * length, bz_center,
                           _ptr(Br), _ptr(Bz))
    return Field(kind=1, nr=nr, nz=nz, r0=0.0, dr=step, z0=-z_half, dz=step, Br=Br, Bz=Bz)


# ----------------------------------------------------------------------------- tracks
@dataclass
class SimParams:
    start: int = 1            # 0: origin on surface 0; 1: vertex (0, 0, z0)
    mom_mode: int = 1         # 0: p uniform; 1: pT log-uniform; 2: p log-uniform
    pmin: float = 0.5
    pmax: float = 100.0
    dir_mode: int = 1         # 0: +-ang about +x; 1: phi U(0, 2pi), eta U(+-eta_max)
    ang: float = 0.1
    eta_max: float = 3.0
    z0_sigma: float = 50.0
    mass: float = PION_MASS
    sigma_hit: float = 0.01   # mm
    sigma_v: float = 0.01     # mm, written into V
    ms: int = 1
    eloss: int = 1
    # seed resolution of a 3-hit seed: 0.05 mm, 1 mrad in phi, 1e-3 in cot(theta), 10 % in q/p
    seed_sigma: tuple = (0.05, 0.05, 0.001, 0.001, 0.1)
    seed_smear: int = 1
    seed_cot: int = 1
    cov_inflate: float = 1.0
    min_hits: int = 6
    max_hits: int = 18
    step: float = 10.0
    r_max: float = 1050.0
    z_max: float = 3050.0
    p_hole: float = 0.0       # probability that a crossing after the first is a hole (no measurement)

    def _c(self) -> _Params:
        p = _Params()
        for name, _ in _Params._fields_:
            val = getattr(self, name)
            if name == "seed_sigma":
                for i in range(5):
                    p.seed_sigma[i] = float(val[i])
            else:
                setattr(p, name, val)
        return p


@dataclass
class Tracks:
    """Simulated tracks. ``meas`` is [m, 5] = (loc0, loc1, V00, V01, V11) in path order;
    ``seed_cov`` is [n, 15], the packed upper triangle (row-major) of the 5x5 covariance."""
    offsets: np.ndarray
    sid: np.ndarray
    meas: np.ndarray
    hit_truth: np.ndarray
    truth: np.ndarray
    seed_par: np.ndarray
    seed_cov: np.ndarray
    truth_last: np.ndarray
    event: np.ndarray
    extra: dict = field(default_factory=dict)

    @property
    def n_tracks(self) -> int:
        return self.offsets.shape[0] - 1

    @property
    def n_hits(self) -> int:
        return self.sid.shape[0]

    def hits_per_track(self) -> np.ndarray:
        return np.diff(self.offsets)

    def subset(self, idx) -> "Tracks":
        """Tracks ``idx`` (an index array), re-packed."""
        idx = np.asarray(idx, dtype=np.int64)
        a, b = self.offsets[idx], self.offsets[idx + 1]
        n = b - a
        offs = np.zeros(len(idx) + 1, dtype=np.uint32)
        offs[1:] = np.cumsum(n)
        hit_idx = np.concatenate([np.arange(x, y) for x, y in zip(a, b)]) if len(idx) else \
            np.zeros(0, dtype=np.int64)
        return Tracks(offs, self.sid[hit_idx], self.meas[hit_idx], self.hit_truth[hit_idx],
                      self.truth[idx], self.seed_par[idx], self.seed_cov[idx],
                      self.truth_last[idx], self.event[idx])


def event_counts(seed: int, n_events: int, lo: int, hi: int) -> np.ndarray:
    out = np.zeros(n_events, dtype=np.uint32)
    lib().syn_event_counts(seed, n_events, lo, hi, _ptr(out))
    return out


def event_counts_loguniform(seed: int, total: int, lo: int = 1000, hi: int = 100000) -> np.ndarray:
    """Track counts of events drawn log-uniform in [lo, hi] until they add up to ``total``
    (the last event is cut to land on it exactly)."""
    rng = np.random.default_rng(seed)
    counts, acc = [], 0
    while acc < total:
        c = int(round(float(np.exp(rng.uniform(np.log(lo), np.log(hi))))))
        c = min(c, total - acc)
        counts.append(c)
        acc += c
    return np.asarray(counts, dtype=np.uint32)


def simulate(geom: Geometry, fld: Field, params: SimParams, seed: int, tracks_per_event,
             n_threads: int | None = None) -> Tracks:
    L = lib()
    tpe = np.ascontiguousarray(np.atleast_1d(np.asarray(tracks_per_event, dtype=np.uint32)))
    nt = n_threads or os.cpu_count() or 1
    cf, cp = fld._c(), params._c()
    h = L.syn_simulate(ctypes.c_void_p(geom._handle), ctypes.byref(cf), ctypes.byref(cp), seed,
                       len(tpe), _ptr(tpe), nt)
    n_t, n_h = ctypes.c_uint64(), ctypes.c_uint64()
    L.syn_result_sizes(h, ctypes.byref(n_t), ctypes.byref(n_h))
    n, m = n_t.value, n_h.value
    out = Tracks(np.zeros(n + 1, np.uint32), np.zeros(m, np.uint32), np.zeros((m, 5)),
                 np.zeros((m, 2)), np.zeros((n, 5)), np.zeros((n, 5)), np.zeros((n, 15)),
                 np.zeros((n, 5)), np.zeros(n, np.uint32))
    L.syn_result_export(h, _ptr(out.offsets), _ptr(out.sid), _ptr(out.meas), _ptr(out.hit_truth),
                        _ptr(out.truth), _ptr(out.seed_par), _ptr(out.seed_cov),
                        _ptr(out.truth_last), _ptr(out.event))
    L.syn_result_free(h)
    return out


# ----------------------------------------------------------------------------- workloads
def telescope_params(**kw) -> SimParams:
    p = SimParams(start=0, mom_mode=0, pmin=1.0, pmax=10.0, dir_mode=0, ang=0.1, mass=MUON_MASS,
                  seed_sigma=(1.0, 1.0, 0.01, 0.01, 0.1), seed_cot=0, min_hits=9, max_hits=9, step=10.0,
                  r_max=1e9, z_max=1e9)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def barrel_params(**kw) -> SimParams:
    p = SimParams()
    for k, v in kw.items():
        setattr(p, k, v)
    return p


@dataclass
class Workload:
    name: str
    geometry: Geometry
    field: Field
    tracks: Tracks
    mass: float = MUON_MASS   # fit hypothesis


def telescope_workload(n_tracks: int = 1000, seed: int = 0, **kw) -> Workload:
    """9-plane telescope, uniform 2 T along z, muons p ~ U(1, 10) GeV."""
    g = telescope_geometry()
    f = uniform_field(2.0)
    t = simulate(g, f, telescope_params(**kw), seed, [n_tracks])
    return Workload("telescope_fp64_1k", g, f, t)


def barrel_workload(n_events: int = 50, lo: int = 2000, hi: int = 20000, seed: int = 2,
                    fld: Field | None = None, geom: Geometry | None = None,
                    **kw) -> Workload:
    """Barrel + endcap batch: n_events events of U{lo..hi} pions (pT log-uniform 0.5-100 GeV,
    eta U(+-3), vertex z ~ N(0, 50 mm)), uniform 2 T along z unless ``fld`` is given."""
    g = geom or barrel_endcap_geometry()
    f = fld or uniform_field(2.0)
    counts = event_counts(seed, n_events, lo, hi)
    p = barrel_params(**kw)
    if f.kind == 0 and "step" not in kw:
        p.step = 40.0  # exact helix segments: the step only bounds the crossing search
    t = simulate(g, f, p, seed, counts)
    return Workload(f"barrel_endcap_{n_events}ev", g, f, t)


def solenoid_muon_workload(n_tracks: int = 100000, seed: int = 3, fld: Field | None = None,
                           geom: Geometry | None = None, **kw) -> Workload:
    """Same geometry in the solenoid map; muons with p log-uniform 1-100 GeV."""
    g = geom or barrel_endcap_geometry()
    f = fld or solenoid_map()
    p = barrel_params(mom_mode=2, pmin=1.0, pmax=100.0, mass=MUON_MASS, step=5.0)
    for k, v in kw.items():
        setattr(p, k, v)
    t = simulate(g, f, p, seed, [n_tracks])
    return Workload(f"solenoid_map_muons_{n_tracks}", g, f, t)


@dataclass
class MeasurementContainer:
    """The measurements of a set of tracks grouped by surface, as a track finder sees them:
    ``meas`` [m, 5] sorted by surface id (stable), surface s owning rows ``offsets[s]`` ..
    ``offsets[s + 1] - 1``; ``track`` and ``hit`` give each row's simulated track and its index
    in the tracks' own measurement arrays (for efficiency and purity)."""
    offsets: np.ndarray
    meas: np.ndarray
    sid: np.ndarray
    track: np.ndarray
    hit: np.ndarray


def measurement_container(tracks: Tracks, n_surfaces: int) -> MeasurementContainer:
    """Groups the tracks' measured hits (holes left out) by surface."""
    hole = (tracks.sid & np.uint32(0x80000000)) != 0
    hit = np.flatnonzero(~hole)
    track_of = np.repeat(np.arange(tracks.n_tracks), np.diff(tracks.offsets.astype(np.int64)))[hit]
    sid = tracks.sid[hit].astype(np.int64)
    order = np.argsort(sid, kind="stable")
    counts = np.bincount(sid, minlength=n_surfaces)
    offsets = np.zeros(n_surfaces + 1, np.uint32)
    offsets[1:] = np.cumsum(counts)
    return MeasurementContainer(offsets, np.ascontiguousarray(tracks.meas[hit][order]), sid[order].astype(np.uint32),
                                track_of[order], hit[order])


def layer_of_surfaces(geom: Geometry) -> np.ndarray:
    """Layer index of every surface (-1 outside the layer structure)."""
    out = np.full(geom.n, -1, dtype=np.int64)
    if geom.layers is None:
        return out
    for li, l in enumerate(geom.layers):
        if l[0] == 0:
            first, cnt = int(l[5]), int(l[2]) * int(l[3])
            out[first:first + cnt] = li
        else:
            for k in range(int(l[2])):
                rg = geom.rings[int(l[3]) + k]
                out[int(rg[2]):int(rg[2]) + int(rg[1])] = li
    return out


def triplet_seed_hits(tracks: Tracks, geom: Geometry):
    """A stand-in for triplet seeding: every track's first measurements on three distinct layers
    (offsets, measurements [m, 5], surface ids), for seed parameter estimation."""
    layer_of = layer_of_surfaces(geom)
    offs, pick = [0], []
    for i in range(tracks.n_tracks):
        seen = []
        for j in range(int(tracks.offsets[i]), int(tracks.offsets[i + 1])):
            if tracks.sid[j] & np.uint32(0x80000000):
                continue
            L = layer_of[tracks.sid[j]]
            if L not in seen:
                seen.append(L)
                pick.append(j)
            if len(seen) == 3:
                break
        offs.append(len(pick))
    pick = np.array(pick, dtype=np.int64)
    return np.array(offs, np.uint32), tracks.meas[pick], tracks.sid[pick]

