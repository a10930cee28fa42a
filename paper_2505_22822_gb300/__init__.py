"""Python binding of libtkf.so, the GB300 (sm_103a) batched Kalman-filter track fitter.

Argument marshalling only: every step of the fit runs in the CUDA kernels behind the C
interface declared in include/tkf.h. PyTorch provides device memory and streams. There is
no CPU fallback: without the compiled library or a GB300 device the calls raise.

    import paper_2505_22822_gb300 as tkf
    ctx = tkf.Context(0)
    geo = tkf.Geometry(ctx, rot, center, thickness, x0)
    fld = tkf.Field.uniform(ctx, (0, 0, 2.0))
    out = tkf.fit(ctx, geo, fld, batch)      # batch: tkf.Batch of CUDA tensors
"""

from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_HERE)
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libtkf.so")
_SOURCES = ["tkf_api.cu", "tkf_order.cu", "tkf_policy.cu", "tkf_fit_fp64.cu", "tkf_fit_fp64_r128.cu",
            "tkf_fit_fp64_r64.cu", "tkf_fit_mixed.cu",
            "tkf_fit_mixed_r128.cu", "tkf_fit_mixed_r64.cu", "tkf_fit_mixed32.cu", "tkf_mlp.cu", "tkf_seed.cu",
            "tkf_fit_group.cu", "tkf_ckf.cu", "tkf_fit_two_filter.cu", "tkf_fit_two_filter_mixed.cu",
            "tkf_fit_two_filter_mixed32.cu", "tkf_fit_two_filter_capped_mixed.cu",
            "tkf_fit_two_filter_capped_fp64.cu", "tkf_states.cu"]
_lib = None

NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo", "-O3", "-std=c++17",
              "-Xcompiler", "-fPIC"]

FP64, MIXED, MIXED_FP32 = 0, 1, 2
STEP_ADAPTIVE, STEP_LEARNED = 0, 1
FIT_AUTOTUNE, FIT_GRAPH, FIT_TEST_PROPOSAL_TIMEOUT = 1, 2, 1 << 31
FIELD_UNIFORM, FIELD_RZ_GRID = 0, 1
SEED_FIRST_MIDDLE_LAST, SEED_FIRST_THREE = 0, 1
SMOOTHER_RTS, SMOOTHER_TWO_FILTER = 0, 1
SID_NO_MEASUREMENT = 0x80000000  # surface-id flag: the track crosses the surface without a measurement
SEED_STATUS = {"TOO_FEW_HITS": 1, "NO_CURVATURE": 2, "BAD_INPUT": 4}

TRACK_STATUS = {
    "MAX_STEPS": 1 << 0, "SURFACE_MISSED": 1 << 1, "PARTICLE_STOPPED": 1 << 2,
    "UPDATE_NOT_SPD": 1 << 3, "SMOOTHER_NOT_SPD": 1 << 4, "TOO_FEW_HITS": 1 << 5,
    "OUT_OF_FIELD": 1 << 6, "BAD_INPUT": 1 << 7, "STEP_UNDERFLOW": 1 << 8, "NON_FINITE": 1 << 9,
    "PROPOSAL_FALLBACK": 1 << 10,
}
FATAL_MASK = ~(TRACK_STATUS["TOO_FEW_HITS"] | TRACK_STATUS["OUT_OF_FIELD"]
               | TRACK_STATUS["PROPOSAL_FALLBACK"]) & 0xFFFFFFFF


class TkfError(RuntimeError):
    pass


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def build(force: bool = False, verbose: bool = False) -> str:
    """Compiles libtkf.so in-tree for sm_103a (translation units in parallel, then linked)."""
    os.makedirs(_BUILD, exist_ok=True)
    csrc = os.path.join(_HERE, "csrc")
    inc = os.path.join(_ROOT, "include")
    deps = [os.path.join(csrc, f) for f in os.listdir(csrc)] + [os.path.join(inc, "tkf.h")]
    newest = max(os.path.getmtime(d) for d in deps)
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= newest:
        return _SO
    nvcc = _nvcc()
    procs, objs = [], []
    for src in _SOURCES:
        obj = os.path.join(_BUILD, src.replace(".cu", ".o"))
        objs.append(obj)
        cmd = [nvcc, *NVCC_FLAGS, "-I", inc, "-c", os.path.join(csrc, src), "-o", obj]
        if verbose:
            cmd += ["-Xptxas", "-v"]
        procs.append(subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT))
    for p, src in zip(procs, _SOURCES):
        out, _ = p.communicate()
        if p.returncode != 0:
            raise TkfError(f"nvcc failed on {src}:\n{out.decode()}")
        if verbose:
            print(out.decode())
    tmp = _SO + ".tmp"
    subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-shared",
                           "-cudart", "shared", "-o", tmp, *objs])
    os.replace(tmp, _SO)
    return _SO


# ---------------------------------------------------------------------------- C structs
class SurfaceDesc(ctypes.Structure):
    _fields_ = [("rot", ctypes.c_double * 9), ("center", ctypes.c_double * 3),
                ("thickness", ctypes.c_double), ("x0", ctypes.c_double)]


class Material(ctypes.Structure):
    _fields_ = [("z_over_a", ctypes.c_double), ("i_ev", ctypes.c_double),
                ("rho_g_cm3", ctypes.c_double), ("hbar_omega_p_ev", ctypes.c_double)]


class FieldDesc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("b_tesla", ctypes.c_double * 3), ("nr", ctypes.c_uint32),
                ("nz", ctypes.c_uint32), ("r0", ctypes.c_double), ("dr", ctypes.c_double),
                ("z0", ctypes.c_double), ("dz", ctypes.c_double), ("br", ctypes.c_void_p),
                ("bz", ctypes.c_void_p)]


class FitOptions(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("step_mode", ctypes.c_int), ("tol", ctypes.c_double),
                ("h_max", ctypes.c_double), ("h_min", ctypes.c_double),
                ("surf_tol", ctypes.c_double), ("max_steps", ctypes.c_uint32),
                ("mass", ctypes.c_double), ("mlp", ctypes.c_void_p), ("records", ctypes.c_void_p),
                ("record_capacity", ctypes.c_uint32), ("record_count", ctypes.c_void_p),
                ("flags", ctypes.c_uint32), ("block_threads", ctypes.c_uint32),
                ("blocks_per_sm", ctypes.c_uint32), ("tracks_per_warp", ctypes.c_uint32),
                ("max_registers", ctypes.c_uint32), ("kernel_events", ctypes.c_void_p),
                ("seed_cov_scale", ctypes.c_double), ("lanes_per_track", ctypes.c_uint32),
                ("smoother", ctypes.c_int), ("backward_inflation", ctypes.c_double)]


class MlpTrainOptions(ctypes.Structure):
    _fields_ = [("batch", ctypes.c_uint32), ("epochs", ctypes.c_uint32), ("lr", ctypes.c_float),
                ("beta1", ctypes.c_float), ("beta2", ctypes.c_float), ("eps", ctypes.c_float)]


class FitInputs(ctypes.Structure):
    _fields_ = [("n_tracks", ctypes.c_uint32), ("n_meas", ctypes.c_uint64),
                ("offsets", ctypes.c_void_p), ("loc0", ctypes.c_void_p), ("loc1", ctypes.c_void_p),
                ("v00", ctypes.c_void_p), ("v01", ctypes.c_void_p), ("v11", ctypes.c_void_p),
                ("sid", ctypes.c_void_p), ("seed_par", ctypes.c_void_p),
                ("seed_cov", ctypes.c_void_p)]


class FitOutputs(ctypes.Structure):
    _fields_ = [("par", ctypes.c_void_p), ("cov", ctypes.c_void_p), ("chi2", ctypes.c_void_p),
                ("ndf", ctypes.c_void_p), ("status", ctypes.c_void_p), ("steps", ctypes.c_void_p),
                ("states_par", ctypes.c_void_p), ("states_cov", ctypes.c_void_p)]


class SeedOutputs(ctypes.Structure):
    _fields_ = [("par", ctypes.c_void_p), ("cov", ctypes.c_void_p), ("status", ctypes.c_void_p)]


class CkfOptions(ctypes.Structure):
    _fields_ = [("chi2_max", ctypes.c_double), ("beam", ctypes.c_uint32), ("max_holes", ctypes.c_uint32),
                ("max_entries", ctypes.c_uint32)]


class CkfInputs(ctypes.Structure):
    _fields_ = [("n_seeds", ctypes.c_uint32), ("seed_sid", ctypes.c_void_p), ("seed_par", ctypes.c_void_p),
                ("seed_cov", ctypes.c_void_p), ("n_meas", ctypes.c_uint32), ("meas_offsets", ctypes.c_void_p),
                ("loc0", ctypes.c_void_p), ("loc1", ctypes.c_void_p), ("v00", ctypes.c_void_p),
                ("v01", ctypes.c_void_p), ("v11", ctypes.c_void_p), ("n_events", ctypes.c_uint32),
                ("seed_event", ctypes.c_void_p)]


class CkfOutputs(ctypes.Structure):
    _fields_ = [("n_entries", ctypes.c_void_p), ("n_meas", ctypes.c_void_p), ("chi2", ctypes.c_void_p),
                ("entry_sid", ctypes.c_void_p), ("entry_meas", ctypes.c_void_p)]


# C entry points and their signatures (argument types), as declared in include/tkf.h.
_VP = ctypes.c_void_p
_SIGNATURES = {
    "tkf_context_create": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(_VP)]),
    "tkf_context_destroy": (None, [_VP]),
    "tkf_last_error": (ctypes.c_char_p, [_VP]),
    "tkf_material_silicon": (None, [ctypes.POINTER(Material)]),
    "tkf_geometry_create": (ctypes.c_int, [_VP, ctypes.POINTER(SurfaceDesc), ctypes.c_uint32,
                                           ctypes.POINTER(Material), ctypes.POINTER(_VP)]),
    "tkf_geometry_destroy": (None, [_VP]),
    "tkf_field_create": (ctypes.c_int, [_VP, ctypes.POINTER(FieldDesc), ctypes.POINTER(_VP)]),
    "tkf_field_destroy": (None, [_VP]),
    "tkf_fit_options_default": (None, [ctypes.POINTER(FitOptions)]),
    "tkf_fit": (ctypes.c_int, [_VP, _VP, _VP, ctypes.POINTER(FitOptions), ctypes.POINTER(FitInputs),
                               ctypes.POINTER(FitOutputs), _VP]),
    "tkf_fit_host": (ctypes.c_int, [_VP, _VP, _VP, ctypes.POINTER(FitOptions),
                                    ctypes.POINTER(FitInputs), ctypes.POINTER(FitOutputs), _VP]),
    "tkf_fit_noalloc": (ctypes.c_int, [_VP, _VP, _VP, ctypes.POINTER(FitOptions),
                                       ctypes.POINTER(FitInputs), ctypes.POINTER(FitOutputs), _VP]),
    "tkf_estimate_seeds": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_uint32, ctypes.POINTER(FitInputs),
                                          ctypes.POINTER(SeedOutputs), _VP]),
    "tkf_geometry_set_layers": (ctypes.c_int, [_VP, _VP, ctypes.c_uint32, _VP, ctypes.c_uint32]),
    "tkf_ckf_options_default": (None, [ctypes.POINTER(CkfOptions)]),
    "tkf_find_tracks": (ctypes.c_int, [_VP, _VP, _VP, ctypes.POINTER(FitOptions), ctypes.POINTER(CkfOptions),
                                       ctypes.POINTER(CkfInputs), ctypes.POINTER(CkfOutputs), _VP]),
    "tkf_propose_start": (ctypes.c_int, [_VP, _VP, _VP, ctypes.POINTER(FitOptions), ctypes.POINTER(FitInputs),
                                         _VP, _VP]),
    "tkf_mlp_load": (ctypes.c_int, [_VP, _VP, ctypes.c_size_t, ctypes.POINTER(_VP)]),
    "tkf_mlp_load_f32": (ctypes.c_int, [_VP, _VP, ctypes.c_size_t, ctypes.POINTER(_VP), _VP]),
    "tkf_mlp_init": (ctypes.c_int, [_VP, _VP, ctypes.c_size_t, ctypes.c_uint64, _VP]),
    "tkf_mlp_calibrate": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_uint32, ctypes.c_double,
                                         ctypes.POINTER(ctypes.c_double), _VP]),
    "tkf_mlp_destroy": (None, [_VP]),
    "tkf_mlp_train": (ctypes.c_int, [_VP, _VP, ctypes.c_uint32, ctypes.POINTER(MlpTrainOptions), _VP, _VP,
                                     ctypes.POINTER(ctypes.c_uint32), _VP, _VP]),
    "tkf_mlp_loss_grad": (ctypes.c_int, [_VP, _VP, _VP, _VP, ctypes.c_uint32, _VP, _VP, _VP]),
    "tkf_mlp_forward": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_uint32, _VP, _VP]),
}

MLP_PARAMS, MLP_INPUTS, MLP_RECORD = 5057, 12, 13

NOALLOC_MAX_TRACKS = 2097152


def lib(build_if_missing: bool = True):
    """Loads libtkf.so (building it first if needed); raises if it cannot be loaded."""
    global _lib
    if _lib is None:
        if build_if_missing:
            build()
        if not os.path.exists(_SO):
            raise TkfError(f"{_SO} is missing: run paper_2505_22822_gb300.build()")
        L = ctypes.CDLL(_SO)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(code: int, ctx_handle=None, what: str = ""):
    if code != 0:
        msg = lib().tkf_last_error(ctx_handle)
        raise TkfError(f"{what} failed with status {code}: {msg.decode() if msg else ''}")


# ---------------------------------------------------------------------------- handles
class Context:
    def __init__(self, device: int = 0):
        h = _VP()
        _check(lib().tkf_context_create(device, ctypes.byref(h)), None, "tkf_context_create")
        self.handle = h
        self.device = device

    def close(self):
        if getattr(self, "handle", None):
            lib().tkf_context_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Geometry:
    """Planar surfaces: ``rot`` [n, 9] row-major (columns u, v, n), ``center`` [n, 3] mm,
    ``thickness`` [n] mm, ``x0`` [n] mm; ``material`` (Z/A, I eV, rho g/cm3, plasma eV)."""

    def __init__(self, ctx: Context, rot, center, thickness, x0, material=None):
        rot = np.ascontiguousarray(rot, dtype=np.float64).reshape(-1, 9)
        n = rot.shape[0]
        center = np.ascontiguousarray(center, dtype=np.float64).reshape(n, 3)
        thickness = np.broadcast_to(np.asarray(thickness, dtype=np.float64), (n,))
        x0 = np.broadcast_to(np.asarray(x0, dtype=np.float64), (n,))
        arr = (SurfaceDesc * n)()
        buf = np.frombuffer(arr, dtype=np.float64).reshape(n, 14)
        buf[:, 0:9] = rot
        buf[:, 9:12] = center
        buf[:, 12] = thickness
        buf[:, 13] = x0
        mat = None
        if material is not None:
            mat = Material(*[float(v) for v in material])
        h = _VP()
        _check(lib().tkf_geometry_create(ctx.handle, arr, n, ctypes.byref(mat) if mat else None,
                                         ctypes.byref(h)), ctx.handle, "tkf_geometry_create")
        self.handle, self.ctx, self.n = h, ctx, n

    def set_layers(self, layers, rings):
        """tkf_geometry_set_layers: the layer structure for track finding (host arrays [n, 8] and
        [m, 4], as the geometry generator exports them)."""
        layers = np.ascontiguousarray(layers, dtype=np.float64)
        rings = np.ascontiguousarray(rings, dtype=np.float64)
        _check(lib().tkf_geometry_set_layers(self.handle, _VP(layers.ctypes.data), layers.shape[0],
                                             _VP(rings.ctypes.data) if rings.size else None, rings.shape[0]),
               self.ctx.handle, "tkf_geometry_set_layers")
        return self

    @classmethod
    def from_table(cls, ctx: Context, table: np.ndarray, material=None) -> "Geometry":
        """From a [n, >=14] table u[3] v[3] n[3] c[3] thickness x0."""
        t = np.asarray(table, dtype=np.float64)
        R = np.stack([t[:, 0:3], t[:, 3:6], t[:, 6:9]], axis=2).reshape(-1, 9)
        return cls(ctx, R, t[:, 9:12], t[:, 12], t[:, 13], material)

    def __del__(self):
        try:
            if getattr(self, "handle", None):
                lib().tkf_geometry_destroy(self.handle)
                self.handle = None
        except Exception:
            pass


class Field:
    def __init__(self, ctx: Context, desc: FieldDesc, keep=()):
        h = _VP()
        _check(lib().tkf_field_create(ctx.handle, ctypes.byref(desc), ctypes.byref(h)), ctx.handle,
               "tkf_field_create")
        self.handle, self.ctx, self.kind = h, ctx, desc.kind

    @classmethod
    def uniform(cls, ctx: Context, b_tesla=(0.0, 0.0, 2.0)) -> "Field":
        d = FieldDesc()
        d.kind = FIELD_UNIFORM
        for i in range(3):
            d.b_tesla[i] = float(b_tesla[i])
        return cls(ctx, d)

    @classmethod
    def rz_grid(cls, ctx: Context, br, bz, r0, dr, z0, dz) -> "Field":
        br = np.ascontiguousarray(br, dtype=np.float32)
        bz = np.ascontiguousarray(bz, dtype=np.float32)
        d = FieldDesc()
        d.kind = FIELD_RZ_GRID
        d.nz, d.nr = br.shape
        d.r0, d.dr, d.z0, d.dz = r0, dr, z0, dz
        d.br = br.ctypes.data_as(_VP)
        d.bz = bz.ctypes.data_as(_VP)
        return cls(ctx, d, keep=(br, bz))

    @classmethod
    def from_desc(cls, ctx: Context, f) -> "Field":
        """From an object with kind, B, nr, nz, r0, dr, z0, dz, Br, Bz attributes."""
        if f.kind == FIELD_UNIFORM:
            return cls.uniform(ctx, f.B)
        return cls.rz_grid(ctx, f.Br, f.Bz, f.r0, f.dr, f.z0, f.dz)

    def __del__(self):
        try:
            if getattr(self, "handle", None):
                lib().tkf_field_destroy(self.handle)
                self.handle = None
        except Exception:
            pass


class Mlp:
    """Step-proposer network handle (BF16 weights on the device): from host BF16 bit patterns
    (tkf_mlp_load), or, with ``from_params``, from trained FP32 parameters in a CUDA tensor that
    the library rounds to BF16 (tkf_mlp_load_f32)."""

    def __init__(self, ctx: Context, bf16_weights=None, params=None, stream=None):
        h = _VP()
        if params is not None:
            import torch
            if stream is None:
                stream = torch.cuda.current_stream(params.device)
            _check(lib().tkf_mlp_load_f32(ctx.handle, _VP(params.data_ptr()), int(params.numel()), ctypes.byref(h),
                                          _VP(stream.cuda_stream)), ctx.handle, "tkf_mlp_load_f32")
        else:
            w = np.ascontiguousarray(bf16_weights, dtype=np.uint16)
            _check(lib().tkf_mlp_load(ctx.handle, w.ctypes.data_as(_VP), w.size, ctypes.byref(h)), ctx.handle,
                   "tkf_mlp_load")
        self.handle, self.ctx = h, ctx

    @classmethod
    def from_params(cls, ctx: Context, params, stream=None) -> "Mlp":
        return cls(ctx, params=params, stream=stream)

    def __del__(self):
        try:
            if getattr(self, "handle", None):
                lib().tkf_mlp_destroy(self.handle)
                self.handle = None
        except Exception:
            pass


@dataclass
class Options:
    precision: int = FP64
    step_mode: int = STEP_ADAPTIVE
    tol: float = 1e-4
    h_max: float = 1000.0
    h_min: float = 1e-4
    surf_tol: float = 1e-2
    max_steps: int = 10000
    mass: float = 0.1056583755
    mlp: object = None            # Mlp for STEP_LEARNED
    records: object = None        # CUDA float tensor [capacity, 13] for record capture
    record_count: object = None   # CUDA int32 tensor [1], zeroed by the caller
    autotune: bool = False        # time the candidate block shapes on the first call of a class
    graph: bool = False           # capture repeated identical calls into a CUDA graph
    test_proposal_timeout: bool = False  # test hook: the pre-pass issues no tensor-core work
    block_threads: int = 0        # explicit block shape (both nonzero), else default or tuned
    blocks_per_sm: int = 0
    tracks_per_warp: int = 0      # explicit tracks a warp takes at a time (1..32), else 32 or tuned
    max_registers: int = 0        # explicit register cap (255; 128 or 64 for MIXED), else default or tuned
    kernel_events: object = None  # (begin, end) torch.cuda.Event pair around the fit kernel
    seed_cov_scale: float = 1.0   # factor on the seed covariance (a refit inflates it)
    lanes_per_track: int = 0      # 0 default / tuned, 1, or 4 (group-per-track)
    smoother: int = 0             # SMOOTHER_RTS or SMOOTHER_TWO_FILTER
    backward_inflation: float = 1e3  # two-filter: factor on the backward filter's starting covariance

    def c(self) -> FitOptions:
        o = FitOptions()
        lib().tkf_fit_options_default(ctypes.byref(o))
        o.precision, o.step_mode = self.precision, self.step_mode
        o.tol, o.h_max, o.h_min, o.surf_tol = self.tol, self.h_max, self.h_min, self.surf_tol
        o.max_steps, o.mass = self.max_steps, self.mass
        if self.mlp is not None:
            o.mlp = self.mlp.handle
        if self.records is not None:
            o.records = self.records.data_ptr()
            o.record_capacity = int(self.records.shape[0])
            o.record_count = self.record_count.data_ptr()
        o.flags = ((FIT_AUTOTUNE if self.autotune else 0) | (FIT_GRAPH if self.graph else 0)
                   | (FIT_TEST_PROPOSAL_TIMEOUT if self.test_proposal_timeout else 0))
        o.block_threads, o.blocks_per_sm = self.block_threads, self.blocks_per_sm
        o.tracks_per_warp = self.tracks_per_warp
        o.max_registers = self.max_registers
        o.seed_cov_scale = self.seed_cov_scale
        o.lanes_per_track = self.lanes_per_track
        o.smoother, o.backward_inflation = self.smoother, self.backward_inflation
        if self.kernel_events is not None:
            # the C array must outlive the call: kept on the options struct
            o._events = (ctypes.c_void_p * 2)(*(ev.cuda_event for ev in self.kernel_events))
            o.kernel_events = ctypes.cast(o._events, ctypes.c_void_p)
        return o


# ---------------------------------------------------------------------------- batches
_IN_FIELDS = ("offsets", "loc0", "loc1", "v00", "v01", "v11", "sid", "seed_par", "seed_cov")


@dataclass
class Batch:
    """Fit inputs in the library's layout: offsets [n+1] u32, loc0/loc1/v00/v01/v11 [m] f64,
    sid [m] u32, seed_par [5, n] f64, seed_cov [15, n] f64 (numpy on the host, or torch)."""
    offsets: object
    loc0: object
    loc1: object
    v00: object
    v01: object
    v11: object
    sid: object
    seed_par: object
    seed_cov: object

    @property
    def n_tracks(self) -> int:
        return int(self.offsets.shape[0]) - 1

    @property
    def n_meas(self) -> int:
        return int(self.loc0.shape[0])

    @classmethod
    def from_arrays(cls, offsets, meas, sid, seed_par, seed_cov) -> "Batch":
        """From track-major arrays: meas [m, 5] (loc0, loc1, V00, V01, V11), seed_par [n, 5],
        seed_cov [n, 15]. Returns host (numpy) arrays in the library layout."""
        meas = np.asarray(meas, dtype=np.float64)
        c = np.ascontiguousarray
        return cls(c(offsets, dtype=np.uint32), c(meas[:, 0]), c(meas[:, 1]), c(meas[:, 2]),
                   c(meas[:, 3]), c(meas[:, 4]), c(sid, dtype=np.uint32),
                   c(np.asarray(seed_par, dtype=np.float64).T), c(np.asarray(seed_cov, dtype=np.float64).T))

    def to(self, device, pin: bool = False) -> "Batch":
        import torch
        vals = {}
        for k in _IN_FIELDS:
            v = getattr(self, k)
            t = torch.from_numpy(np.ascontiguousarray(v)) if isinstance(v, np.ndarray) else v
            if t.dtype == torch.uint32:
                t = t.view(torch.int32)
            if device == "cpu" and pin:
                t = t.pin_memory()
            else:
                t = t.to(device)
            vals[k] = t
        return Batch(**vals)

    def nbytes(self) -> int:
        return int(sum(getattr(self, k).nbytes if isinstance(getattr(self, k), np.ndarray)
                       else getattr(self, k).numel() * getattr(self, k).element_size()
                       for k in _IN_FIELDS))


def _ptr(x) -> int | None:
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


def _inputs_struct(b: Batch) -> FitInputs:
    s = FitInputs()
    s.n_tracks = b.n_tracks
    s.n_meas = b.n_meas
    for k in _IN_FIELDS:
        setattr(s, k, _ptr(getattr(b, k)))
    return s


@dataclass
class Result:
    par: object      # [5, n]
    cov: object      # [15, n]
    chi2: object     # [n]
    ndf: object      # [n]
    status: object   # [n]
    steps: object    # [2, n] or None
    states_par: object = None  # [5, n_meas]: every entry's smoothed parameters, or None
    states_cov: object = None  # [15, n_meas]: every entry's smoothed covariance (packed), or None


def alloc_outputs(n: int, device, steps: bool = True, states_meas: int | None = None) -> Result:
    """Output tensors for n tracks; with ``states_meas`` also the all-states arrays for that many
    measurement rows."""
    import torch
    kw = dict(device=device)
    st = states_meas is not None
    return Result(torch.empty((5, n), dtype=torch.float64, **kw),
                  torch.empty((15, n), dtype=torch.float64, **kw),
                  torch.empty((n,), dtype=torch.float64, **kw),
                  torch.empty((n,), dtype=torch.int32, **kw),
                  torch.empty((n,), dtype=torch.int32, **kw),
                  torch.empty((2, n), dtype=torch.int32, **kw) if steps else None,
                  torch.empty((5, states_meas), dtype=torch.float64, **kw) if st else None,
                  torch.empty((15, states_meas), dtype=torch.float64, **kw) if st else None)


def _outputs_struct(r: Result) -> FitOutputs:
    s = FitOutputs()
    s.par, s.cov, s.chi2 = _ptr(r.par), _ptr(r.cov), _ptr(r.chi2)
    s.ndf, s.status, s.steps = _ptr(r.ndf), _ptr(r.status), _ptr(r.steps)
    s.states_par, s.states_cov = _ptr(r.states_par), _ptr(r.states_cov)
    return s


def fit(ctx: Context, geo: Geometry, field: Field, batch: Batch, opts: Options | None = None,
        out: Result | None = None, stream=None, steps: bool = True, states: bool = False) -> Result:
    """Enqueues the fit of a batch of CUDA tensors on ``stream`` (default: torch's current
    stream) and returns the output tensors (valid once the stream reaches the work). With
    ``states`` the result also holds every entry's smoothed state (``states_par``,
    ``states_cov``)."""
    import torch
    dev = batch.offsets.device
    if dev.type != "cuda":
        raise TkfError("fit() needs CUDA tensors; use fit_host() for host arrays")
    out = out or alloc_outputs(batch.n_tracks, dev, steps, batch.n_meas if states else None)
    if stream is None:
        stream = torch.cuda.current_stream(dev)
    o = (opts or Options()).c()
    _check(lib().tkf_fit(ctx.handle, geo.handle, field.handle, ctypes.byref(o),
                         ctypes.byref(_inputs_struct(batch)), ctypes.byref(_outputs_struct(out)),
                         _VP(stream.cuda_stream)), ctx.handle, "tkf_fit")
    return out


def fit_host(ctx: Context, geo: Geometry, field: Field, batch: Batch, opts: Options | None = None,
             out: Result | None = None, stream=None, steps: bool = True) -> Result:
    """Fits a batch of host arrays (numpy or pinned CPU tensors) through tkf_fit_host:
    host-to-device copies, the fit and device-to-host copies, pipelined in chunks for large
    batches (the copies overlap the fits); returns when the results are in the host buffers."""
    n = batch.n_tracks
    if out is None:
        out = Result(np.empty((5, n)), np.empty((15, n)), np.empty(n), np.empty(n, np.int32),
                     np.empty(n, np.uint32), np.empty((2, n), np.uint32) if steps else None)
    o = (opts or Options()).c()
    s = stream.cuda_stream if stream is not None else None
    _check(lib().tkf_fit_host(ctx.handle, geo.handle, field.handle, ctypes.byref(o),
                              ctypes.byref(_inputs_struct(batch)), ctypes.byref(_outputs_struct(out)),
                              _VP(s) if s else None), ctx.handle, "tkf_fit_host")
    return out


def propose_start(ctx: Context, geo: Geometry, field: Field, batch: Batch, opts: Options, stream=None):
    """tkf_propose_start: the learned mode's starting step-size control of every track (CUDA
    float32 tensor [n]), as the fit computes it with ``opts`` (STEP_LEARNED, ``opts.mlp``)."""
    import torch
    dev = batch.offsets.device
    h0 = torch.empty(batch.n_tracks, dtype=torch.float32, device=dev)
    if stream is None:
        stream = torch.cuda.current_stream(dev)
    o = opts.c()
    _check(lib().tkf_propose_start(ctx.handle, geo.handle, field.handle, ctypes.byref(o),
                                   ctypes.byref(_inputs_struct(batch)), _VP(h0.data_ptr()),
                                   _VP(stream.cuda_stream)), ctx.handle, "tkf_propose_start")
    return h0


@dataclass
class SeedResult:
    par: object     # [5, n] f64: loc0, loc1, phi, theta, q/p on the first measurement's surface
    cov: object     # [15, n] f64, packed upper triangle
    status: object  # [n] (SEED_STATUS bits)


def estimate_seeds(ctx: Context, geo: Geometry, field: Field, batch: Batch,
                   which: int = SEED_FIRST_MIDDLE_LAST, out: SeedResult | None = None, stream=None) -> SeedResult:
    """tkf_estimate_seeds: every track's starting parameters and prior covariance from the helix
    through three of its measurements (the first, middle and last, or the first three), in the
    layout of ``Batch.seed_par`` / ``seed_cov``; enqueued on ``stream`` (default: torch's current
    stream). The batch's own seeds are not read."""
    import torch
    dev = batch.offsets.device
    if dev.type != "cuda":
        raise TkfError("estimate_seeds() needs CUDA tensors")
    n = batch.n_tracks
    if out is None:
        out = SeedResult(torch.empty((5, n), dtype=torch.float64, device=dev),
                         torch.empty((15, n), dtype=torch.float64, device=dev),
                         torch.empty((n,), dtype=torch.int32, device=dev))
    if stream is None:
        stream = torch.cuda.current_stream(dev)
    so = SeedOutputs()
    so.par, so.cov, so.status = _ptr(out.par), _ptr(out.cov), _ptr(out.status)
    _check(lib().tkf_estimate_seeds(ctx.handle, geo.handle, field.handle, int(which),
                                    ctypes.byref(_inputs_struct(batch)), ctypes.byref(so),
                                    _VP(stream.cuda_stream)), ctx.handle, "tkf_estimate_seeds")
    return out


@dataclass
class CkfResult:
    n_entries: object   # [n] i32
    n_meas: object      # [n] i32
    chi2: object        # [n] f64
    entry_sid: object   # [max_entries, n] i32 (bit 31: hole)
    entry_meas: object  # [max_entries, n] i32 (-1: hole)


def find_tracks(ctx: Context, geo: Geometry, field: Field, seed_sid, seed_par, seed_cov, meas_offsets, loc0, loc1, v00,
                v01, v11, opts: Options | None = None, chi2_max: float = 15.0, beam: int = 3, max_holes: int = 2,
                max_entries: int = 24, stream=None, seed_event=None) -> CkfResult:
    """tkf_find_tracks on CUDA tensors: seeds (surface ids [n], parameters [5, n], covariances
    [15, n]) and the event's measurements grouped by surface (offsets [n_surfaces + 1] and the
    SoA measurement arrays). Several events in one launch: ``meas_offsets`` [n_events,
    n_surfaces + 1] into shared measurement arrays and ``seed_event`` [n] (int32) the event of
    each seed. Enqueued on ``stream`` (default: torch's current stream)."""
    import torch
    dev = seed_par.device
    n = int(seed_sid.shape[0])
    out = CkfResult(torch.empty(n, dtype=torch.int32, device=dev), torch.empty(n, dtype=torch.int32, device=dev),
                    torch.empty(n, dtype=torch.float64, device=dev),
                    torch.empty((max_entries, n), dtype=torch.int32, device=dev),
                    torch.empty((max_entries, n), dtype=torch.int32, device=dev))
    if stream is None:
        stream = torch.cuda.current_stream(dev)
    co = CkfOptions()
    lib().tkf_ckf_options_default(ctypes.byref(co))
    co.chi2_max, co.beam, co.max_holes, co.max_entries = chi2_max, beam, max_holes, max_entries
    ci = CkfInputs()
    ci.n_seeds, ci.n_meas = n, int(loc0.shape[0])
    ci.seed_sid, ci.seed_par, ci.seed_cov = _ptr(seed_sid), _ptr(seed_par), _ptr(seed_cov)
    ci.meas_offsets, ci.loc0, ci.loc1 = _ptr(meas_offsets), _ptr(loc0), _ptr(loc1)
    ci.v00, ci.v01, ci.v11 = _ptr(v00), _ptr(v01), _ptr(v11)
    if seed_event is not None:
        ci.n_events = int(meas_offsets.shape[0]) if meas_offsets.dim() == 2 else 1
        ci.seed_event = _ptr(seed_event)
    cout = CkfOutputs()
    cout.n_entries, cout.n_meas, cout.chi2 = _ptr(out.n_entries), _ptr(out.n_meas), _ptr(out.chi2)
    cout.entry_sid, cout.entry_meas = _ptr(out.entry_sid), _ptr(out.entry_meas)
    o = (opts or Options()).c()
    _check(lib().tkf_find_tracks(ctx.handle, geo.handle, field.handle, ctypes.byref(o), ctypes.byref(co),
                                 ctypes.byref(ci), ctypes.byref(cout), _VP(stream.cuda_stream)),
           ctx.handle, "tkf_find_tracks")
    return out


def with_seeds(batch: Batch, seed_par, seed_cov) -> Batch:
    """The batch with other seeds (for example those of estimate_seeds, or a fit's result for a
    refit); the measurement arrays are shared, not copied."""
    return Batch(batch.offsets, batch.loc0, batch.loc1, batch.v00, batch.v01, batch.v11, batch.sid,
                 seed_par, seed_cov)


def fit_noalloc(ctx: Context, geo: Geometry, field: Field, batch: Batch, out: Result,
                opts: Options | None = None, stream=None) -> Result:
    """tkf_fit_noalloc: the fit of ``fit`` for callers that may not allocate device memory while
    running; its scratch is a static array of the library (at most NOALLOC_MAX_TRACKS tracks per
    call). ``out`` must be preallocated CUDA tensors. Calls that overlap on the GPU race."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream(batch.offsets.device)
    o = (opts or Options()).c()
    _check(lib().tkf_fit_noalloc(ctx.handle, geo.handle, field.handle, ctypes.byref(o),
                                 ctypes.byref(_inputs_struct(batch)), ctypes.byref(_outputs_struct(out)),
                                 _VP(stream.cuda_stream)), ctx.handle, "tkf_fit_noalloc")
    return out


def mlp_train(ctx: Context, records, params, moments, adam_t: int, batch: int, epochs: int, lr=1e-3,
              beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    """Trains FP32 params (CUDA tensor [5057]) in place on records (CUDA [n, 13]) with the library's
    kernels; moments is a CUDA tensor [2, 5057]. Returns (per-epoch mean loss tensor, new adam_t)."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream(records.device)
    loss = torch.zeros(epochs, dtype=torch.float32, device=records.device)
    t = ctypes.c_uint32(adam_t)
    o = MlpTrainOptions(batch, epochs, lr, beta1, beta2, eps)
    _check(lib().tkf_mlp_train(ctx.handle, _VP(records.data_ptr()), records.shape[0], ctypes.byref(o),
                               _VP(params.data_ptr()), _VP(moments.data_ptr()), ctypes.byref(t),
                               _VP(loss.data_ptr()), _VP(stream.cuda_stream)), ctx.handle, "tkf_mlp_train")
    return loss, t.value


def mlp_loss_grad(ctx: Context, params, x, y, stream=None):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream(x.device)
    grad = torch.empty(MLP_PARAMS, dtype=torch.float32, device=x.device)
    loss = torch.empty(1, dtype=torch.float32, device=x.device)
    _check(lib().tkf_mlp_loss_grad(ctx.handle, _VP(params.data_ptr()), _VP(x.data_ptr()), _VP(y.data_ptr()),
                                   x.shape[0], _VP(grad.data_ptr()), _VP(loss.data_ptr()),
                                   _VP(stream.cuda_stream)), ctx.handle, "tkf_mlp_loss_grad")
    return loss, grad


def mlp_forward(ctx: Context, params, x, stream=None):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream(x.device)
    out = torch.empty(x.shape[0], dtype=torch.float32, device=x.device)
    _check(lib().tkf_mlp_forward(ctx.handle, _VP(params.data_ptr()), _VP(x.data_ptr()), x.shape[0],
                                 _VP(out.data_ptr()), _VP(stream.cuda_stream)), ctx.handle, "tkf_mlp_forward")
    return out


def mlp_init(ctx: Context, params, seed: int, stream=None):
    """tkf_mlp_init: seeded initial FP32 parameters into ``params`` (CUDA tensor [5057])."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream(params.device)
    _check(lib().tkf_mlp_init(ctx.handle, _VP(params.data_ptr()), int(params.numel()), int(seed),
                              _VP(stream.cuda_stream)), ctx.handle, "tkf_mlp_init")
    return params


def mlp_calibrate(ctx: Context, params, records, quantile: float, stream=None) -> float:
    """tkf_mlp_calibrate: shifts the output bias of ``params`` (CUDA [5057], in place) by the
    ``quantile`` of the residuals over ``records`` (CUDA [n, 13]); returns the shift."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream(params.device)
    shift = ctypes.c_double()
    _check(lib().tkf_mlp_calibrate(ctx.handle, _VP(params.data_ptr()), _VP(records.data_ptr()), records.shape[0],
                                   float(quantile), ctypes.byref(shift), _VP(stream.cuda_stream)), ctx.handle,
           "tkf_mlp_calibrate")
    return shift.value


def exported_symbols() -> list[str]:
    return sorted(_SIGNATURES)
