"""Thin ctypes binding of the C ABI in include/lbve.h (argument marshalling only).

Every step of the method runs in the CUDA kernels of liblbve.so; this module only
converts numpy arrays and Python numbers into the ABI's plain pointers and sizes.
If the library is missing it raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as ct
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblbve.so")

F64, F32, F16_SHIFTED, BF16_SHIFTED = 0, 1, 2, 3
PRECISIONS = {"f64": F64, "f32": F32, "f16": F16_SHIFTED, "bf16": BF16_SHIFTED}
FV_FLUX, FV_SOURCE = 1, 2
FV_CTU, FV_DIVU = 4, 8  # variants: transverse CTU overlap on the face fluxes; tau div(u) source
SCHED_AUTO, SCHED_SPLIT, SCHED_FUSED, SCHED_PIPELINED = 0, 1, 2, 3
FLAG_FLUID, FLAG_NOSLIP, FLAG_WALL0, FLAG_PARTICLE0 = 0, 1, 2, 64
KERNEL_KINDS = ["lb", "fv", "fused", "momentum_exchange", "particle", "", "", ""]
EUNSTABLE = 4
HALO_F, HALO_U, HALO_TAU = 0, 1, 2
LB_CELLS, LB_ROWS = 0, 1
FV_TILES, FV_PAIRS = 0, 1
STATUS = ["LBVE_OK", "LBVE_EINVAL", "LBVE_ENOMEM", "LBVE_ECUDA", "LBVE_EUNSTABLE", "LBVE_ETIMEOUT", "LBVE_ESTATE"]

# every entry point declared in include/lbve.h
EXPORTS = [
    "lbve_default_params", "lbve_device_bytes", "lbve_create", "lbve_create_with_allocator", "lbve_destroy",
    "lbve_set_geometry", "lbve_init_fields", "lbve_init_fields_device", "lbve_probe", "lbve_add_particle", "lbve_step", "lbve_read_fields",
    "lbve_read_fields_device", "lbve_read_pdfs", "lbve_write_pdfs", "lbve_read_particle", "lbve_read_conversions", "lbve_read_body_forces",
    "lbve_reduce", "lbve_residual", "lbve_pool_create", "lbve_pool_destroy", "lbve_pool_fits", "lbve_pool_admit",
    "lbve_pool_remove", "lbve_pool_step", "lbve_pool_residuals", "lbve_pool_size", "lbve_pool_bytes_in_use",
    "lbve_pool_set_graphs", "lbve_pool_last_error", "lbve_step_noalloc", "lbve_noalloc_last_error", "lbve_set_kernel_timing", "lbve_read_kernel_times", "lbve_time", "lbve_synchronize", "lbve_is_unstable", "lbve_stream_collide_kernel", "lbve_stress_kernel", "lbve_checkpoint_bytes", "lbve_save", "lbve_restore",
    "lbve_set_z_range", "lbve_step_phase", "lbve_halo_bytes", "lbve_halo_pack", "lbve_halo_unpack", "lbve_last_error", "lbve_status_string",
    "lbve_autotune", "lbve_pool_autotune",
    # include/lbve2d.h
    "lbve2d_default_params", "lbve2d_create", "lbve2d_destroy", "lbve2d_set_geometry", "lbve2d_set_force_field",
    "lbve2d_init_fields", "lbve2d_step", "lbve2d_read_fields", "lbve2d_read_pdfs", "lbve2d_time", "lbve2d_last_error",
]


class Tuning(ct.Structure):
    """lbve_tuning: the schedule lbve_autotune chose and what it measured."""

    _fields_ = [("block_x", ct.c_int), ("fv_zchunk", ct.c_int), ("candidates", ct.c_int),
                ("steps_taken", ct.c_longlong), ("ms_per_step", ct.c_double), ("ms_per_step_default", ct.c_double)]


class Params2D(ct.Structure):
    """lbve2d_params (include/lbve2d.h)."""

    _fields_ = [
        ("nx", ct.c_int), ("ny", ct.c_int), ("periodic", ct.c_int * 2),
        ("eta", ct.c_double), ("beta", ct.c_double), ("lambda_p", ct.c_double), ("rho0", ct.c_double),
        ("body_force", ct.c_double * 2), ("magic", ct.c_double), ("pdf_prec", ct.c_int), ("fv_terms", ct.c_int),
    ]


class LbveError(RuntimeError):
    def __init__(self, status: int, msg: str):
        self.status = status
        name = STATUS[status] if 0 <= status < len(STATUS) else str(status)
        super().__init__(f"{name}: {msg}")


class Params(ct.Structure):
    _fields_ = [
        ("nx", ct.c_int), ("ny", ct.c_int), ("nz", ct.c_int),
        ("periodic", ct.c_int * 3),
        ("eta", ct.c_double), ("beta", ct.c_double), ("lambda_p", ct.c_double), ("rho0", ct.c_double),
        ("body_force", ct.c_double * 3),
        ("magic", ct.c_double),
        ("pdf_prec", ct.c_int), ("pdf_scale_log2", ct.c_int), ("fv_terms", ct.c_int),
        ("schedule", ct.c_int), ("block_x", ct.c_int),
        ("giesekus_alpha", ct.c_double),
        ("fene_L2", ct.c_double),
    ]


ALLOC_FN = ct.CFUNCTYPE(ct.c_void_p, ct.c_size_t, ct.c_void_p, ct.c_void_p)
FREE_FN = ct.CFUNCTYPE(None, ct.c_void_p, ct.c_size_t, ct.c_void_p, ct.c_void_p)

_lock = threading.Lock()
_lib = None


def load(path: str | None = None):
    """Load liblbve.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or os.environ.get("LBVE_LIB") or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"CUDA library {p} is missing; build it with paper_2009_12279_gb300.build.build()")
        L = ct.CDLL(p)
        vp, dp = ct.c_void_p, ct.POINTER(ct.c_double)
        L.lbve_default_params.argtypes = [ct.POINTER(Params)]
        L.lbve_device_bytes.argtypes = [ct.POINTER(Params)]
        L.lbve_device_bytes.restype = ct.c_size_t
        L.lbve_create.argtypes = [ct.POINTER(Params), vp, ct.POINTER(vp)]
        L.lbve_create_with_allocator.argtypes = [ct.POINTER(Params), vp, ALLOC_FN, FREE_FN, vp, ct.POINTER(vp)]
        L.lbve_destroy.argtypes = [vp]
        L.lbve_set_geometry.argtypes = [vp, vp, dp, ct.c_int]
        L.lbve_init_fields.argtypes = [vp, vp, vp, vp]
        L.lbve_init_fields_device.argtypes = [vp, vp, vp, vp]
        L.lbve_probe.argtypes = [vp, vp, ct.c_int, dp]
        L.lbve_add_particle.argtypes = [vp, dp, ct.c_double, ct.c_double, dp, dp, dp, dp, ct.POINTER(ct.c_int)]
        L.lbve_step.argtypes = [vp, ct.c_int]
        L.lbve_read_fields.argtypes = [vp, vp, vp, vp, vp]
        L.lbve_read_fields_device.argtypes = [vp, vp, vp, vp]
        L.lbve_read_pdfs.argtypes = [vp, vp]
        L.lbve_write_pdfs.argtypes = [vp, vp]
        L.lbve_read_particle.argtypes = [vp, ct.c_int, dp]
        L.lbve_read_body_forces.argtypes = [vp, dp]
        L.lbve_read_conversions.argtypes = [vp, dp]
        L.lbve_reduce.argtypes = [vp, dp]
        L.lbve_residual.argtypes = [vp, dp]
        L.lbve_pool_create.argtypes = [ct.c_int, ct.c_size_t, vp, ct.POINTER(vp)]
        L.lbve_pool_destroy.argtypes = [vp]
        L.lbve_pool_fits.argtypes = [vp, ct.POINTER(Params)]
        L.lbve_pool_admit.argtypes = [vp, vp]
        L.lbve_pool_remove.argtypes = [vp, vp]
        L.lbve_pool_step.argtypes = [vp, ct.c_int]
        L.lbve_pool_residuals.argtypes = [vp, dp]
        L.lbve_pool_size.argtypes = [vp]
        L.lbve_pool_bytes_in_use.argtypes = [vp]
        L.lbve_pool_bytes_in_use.restype = ct.c_size_t
        L.lbve_pool_set_graphs.argtypes = [vp, ct.c_int]
        L.lbve_pool_last_error.argtypes = [vp]
        L.lbve_pool_last_error.restype = ct.c_char_p
        L.lbve_step_noalloc.argtypes = [ct.POINTER(Params), vp, vp, vp, vp, dp, ct.c_int, ct.c_longlong, ct.c_int, vp]
        L.lbve_noalloc_last_error.argtypes = []
        L.lbve_noalloc_last_error.restype = ct.c_char_p
        L.lbve_set_kernel_timing.argtypes = [vp, ct.c_int]
        L.lbve_read_kernel_times.argtypes = [vp, dp, ct.POINTER(ct.c_longlong)]
        L.lbve_time.argtypes = [vp]
        L.lbve_time.restype = ct.c_longlong
        L.lbve_synchronize.argtypes = [vp]
        L.lbve_is_unstable.argtypes = [vp]
        L.lbve_stream_collide_kernel.argtypes = [vp]
        L.lbve_stress_kernel.argtypes = [vp]
        L.lbve_set_z_range.argtypes = [vp, ct.c_int, ct.c_int, ct.c_int]
        L.lbve_step_phase.argtypes = [vp, ct.c_int]
        L.lbve_halo_bytes.argtypes = [vp, ct.c_int]
        L.lbve_halo_bytes.restype = ct.c_size_t
        L.lbve_halo_pack.argtypes = [vp, ct.c_int, ct.c_int, vp]
        L.lbve_halo_unpack.argtypes = [vp, ct.c_int, ct.c_int, vp]
        L.lbve_checkpoint_bytes.argtypes = [vp]
        L.lbve_checkpoint_bytes.restype = ct.c_size_t
        L.lbve_save.argtypes = [vp, vp, ct.c_size_t]
        L.lbve_restore.argtypes = [vp, vp, ct.c_size_t]
        L.lbve_last_error.argtypes = [vp]
        L.lbve_last_error.restype = ct.c_char_p
        L.lbve_status_string.argtypes = [ct.c_int]
        L.lbve_status_string.restype = ct.c_char_p
        L.lbve_autotune.argtypes = [vp, ct.c_int, ct.POINTER(Tuning)]
        ip = ct.POINTER(ct.c_int)
        L.lbve_pool_autotune.argtypes = [vp, ct.c_int, ct.c_int, ip, ip, ip, ip, dp, dp]
        p2 = ct.POINTER(Params2D)
        L.lbve2d_default_params.argtypes = [p2]
        L.lbve2d_create.argtypes = [p2, vp, ct.POINTER(vp)]
        L.lbve2d_destroy.argtypes = [vp]
        L.lbve2d_set_geometry.argtypes = [vp, vp, vp]
        L.lbve2d_set_force_field.argtypes = [vp, vp]
        L.lbve2d_init_fields.argtypes = [vp, vp, vp, vp]
        L.lbve2d_step.argtypes = [vp, ct.c_int]
        L.lbve2d_read_fields.argtypes = [vp, vp, vp, vp]
        L.lbve2d_read_pdfs.argtypes = [vp, vp]
        L.lbve2d_time.argtypes = [vp]
        L.lbve2d_time.restype = ct.c_longlong
        L.lbve2d_last_error.argtypes = [vp]
        L.lbve2d_last_error.restype = ct.c_char_p
        _lib = L
        return L


def _dp(a):
    return a.ctypes.data_as(ct.POINTER(ct.c_double))


def _vec3(v):
    return np.ascontiguousarray(np.asarray(v if v is not None else (0.0, 0.0, 0.0), dtype=np.float64).reshape(3))


def default_params() -> Params:
    p = Params()
    load().lbve_default_params(ct.byref(p))
    return p


def make_params(shape, *, periodic=(1, 1, 1), eta=1.0 / 6.0, beta=0.5, lambda_p=1000.0, rho0=1.0,
                body_force=(0.0, 0.0, 0.0), magic=3.0 / 16.0, precision="f32", pdf_scale_log2=-1,
                fv_terms=FV_FLUX | FV_SOURCE, schedule=SCHED_AUTO, block_x=0, giesekus_alpha=0.0,
                fene_L2=0.0) -> Params:
    p = default_params()
    p.nx, p.ny, p.nz = (int(v) for v in shape)
    for a in range(3):
        p.periodic[a] = int(periodic[a])
        p.body_force[a] = float(body_force[a])
    p.eta, p.beta, p.lambda_p, p.rho0, p.magic = float(eta), float(beta), float(lambda_p), float(rho0), float(magic)
    p.pdf_prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    p.pdf_scale_log2, p.fv_terms, p.schedule, p.block_x = int(pdf_scale_log2), int(fv_terms), int(schedule), int(block_x)
    p.giesekus_alpha = float(giesekus_alpha)
    p.fene_L2 = float(fene_L2)
    return p


NOALLOC_MAX_CELLS = 1 << 19


def step_noalloc(params: Params, f_ptr, tau_a_ptr, tau_b_ptr, flags_ptr, wall_vel=(), t0=0, nsteps=1, stream=0):
    """Advance caller-owned device buffers (raw pointers) without device allocation."""
    L = load()
    wv = np.ascontiguousarray(np.asarray(wall_vel, dtype=np.float64).reshape(-1, 3)) if len(wall_vel) else None
    rc = L.lbve_step_noalloc(ct.byref(params), f_ptr, tau_a_ptr, tau_b_ptr, flags_ptr,
                             _dp(wv) if wv is not None else None, 0 if wv is None else wv.shape[0],
                             int(t0), int(nsteps), ct.c_void_p(stream or 0))
    if rc != 0:
        raise LbveError(rc, L.lbve_noalloc_last_error().decode())


def device_bytes(params: Params) -> int:
    return int(load().lbve_device_bytes(ct.byref(params)))


class Solver:
    """One solve on the current CUDA device.  Host arrays are numpy, shape (..., nz, ny, nx)."""

    def __init__(self, shape=None, *, params: Params | None = None, stream: int | None = None,
                 allocator=None, **kw):
        self._L = load()
        self.params = params if params is not None else make_params(shape, **kw)
        self.shape = (self.params.nx, self.params.ny, self.params.nz)
        self.n = self.shape[0] * self.shape[1] * self.shape[2]
        h = ct.c_void_p()
        s = ct.c_void_p(stream or 0)
        self._cb = None
        if allocator is not None:
            alloc, free = allocator
            self._cb = (ALLOC_FN(lambda b, st, u: alloc(int(b), st) or 0),
                        FREE_FN(lambda ptr, b, st, u: free(ptr, int(b), st)))
            rc = self._L.lbve_create_with_allocator(ct.byref(self.params), s, self._cb[0], self._cb[1], None, ct.byref(h))
        else:
            rc = self._L.lbve_create(ct.byref(self.params), s, ct.byref(h))
        if rc != 0:
            raise LbveError(rc, self._L.lbve_last_error(None).decode())
        self._h = h

    # -- plumbing -------------------------------------------------------------
    def _check(self, rc):
        if rc != 0:
            raise LbveError(rc, self._L.lbve_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._L.lbve_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _grid(self, k=None):
        nx, ny, nz = self.shape
        return (nz, ny, nx) if k is None else (k, nz, ny, nx)

    # -- API ------------------------------------------------------------------
    def set_geometry(self, flags, wall_vel=()):
        fl = np.ascontiguousarray(flags, dtype=np.uint8).reshape(self._grid())
        wv = np.ascontiguousarray(np.asarray(wall_vel, dtype=np.float64).reshape(-1, 3)) if len(wall_vel) else None
        self._check(self._L.lbve_set_geometry(self._h, fl.ctypes.data, _dp(wv) if wv is not None else None,
                                              0 if wv is None else wv.shape[0]))

    def init_fields(self, rho=None, u=None, tau=None):
        keep = []

        def ptr(a, k):
            if a is None:
                return None
            a = np.ascontiguousarray(a, dtype=np.float64).reshape(self._grid(k))
            keep.append(a)
            return a.ctypes.data

        self._check(self._L.lbve_init_fields(self._h, ptr(rho, None), ptr(u, 3), ptr(tau, 6)))

    def init_fields_ptr(self, rho_ptr, u_ptr, tau_ptr):
        """Initial fields from host pointers (e.g. pinned buffers); each may be 0."""
        self._check(self._L.lbve_init_fields(self._h, rho_ptr or None, u_ptr or None, tau_ptr or None))

    def init_fields_device(self, rho_ptr=0, u_ptr=0, tau_ptr=0):
        """Initial fields from device pointers (FP64), e.g. torch tensors' data_ptr()."""
        self._check(self._L.lbve_init_fields_device(self._h, rho_ptr or None, u_ptr or None, tau_ptr or None))

    def probe(self, cells) -> np.ndarray:
        """(count, 29): f_0..f_18, rho, u_x, u_y, u_z, tau_xx..tau_yz of the listed cells."""
        idx = np.ascontiguousarray(np.asarray(cells, dtype=np.int64).reshape(-1))
        out = np.zeros((idx.size, 29))
        self._check(self._L.lbve_probe(self._h, idx.ctypes.data, int(idx.size), _dp(out)))
        return out

    def add_particle(self, X, R, rho_p, v=None, w=None, Fext=None, Text=None) -> int:
        pid = ct.c_int(-1)
        self._check(self._L.lbve_add_particle(self._h, _dp(_vec3(X)), float(R), float(rho_p), _dp(_vec3(v)),
                                              _dp(_vec3(w)), _dp(_vec3(Fext)), _dp(_vec3(Text)), ct.byref(pid)))
        return pid.value

    def step(self, n: int = 1):
        self._check(self._L.lbve_step(self._h, int(n)))

    def synchronize(self):
        self._check(self._L.lbve_synchronize(self._h))

    # -- z-slab decomposition (see lbve_set_z_range in include/lbve.h) ------------------
    def set_z_range(self, z_lo: int, z_hi: int, z_origin: int = 0):
        self._check(self._L.lbve_set_z_range(self._h, int(z_lo), int(z_hi), int(z_origin)))

    def step_phase(self, phase: int):
        self._check(self._L.lbve_step_phase(self._h, int(phase)))

    def halo_bytes(self, what: int) -> int:
        return int(self._L.lbve_halo_bytes(self._h, int(what)))

    def halo_pack(self, what: int, side: int, dev_ptr: int):
        self._check(self._L.lbve_halo_pack(self._h, int(what), int(side), ct.c_void_p(dev_ptr)))

    def halo_unpack(self, what: int, side: int, dev_ptr: int):
        self._check(self._L.lbve_halo_unpack(self._h, int(what), int(side), ct.c_void_p(dev_ptr)))

    def save(self) -> bytes:
        """Checkpoint record of the solve's state at this step boundary (lbve_save)."""
        n = int(self._L.lbve_checkpoint_bytes(self._h))
        buf = ct.create_string_buffer(n)
        self._check(self._L.lbve_save(self._h, buf, n))
        return buf.raw

    def restore(self, record: bytes):
        """Overwrite the state from a record of lbve_save (same parameters, geometry and
        particle count; see lbve_restore)."""
        buf = ct.create_string_buffer(record, len(record))
        self._check(self._L.lbve_restore(self._h, buf, len(record)))

    def is_unstable(self) -> bool:
        """True once a stream-collide has flagged rho <= 0, |u|^2 >= 1/3 or a NaN (no sync)."""
        return self._L.lbve_is_unstable(self._h) == 1

    @property
    def stream_collide_kernel(self) -> str:
        """'rows' (row pipeline) or 'cells' (per-cell kernel): see lbve_stream_collide_kernel."""
        return {LB_CELLS: "cells", LB_ROWS: "rows"}[int(self._L.lbve_stream_collide_kernel(self._h))]

    @property
    def stress_kernel(self) -> str:
        """'pairs' (two cells per thread) or 'tiles' (one): see lbve_stress_kernel."""
        return {FV_TILES: "tiles", FV_PAIRS: "pairs"}[int(self._L.lbve_stress_kernel(self._h))]

    @property
    def time(self) -> int:
        return int(self._L.lbve_time(self._h))

    def read_fields(self):
        rho = np.zeros(self._grid())
        u = np.zeros(self._grid(3))
        tau = np.zeros(self._grid(6))
        flags = np.zeros(self._grid(), dtype=np.uint8)
        self._check(self._L.lbve_read_fields(self._h, rho.ctypes.data, u.ctypes.data, tau.ctypes.data, flags.ctypes.data))
        return rho, u, tau, flags

    def read_fields_ptr(self, rho_ptr, u_ptr, tau_ptr, flags_ptr=0):
        self._check(self._L.lbve_read_fields(self._h, rho_ptr or None, u_ptr or None, tau_ptr or None, flags_ptr or None))

    def read_fields_device(self, rho_ptr, u_ptr, tau_ptr):
        self._check(self._L.lbve_read_fields_device(self._h, rho_ptr or None, u_ptr or None, tau_ptr or None))

    def read_pdfs(self) -> np.ndarray:
        f = np.zeros(self._grid(19))
        self._check(self._L.lbve_read_pdfs(self._h, f.ctypes.data))
        return f

    def write_pdfs(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(self._grid(19))
        self._check(self._L.lbve_write_pdfs(self._h, f.ctypes.data))

    def read_particle(self, pid=0) -> dict:
        o = np.zeros(24)
        self._check(self._L.lbve_read_particle(self._h, int(pid), _dp(o)))
        return {"X": o[0:3].copy(), "v": o[3:6].copy(), "w": o[6:9].copy(), "F": o[9:12].copy(),
                "T": o[12:15].copy(), "dP": o[15:18].copy(), "dL": o[18:21].copy(),
                "m": o[21], "I": o[22], "R": o[23]}

    def conversions(self) -> dict:
        o = np.zeros(8)
        self._check(self._L.lbve_read_conversions(self._h, _dp(o)))
        return {"dropped_tau": o[:6].copy(), "destroyed": int(o[6]), "created": int(o[7])}

    def body_forces(self) -> np.ndarray:
        o = np.zeros((256, 3))
        self._check(self._L.lbve_read_body_forces(self._h, _dp(o)))
        return o

    def set_kernel_timing(self, enable: bool = True):
        self._check(self._L.lbve_set_kernel_timing(self._h, int(bool(enable))))

    def kernel_times(self) -> dict:
        """{kind: (total_ms, launches)} of the kernels launched while timing was on."""
        ms = np.zeros(8)
        cnt = (ct.c_longlong * 8)()
        self._check(self._L.lbve_read_kernel_times(self._h, _dp(ms), cnt))
        return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(KERNEL_KINDS) if k and cnt[i] > 0}

    def autotune(self, steps: int = 20) -> dict:
        """Pick the stream-collide block width and stress z-chunk by timing candidates on
        this solve's own steps (it advances by them); see lbve_autotune."""
        t = Tuning()
        self._check(self._L.lbve_autotune(self._h, int(steps), ct.byref(t)))
        return {f: getattr(t, f) for f, _ in Tuning._fields_}

    def residual(self) -> tuple:
        """(|u - u_prev| / |u|, |u|) since the previous call (see lbve_residual)."""
        o = np.zeros(2)
        self._check(self._L.lbve_residual(self._h, _dp(o)))
        return float(o[0]), float(o[1])

    def reduce(self) -> dict:
        o = np.zeros(6)
        self._check(self._L.lbve_reduce(self._h, _dp(o)))
        return {"mass": o[0], "momentum": o[1:4].copy(), "fluid_cells": int(o[4]), "bad": bool(o[5] > 0)}


class Pool:
    """Resident solves stepped together by the batched persistent kernels (lbve_pool_*)."""

    def __init__(self, precision="bf16", budget_bytes=150 * 10**9, stream: int | None = None, graphs=True):
        self._L = load()
        self.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        h = ct.c_void_p()
        rc = self._L.lbve_pool_create(self.precision, int(budget_bytes), ct.c_void_p(stream or 0), ct.byref(h))
        if rc != 0:
            raise LbveError(rc, "pool creation failed")
        self._h = h
        self.members = []
        if not graphs:
            self._L.lbve_pool_set_graphs(self._h, 0)

    def _check(self, rc):
        if rc != 0:
            raise LbveError(rc, self._L.lbve_pool_last_error(self._h).decode())

    def fits(self, params: Params) -> bool:
        return bool(self._L.lbve_pool_fits(self._h, ct.byref(params)))

    def admit(self, solver: "Solver"):
        self._check(self._L.lbve_pool_admit(self._h, solver._h))
        self.members.append(solver)

    def remove(self, solver: "Solver"):
        self._check(self._L.lbve_pool_remove(self._h, solver._h))
        self.members.remove(solver)

    def step(self, n: int = 1):
        self._check(self._L.lbve_pool_step(self._h, int(n)))

    def autotune(self, steps: int = 10, max_classes: int = 64) -> dict:
        """Per-class (by nx) tile widths of the batched kernels, chosen by timing candidates
        on the members' own steps (they advance by them); see lbve_pool_autotune."""
        n = ct.c_int(0)
        nx = (ct.c_int * max_classes)()
        lb = (ct.c_int * max_classes)()
        fv = (ct.c_int * max_classes)()
        before, after = ct.c_double(0.0), ct.c_double(0.0)
        self._check(self._L.lbve_pool_autotune(self._h, int(steps), int(max_classes), ct.byref(n), nx, lb, fv,
                                               ct.byref(before), ct.byref(after)))
        k = min(n.value, max_classes)
        return {"classes": [{"nx": nx[i], "lb_tx": lb[i], "fv_tx": fv[i]} for i in range(k)],
                "ms_per_step_before": before.value, "ms_per_step_after": after.value}

    def residuals(self) -> np.ndarray:
        o = np.zeros((max(len(self.members), 1), 2))
        if self.members:
            self._check(self._L.lbve_pool_residuals(self._h, _dp(o)))
        return o[: len(self.members)]

    @property
    def bytes_in_use(self) -> int:
        return int(self._L.lbve_pool_bytes_in_use(self._h))

    def __len__(self):
        return int(self._L.lbve_pool_size(self._h))

    def close(self):
        if getattr(self, "_h", None):
            self._L.lbve_pool_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Solver2D:
    """One two-dimensional solve (include/lbve2d.h).  Host arrays are numpy, (..., ny, nx)."""

    def __init__(self, shape, *, periodic=(1, 1), eta=1.0 / 6.0, beta=0.5, lambda_p=1000.0, rho0=1.0,
                 body_force=(0.0, 0.0), magic=3.0 / 16.0, precision="f32", fv_terms=FV_FLUX | FV_SOURCE,
                 stream: int | None = None):
        self._L = load()
        p = Params2D()
        self._L.lbve2d_default_params(ct.byref(p))
        p.nx, p.ny = (int(v) for v in shape)
        for a in range(2):
            p.periodic[a] = int(periodic[a])
            p.body_force[a] = float(body_force[a])
        p.eta, p.beta, p.lambda_p, p.rho0, p.magic = float(eta), float(beta), float(lambda_p), float(rho0), float(magic)
        p.pdf_prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        p.fv_terms = int(fv_terms)
        self.params = p
        self.shape = (p.nx, p.ny)
        h = ct.c_void_p()
        rc = self._L.lbve2d_create(ct.byref(p), ct.c_void_p(stream or 0), ct.byref(h))
        if rc != 0:
            raise LbveError(rc, self._L.lbve2d_last_error(None).decode())
        self._h = h

    def _check(self, rc):
        if rc != 0:
            raise LbveError(rc, self._L.lbve2d_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._L.lbve2d_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _grid(self, k=None):
        nx, ny = self.shape
        return (ny, nx) if k is None else (k, ny, nx)

    def _arr(self, a, k):
        return None if a is None else np.ascontiguousarray(a, dtype=np.float64).reshape(self._grid(k))

    def set_geometry(self, flags, ub=None):
        fl = np.ascontiguousarray(flags, dtype=np.uint8).reshape(self._grid())
        u = self._arr(ub, 2)
        self._check(self._L.lbve2d_set_geometry(self._h, fl.ctypes.data, None if u is None else u.ctypes.data))

    def set_force_field(self, F=None):
        a = self._arr(F, 2)
        self._check(self._L.lbve2d_set_force_field(self._h, None if a is None else a.ctypes.data))

    def init_fields(self, rho=None, u=None, tau=None):
        arrs = [self._arr(rho, None), self._arr(u, 2), self._arr(tau, 3)]
        self._check(self._L.lbve2d_init_fields(self._h, *[None if a is None else a.ctypes.data for a in arrs]))

    def step(self, n=1):
        self._check(self._L.lbve2d_step(self._h, int(n)))

    @property
    def time(self) -> int:
        return int(self._L.lbve2d_time(self._h))

    def read_fields(self):
        rho, u, tau = np.zeros(self._grid()), np.zeros(self._grid(2)), np.zeros(self._grid(3))
        self._check(self._L.lbve2d_read_fields(self._h, rho.ctypes.data, u.ctypes.data, tau.ctypes.data))
        return rho, u, tau

    def read_pdfs(self):
        f = np.zeros(self._grid(9))
        self._check(self._L.lbve2d_read_pdfs(self._h, f.ctypes.data))
        return f
