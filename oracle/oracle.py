"""Python handle on the FP64 CPU oracle (``lbve_oracle.c``).

TEST INFRASTRUCTURE ONLY.  The oracle is the plain reference that the CUDA library
is checked against; only the tests, the package smoke check and the benchmark's
CPU-baseline leg may import this module.  It shares no code with the CUDA path.
"""
from __future__ import annotations

import ctypes as ct
import fcntl
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "lbve_oracle.c")
LIB = os.path.join(HERE, "liblbve_oracle.so")
SRC2D = os.path.join(HERE, "lbve2d_oracle.c")
LIB2D = os.path.join(HERE, "liblbve2d_oracle.so")

FLUID, NOSLIP, WALL0, PART0 = 0, 1, 2, 64
FV_FLUX, FV_SOURCE = 1, 2
FV_CTU, FV_DIVU = 4, 8  # variants: transverse CTU overlap on the face fluxes; tau div(u) source

_lock = threading.Lock()
_lib = None


def _fresh() -> bool:
    def ok(lib, src, hdr):
        return os.path.exists(lib) and os.path.getmtime(lib) >= max(os.path.getmtime(src),
                                                                     os.path.getmtime(os.path.join(HERE, hdr)))
    return ok(LIB, SRC, "lbve_oracle.h") and ok(LIB2D, SRC2D, "lbve2d_oracle.h")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP contraction off so that a*b+c is never fused)."""
    if not force and _fresh():
        return LIB
    with open(LIB + ".lock", "w") as lk:
        fcntl.flock(lk, fcntl.LOCK_EX)
        try:
            if not force and _fresh():
                return LIB
            return _compile()
        finally:
            fcntl.flock(lk, fcntl.LOCK_UN)


def _compile() -> str:
    for src, lib in ((SRC, LIB), (SRC2D, LIB2D)):
        tmp = lib + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off", "-fopenmp",
               src, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, lib)
    return LIB


class _Params(ct.Structure):
    _fields_ = [
        ("nx", ct.c_int), ("ny", ct.c_int), ("nz", ct.c_int),
        ("periodic", ct.c_int * 3),
        ("eta", ct.c_double), ("beta", ct.c_double), ("lambda_p", ct.c_double), ("rho0", ct.c_double),
        ("g", ct.c_double * 3),
        ("magic", ct.c_double),
        ("n_wall", ct.c_int),
        ("wall_vel", (ct.c_double * 3) * 16),
        ("fv_terms", ct.c_int),
        ("giesekus_alpha", ct.c_double),
        ("fene_L2", ct.c_double),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            # a test may point this at a deliberately mutated copy of the oracle
            path = os.environ.get("LBVE_ORACLE_LIB") or build()
            L = ct.CDLL(path)
            dp = ct.POINTER(ct.c_double)
            L.orc_create.restype = ct.c_void_p
            L.orc_create.argtypes = [ct.POINTER(_Params)]
            L.orc_destroy.argtypes = [ct.c_void_p]
            L.orc_set_flags.argtypes = [ct.c_void_p, ct.c_void_p]
            L.orc_init_fields.argtypes = [ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p]
            L.orc_add_particle.argtypes = [ct.c_void_p, dp, ct.c_double, ct.c_double, dp, dp, dp, dp]
            L.orc_set_particle.argtypes = [ct.c_void_p, ct.c_int, dp, dp, dp]
            L.orc_step.argtypes = [ct.c_void_p, ct.c_int]
            L.orc_time.argtypes = [ct.c_void_p]
            L.orc_time.restype = ct.c_long
            L.orc_read_fields.argtypes = [ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p]
            L.orc_read_pdfs.argtypes = [ct.c_void_p, ct.c_void_p]
            L.orc_write_pdfs.argtypes = [ct.c_void_p, ct.c_void_p]
            L.orc_write_tau.argtypes = [ct.c_void_p, ct.c_void_p]
            L.orc_read_particle.argtypes = [ct.c_void_p, ct.c_int, dp]
            L.orc_read_body_forces.argtypes = [ct.c_void_p, dp]
            L.orc_read_diag.argtypes = [ct.c_void_p, dp]
            L.orc_rates.argtypes = [ct.c_void_p, dp]
            L.orc_lattice.argtypes = [ct.c_void_p, dp, ct.c_void_p]
            L.orc_equilibrium.argtypes = [ct.c_double, dp, dp]
            L.orc_forcing.argtypes = [dp, dp, ct.c_double, ct.c_double, dp]
            L.orc_collide.argtypes = [dp, dp, ct.c_double, ct.c_double, dp]
            L.orc_source.argtypes = [dp, dp, ct.c_double, ct.c_double, dp]
            L.orc_fene_stress.argtypes = [dp, ct.c_double, ct.c_double, ct.c_double, dp]
            L.orc_fene_conformation.argtypes = [dp, ct.c_double, ct.c_double, ct.c_double, dp]
            L.orc_polymer_force_field.argtypes = [ct.c_void_p, ct.c_void_p]
            L.orc_velocity_field.argtypes = [ct.c_void_p, ct.c_void_p]
            L.orc_fv_update_field.argtypes = [ct.c_void_p, ct.c_void_p, ct.c_void_p]
            L.orc_fill_drain.argtypes = [ct.c_void_p]
            _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ct.POINTER(ct.c_double))


def _vec3(v):
    return np.ascontiguousarray(np.asarray(v if v is not None else (0.0, 0.0, 0.0), dtype=np.float64))


def lattice():
    """(c[19,3] int, w[19], opp[19]) of the D3Q19 set."""
    c = np.zeros((19, 3), dtype=np.int32)
    w = np.zeros(19)
    opp = np.zeros(19, dtype=np.int32)
    lib().orc_lattice(c.ctypes.data, _dp(w), opp.ctypes.data)
    return c.astype(np.int64), w, opp.astype(np.int64)


def equilibrium(rho: float, u) -> np.ndarray:
    out = np.zeros(19)
    lib().orc_equilibrium(float(rho), _dp(_vec3(u)), _dp(out))
    return out


def forcing(u, F, omega_p: float, omega_m: float) -> np.ndarray:
    out = np.zeros(19)
    lib().orc_forcing(_dp(_vec3(u)), _dp(_vec3(F)), float(omega_p), float(omega_m), _dp(out))
    return out


def collide(f, F, omega_p: float, omega_m: float) -> np.ndarray:
    f = np.ascontiguousarray(np.asarray(f, dtype=np.float64))
    out = np.zeros(19)
    lib().orc_collide(_dp(f), _dp(_vec3(F)), float(omega_p), float(omega_m), _dp(out))
    return out


def source(tau6, G, ep_l: float, inv_l: float) -> np.ndarray:
    """S of Eq. (source); G[k, j] = d_k u_j."""
    t = np.ascontiguousarray(np.asarray(tau6, dtype=np.float64))
    g = np.ascontiguousarray(np.asarray(G, dtype=np.float64).reshape(9))
    out = np.zeros(6)
    lib().orc_source(_dp(t), _dp(g), float(ep_l), float(inv_l), _dp(out))
    return out


def fene_stress(A6, eta_p, lambda_p, L2):
    a = np.ascontiguousarray(np.asarray(A6, dtype=np.float64))
    out = np.zeros(6)
    lib().orc_fene_stress(_dp(a), float(eta_p), float(lambda_p), float(L2), _dp(out))
    return out


def fene_conformation(tau6, eta_p, lambda_p, L2):
    t = np.ascontiguousarray(np.asarray(tau6, dtype=np.float64))
    out = np.zeros(6)
    lib().orc_fene_conformation(_dp(t), float(eta_p), float(lambda_p), float(L2), _dp(out))
    return out


class Oracle:
    """One solve held by the CPU oracle.  Arrays are numpy, shape (..., nz, ny, nx)."""

    def __init__(self, shape, *, periodic=(1, 1, 1), eta=1.0 / 6.0, beta=0.5, lambda_p=3000.0,
                 rho0=1.0, g=(0.0, 0.0, 0.0), magic=3.0 / 16.0, wall_vel=(), fv_terms=FV_FLUX | FV_SOURCE,
                 giesekus_alpha=0.0, fene_L2=0.0):
        nx, ny, nz = (int(v) for v in shape)
        p = _Params()
        p.nx, p.ny, p.nz = nx, ny, nz
        for a in range(3):
            p.periodic[a] = int(periodic[a])
            p.g[a] = float(g[a])
        p.eta, p.beta, p.lambda_p, p.rho0, p.magic = float(eta), float(beta), float(lambda_p), float(rho0), float(magic)
        p.n_wall = len(wall_vel)
        for k, v in enumerate(wall_vel):
            for a in range(3):
                p.wall_vel[k][a] = float(v[a])
        p.fv_terms = int(fv_terms)
        p.giesekus_alpha = float(giesekus_alpha)
        p.fene_L2 = float(fene_L2)
        self._p = p
        self.shape = (nx, ny, nz)
        self.n = nx * ny * nz
        self._h = lib().orc_create(ct.byref(p))
        if not self._h:
            raise ValueError("oracle rejected the parameters")

    def close(self):
        if getattr(self, "_h", None):
            lib().orc_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def _grid(self, k=None):
        nx, ny, nz = self.shape
        return (nz, ny, nx) if k is None else (k, nz, ny, nx)

    def set_flags(self, flags: np.ndarray):
        fl = np.ascontiguousarray(flags, dtype=np.uint8).reshape(self._grid())
        rc = lib().orc_set_flags(self._h, fl.ctypes.data)
        if rc != 0:
            raise ValueError(f"oracle rejected the flag field ({rc})")

    def init_fields(self, rho=None, u=None, tau=None):
        keep = []

        def ptr(a, k):
            if a is None:
                return None
            a = np.ascontiguousarray(a, dtype=np.float64).reshape(self._grid(k))
            keep.append(a)
            return a.ctypes.data

        lib().orc_init_fields(self._h, ptr(rho, None), ptr(u, 3), ptr(tau, 6))

    def add_particle(self, X, R, rho_p, v=None, w=None, Fext=None, Text=None) -> int:
        pid = lib().orc_add_particle(self._h, _dp(_vec3(X)), float(R), float(rho_p), _dp(_vec3(v)),
                                     _dp(_vec3(w)), _dp(_vec3(Fext)), _dp(_vec3(Text)))
        if pid < 0:
            raise ValueError("oracle rejected the particle")
        return pid

    def set_particle(self, pid, X=None, v=None, w=None):
        args = [(_dp(_vec3(a)) if a is not None else None) for a in (X, v, w)]
        lib().orc_set_particle(self._h, int(pid), *args)

    def step(self, n: int = 1):
        lib().orc_step(self._h, int(n))

    @property
    def time(self) -> int:
        return int(lib().orc_time(self._h))

    def read_fields(self):
        rho = np.zeros(self._grid())
        u = np.zeros(self._grid(3))
        tau = np.zeros(self._grid(6))
        flags = np.zeros(self._grid(), dtype=np.uint8)
        lib().orc_read_fields(self._h, rho.ctypes.data, u.ctypes.data, tau.ctypes.data, flags.ctypes.data)
        return rho, u, tau, flags

    def read_pdfs(self) -> np.ndarray:
        f = np.zeros(self._grid(19))
        lib().orc_read_pdfs(self._h, f.ctypes.data)
        return f

    def write_pdfs(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(self._grid(19))
        lib().orc_write_pdfs(self._h, f.ctypes.data)

    def write_tau(self, tau):
        """Overwrite the stored tensor (the stress; the conformation A in FENE-P mode)."""
        t = np.ascontiguousarray(tau, dtype=np.float64).reshape(self._grid(6))
        lib().orc_write_tau(self._h, t.ctypes.data)

    def read_particle(self, pid=0) -> dict:
        o = np.zeros(24)
        if lib().orc_read_particle(self._h, int(pid), _dp(o)) != 0:
            raise IndexError(pid)
        return {"X": o[0:3].copy(), "v": o[3:6].copy(), "w": o[6:9].copy(), "F": o[9:12].copy(),
                "T": o[12:15].copy(), "dP": o[15:18].copy(), "dL": o[18:21].copy(),
                "m": o[21], "I": o[22], "R": o[23]}

    def body_forces(self) -> np.ndarray:
        o = np.zeros((256, 3))
        lib().orc_read_body_forces(self._h, _dp(o))
        return o

    def diag(self) -> dict:
        o = np.zeros(8)
        lib().orc_read_diag(self._h, _dp(o))
        return {"dropped_tau": o[:6].copy(), "destroyed": int(o[6]), "created": int(o[7])}

    def rates(self) -> dict:
        o = np.zeros(5)
        lib().orc_rates(self._h, _dp(o))
        return {"omega_p": o[0], "omega_m": o[1], "eta_p": o[2], "ep_l": o[3], "inv_l": o[4]}

    def polymer_force(self) -> np.ndarray:
        o = np.zeros(self._grid(3))
        lib().orc_polymer_force_field(self._h, o.ctypes.data)
        return o

    def velocity(self) -> np.ndarray:
        o = np.zeros(self._grid(3))
        lib().orc_velocity_field(self._h, o.ctypes.data)
        return o

    def fv_update(self, u) -> np.ndarray:
        uu = np.ascontiguousarray(u, dtype=np.float64).reshape(self._grid(3))
        o = np.zeros(self._grid(6))
        lib().orc_fv_update_field(self._h, uu.ctypes.data, o.ctypes.data)
        return o

    def fill_drain(self):
        lib().orc_fill_drain(self._h)


# ---------------------------------------------------------------------------------
# two-dimensional form (D2Q9 lattice Boltzmann, D2Q5 finite-volume stress)
# ---------------------------------------------------------------------------------
class _Params2D(ct.Structure):
    _fields_ = [
        ("nx", ct.c_int), ("ny", ct.c_int), ("periodic", ct.c_int * 2),
        ("eta", ct.c_double), ("beta", ct.c_double), ("lambda_p", ct.c_double), ("rho0", ct.c_double),
        ("g", ct.c_double * 2), ("magic", ct.c_double), ("fv_terms", ct.c_int),
    ]


_lib2d = None


def lib2d():
    global _lib2d
    with _lock:
        if _lib2d is None:
            build()
            L = ct.CDLL(os.environ.get("LBVE_ORACLE2D_LIB") or LIB2D)
            vp = ct.c_void_p
            L.orc2_create.restype = vp
            L.orc2_create.argtypes = [ct.POINTER(_Params2D)]
            L.orc2_destroy.argtypes = [vp]
            L.orc2_set_flags.argtypes = [vp, vp, vp]
            L.orc2_set_force.argtypes = [vp, vp]
            L.orc2_init_fields.argtypes = [vp, vp, vp, vp]
            L.orc2_step.argtypes = [vp, ct.c_int]
            L.orc2_time.argtypes = [vp]
            L.orc2_time.restype = ct.c_long
            L.orc2_read_fields.argtypes = [vp, vp, vp, vp]
            L.orc2_read_pdfs.argtypes = [vp, vp]
            L.orc2_write_pdfs.argtypes = [vp, vp]
            L.orc2_write_tau.argtypes = [vp, vp]
            L.orc2_lattice.argtypes = [vp, vp, vp]
            L.orc2_fv_update_field.argtypes = [vp, vp, vp]
            _lib2d = L
    return _lib2d


def lattice2d():
    """(c[9,2] int, w[9], opp[9]) of the D2Q9 set."""
    c = np.zeros((9, 2), dtype=np.int32)
    w = np.zeros(9)
    opp = np.zeros(9, dtype=np.int32)
    lib2d().orc2_lattice(c.ctypes.data, w.ctypes.data, opp.ctypes.data)
    return c.astype(np.int64), w, opp.astype(np.int64)


class Oracle2D:
    """One two-dimensional solve held by the CPU oracle.  Arrays (..., ny, nx)."""

    def __init__(self, shape, *, periodic=(1, 1), eta=1.0 / 6.0, beta=0.5, lambda_p=3000.0, rho0=1.0,
                 g=(0.0, 0.0), magic=3.0 / 16.0, fv_terms=FV_FLUX | FV_SOURCE):
        p = _Params2D()
        p.nx, p.ny = (int(v) for v in shape)
        for a in range(2):
            p.periodic[a] = int(periodic[a])
            p.g[a] = float(g[a])
        p.eta, p.beta, p.lambda_p, p.rho0, p.magic = float(eta), float(beta), float(lambda_p), float(rho0), float(magic)
        p.fv_terms = int(fv_terms)
        self.shape = (p.nx, p.ny)
        self._h = lib2d().orc2_create(ct.byref(p))
        if not self._h:
            raise ValueError("oracle rejected the parameters")

    def close(self):
        if getattr(self, "_h", None):
            lib2d().orc2_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def _grid(self, k=None):
        nx, ny = self.shape
        return (ny, nx) if k is None else (k, ny, nx)

    def set_geometry(self, flags, ub=None):
        fl = np.ascontiguousarray(flags, dtype=np.uint8).reshape(self._grid())
        u = None if ub is None else np.ascontiguousarray(ub, dtype=np.float64).reshape(self._grid(2))
        if lib2d().orc2_set_flags(self._h, fl.ctypes.data, None if u is None else u.ctypes.data) != 0:
            raise ValueError("oracle rejected the flag field")

    def set_force(self, F=None):
        a = None if F is None else np.ascontiguousarray(F, dtype=np.float64).reshape(self._grid(2))
        lib2d().orc2_set_force(self._h, None if a is None else a.ctypes.data)

    def init_fields(self, rho=None, u=None, tau=None):
        keep = [None if a is None else np.ascontiguousarray(a, dtype=np.float64).reshape(self._grid(k))
                for a, k in ((rho, None), (u, 2), (tau, 3))]
        lib2d().orc2_init_fields(self._h, *[None if a is None else a.ctypes.data for a in keep])

    def step(self, n=1):
        lib2d().orc2_step(self._h, int(n))

    @property
    def time(self):
        return int(lib2d().orc2_time(self._h))

    def read_fields(self):
        rho, u, tau = np.zeros(self._grid()), np.zeros(self._grid(2)), np.zeros(self._grid(3))
        lib2d().orc2_read_fields(self._h, rho.ctypes.data, u.ctypes.data, tau.ctypes.data)
        return rho, u, tau

    def read_pdfs(self):
        f = np.zeros(self._grid(9))
        lib2d().orc2_read_pdfs(self._h, f.ctypes.data)
        return f

    def write_pdfs(self, f):
        a = np.ascontiguousarray(f, dtype=np.float64).reshape(self._grid(9))
        lib2d().orc2_write_pdfs(self._h, a.ctypes.data)

    def write_tau(self, tau):
        a = np.ascontiguousarray(tau, dtype=np.float64).reshape(self._grid(3))
        lib2d().orc2_write_tau(self._h, a.ctypes.data)

    def fv_update(self, u):
        uu = np.ascontiguousarray(u, dtype=np.float64).reshape(self._grid(2))
        o = np.zeros(self._grid(3))
        lib2d().orc2_fv_update_field(self._h, uu.ctypes.data, o.ctypes.data)
        return o
