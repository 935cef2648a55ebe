"""Plain FP64 CPU oracle for the two-range pseudopotential lattice Boltzmann
method (Fei et al., arXiv:1806.06943).

TEST INFRASTRUCTURE ONLY: the test suite, the package smoke check and the
benchmark's CPU-baseline leg are the only callers.  The method itself lives in
``oracle.c`` (no fused multiply-add, libm ``exp``; the row loops of a time
step optionally on several OpenMP threads, with results bitwise those of one
thread); this file
compiles it with the host C compiler and marshals arguments through ctypes.
It shares no code with the CUDA path.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-ffp-contract=off", "-std=c99", "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (only when stale), with
    OpenMP where the compiler offers it (the row loops may then run on several
    threads, with bitwise the same results), else without."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cc = os.environ.get("CC", "cc")
        r = subprocess.run([cc, *CFLAGS, "-fopenmp", _SRC, "-o", tmp, "-lm"], capture_output=True, text=True)
        if r.returncode != 0:
            subprocess.run([cc, *CFLAGS, _SRC, "-o", tmp, "-lm"], check=True)
        os.replace(tmp, _LIB)
    return _LIB


def set_threads(n: int = 0) -> int:
    """Threads of the oracle's row loops (n <= 0: keep); returns the count in
    use, 1 when built without OpenMP."""
    return int(_load().orc_set_threads(int(n)))


class OrcParams(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("tau", ctypes.c_double * 2),
        ("G_AB", ctypes.c_double), ("G1", ctypes.c_double), ("G2", ctypes.c_double),
        ("g", ctypes.c_double * 2),
        ("walls", ctypes.c_int32), ("wall_mode", ctypes.c_int32),
        ("wall_rho", ctypes.c_double * 2),
        ("forcing", ctypes.c_int32), ("pad", ctypes.c_int32),
    ]


class Orc3Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32), ("pad", ctypes.c_int32),
        ("tau", ctypes.c_double * 2),
        ("G_AB", ctypes.c_double), ("G1", ctypes.c_double), ("G2", ctypes.c_double),
        ("g", ctypes.c_double * 3),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.POINTER
            d = ctypes.c_double
            dp = P(d)
            lib.orc_create.restype = ctypes.c_void_p
            lib.orc_create.argtypes = [P(OrcParams)]
            lib.orc_destroy.argtypes = [ctypes.c_void_p]
            lib.orc_step.argtypes = [ctypes.c_void_p, ctypes.c_long]
            lib.orc_time.restype = ctypes.c_long
            lib.orc_time.argtypes = [ctypes.c_void_p]
            lib.orc_set_fields.argtypes = [ctypes.c_void_p, dp, dp]
            lib.orc_get_f.argtypes = [ctypes.c_void_p, dp]
            lib.orc_set_f.argtypes = [ctypes.c_void_p, dp, ctypes.c_long]
            lib.orc_fields.argtypes = [ctypes.c_void_p, dp, dp, dp, dp, dp]
            lib.orc_observables.argtypes = [ctypes.c_void_p, d, d, d, dp]
            lib.orc_psi.restype = d
            lib.orc_psi.argtypes = [d]
            lib.orc_equilibrium.argtypes = [d, d, d, dp]
            lib.orc_guo.argtypes = [d, d, d, d, d, dp]
            lib.orc_tables.argtypes = [dp, P(ctypes.c_int32), P(ctypes.c_int32), dp,
                                       P(ctypes.c_int32), P(ctypes.c_int32)]
            lib.orc_shift_forcing.argtypes = [d, d, d, d, d, d, dp]
            lib.orc_pressure_tensor.argtypes = [ctypes.c_void_p, dp]
            lib.orc3_create.restype = ctypes.c_void_p
            lib.orc3_create.argtypes = [P(Orc3Params)]
            lib.orc3_destroy.argtypes = [ctypes.c_void_p]
            lib.orc3_step.argtypes = [ctypes.c_void_p, ctypes.c_long]
            lib.orc3_set_fields.argtypes = [ctypes.c_void_p, dp, dp]
            lib.orc3_get_f.argtypes = [ctypes.c_void_p, dp]
            lib.orc3_fields.argtypes = [ctypes.c_void_p, dp, dp, dp]
            lib.orc3_observables.argtypes = [ctypes.c_void_p, d, d, d, d, dp]
            lib.orc3_tables.argtypes = [dp, P(ctypes.c_int32), dp]
            lib.orc_set_threads.restype = ctypes.c_int
            lib.orc_set_threads.argtypes = [ctypes.c_int]
            lib.orc_bulk_pressure.restype = d
            lib.orc_bulk_pressure.argtypes = [P(OrcParams), d, d]
            _lib = lib
    return _lib


def _dptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


FORCING_GUO, FORCING_SHIFT = 0, 1


def make_params(nx, ny, tau=(1.0, 1.0), G_AB=3.0, G1=-7.4, G2=6.4, g=(0.0, 0.0),
                walls=0, wall_mode=0, wall_rho=(0.0, 0.0), forcing=FORCING_GUO) -> OrcParams:
    p = OrcParams()
    p.nx, p.ny = int(nx), int(ny)
    p.tau[0], p.tau[1] = float(tau[0]), float(tau[1])
    p.G_AB, p.G1, p.G2 = float(G_AB), float(G1), float(G2)
    p.g[0], p.g[1] = float(g[0]), float(g[1])
    p.walls, p.wall_mode = int(walls), int(wall_mode)
    p.wall_rho[0], p.wall_rho[1] = float(wall_rho[0]), float(wall_rho[1])
    p.forcing = int(forcing)
    return p


OBS_KEYS = ("massA", "massB", "momAx", "momAy", "momBx", "momBy", "Q", "mu_r",
            "dp", "R_eff", "umax", "finite")


class OracleSim:
    """One lattice advanced by the oracle.  Populations are [2][9][ny][nx]."""

    def __init__(self, nx, ny, **kw):
        self.lib = _load()
        self.params = make_params(nx, ny, **kw)
        self.nx, self.ny = int(nx), int(ny)
        self.h = self.lib.orc_create(ctypes.byref(self.params))
        if not self.h:
            raise ValueError("oracle rejected the parameters")

    def close(self):
        if self.h:
            self.lib.orc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def t(self) -> int:
        return self.lib.orc_time(self.h)

    def set_fields(self, rho: np.ndarray, u: np.ndarray | None = None):
        rho = np.ascontiguousarray(rho, dtype=np.float64)
        assert rho.shape == (2, self.ny, self.nx)
        up = None
        if u is not None:
            u = np.ascontiguousarray(u, dtype=np.float64)
            assert u.shape == (2, self.ny, self.nx)
            up = _dptr(u)
        self.lib.orc_set_fields(self.h, _dptr(rho), up)

    def step(self, n: int = 1):
        self.lib.orc_step(self.h, int(n))

    def get_f(self) -> np.ndarray:
        f = np.empty((2, 9, self.ny, self.nx))
        self.lib.orc_get_f(self.h, _dptr(f))
        return f

    def set_f(self, f: np.ndarray, t: int = 0):
        f = np.ascontiguousarray(f, dtype=np.float64)
        assert f.shape == (2, 9, self.ny, self.nx)
        self.lib.orc_set_f(self.h, _dptr(f), int(t))

    def fields(self) -> dict:
        n = (self.ny, self.nx)
        rho = np.empty((2,) + n)
        mom = np.empty((2, 2) + n)
        force = np.empty((2, 2) + n)
        ueq = np.empty((2,) + n)
        ubar = np.empty((2,) + n)
        self.lib.orc_fields(self.h, _dptr(rho), _dptr(mom), _dptr(force), _dptr(ueq), _dptr(ubar))
        return {"rho": rho, "mom": mom, "force": force, "ueq": ueq, "ubar": ubar}

    def pressure_tensor(self) -> np.ndarray:
        """[2][3][ny][nx]: kinetic and interaction parts (Eqs. 10, 13), xx, yy, xy."""
        out = np.empty((2, 3, self.ny, self.nx))
        self.lib.orc_pressure_tensor(self.h, _dptr(out))
        return out

    def observables(self, probe=(0.0, 0.0, 0.0)) -> dict:
        out = np.empty(12)
        cx, cy, R = probe
        self.lib.orc_observables(self.h, float(cx), float(cy), float(R), _dptr(out))
        return dict(zip(OBS_KEYS, out.tolist()))


def equilibrium(rho, ux, uy) -> np.ndarray:
    out = np.empty(9)
    _load().orc_equilibrium(float(rho), float(ux), float(uy), _dptr(out))
    return out


def guo(tau, ux, uy, Fx, Fy) -> np.ndarray:
    out = np.empty(9)
    _load().orc_guo(float(tau), float(ux), float(uy), float(Fx), float(Fy), _dptr(out))
    return out


def shift_forcing(tau, rho, ux, uy, Fx, Fy) -> np.ndarray:
    out = np.empty(9)
    _load().orc_shift_forcing(float(tau), float(rho), float(ux), float(uy), float(Fx), float(Fy), _dptr(out))
    return out


def psi(rho) -> float:
    return _load().orc_psi(float(rho))


def bulk_pressure(params: OrcParams, rhoA, rhoB) -> float:
    return _load().orc_bulk_pressure(ctypes.byref(params), float(rhoA), float(rhoB))


def tables() -> dict:
    w = np.empty(9)
    ex = np.empty(9, np.int32)
    ey = np.empty(9, np.int32)
    p = np.empty(25)
    jx = np.empty(25, np.int32)
    jy = np.empty(25, np.int32)
    I = ctypes.POINTER(ctypes.c_int32)
    _load().orc_tables(_dptr(w), ex.ctypes.data_as(I), ey.ctypes.data_as(I), _dptr(p),
                       jx.ctypes.data_as(I), jy.ctypes.data_as(I))
    return {"w": w, "ex": ex, "ey": ey, "p": p, "jx": jx, "jy": jy}


def disjoining_pressure(h, s) -> np.ndarray:
    """Disjoining pressure of Eq. (18), Pi(h) = s(h)/h - int_h^inf s(t)/t^2 dt,
    from samples s(h_i) = gamma_f(h_i) - 2 gamma (Eq. 17) at increasing h_i:
    the integral by the trapezoid rule over the samples, s taken as zero
    beyond the last one (the boundary condition Pi(inf) = 0)."""
    h = np.asarray(h, dtype=np.float64)
    s = np.asarray(s, dtype=np.float64)
    g = s / (h * h)
    out = np.empty_like(h)
    for i in range(len(h)):
        tail = 0.0
        for j in range(i, len(h) - 1):
            tail += 0.5 * (g[j] + g[j + 1]) * (h[j + 1] - h[j])
        out[i] = s[i] / h[i] - tail
    return out


OBS3_KEYS = ("massA", "massB", "momAx", "momAy", "momAz", "momBx", "momBy", "momBz", "dp", "R_eff", "umax",
             "finite")


class OracleSim3:
    """The 3-D extension (D3Q19, 5^3 mid-range stencil), periodic in x, y, z.
    Fields are [..][nz][ny][nx], populations [2][19][nz][ny][nx]."""

    def __init__(self, nx, ny, nz, tau=(1.0, 1.0), G_AB=3.0, G1=-7.4, G2=6.4, g=(0.0, 0.0, 0.0)):
        self.lib = _load()
        p = Orc3Params()
        p.nx, p.ny, p.nz = int(nx), int(ny), int(nz)
        p.tau[0], p.tau[1] = float(tau[0]), float(tau[1])
        p.G_AB, p.G1, p.G2 = float(G_AB), float(G1), float(G2)
        for a in range(3):
            p.g[a] = float(g[a])
        self.params = p
        self.shape = (int(nz), int(ny), int(nx))
        self.h = self.lib.orc3_create(ctypes.byref(p))
        if not self.h:
            raise ValueError("oracle rejected the parameters")

    def close(self):
        if self.h:
            self.lib.orc3_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_fields(self, rho, u=None):
        rho = np.ascontiguousarray(rho, dtype=np.float64)
        assert rho.shape == (2,) + self.shape
        up = None
        if u is not None:
            u = np.ascontiguousarray(u, dtype=np.float64)
            assert u.shape == (3,) + self.shape
            up = _dptr(u)
        self.lib.orc3_set_fields(self.h, _dptr(rho), up)

    def step(self, n=1):
        self.lib.orc3_step(self.h, int(n))

    def get_f(self):
        f = np.empty((2, 19) + self.shape)
        self.lib.orc3_get_f(self.h, _dptr(f))
        return f

    def fields(self):
        rho = np.empty((2,) + self.shape)
        force = np.empty((2, 3) + self.shape)
        ubar = np.empty((3,) + self.shape)
        self.lib.orc3_fields(self.h, _dptr(rho), _dptr(force), _dptr(ubar))
        return {"rho": rho, "force": force, "ubar": ubar}

    def observables(self, probe=(0.0, 0.0, 0.0, 0.0)):
        out = np.empty(12)
        cx, cy, cz, R = probe
        self.lib.orc3_observables(self.h, float(cx), float(cy), float(cz), float(R), _dptr(out))
        return dict(zip(OBS3_KEYS, out.tolist()))


def tables3() -> dict:
    w = np.empty(19)
    e = np.empty(57, np.int32)
    q = np.empty(13)
    _load().orc3_tables(_dptr(w), e.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _dptr(q))
    return {"w": w, "e": e.reshape(19, 3), "q": q}
