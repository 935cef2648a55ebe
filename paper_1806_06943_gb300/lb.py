"""ctypes binding of the C-ABI in include/lb.h (argument marshalling only).

Every function of the header is bound under the same name on the module
object ``LIB``; the classes ``Lattice`` and ``Batch`` wrap a handle and turn
error codes into ``LBError``.  Host arrays are numpy float64 in the header's
layouts; device arrays may be torch CUDA tensors (float64, contiguous), whose
data pointers are passed through unchanged.  The library must have been built
(``paper_1806_06943_gb300.build.build()``); there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "liblb.so")
HEADER = os.path.join(os.path.dirname(_PKG), "include", "lb.h")

LB_OK, LB_EINVAL, LB_ENOMEM, LB_ECUDA, LB_EUNSTABLE, LB_ETIMEOUT = 0, -1, -2, -3, -4, -5
LB_FP64, LB_FP32 = 0, 1
LB_PERIODIC, LB_WALLS_Y = 0, 1
LB_WALL_MIRROR, LB_WALL_FIXED = 0, 1
LB_STATIC_MAX_TILES = 32768
LB_MODE_LAUNCH, LB_MODE_PERSISTENT, LB_MODE_FUSED, LB_MODE_TMA = 0, 1, 2, 3
LB_OBJ_MU_R, LB_OBJ_DP = 0, 1
LB_FORCING_GUO, LB_FORCING_SHIFT = 0, 1


class LBError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"lb error {code}: {msg}")
        self.code = code


class lb_params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("tau", ctypes.c_double * 2),
        ("G_AB", ctypes.c_double), ("G1", ctypes.c_double), ("G2", ctypes.c_double),
        ("g", ctypes.c_double * 2),
        ("walls", ctypes.c_int32), ("wall_mode", ctypes.c_int32),
        ("wall_rho", ctypes.c_double * 2),
        ("precision", ctypes.c_int32), ("forcing", ctypes.c_int32),
        ("stream", ctypes.c_void_p),
    ]


class lb_obs(ctypes.Structure):
    _fields_ = [
        ("t", ctypes.c_int64),
        ("mass", ctypes.c_double * 2),
        ("mom", (ctypes.c_double * 2) * 2),
        ("flux_Q", ctypes.c_double), ("mu_r", ctypes.c_double),
        ("dp_laplace", ctypes.c_double), ("R_eff", ctypes.c_double),
        ("umax", ctypes.c_double),
        ("finite", ctypes.c_int32), ("reserved", ctypes.c_int32),
    ]

    def to_dict(self) -> dict:
        return {
            "t": self.t, "massA": self.mass[0], "massB": self.mass[1],
            "momAx": self.mom[0][0], "momAy": self.mom[0][1], "momBx": self.mom[1][0], "momBy": self.mom[1][1],
            "Q": self.flux_Q, "mu_r": self.mu_r, "dp": self.dp_laplace, "R_eff": self.R_eff,
            "umax": self.umax, "finite": float(self.finite),
        }


class lb3_params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32), ("precision", ctypes.c_int32),
        ("tau", ctypes.c_double * 2),
        ("G_AB", ctypes.c_double), ("G1", ctypes.c_double), ("G2", ctypes.c_double),
        ("g", ctypes.c_double * 3),
        ("stream", ctypes.c_void_p),
    ]


class lb3_obs(ctypes.Structure):
    _fields_ = [
        ("t", ctypes.c_int64),
        ("mass", ctypes.c_double * 2),
        ("mom", (ctypes.c_double * 3) * 2),
        ("dp_laplace", ctypes.c_double), ("R_eff", ctypes.c_double), ("umax", ctypes.c_double),
        ("finite", ctypes.c_int32), ("reserved", ctypes.c_int32),
    ]

    def to_dict(self) -> dict:
        d = {"t": self.t, "massA": self.mass[0], "massB": self.mass[1], "dp": self.dp_laplace, "R_eff": self.R_eff,
             "umax": self.umax, "finite": float(self.finite)}
        for k, sp in enumerate("AB"):
            for a, ax in enumerate("xyz"):
                d["mom" + sp + ax] = self.mom[k][a]
        return d


_P = ctypes.POINTER
_d = ctypes.c_double
_dp = _P(_d)
_vp = ctypes.c_void_p
_i32, _i64, _sz = ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t

# name -> (restype, argtypes); mirrors include/lb.h
SIGNATURES = {
    "lb_last_error": (ctypes.c_char_p, []),
    "lb_create": (ctypes.c_int, [_P(lb_params), _P(_vp)]),
    "lb_destroy": (None, [_vp]),
    "lb_set_fields": (ctypes.c_int, [_vp, _vp, _vp]),
    "lb_set_fields_device": (ctypes.c_int, [_vp, _vp, _vp]),
    "lb_step": (ctypes.c_int, [_vp, _i64]),
    "lb_synchronize": (ctypes.c_int, [_vp]),
    "lb_time": (_i64, [_vp]),
    "lb_set_probe": (ctypes.c_int, [_vp, _d, _d, _d]),
    "lb_observables": (ctypes.c_int, [_vp, _P(lb_obs)]),
    "lb_get_fields": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "lb_get_populations": (ctypes.c_int, [_vp, _vp]),
    "lb_step_vjp": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "lb_set_populations": (ctypes.c_int, [_vp, _vp, _i64]),
    "lb_save": (ctypes.c_int, [_vp, _vp, _P(_sz)]),
    "lb_load": (ctypes.c_int, [_vp, _vp, _sz]),
    "lb_profile": (ctypes.c_int, [_vp, _i32, _vp, _sz, _dp]),
    "lb_grad": (ctypes.c_int, [_vp, _i64, _i32, _i32, _dp, _dp]),
    "lb_set_config": (ctypes.c_int, [_vp, _i32, _i32]),
    "lb_get_config": (ctypes.c_int, [_vp, _P(_i32), _P(_i32)]),
    "lb_autotune": (ctypes.c_int, [_vp, _i32, ctypes.c_char_p, _dp]),
    "lb_batch_create": (ctypes.c_int, [_P(lb_params), _i32, _P(_vp)]),
    "lb_batch_destroy": (None, [_vp]),
    "lb_batch_size": (ctypes.c_int, [_vp]),
    "lb_batch_set_fields": (ctypes.c_int, [_vp, _i32, _vp, _vp]),
    "lb_batch_step": (ctypes.c_int, [_vp, _i64]),
    "lb_batch_synchronize": (ctypes.c_int, [_vp]),
    "lb_batch_set_probe": (ctypes.c_int, [_vp, _i32, _d, _d, _d]),
    "lb_batch_observables": (ctypes.c_int, [_vp, _P(lb_obs)]),
    "lb_batch_get_fields": (ctypes.c_int, [_vp, _i32, _vp, _vp, _vp]),
    "lb_batch_profile": (ctypes.c_int, [_vp, _i32, _vp, _sz, _dp]),
    "lb_batch_set_config": (ctypes.c_int, [_vp, _i32, _i32]),
    "lb_batch_get_config": (ctypes.c_int, [_vp, _P(_i32), _P(_i32)]),
    "lb_batch_autotune": (ctypes.c_int, [_vp, _i32, ctypes.c_char_p, _dp]),
    "lb_batch_set_wait_limit": (ctypes.c_int, [_vp, _d, _i32]),
    "lb_observables_static": (ctypes.c_int, [_P(lb_params), _vp, _d, _d, _d, _vp]),
    "lb_device_fp64_peak": (ctypes.c_int, [_i32, _dp]),
    "lb_pressure_tensor": (ctypes.c_int, [_vp, _vp, _vp]),
    "lb3_create": (ctypes.c_int, [_P(lb3_params), _P(_vp)]),
    "lb3_destroy": (None, [_vp]),
    "lb3_set_fields": (ctypes.c_int, [_vp, _vp, _vp]),
    "lb3_step": (ctypes.c_int, [_vp, _i64]),
    "lb3_time": (_i64, [_vp]),
    "lb3_set_probe": (ctypes.c_int, [_vp, _d, _d, _d, _d]),
    "lb3_observables": (ctypes.c_int, [_vp, _P(lb3_obs)]),
    "lb3_get_fields": (ctypes.c_int, [_vp, _vp, _vp]),
    "lb3_get_populations": (ctypes.c_int, [_vp, _vp]),
    "lb3_profile": (ctypes.c_int, [_vp, _i32, _vp, _sz, _dp]),
    "lb_batch_pressure_tensor": (ctypes.c_int, [_vp, _i32, _vp, _vp]),
}


def device_fp64_peak(trips: int = 4096) -> float:
    """Measured FP64 FMA throughput of the current device, TFLOP/s."""
    v = ctypes.c_double()
    _check(LIB.lb_device_fp64_peak(int(trips), ctypes.byref(v)))
    return v.value


def header_functions() -> list[str]:
    """Names of the functions include/lb.h declares."""
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lb3?_[a-z0-9_]+)\s*\(", src)))


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with paper_1806_06943_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


LIB = load()


def _check(rc: int):
    if rc != LB_OK:
        raise LBError(rc, LIB.lb_last_error().decode())


def _host_ptr(a: np.ndarray | None, shape, writable=False):
    if a is None:
        return None
    if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]):
        raise TypeError("expected a C-contiguous float64 numpy array")
    if a.shape != tuple(shape):
        raise ValueError(f"expected shape {tuple(shape)}, got {a.shape}")
    if writable and not a.flags["WRITEABLE"]:
        raise ValueError("array is read-only")
    return a.ctypes.data


def make_params(nx, ny, tau=(1.0, 1.0), G_AB=3.0, G1=-7.4, G2=6.4, g=(0.0, 0.0), walls=0, wall_mode=0,
                wall_rho=(0.0, 0.0), precision=LB_FP64, stream=None, forcing=LB_FORCING_GUO) -> lb_params:
    p = lb_params()
    p.nx, p.ny = int(nx), int(ny)
    p.tau[0], p.tau[1] = float(tau[0]), float(tau[1])
    p.G_AB, p.G1, p.G2 = float(G_AB), float(G1), float(G2)
    p.g[0], p.g[1] = float(g[0]), float(g[1])
    p.walls, p.wall_mode = int(walls), int(wall_mode)
    p.wall_rho[0], p.wall_rho[1] = float(wall_rho[0]), float(wall_rho[1])
    p.precision = int(precision)
    p.forcing = int(forcing)
    p.stream = stream
    return p


def current_stream():
    """The raw cudaStream_t of torch's current stream (None for the legacy
    default stream)."""
    import torch
    s = torch.cuda.current_stream().cuda_stream
    return s or None


class Lattice:
    """One lattice behind an lb_handle."""

    def __init__(self, nx, ny, **kw):
        self.params = make_params(nx, ny, **kw)
        self.nx, self.ny = int(nx), int(ny)
        h = _vp()
        _check(LIB.lb_create(ctypes.byref(self.params), ctypes.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            LIB.lb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def t(self) -> int:
        return LIB.lb_time(self.h)

    def set_fields(self, rho: np.ndarray, u: np.ndarray | None = None):
        shp = (2, self.ny, self.nx)
        _check(LIB.lb_set_fields(self.h, _host_ptr(rho, shp), _host_ptr(u, shp)))

    def set_fields_device(self, rho, u=None):
        """rho, u: contiguous float64 CUDA tensors of shape (2, ny, nx)."""
        for a in (rho, u):
            if a is not None:
                if not (a.is_cuda and a.is_contiguous() and str(a.dtype) == "torch.float64"):
                    raise TypeError("expected a contiguous float64 CUDA tensor")
                if tuple(a.shape) != (2, self.ny, self.nx):
                    raise ValueError("bad shape")
        _check(LIB.lb_set_fields_device(self.h, rho.data_ptr(), u.data_ptr() if u is not None else None))

    def step(self, n: int = 1):
        _check(LIB.lb_step(self.h, int(n)))

    def synchronize(self):
        _check(LIB.lb_synchronize(self.h))

    def set_probe(self, cx, cy, R):
        _check(LIB.lb_set_probe(self.h, float(cx), float(cy), float(R)))

    def observables(self, check: bool = True) -> dict:
        o = lb_obs()
        rc = LIB.lb_observables(self.h, ctypes.byref(o))
        if check or rc != LB_EUNSTABLE:
            _check(rc)
        return o.to_dict()

    def fields(self) -> dict:
        n = (self.ny, self.nx)
        rho, mom, ubar = np.empty((2,) + n), np.empty((2, 2) + n), np.empty((2,) + n)
        _check(LIB.lb_get_fields(self.h, rho.ctypes.data, mom.ctypes.data, ubar.ctypes.data))
        return {"rho": rho, "mom": mom, "ubar": ubar}

    def pressure_tensor(self, field: bool = False):
        """(sums[6], P or None): lattice sums of the kinetic and interaction
        xx, yy, xy components, and optionally the field [2][3][ny][nx]."""
        sums = np.empty(6)
        P = np.empty((2, 3, self.ny, self.nx)) if field else None
        _check(LIB.lb_pressure_tensor(self.h, P.ctypes.data if field else None, sums.ctypes.data))
        return sums, P

    def step_vjp(self, w: np.ndarray) -> tuple:
        """((dStep/df)^T w, <w, dStep/dtheta>) at the current state (FP64)."""
        ny, nx = self.ny, self.nx
        wa = np.ascontiguousarray(w, dtype=np.float64)   # kept alive across the call
        out = np.empty((2, 9, ny, nx))
        dth = (ctypes.c_double * 5)()
        _check(LIB.lb_step_vjp(self.h, _host_ptr(wa, (2, 9, ny, nx)), out.ctypes.data, dth))
        return out, np.array(list(dth))

    def get_populations(self) -> np.ndarray:
        f = np.empty((2, 9, self.ny, self.nx))
        _check(LIB.lb_get_populations(self.h, f.ctypes.data))
        return f

    def set_populations(self, f: np.ndarray, t: int = 0):
        _check(LIB.lb_set_populations(self.h, _host_ptr(f, (2, 9, self.ny, self.nx)), int(t)))

    def profile(self, nsteps: int, flush_ptr=None, flush_bytes: int = 0) -> tuple:
        """Mean (density, fused, whole-step) kernel milliseconds over nsteps."""
        ms = (ctypes.c_double * 3)()
        _check(LIB.lb_profile(self.h, int(nsteps), flush_ptr, int(flush_bytes), ms))
        return tuple(ms)

    def grad(self, nsteps: int, ckpt_every: int, objective: int = LB_OBJ_MU_R):
        """(J, dJ/d(G_AB, G1, G2, tau_A, tau_B)) after nsteps steps from the current state."""
        J = ctypes.c_double()
        dJ = (ctypes.c_double * 5)()
        _check(LIB.lb_grad(self.h, int(nsteps), int(ckpt_every), int(objective), ctypes.byref(J), dJ))
        return J.value, np.array(list(dJ))

    def set_config(self, mode: int, tile_height: int):
        _check(LIB.lb_set_config(self.h, int(mode), int(tile_height)))

    def config(self) -> tuple:
        m, t = ctypes.c_int32(), ctypes.c_int32()
        _check(LIB.lb_get_config(self.h, ctypes.byref(m), ctypes.byref(t)))
        return m.value, t.value

    def autotune(self, trial_steps: int = 64, cache_path: str | None = None) -> float:
        ms = ctypes.c_double()
        _check(LIB.lb_autotune(self.h, int(trial_steps), cache_path.encode() if cache_path else None,
                               ctypes.byref(ms)))
        return ms.value

    def save(self) -> bytes:
        n = ctypes.c_size_t(0)
        _check(LIB.lb_save(self.h, None, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        _check(LIB.lb_save(self.h, buf, ctypes.byref(n)))
        return buf.raw[: n.value]

    def load(self, blob: bytes):
        buf = ctypes.create_string_buffer(blob, len(blob))
        _check(LIB.lb_load(self.h, buf, len(blob)))


class Batch:
    """Several independent lattices stepped together behind an lb_batch."""

    def __init__(self, specs: list[dict], **common):
        arr = (lb_params * len(specs))()
        self.shapes = []
        for i, s in enumerate(specs):
            kw = dict(common)
            kw.update({k: v for k, v in s.items() if k in (
                "tau", "G_AB", "G1", "G2", "g", "walls", "wall_mode", "wall_rho", "precision", "stream",
                "forcing")})
            arr[i] = make_params(s["nx"], s["ny"], **kw)
            self.shapes.append((int(s["ny"]), int(s["nx"])))
        self.params = arr
        b = _vp()
        _check(LIB.lb_batch_create(arr, len(specs), ctypes.byref(b)))
        self.b = b
        self.n = len(specs)

    def close(self):
        if getattr(self, "b", None):
            LIB.lb_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_fields(self, i, rho, u=None):
        shp = (2,) + self.shapes[i]
        _check(LIB.lb_batch_set_fields(self.b, int(i), _host_ptr(rho, shp), _host_ptr(u, shp)))

    def step(self, n: int = 1):
        _check(LIB.lb_batch_step(self.b, int(n)))

    def synchronize(self):
        _check(LIB.lb_batch_synchronize(self.b))

    def set_probe(self, i, cx, cy, R):
        _check(LIB.lb_batch_set_probe(self.b, int(i), float(cx), float(cy), float(R)))

    def observables(self, check: bool = True) -> list[dict]:
        o = (lb_obs * self.n)()
        rc = LIB.lb_batch_observables(self.b, o)
        if check or rc != LB_EUNSTABLE:
            _check(rc)
        return [x.to_dict() for x in o]

    def profile(self, nsteps: int, flush_ptr=None, flush_bytes: int = 0) -> tuple:
        ms = (ctypes.c_double * 3)()
        _check(LIB.lb_batch_profile(self.b, int(nsteps), flush_ptr, int(flush_bytes), ms))
        return tuple(ms)

    def set_config(self, mode: int, tile_height: int):
        _check(LIB.lb_batch_set_config(self.b, int(mode), int(tile_height)))

    def config(self) -> tuple:
        m, t = ctypes.c_int32(), ctypes.c_int32()
        _check(LIB.lb_batch_get_config(self.b, ctypes.byref(m), ctypes.byref(t)))
        return m.value, t.value

    def autotune(self, trial_steps: int = 64, cache_path: str | None = None) -> float:
        ms = ctypes.c_double()
        _check(LIB.lb_batch_autotune(self.b, int(trial_steps), cache_path.encode() if cache_path else None,
                                     ctypes.byref(ms)))
        return ms.value

    def set_wait_limit(self, seconds: float, drop_tile: int = -1):
        _check(LIB.lb_batch_set_wait_limit(self.b, float(seconds), int(drop_tile)))

    def pressure_tensor(self, i, field: bool = False):
        """As Lattice.pressure_tensor, for lattice i."""
        sums = np.empty(6)
        P = np.empty((2, 3) + self.shapes[i]) if field else None
        _check(LIB.lb_batch_pressure_tensor(self.b, int(i), P.ctypes.data if field else None, sums.ctypes.data))
        return sums, P

    def fields(self, i) -> dict:
        n = self.shapes[i]
        rho, mom, ubar = np.empty((2,) + n), np.empty((2, 2) + n), np.empty((2,) + n)
        _check(LIB.lb_batch_get_fields(self.b, int(i), rho.ctypes.data, mom.ctypes.data, ubar.ctypes.data))
        return {"rho": rho, "mom": mom, "ubar": ubar}


class Lattice3:
    """One 3-D lattice (D3Q19, 5^3 mid-range stencil, periodic) behind an
    lb3_handle.  Fields are numpy float64 [..][nz][ny][nx]."""

    def __init__(self, nx, ny, nz, tau=(1.0, 1.0), G_AB=3.0, G1=-7.4, G2=6.4, g=(0.0, 0.0, 0.0),
                 precision=LB_FP64, stream=None):
        p = lb3_params()
        p.nx, p.ny, p.nz, p.precision = int(nx), int(ny), int(nz), int(precision)
        p.tau[0], p.tau[1] = float(tau[0]), float(tau[1])
        p.G_AB, p.G1, p.G2 = float(G_AB), float(G1), float(G2)
        for a in range(3):
            p.g[a] = float(g[a])
        p.stream = stream
        self.params = p
        self.shape = (int(nz), int(ny), int(nx))
        h = _vp()
        _check(LIB.lb3_create(ctypes.byref(p), ctypes.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            LIB.lb3_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def t(self) -> int:
        return LIB.lb3_time(self.h)

    def set_fields(self, rho, u=None):
        _check(LIB.lb3_set_fields(self.h, _host_ptr(rho, (2,) + self.shape), _host_ptr(u, (3,) + self.shape)))

    def step(self, n: int = 1):
        _check(LIB.lb3_step(self.h, int(n)))

    def set_probe(self, cx, cy, cz, R):
        _check(LIB.lb3_set_probe(self.h, float(cx), float(cy), float(cz), float(R)))

    def observables(self, check: bool = True) -> dict:
        o = lb3_obs()
        rc = LIB.lb3_observables(self.h, ctypes.byref(o))
        if check or rc != LB_EUNSTABLE:
            _check(rc)
        return o.to_dict()

    def fields(self) -> dict:
        rho, ubar = np.empty((2,) + self.shape), np.empty((3,) + self.shape)
        _check(LIB.lb3_get_fields(self.h, rho.ctypes.data, ubar.ctypes.data))
        return {"rho": rho, "ubar": ubar}

    def get_populations(self) -> np.ndarray:
        f = np.empty((2, 19) + self.shape)
        _check(LIB.lb3_get_populations(self.h, f.ctypes.data))
        return f

    def profile(self, nsteps: int, flush_ptr=None, flush_bytes: int = 0) -> tuple:
        ms = (ctypes.c_double * 3)()
        _check(LIB.lb3_profile(self.h, int(nsteps), flush_ptr, int(flush_bytes), ms))
        return tuple(ms)
