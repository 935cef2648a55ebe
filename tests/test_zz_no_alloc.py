"""The allocation-free observables entry point, lb_observables_static.

Callers that may not allocate device memory once they run (a fixed memory
budget, a step that must stay out of the allocator) hand it the populations
and an output array in their own device memory; its scratch is a fixed
file-scope device array.  This file is collected last so that a run stopping
at the first failure has already run every other test; it also passes on
its own in a fresh process."""
import ctypes

import numpy as np
import pytest

from paper_1806_06943_gb300 import workloads as W

C6 = dict(G_AB=3.0, G1=-7.4, G2=6.4)
KEYS = ("massA", "massB", "momAx", "momAy", "momBx", "momBy", "Q", "mu_r", "dp", "R_eff", "umax", "finite")


@pytest.fixture(scope="module")
def lbmod():
    from paper_1806_06943_gb300 import build
    build.build()
    from paper_1806_06943_gb300 import lb
    return lb


def test_rejects_oversized_and_invalid_without_a_gpu_call(lbmod):
    out = ctypes.c_void_p(16)   # never dereferenced: the call fails validation first
    big = lbmod.make_params(4096, 4096)
    rc = lbmod.LIB.lb_observables_static(ctypes.byref(big), out, 0.0, 0.0, 0.0, out)
    assert rc == lbmod.LB_EINVAL and b"LB_STATIC_MAX_TILES" in lbmod.LIB.lb_last_error()
    p32 = lbmod.make_params(64, 64, precision=lbmod.LB_FP32)
    assert lbmod.LIB.lb_observables_static(ctypes.byref(p32), out, 0.0, 0.0, 0.0, out) == lbmod.LB_EINVAL
    p = lbmod.make_params(64, 64)
    assert lbmod.LIB.lb_observables_static(ctypes.byref(p), None, 0.0, 0.0, 0.0, out) == lbmod.LB_EINVAL
    assert lbmod.LIB.lb_observables_static(ctypes.byref(p), out, 0.0, 0.0, 0.0, None) == lbmod.LB_EINVAL
    assert lbmod.LIB.lb_observables_static(None, out, 0.0, 0.0, 0.0, out) == lbmod.LB_EINVAL
    assert lbmod.LIB.lb_observables_static(ctypes.byref(p), out, float("nan"), 0.0, 4.0, out) == lbmod.LB_EINVAL


@pytest.mark.parametrize("kw,needle", [
    (dict(walls=1, wall_mode=5), b"wall_mode"),          # not LB_WALL_MIRROR or LB_WALL_FIXED
    (dict(G1=float("nan")), b"non-finite"),
    (dict(g=(float("inf"), 0.0)), b"non-finite"),
    (dict(wall_rho=(float("nan"), 1.0)), b"non-finite"),
    (dict(tau=(0.5, 1.0)), b"tau[0]"),
    (dict(walls=3), b"walls"),
])
def test_rejects_what_lb_create_rejects(lbmod, kw, needle):
    """The entry point checks its parameters as lb_create does, before any
    CUDA call."""
    out = ctypes.c_void_p(16)
    p = lbmod.make_params(64, 40, **kw)
    assert lbmod.LIB.lb_observables_static(ctypes.byref(p), out, 0.0, 0.0, 0.0, out) == lbmod.LB_EINVAL
    assert needle in lbmod.LIB.lb_last_error()


@pytest.mark.gpu
@pytest.mark.parametrize("nx,ny,walls,wall_mode,centre", [
    (96, 80, 0, 1, (48.0, 40.0)),
    (96, 80, 0, 1, (3.0, 77.5)),      # drop and probe across the periodic corner: wrapped distances
    (70, 37, 1, 1, (35.0, 18.5)),     # fixed (non-wetting) wall ghosts
    (70, 37, 1, 0, (35.0, 18.5)),     # mirrored wall ghosts
])
def test_matches_lb_observables_on_two_calls_in_a_row(lbmod, nx, ny, walls, wall_mode, centre):
    """Same record as lb_observables on the library's own lattice, twice in a
    row on the shared scratch, within the tolerances of the FP64 parity
    tests (reductions 1e-12 of their scale, derived observables 1e-10)."""
    torch = pytest.importorskip("torch")
    # set-up form: loads the array on this device before anything else
    assert lbmod.LIB.lb_observables_static(None, None, 0.0, 0.0, 0.0, None) == lbmod.LB_OK
    kw = dict(walls=walls, wall_mode=wall_mode, wall_rho=(0.03, 1.0), g=(1e-5, 0.0)) if walls else {}
    R = min(nx, ny) / 4.0
    cx, cy = centre
    L = lbmod.Lattice(nx, ny, tau=(1.3, 0.8), **kw, **C6)
    L.set_fields(W.droplet(nx, ny, R, cx=cx, cy=cy, seed=31 + nx, periodic=not walls))
    L.step(150)
    L.set_probe(cx, cy, R)
    ref = L.observables()
    f = torch.from_numpy(L.get_populations()).cuda()
    p = lbmod.make_params(nx, ny, tau=(1.3, 0.8), **kw, **C6)
    outs = []
    for _ in range(2):
        out = torch.full((16,), float("nan"), dtype=torch.float64, device="cuda")
        rc = lbmod.LIB.lb_observables_static(ctypes.byref(p), f.data_ptr(), cx, cy, R, out.data_ptr())
        assert rc == lbmod.LB_OK, lbmod.LIB.lb_last_error()
        torch.cuda.synchronize()
        outs.append(dict(zip(KEYS, out.cpu().numpy().tolist())))
    M = ref["massA"] + ref["massB"]
    for got in outs:
        for k in ("massA", "massB"):
            assert abs(got[k] - ref[k]) <= 1e-12 * abs(ref[k]), k
        for k in ("momAx", "momAy", "momBx", "momBy"):
            assert abs(got[k] - ref[k]) <= 1e-12 * M, k
        assert abs(got["Q"] - ref["Q"]) <= 1e-12 * max(1e-3, ref["umax"]) * ny
        for k in ("dp", "R_eff", "umax"):
            assert abs(got[k] - ref[k]) <= 1e-10 * abs(ref[k]), k
        if walls:
            assert abs(got["mu_r"] - ref["mu_r"]) <= 1e-10 * abs(ref["mu_r"])
        else:
            assert np.isnan(got["mu_r"])
        assert got["finite"] == 1.0
    # the second call over the leftovers of the first gives the same bits
    for k in KEYS:
        assert outs[0][k] == outs[1][k] or (np.isnan(outs[0][k]) and np.isnan(outs[1][k])), k
