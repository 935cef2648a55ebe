"""The TMA-staged one-pass step (LB_MODE_TMA, FP32): the same populations as
the plain one-pass step on lattices that mix tiles staged by TMA (box inside
the lattice) with tiles that load directly (periodic edges, wall rows, ragged
tiles), for every tile height; rejected for FP64; its bounded wait for a copy
ends with LB_ETIMEOUT and leaves the device usable."""
import numpy as np
import pytest

from paper_1806_06943_gb300 import workloads as W

pytestmark = pytest.mark.gpu

C6 = dict(G_AB=3.0, G1=-7.4, G2=6.4)
SPECS = [
    dict(nx=256, ny=96, tau=(1.0, 1.0)),                                          # periodic, all heights full
    dict(nx=200, ny=70, tau=(2.0, 1.0), walls=1, wall_mode=1, wall_rho=(0.03, 1.0), g=(1e-5, 0.0)),
    dict(nx=177, ny=45, tau=(0.7, 1.3)),                                          # ragged in x and y
    dict(nx=96, ny=41, tau=(1.5, 1.0), walls=1, wall_mode=0, g=(2e-5, 0.0)),      # few TMA tiles
]
STEPS = 3 * 32 + 5


@pytest.fixture(scope="module")
def lbmod():
    from paper_1806_06943_gb300 import build
    build.build()
    from paper_1806_06943_gb300 import lb
    return lb


def fields_for(specs):
    out = []
    for i, s in enumerate(specs):
        periodic = not s.get("walls", 0)
        n = max(1, s["nx"] * s["ny"] // 900)
        rng = np.random.default_rng(40 + i)
        centres = [(rng.uniform(0, s["nx"]), rng.uniform(6, s["ny"] - 6)) for _ in range(n)]
        out.append(W.droplets(s["nx"], s["ny"], centres, [7.0] * n, seed=300 + i, periodic=periodic))
    return out


def run(lbmod, mode, ty, rhos, steps=STEPS):
    b = lbmod.Batch(SPECS, precision=lbmod.LB_FP32, **C6)
    b.set_config(mode, ty)
    for i, r in enumerate(rhos):
        b.set_fields(i, r)
    b.step(steps)
    b.synchronize()
    return b


@pytest.mark.parametrize("ty", [2, 4, 8])
def test_tma_step_equals_plain_one_pass(lbmod, ty):
    rhos = fields_for(SPECS)
    ref = run(lbmod, lbmod.LB_MODE_FUSED, ty, rhos)
    got = run(lbmod, lbmod.LB_MODE_TMA, ty, rhos)
    assert got.config() == (lbmod.LB_MODE_TMA, ty)
    for i in range(len(SPECS)):
        a, b = got.fields(i), ref.fields(i)
        for k in ("rho", "mom", "ubar"):
            assert np.all(np.isfinite(a[k]))
            # same arithmetic in the same order: bit for bit
            assert np.array_equal(a[k], b[k]), (i, k, np.max(np.abs(a[k] - b[k])))


def test_tma_mode_rejected_for_fp64(lbmod):
    b = lbmod.Batch(SPECS[:1], precision=lbmod.LB_FP64, **C6)
    with pytest.raises(lbmod.LBError) as ei:
        b.set_config(lbmod.LB_MODE_TMA, 8)
    assert ei.value.code == lbmod.LB_EINVAL


def test_tma_wait_times_out_and_device_recovers(lbmod):
    rhos = fields_for(SPECS)
    b = lbmod.Batch(SPECS, precision=lbmod.LB_FP32, **C6)
    b.set_config(lbmod.LB_MODE_TMA, 8)
    for i, r in enumerate(rhos):
        b.set_fields(i, r)
    # tile 18 of the height-8 list: lattice 0, x0 = 64, y0 = 16, box inside;
    # its copy is never started, so its wait runs out after 50 ms
    b.set_wait_limit(0.05, drop_tile=18)
    b.step(4)
    with pytest.raises(lbmod.LBError) as ei:
        b.synchronize()
    assert ei.value.code == lbmod.LB_ETIMEOUT
    b.set_wait_limit(2.0, drop_tile=-1)
    for i, r in enumerate(rhos):
        b.set_fields(i, r)
    b.step(40)
    b.synchronize()
    assert all(o["finite"] == 1.0 for o in b.observables())
    ref = run(lbmod, lbmod.LB_MODE_FUSED, 8, rhos, steps=40)
    for i in range(len(SPECS)):
        a, r = b.fields(i), ref.fields(i)
        assert np.array_equal(a["rho"], r["rho"]) and np.array_equal(a["mom"], r["mom"]), i
