"""Batched form: every execution configuration (two-launch steps, one
persistent launch per 64 steps, one-pass steps, or TMA-staged one-pass steps
in FP32; tile heights 2, 4, 8) gives the same populations bit for bit, in
FP64 (the plain evaluation order) and in FP32 (every rounding spelled out,
the same in every kernel); a batch stepped in the two chains of its step
graph matches its lattices stepped alone; the persistent kernel's bounded
waits end with LB_ETIMEOUT when a tile never reports; the autotuner leaves
the state untouched and caches its choice."""
import numpy as np
import pytest

from paper_1806_06943_gb300 import workloads as W

pytestmark = pytest.mark.gpu

C6 = dict(G_AB=3.0, G1=-7.4, G2=6.4)
SPECS = [
    dict(nx=64, ny=64, tau=(1.0, 1.0)),
    dict(nx=37, ny=50, tau=(2.0, 1.0)),
    dict(nx=96, ny=33, tau=(0.6, 1.2), walls=1, wall_mode=1, wall_rho=(0.03, 1.0), g=(1e-5, 0.0)),
    dict(nx=130, ny=6, tau=(1.3, 0.9), walls=1, wall_mode=0, g=(2e-5, 0.0)),
]
CONFIGS = [(m, ty) for m in (0, 1, 2) for ty in (2, 4, 8)]
TMA_CONFIGS = [(3, ty) for ty in (2, 4, 8)]    # FP32 only


@pytest.fixture(scope="module")
def lbmod():
    from paper_1806_06943_gb300 import build
    build.build()
    from paper_1806_06943_gb300 import lb
    return lb


def fields_for(specs):
    return [W.droplet(s["nx"], s["ny"], min(s["nx"], s["ny"]) / 4, seed=200 + i, periodic=not s.get("walls", 0))
            for i, s in enumerate(specs)]


def run_batch(lbmod, precision, config, steps, rhos):
    b = lbmod.Batch(SPECS, precision=precision, **C6)
    b.set_config(*config)
    assert b.config() == config
    for i, r in enumerate(rhos):
        b.set_fields(i, r)
    b.step(steps)
    b.synchronize()
    return b


@pytest.mark.parametrize("precision", [0, 1])
def test_all_configurations_agree(lbmod, oracle_mod, precision):
    rhos = fields_for(SPECS)
    steps = 3 * 64 + 5          # graph replays plus a ragged remainder
    ref = run_batch(lbmod, precision, (0, 4), steps, rhos)
    ref_fields = [ref.fields(i) for i in range(len(SPECS))]
    for cfg in CONFIGS + (TMA_CONFIGS if precision == 1 else []):
        b = run_batch(lbmod, precision, cfg, steps, rhos)
        for i in range(len(SPECS)):
            got = b.fields(i)
            for k in ("rho", "mom"):
                assert np.array_equal(got[k], ref_fields[i][k]), (cfg, i, k)
    if precision == 0:
        # and the reference configuration against the oracle
        for i, s in enumerate(SPECS):
            kw = {k: v for k, v in s.items() if k not in ("nx", "ny")}
            o = oracle_mod.OracleSim(s["nx"], s["ny"], **kw, **C6)
            o.set_fields(rhos[i])
            o.step(steps)
            fo = o.fields()
            den = np.max(np.abs(fo["rho"]))
            assert np.max(np.abs(ref_fields[i]["rho"] - fo["rho"])) <= 1e-12 * den, i


@pytest.mark.parametrize("config", [(3, 8), (2, 4), (0, 4)])
def test_batch_in_two_chains_equals_single_lattices(lbmod, config):
    """A batch's step graph runs its lattices as two chains on two streams
    (groups of about equal node counts); every lattice ends with the same
    populations as the same lattice stepped alone, in one chain, bit for bit
    (FP32; graph replays plus single steps)."""
    rhos = fields_for(SPECS)
    steps = 2 * 32 + 3
    b = run_batch(lbmod, 1, config, steps, rhos)
    for i, s in enumerate(SPECS):
        kw = {k: v for k, v in s.items() if k not in ("nx", "ny")}
        L = lbmod.Lattice(s["nx"], s["ny"], precision=1, **kw, **C6)
        L.set_config(*config)
        L.set_fields(rhos[i])
        L.step(steps)
        got, ref = b.fields(i), L.fields()
        for k in ("rho", "mom"):
            assert np.array_equal(got[k], ref[k]), (config, i, k)


def test_persistent_wait_times_out_and_device_recovers(lbmod):
    rhos = fields_for(SPECS)
    b = lbmod.Batch(SPECS, precision=1, **C6)
    b.set_config(lbmod.LB_MODE_PERSISTENT, 4)
    for i, r in enumerate(rhos):
        b.set_fields(i, r)
    b.set_wait_limit(0.05, drop_tile=3)     # tile 3 never reports completion
    b.step(64)
    with pytest.raises(lbmod.LBError) as ei:
        b.synchronize()
    assert ei.value.code == lbmod.LB_ETIMEOUT
    # the flag is reported once; restore the state and run normally
    b.set_wait_limit(2.0, drop_tile=-1)
    for i, r in enumerate(rhos):
        b.set_fields(i, r)
    b.step(64)
    b.synchronize()
    assert all(o["finite"] == 1.0 for o in b.observables())


def test_autotune_keeps_state_and_caches(lbmod, tmp_path):
    rhos = fields_for(SPECS)
    b = lbmod.Batch(SPECS, precision=1, **C6)
    for i, r in enumerate(rhos):
        b.set_fields(i, r)
    b.step(10)
    before = [b.fields(i) for i in range(len(SPECS))]
    cache = str(tmp_path / "tune.txt")
    ms = b.autotune(16, cache)
    assert ms > 0
    cfg = b.config()
    assert cfg in CONFIGS + TMA_CONFIGS
    after = [b.fields(i) for i in range(len(SPECS))]
    for x, y in zip(before, after):
        assert np.array_equal(x["rho"], y["rho"]) and np.array_equal(x["mom"], y["mom"])
    text = open(cache).read().split()
    assert len(text) == 4 and int(text[1]) == cfg[0] and int(text[2]) == cfg[1]
    b2 = lbmod.Batch(SPECS, precision=1, **C6)
    ms2 = b2.autotune(16, cache)          # cache hit: no trials
    assert b2.config() == cfg and ms2 == pytest.approx(float(text[3]))
