"""Parity of the CUDA path (through the C-ABI) with the FP64 oracle on the
same seeded inputs.

Tolerances (normwise relative error, ||x_gpu - x_ref||_inf / ||x_ref||_inf,
per field, because velocities are near zero at many nodes):
  FP64 populations, densities and velocities ........ 1e-12
  FP32 densities .................................... 1e-5
  FP32 velocities ................................... 1e-5
  FP32 Laplace pressure jump and effective viscosity  1e-3 relative
FP64 reductions (mass, momentum, flux) are compared at 1e-12 relative to
their scale; derived observables at 1e-10.

FP32 velocity error: at an interface node the momentum balance is a
difference of a pressure-gradient flux cs^2 |grad rho| ~ 0.03 and the forces;
single-precision densities (half ulp ~ 3e-8 near rho = 1) make that balance
err by ~1e-8 per step, a random forcing whose effect accumulates over the
viscous relaxation time of the drop (R^2/nu ~ 900 steps): sqrt(900) * 1e-8 ~
3e-7, i.e. 3e-5 of the 0.0095 spurious-current maximum at worst.  With the
node's density split exactly into reference and offsets (no mass drift) the
C1 droplet lands just under 1e-5.  Where a body force drives the flow (the
channel) the FP32 velocity also carries a systematic rounding bias growing
with g t (see that test), and the fields are held to 5e-5 (u) and 2e-5
(rho) there."""
import numpy as np
import pytest

from paper_1806_06943_gb300 import workloads as W

pytestmark = pytest.mark.gpu

C6 = dict(G_AB=3.0, G1=-7.4, G2=6.4)


@pytest.fixture(scope="module")
def lbmod():
    from paper_1806_06943_gb300 import build
    build.build()
    from paper_1806_06943_gb300 import lb
    return lb


def nrel(a, b, floor=0.0):
    """||a - b||_inf / max(||b||_inf, floor)."""
    den = max(np.max(np.abs(b)), floor)
    return np.max(np.abs(a - b)) / (den if den > 0 else 1.0)


def run_pair(oracle_mod, lbmod, rho, steps, u=None, precision=0, probe=None, **kw):
    ny, nx = rho.shape[1:]
    o = oracle_mod.OracleSim(nx, ny, **kw)
    o.set_fields(rho, u)
    o.step(steps)
    g = lbmod.Lattice(nx, ny, precision=precision, **kw)
    g.set_fields(rho, u)
    g.step(steps)
    if probe is not None:
        g.set_probe(*probe)
    return o, g


def test_c1_droplet_fp64_2000_steps(oracle_mod, lbmod):
    """64x64 periodic droplet R=12, tau_A=tau_B=1, 2000 steps: rho and u
    within 1e-12 of the oracle."""
    rho = W.c1_droplet_64()
    o, g = run_pair(oracle_mod, lbmod, rho, 2000, **C6)
    fo, fg = o.fields(), g.fields()
    assert nrel(fg["rho"], fo["rho"]) <= 1e-12
    assert nrel(fg["ubar"], fo["ubar"]) <= 1e-12
    assert nrel(fg["mom"], fo["mom"]) <= 1e-12
    assert nrel(g.get_populations(), o.get_f()) <= 1e-12
    oo, og = o.observables((32, 32, 12)), None
    g.set_probe(32, 32, 12)
    og = g.observables()
    for k in ("massA", "massB"):
        assert abs(og[k] - oo[k]) <= 1e-12 * abs(oo[k])
    for k in ("dp", "R_eff", "umax"):
        assert abs(og[k] - oo[k]) <= 1e-10 * abs(oo[k]), k
    M = oo["massA"] + oo["massB"]
    for k in ("momAx", "momAy", "momBx", "momBy"):
        assert abs(og[k] - oo[k]) <= 1e-12 * M, k
    assert og["t"] == 2000 and og["finite"] == 1.0


@pytest.mark.parametrize("nx,ny,walls,wall_mode,tau,g", [
    (45, 37, 1, 0, (0.7, 1.6), (2e-5, 0.0)),      # ragged tiles, mirror walls, body force
    (70, 19, 1, 1, (1.0, 3.0), (1e-5, 0.0)),      # fixed (non-wetting) walls
    (33, 41, 0, 0, (2.0, 0.6), (0.0, 3e-6)),      # periodic, force along y
    (5, 5, 0, 0, (1.0, 1.0), (0.0, 0.0)),         # smallest lattice: stencil wraps several times
    (5, 9, 1, 0, (0.8, 1.2), (1e-5, 0.0)),        # smallest channel
    (130, 6, 1, 1, (1.3, 0.9), (1e-5, 0.0)),      # one tile row, ragged in x
])
def test_fp64_parity_shapes(oracle_mod, lbmod, nx, ny, walls, wall_mode, tau, g):
    rho = W.droplet(nx, ny, min(nx, ny) / 3.0, seed=7 + nx, periodic=not walls)
    kw = dict(tau=tau, g=g, walls=walls, wall_mode=wall_mode, wall_rho=(0.03, 1.0), **C6)
    o, gl = run_pair(oracle_mod, lbmod, rho, 300, **kw)
    fo, fg = o.fields(), gl.fields()
    assert nrel(fg["rho"], fo["rho"]) <= 1e-12
    # the 5x5 drop dissolves and its velocities fall to ~1e-7: compare those
    # against a velocity scale of 1e-3 instead of their own round-off size
    assert nrel(fg["ubar"], fo["ubar"], floor=1e-3) <= 1e-12
    assert nrel(gl.get_populations(), o.get_f()) <= 1e-12
    oo, og = o.observables(), gl.observables()
    if walls and g[0] != 0.0:
        assert abs(og["mu_r"] - oo["mu_r"]) <= 1e-10 * abs(oo["mu_r"])
    assert abs(og["Q"] - oo["Q"]) <= 1e-12 * max(1e-3, np.abs(fo["ubar"][0]).max()) * ny


def test_fp64_initial_velocity_and_single_step(oracle_mod, lbmod):
    nx, ny = 40, 24
    rho = W.droplet(nx, ny, 7.0, seed=3)
    rng = np.random.default_rng(5)
    u = 0.02 * rng.standard_normal((2, ny, nx))
    o, g = run_pair(oracle_mod, lbmod, rho, 1, u=u, tau=(0.9, 1.4), **C6)
    assert nrel(g.get_populations(), o.get_f()) <= 1e-13


def test_fp32_offset_c1_droplet(oracle_mod, lbmod):
    """FP32 offset populations against the FP64 oracle, 2000 steps."""
    rho = W.c1_droplet_64()
    o, g = run_pair(oracle_mod, lbmod, rho, 2000, precision=1, **C6)
    fo, fg = o.fields(), g.fields()
    er, eu = nrel(fg["rho"], fo["rho"]), nrel(fg["ubar"], fo["ubar"])
    print(f"C1 FP32 2000 steps: rho {er:.2e} u {eu:.2e}")
    assert er <= 1e-5, er
    assert eu <= 1e-5, eu
    oo = o.observables((32, 32, 12))
    g.set_probe(32, 32, 12)
    og = g.observables()
    assert abs(og["dp"] - oo["dp"]) <= 1e-3 * abs(oo["dp"])
    assert abs(og["massA"] - oo["massA"]) <= 1e-5 * oo["massA"]


def test_fp32_offset_channel_mu_r(oracle_mod, lbmod):
    """Body-forced channel with non-wetting walls (g = 1e-5, ten times the
    emulsion workloads' forcing): mu_r of FP32 within 1e-3 of the oracle
    (measured 3.2e-6).  The FP32 velocity carries the systematic rounding bias
    of the momentum-carrying terms under a body force, which grows with g t:
    measured 3.5e-5 on u and 9.4e-6 on rho (the drops advect with the biased
    flow), while an FP64 run with its initial densities perturbed by 1e-7
    moves by only 2.9e-7 and 1.3e-7, so the excess is FP32 arithmetic, not
    amplification; held to 5e-5 (u) and 2e-5 (rho)."""
    nx, ny = 96, 48
    rho, _, _, _ = W.hex_emulsion(nx, ny, 0.4, R=7.0, spread=1.0, gap=3.0, walls=True, seed=21)
    kw = dict(tau=(2.0, 1.0), g=(1e-5, 0.0), walls=1, wall_mode=1, wall_rho=(0.03, 1.0), **C6)
    o, g = run_pair(oracle_mod, lbmod, rho, 1500, precision=1, **kw)
    oo, og = o.observables(), g.observables()
    assert abs(og["mu_r"] - oo["mu_r"]) <= 1e-3 * abs(oo["mu_r"])
    fo, fg = o.fields(), g.fields()
    er, eu = nrel(fg["rho"], fo["rho"]), nrel(fg["ubar"], fo["ubar"])
    print(f"channel 96x48 FP32 1500 steps: rho {er:.2e} u {eu:.2e} mu_r {abs(og['mu_r'] - oo['mu_r']) / abs(oo['mu_r']):.2e}")
    assert er <= 2e-5
    assert eu <= 5e-5


def test_batch_matches_oracle_per_lattice(oracle_mod, lbmod):
    specs = [
        dict(nx=64, ny=64, tau=(1.0, 1.0)),
        dict(nx=37, ny=50, tau=(2.0, 1.0)),
        dict(nx=96, ny=33, tau=(0.6, 1.2), walls=1, wall_mode=1, wall_rho=(0.03, 1.0), g=(1e-5, 0.0)),
    ]
    b = lbmod.Batch(specs, **C6)
    rhos = []
    for i, s in enumerate(specs):
        r = W.droplet(s["nx"], s["ny"], min(s["nx"], s["ny"]) / 4, seed=100 + i, periodic=not s.get("walls", 0))
        rhos.append(r)
        b.set_fields(i, r)
    b.step(200)
    for i, s in enumerate(specs):
        kw = {k: v for k, v in s.items() if k not in ("nx", "ny")}
        o = oracle_mod.OracleSim(s["nx"], s["ny"], **kw, **C6)
        o.set_fields(rhos[i])
        o.step(200)
        fo, fg = o.fields(), b.fields(i)
        assert nrel(fg["rho"], fo["rho"]) <= 1e-12, i
        assert nrel(fg["ubar"], fo["ubar"]) <= 1e-12, i
    obs = b.observables()
    assert len(obs) == 3 and all(x["finite"] == 1.0 for x in obs)


def test_graph_replay_equals_single_steps(lbmod):
    rho = W.droplet(48, 40, 10.0, seed=9)
    a = lbmod.Lattice(48, 40, **C6)
    a.set_fields(rho)
    a.step(64)          # two captured 32-step graphs
    b = lbmod.Lattice(48, 40, **C6)
    b.set_fields(rho)
    for _ in range(64):
        b.step(1)       # direct launches
    assert np.array_equal(a.get_populations(), b.get_populations())
    c = lbmod.Lattice(48, 40, **C6)
    c.set_fields(rho)
    c.step(1)
    c.step(63)          # odd start: one direct step, graph, remainder
    assert np.array_equal(a.get_populations(), c.get_populations())


def test_checkpoint_roundtrip_is_bitwise(lbmod):
    rho = W.droplet(40, 40, 9.0, seed=10)
    for prec in (0, 1):
        a = lbmod.Lattice(40, 40, precision=prec, **C6)
        a.set_fields(rho)
        a.step(200)
        b = lbmod.Lattice(40, 40, precision=prec, **C6)
        b.set_fields(rho)
        b.step(100)
        blob = b.save()
        c = lbmod.Lattice(40, 40, precision=prec, **C6)
        c.load(blob)
        assert c.t == 100
        c.step(100)
        assert np.array_equal(a.get_populations(), c.get_populations())


def test_runs_are_deterministic(lbmod):
    rho = W.droplet(64, 48, 11.0, seed=12)
    out = []
    for _ in range(2):
        a = lbmod.Lattice(64, 48, precision=1, **C6)
        a.set_fields(rho)
        a.step(100)
        a.set_probe(32, 24, 11)
        out.append((a.get_populations(), a.observables()))
    assert np.array_equal(out[0][0], out[1][0])
    a, b = out[0][1], out[1][1]
    assert a.keys() == b.keys()
    for k in a:   # bitwise, NaN (no walls: mu_r) equal to NaN
        assert (a[k] == b[k]) or (np.isnan(a[k]) and np.isnan(b[k])), k


def test_unstable_run_reports_error_without_fault(lbmod):
    """A wildly unstable setting produces non-finite values; the library
    reports LB_EUNSTABLE from the observables, the context stays usable."""
    rho = W.droplet(32, 32, 8.0, seed=13)
    a = lbmod.Lattice(32, 32, tau=(0.5001, 0.5001), G_AB=40.0, G1=-80.0, G2=60.0)
    a.set_fields(rho)
    a.step(400)
    with pytest.raises(lbmod.LBError) as ei:
        a.observables()
    assert ei.value.code == lbmod.LB_EUNSTABLE
    o = a.observables(check=False)
    assert o["finite"] == 0.0
    b = lbmod.Lattice(32, 32, **C6)        # the device still works
    b.set_fields(rho)
    b.step(10)
    assert b.observables()["finite"] == 1.0


def test_device_pointer_init_matches_host_init(lbmod):
    torch = pytest.importorskip("torch")
    rho = W.droplet(40, 30, 8.0, seed=14)
    a = lbmod.Lattice(40, 30, stream=lbmod.current_stream(), **C6)
    a.set_fields_device(torch.from_numpy(rho).cuda())
    b = lbmod.Lattice(40, 30, **C6)
    b.set_fields(rho)
    a.step(50)
    b.step(50)
    assert np.array_equal(a.get_populations(), b.get_populations())
