"""The batched Laplace sweep and the channel emulsions at their full sizes and
step counts: the FP32 offset form against the FP64 form (whose arithmetic the
FP64 parity tests tie to the oracle), at the tolerance stated for the
observables, 1e-3 relative on the Laplace pressure jump and on the relative
effective viscosity, and the Laplace law across the sweep.

The pressure jump of the largest drops is only ~1e-3 of the ~0.35 bulk
pressure, and after 20000 steps the FP32 bulk pressures carry a bias of
~1e-6 (a density bias of that size): the relative bound is asserted where
dp >= 2e-3 (R <= 20), and for every drop the absolute error is held under
2e-6; the surface tension fitted over each ratio's eight drops agrees to
1e-3.  The channel emulsions are compared where mu_r is well conditioned (see
the test's own note)."""
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


def bench_mode(lbmod, precision):
    """The benchmark's configuration: FP32 staged by TMA, FP64 one-pass."""
    return lbmod.LB_MODE_TMA if precision == lbmod.LB_FP32 else lbmod.LB_MODE_FUSED


def sweep(lbmod, precision, steps):
    specs = W.laplace_sweep_specs()
    b = lbmod.Batch([dict(nx=s["nx"], ny=s["ny"], tau=s["tau"]) for s in specs], precision=precision, **C6)
    b.set_config(bench_mode(lbmod, precision), 8)
    for i, s in enumerate(specs):
        b.set_fields(i, W.droplet(s["nx"], s["ny"], s["R"], seed=W.BASE_SEED + 1 + i))
        b.set_probe(i, s["nx"] / 2, s["ny"] / 2, s["R"])
    b.step(steps)
    return specs, b.observables()


def test_laplace_sweep_fp32_vs_fp64_20k_steps(lbmod):
    steps = 20000
    specs, o32 = sweep(lbmod, lbmod.LB_FP32, steps)
    _, o64 = sweep(lbmod, lbmod.LB_FP64, steps)
    for s, a, b in zip(specs, o32, o64):
        assert a["finite"] == 1.0 and b["finite"] == 1.0
        err = abs(a["dp"] - b["dp"])
        assert err <= 2e-6, (s, a["dp"], b["dp"])
        if abs(b["dp"]) >= 2e-3:
            assert err <= 1e-3 * abs(b["dp"]), (s, a["dp"], b["dp"])
        assert abs(a["massA"] - b["massA"]) <= 1e-5 * b["massA"]

    def fit(obs, ratio):
        pts = np.array([(1.0 / o["R_eff"], o["dp"]) for s, o in zip(specs, obs) if s["ratio"] == ratio])
        A = np.vstack([pts[:, 0], np.ones(len(pts))]).T
        (gamma, c), *_ = np.linalg.lstsq(A, pts[:, 1], rcond=None)
        f = A @ np.array([gamma, c])
        r2 = 1 - ((pts[:, 1] - f) ** 2).sum() / ((pts[:, 1] - pts[:, 1].mean()) ** 2).sum()
        return gamma, r2

    # Laplace law per viscosity ratio: dp linear in 1/R_eff, same surface tension
    for ratio in (1.0, 3.0, 10.0):
        g64, r2 = fit(o64, ratio)
        g32, _ = fit(o32, ratio)
        assert r2 > 0.99 and 0.02 < g64 < 0.07, (ratio, g64, r2)
        assert abs(g32 - g64) <= 1e-3 * g64, (ratio, g32, g64)


NX, NY = 1024, 256
CHECKPOINTS = (10000, 20000, 30000, 40000, 50000)
CASES = [(phi, tau_d) for phi in (0.3, 0.5, 0.7) for tau_d in (2.0 / 3.0, 2.0)]
DTAU_B = 1e-5      # a relative change of 2e-5 in the continuous phase's viscosity


def channel_spec(tau_d, tau_b=1.0):
    return dict(nx=NX, ny=NY, tau=(tau_d, tau_b), walls=1, wall_mode=1, wall_rho=(0.03, 1.0), g=(1e-6, 0.0))


def channel_emulsion(phi):
    return W.hex_emulsion(NX, NY, phi, R=12.0, spread=2.0, gap=3.0, walls=True, seed=W.BASE_SEED + 2)


def channel_field(phi):
    return channel_emulsion(phi)[0]


# area fraction each configured one reaches (within 0.01), for the test ids
PHI_ACHIEVED = {phi: channel_emulsion(phi)[3] for phi in (0.3, 0.5, 0.7)}


def run_series(lbmod, precision, specs, fields):
    """mu_r of every lattice at every checkpoint, all lattices in one batch."""
    b = lbmod.Batch(specs, precision=precision, **C6)
    b.set_config(bench_mode(lbmod, precision), 8)
    for i, r in enumerate(fields):
        b.set_fields(i, r)
    out, t = [], 0
    for T in CHECKPOINTS:
        b.step(T - t)
        t = T
        obs = b.observables()
        assert all(o["finite"] == 1.0 for o in obs)
        out.append([o["mu_r"] for o in obs])
    return np.array(out).T          # (lattice, checkpoint)


@pytest.fixture(scope="module")
def channel_runs(lbmod):
    """The six emulsions (area fraction 0.3, 0.5, 0.7; viscosity ratio 1/3, 3)
    in FP32, and in FP64 at tau_B = 1 and at tau_B = 1 -+ 1e-5."""
    fields = [channel_field(phi) for phi, _ in CASES]
    mu32 = run_series(lbmod, lbmod.LB_FP32, [channel_spec(td) for _, td in CASES], fields)
    specs64 = [channel_spec(td, tb) for tb in (1.0, 1.0 - DTAU_B, 1.0 + DTAU_B) for _, td in CASES]
    mu64 = run_series(lbmod, lbmod.LB_FP64, specs64, fields * 3).reshape(3, len(CASES), len(CHECKPOINTS))
    return mu32, mu64


@pytest.mark.parametrize("case", range(len(CASES)),
                         ids=["phi%.1f(%.3f)-M%s" % (p, PHI_ACHIEVED[p], "3" if t > 1 else "1/3") for p, t in CASES])
def test_channel_emulsion_fp32_vs_fp64_50k_steps(channel_runs, case):
    """1024 x 256 channel, non-wetting walls, g = 1e-6, droplets of radius
    12 +- 2 on a jittered hexagonal lattice (clipped to keep the gaps: at 0.7
    the radii are 10-10.7 with 2.5-node gaps), the id giving the area
    fraction reached; viscosity ratio mu_d/mu_c = 3
    (tau_d = 2) or 1/3 (tau_d = 2/3); mu_r every 10000 steps up to 50000.

    Where mu_r is well conditioned (the FP64 runs at tau_B -+ 1e-5 move it by
    less than 1e-4) FP32 agrees with FP64 to 1e-3.  Where a coalescence sits
    so close to its threshold that the 2e-5 change of the continuous phase's
    viscosity moves mu_r by more (an FP32 flux bias of 1e-5..1e-4 is of that
    order), FP32 lies inside the FP64 runs' spread widened by 1e-3.  The first
    checkpoint is required to be well conditioned."""
    mu32, mu64 = channel_runs
    a, (b, bm, bp) = mu32[case], mu64[:, case]
    assert np.all(b > 1.0)                # droplets raise the effective viscosity
    for j, t in enumerate(CHECKPOINTS):
        spread = max(abs(bm[j] - b[j]), abs(bp[j] - b[j]))
        print("step %d mu_r fp32 %.6f fp64 %.6f (tau_B -+1e-5: %.6f %.6f) rel err %.1e spread %.1e" %
              (t, a[j], b[j], bm[j], bp[j], abs(a[j] / b[j] - 1), spread / b[j]))
        if j == 0:
            assert spread <= 1e-4 * b[j], (t, b[j], bm[j], bp[j])
        if spread <= 1e-4 * b[j]:
            assert abs(a[j] - b[j]) <= 1e-3 * b[j], (t, a[j], b[j])
        else:
            lo, hi = min(b[j], bm[j], bp[j]), max(b[j], bm[j], bp[j])
            assert lo - 1e-3 * b[j] <= a[j] <= hi + 1e-3 * b[j], (t, a[j], b[j], bm[j], bp[j])


def test_single_phase_channel_fp32_vs_fp64_50k_steps(lbmod):
    """No droplets (species A only at its dissolved density): the flux of the
    body-force-driven channel, FP32 against FP64 after 50000 steps, 1e-3 on
    mu_r; the FP32 flux error is an accumulation of roundings of the
    momentum-carrying terms, ~4e-4 here."""
    rho = np.empty((2, NY, NX))
    rho[0], rho[1] = 0.03, 1.0
    mu = {}
    for prec in (lbmod.LB_FP32, lbmod.LB_FP64):
        L = lbmod.Lattice(NX, NY, tau=(2.0, 1.0), g=(1e-6, 0.0), walls=1, wall_mode=1, wall_rho=(0.03, 1.0),
                          precision=prec, **C6)
        L.set_config(bench_mode(lbmod, prec), 8)
        L.set_fields(rho)
        L.step(50000)
        mu[prec] = L.observables()["mu_r"]
    assert abs(mu[lbmod.LB_FP32] - mu[lbmod.LB_FP64]) <= 1e-3 * mu[lbmod.LB_FP64]
