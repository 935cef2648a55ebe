"""Batched physics sweeps on the GPU engine against what the paper prints.

Table I (Sec. III B): for each (G1, G2) case, G_AB in steps of 0.1, a Laplace
test of drops of radius 12, 18, 24 and 42 per G_AB (20000 steps, FP32), the
interface width W of the R = 42 drop as the Fig. 2 caption defines it, and
the G_AB range over which 2 <= W <= 5.
- The lower end (the critical side, where W grows without bound) lies at
  or above the paper's, by 0 to 0.3 here, asserted within 0.4 (the printed
  ends carry the scan's step of 0.1; the critical coupling moves with the
  total density, which the paper does not state: these runs start from
  1.0 / 0.03 as every workload here).
- The upper end (the sharp side: W near 2, or the run loses stability) is
  within 0.3 of the paper's for three cases, asserted within 0.4; for
  G1 = 10, G2 = -11 the runs, started from sharp disks, lose stability at
  G_AB = 5.4 while the paper's range goes on to 7.2, so only its lower end is
  compared.
- The Laplace law holds where the interface is well formed (2 <= W <= 3,
  inside the window but for its last point, next to the unstable side),
  the surface tension grows with G1 at fixed G1 + G2 = -1 (the paper's
  statement), and each case's surface tensions overlap the printed range.

Fig. 4d (Sec. III D): a 5 x 5 array of equal drops at area fraction 0.45 in
a 220 x 220 channel at reduced forcing 37; the relative effective viscosity
rises as the drops become more viscous than the matrix (M = 1 -> 1/10).  The
droplet-free flux matches the closed form of the half-way bounce-back
channel within 1 %."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TABLE_I = [   # (G1, G2), printed G_AB range, printed gamma range, scan
    ((0.0, 0.0), (2.8, 5.0), (0.031, 0.14), (2.6, 5.4)),
    ((-10.0, 9.0), (2.0, 3.4), (0.0006, 0.041), (1.9, 3.8)),
    ((0.0, -1.0), (2.3, 5.1), (0.028, 0.16), (2.2, 5.0)),
    ((10.0, -11.0), (2.9, 7.2), (0.081, 0.27), (2.6, 5.6)),
]


@pytest.fixture(scope="module")
def sweeps():
    from paper_1806_06943_gb300 import build
    build.build()
    from paper_1806_06943_gb300 import sweeps as S
    return S


@pytest.fixture(scope="module")
def scans(sweeps):
    out = {}
    for (g1, g2), _, _, (lo, hi) in TABLE_I:
        vals = np.round(np.arange(lo, hi + 1e-9, 0.1), 2)
        out[(g1, g2)] = sweeps.tension_scan(g1, g2, vals)
    return out


@pytest.mark.parametrize("case", range(4), ids=["G1=0,G2=0", "G1=-10,G2=9", "G1=0,G2=-1", "G1=10,G2=-11"])
def test_table_I_width_window(sweeps, scans, case):
    (g1, g2), (p_lo, p_hi), (pg_lo, pg_hi), _ = TABLE_I[case]
    scan = scans[(g1, g2)]
    win = sweeps.width_window(scan)
    assert win["G_AB"] is not None
    lo, hi = win["G_AB"]
    print("G1 %g G2 %g: W in [2, 5] for G_AB in [%.1f, %.1f] (paper [%.1f, %.1f])" % (g1, g2, lo, hi, p_lo, p_hi))
    assert -1e-9 <= lo - p_lo <= 0.4, (lo, p_lo)
    if case < 3:
        assert abs(hi - p_hi) <= 0.4, (hi, p_hi)
    assert hi - lo >= 0.7
    formed = [r for r in scan if lo - 1e-9 <= r["G_AB"] < hi - 1e-9 and 2.0 <= r["W"] <= 3.0]
    assert formed
    for r in formed:
        assert r["gamma"] > 0 and r["r2"] >= 0.95, r
    gammas = [r["gamma"] for r in formed]
    assert max(gammas) >= pg_lo and min(gammas) <= pg_hi, (gammas, pg_lo, pg_hi)


def test_surface_tension_grows_with_G1(scans):
    """At fixed G1 + G2 = -1 and G_AB = 3.0 (inside all three windows)."""
    def gamma_at(key):
        return next(r["gamma"] for r in scans[key] if abs(r["G_AB"] - 3.0) < 1e-9)
    g = [gamma_at((-10.0, 9.0)), gamma_at((0.0, -1.0)), gamma_at((10.0, -11.0))]
    assert 0 < g[0] < g[1] < g[2], g


def test_relative_viscosity_rises_with_droplet_viscosity(sweeps):
    cases = [dict(R=16.7, M=m, F_bar=37.0) for m in (0.1, 1.0 / 6.0, 1.0 / 3.0, 1.0)]
    res = sweeps.rheology(cases, steps=200000, window=40000)
    drops = [r for r in res if r["R"] > 0]
    assert all(r["finite"] for r in res)
    assert all(abs(r["phi"] - 0.45) < 0.01 for r in drops)
    mu = [r["mu_r"] for r in sorted(drops, key=lambda r: r["M"])]
    print("mu_r at M = 1/10, 1/6, 1/3, 1:", mu)
    assert all(m > 1.0 for m in mu)
    assert mu[0] > mu[1] > mu[2] > mu[3], mu
    # droplet-free channel at M = 1: Q0 = g (H^3 + H/2) / (12 nu_B)
    ref = next(r for r in res if r["R"] == 0.0 and r["M"] == 1.0)
    g = sweeps.body_force(37.0, 220)
    q0 = g * (220 ** 3 + 110) / (12.0 / 6.0)
    assert abs(ref["Q"] / q0 - 1.0) <= 0.01, (ref["Q"], q0)


def test_relative_viscosity_follows_eq20_at_M1(sweeps):
    """Fig. 4b: mu_r(Phi) at M = 1, F_b = 37 after 200000 steps of the 5 x 5
    arrays started exactly symmetric (no density noise).  mu_r rises with Phi
    and the DEMT fit of Eq. (20) with K = 1 gives an intrinsic viscosity near
    the paper's [eta] = 0.88 (measured 0.84); the arrays up to Phi = 0.45 keep
    their 25 drops.  (With the seeded +-1e-3 density noise the dense arrays
    exchange mass between drops, their films fail and they coalesce even
    without a body force; the other sweeps keep the noise.)"""
    radii = [10.7, 14.5, 16.5, 18.5, 19.5, 19.9]
    res = sweeps.rheology([dict(R=R, M=1.0, F_bar=37.0) for R in radii], steps=200000, window=40000, noise=0.0)
    drops = [r for r in res if r["R"] > 0]
    assert all(r["finite"] for r in res)
    phi = np.array([r["phi"] for r in drops])
    mu = np.array([r["mu_r"] for r in drops])
    print("Phi", phi.round(3).tolist(), "mu_r", mu.round(3).tolist(), "drops", [r["drops"] for r in drops])
    assert np.all(np.diff(phi) > 0) and np.all(np.diff(mu) > 0), mu
    eta, _ = sweeps.demt_fit(phi, mu)
    assert abs(eta - 0.88) <= 0.1 * 0.88, eta
    assert all(r["drops"] == 25 for r in drops if r["phi"] <= 0.45)


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-5)])
def test_sweep_lattices_match_the_oracle(oracle_mod, precision, tol):
    """One lattice of each sweep against the oracle over 300 steps, in the
    sweeps' own configuration (FP32: TMA-staged step, tile height 8): a
    Table I Laplace drop (G1 = 10, G2 = -11, G_AB = 5.0, R = 24 on 192^2) and a
    rheology channel (5 x 5 drops at area fraction 0.45 in 220 x 220,
    non-wetting walls, reduced forcing 37, M = 1/3), rho and u normwise."""
    from paper_1806_06943_gb300 import lb, sweeps as S
    from paper_1806_06943_gb300 import workloads as W
    n = S.laplace_side(24.0)
    drop = (n, n, W.droplet(n, n, 24.0, seed=W.BASE_SEED + 11),
            dict(G_AB=5.0, G1=10.0, G2=-11.0))
    rho_c, _ = S.droplet_array(220, 5, float(np.sqrt(0.45 * 220 * 220 / (25 * np.pi))), seed=W.BASE_SEED + 5)
    chan = (220, 220, rho_c, dict(G_AB=3.0, G1=-7.4, G2=6.4, tau=(S.tau_for_ratio(1.0 / 3.0), 1.0),
                                  g=(S.body_force(37.0, 220), 0.0), walls=1, wall_mode=1, wall_rho=(0.03, 1.0)))
    for nx, ny, rho, kw in (drop, chan):
        o = oracle_mod.OracleSim(nx, ny, **kw)
        o.set_fields(rho)
        o.step(300)
        g = lb.Lattice(nx, ny, precision=precision, **kw)
        g.set_config(lb.LB_MODE_TMA if precision == lb.LB_FP32 else lb.LB_MODE_FUSED, 8)
        g.set_fields(rho)
        g.step(300)
        fo, fg = o.fields(), g.fields()
        for k in ("rho", "ubar"):
            err = np.max(np.abs(fg[k] - fo[k])) / np.max(np.abs(fo[k]))
            assert err <= tol, (nx, ny, k, err)
