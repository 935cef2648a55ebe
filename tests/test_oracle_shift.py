"""Pins of the oracle's velocity-shift forcing, the original two-range
model the paper compares with (Sec. II A, Eq. 4).

- C^SC = (1/tau) [f^eq(rho, u + F tau / rho) - f^eq(rho, u)] has the moments
  sum_i C = 0, sum_i C e_i = F and sum_i C e_i e_i = u F + F u + tau F F / rho
  (from the moments of Eq. 2), the last being the source of the
  tau-dependent kinetic terms of Eq. (14);
- without any force both collisions are the same map, bit for bit;
- mass is conserved and the total momentum budget is n M g, as with Guo
  forcing (the momenta of Eq. 3 without the force are relaxed to a common
  velocity that keeps their weighted sum);
- in the single-phase limit a body-forced channel reaches the plane
  Poiseuille parabola (velocity with half the force, Eq. 6)."""
import numpy as np
import pytest

from paper_1806_06943_gb300 import workloads as W

C6 = dict(G_AB=3.0, G1=-7.4, G2=6.4)


@pytest.mark.parametrize("tau,rho,ux,uy,Fx,Fy", [(1.0, 1.0, 0.0, 0.0, 1e-3, 0.0), (0.7, 0.4, 0.03, -0.02, 2e-3, -1e-3),
                                                 (2.5, 0.03, -0.01, 0.05, -4e-4, 6e-4)])
def test_shift_forcing_moments(oracle_mod, tau, rho, ux, uy, Fx, Fy):
    t = oracle_mod.tables()
    ex, ey = t["ex"].astype(float), t["ey"].astype(float)
    C = oracle_mod.shift_forcing(tau, rho, ux, uy, Fx, Fy)
    sc = max(abs(Fx), abs(Fy))
    assert abs(C.sum()) < 1e-17
    assert abs((C * ex).sum() - Fx) < 1e-13 * sc / min(rho, 1.0) and abs((C * ey).sum() - Fy) < 1e-13 * sc / min(rho, 1.0)
    want_xx = 2 * ux * Fx + tau * Fx * Fx / rho
    want_yy = 2 * uy * Fy + tau * Fy * Fy / rho
    want_xy = ux * Fy + uy * Fx + tau * Fx * Fy / rho
    assert abs((C * ex * ex).sum() - want_xx) < 1e-14
    assert abs((C * ey * ey).sum() - want_yy) < 1e-14
    assert abs((C * ex * ey).sum() - want_xy) < 1e-14


def test_without_force_both_collisions_are_the_same(oracle_mod):
    rho = W.droplet(30, 24, 7.0, seed=3)
    rng = np.random.default_rng(2)
    u = 0.02 * rng.standard_normal((2, 24, 30))
    out = []
    for forcing in (0, 1):
        s = oracle_mod.OracleSim(30, 24, tau=(0.7, 1.9), G_AB=0.0, G1=0.0, G2=0.0, forcing=forcing)
        s.set_fields(rho, u)
        s.step(40)
        out.append(s.get_f())
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("walls,g", [(0, (3e-6, -1e-6)), (1, (1e-5, 0.0))])
def test_shift_model_mass_and_momentum_budget(oracle_mod, walls, g):
    rho = W.droplet(36, 30, 8.0, cx=15.3, cy=13.1, seed=12, periodic=not walls)
    s = oracle_mod.OracleSim(36, 30, tau=(1.0, 1.4), g=g, walls=walls, wall_mode=0, forcing=1, **C6)
    s.set_fields(rho)
    o0 = s.observables()
    s.step(300)
    o1 = s.observables()
    assert o1["finite"] == 1.0
    for k in ("massA", "massB"):
        assert abs(o1[k] - o0[k]) / o0[k] < 2e-13
    if not walls:
        M = o0["massA"] + o0["massB"]
        for a, ga in zip("xy", g):
            p0 = o0["momA" + a] + o0["momB" + a]
            p1 = o1["momA" + a] + o1["momB" + a]
            assert abs((p1 - p0) - 300 * M * ga) < 1e-13 * M


@pytest.mark.parametrize("tau", [0.8, 1.0])
def test_shift_model_single_phase_poiseuille(oracle_mod, tau):
    nx, ny, g = 5, 32, 1e-6
    nu = (tau - 0.5) / 3.0
    y = np.arange(ny)
    ua = g / (2 * nu) * (y + 0.5) * (ny - 0.5 - y)
    rho = np.zeros((2, ny, nx))
    rho[0] = 0.03                # the shift tau F_k / rho_k needs rho_k > 0: A dissolved, not absent
    rho[1] = 1.0
    u = np.zeros((2, ny, nx))
    u[0] = ua[:, None]
    s = oracle_mod.OracleSim(nx, ny, tau=(tau, tau), G_AB=0.0, G1=0.0, G2=0.0, g=(g, 0.0), walls=1, forcing=1)
    s.set_fields(rho, u)
    s.step(3000)
    ux = s.fields()["ubar"][0][:, 2]
    assert np.max(np.abs(ux - ua)) / ua.max() < 2e-3
    assert abs(s.observables()["mu_r"] - 1.0) < 2e-3
