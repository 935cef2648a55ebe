"""Invariants the method fixes exactly, and textbook closed forms in its
single-phase limit, checked on the oracle.

- per-species mass is conserved to round-off (Sec. II B, last sentence);
- total momentum changes per step by exactly sum_x rho g (Guo forcing:
  sum_i C_i e_i = (1 - 1/2tau) F and the relaxation term sum to F per site,
  the pair forces of Eqs. 8-9 cancel over a periodic lattice);
- with every coupling off, a body-forced channel with half-way bounce-back
  walls relaxes to the plane Poiseuille parabola u = g/(2 nu)(y+1/2)(H-1/2-y),
  nu = (tau - 1/2)/3 (Sec. II A after Eq. 1), and its flux Q gives mu_r = 1
  against the closed form Q0 = g (H^3 + H/2)/(12 nu)."""
import numpy as np
import pytest

from paper_1806_06943_gb300 import workloads as W


@pytest.mark.parametrize("walls,wall_mode,g", [(0, 0, (0.0, 0.0)), (1, 0, (1e-5, 0.0)), (1, 1, (2e-5, 0.0)),
                                               (0, 0, (1e-5, -2e-5))])
def test_mass_conserved(oracle_mod, walls, wall_mode, g):
    rho = W.droplet(40, 32, 9.0, seed=11, periodic=not walls)
    s = oracle_mod.OracleSim(40, 32, tau=(0.7, 1.6), walls=walls, wall_mode=wall_mode,
                             wall_rho=(0.03, 1.0), g=g)
    s.set_fields(rho)
    o0 = s.observables()
    s.step(400)
    o1 = s.observables()
    assert o1["finite"] == 1.0
    for k in ("massA", "massB"):
        assert abs(o1[k] - o0[k]) / o0[k] < 2e-13, (k, o0[k], o1[k])


@pytest.mark.parametrize("g", [(0.0, 0.0), (3e-6, -1e-6)])
def test_total_momentum_budget_periodic(oracle_mod, g):
    rho = W.droplet(36, 30, 8.0, cx=15.3, cy=13.1, seed=12)
    s = oracle_mod.OracleSim(36, 30, tau=(0.6, 1.9), g=g)
    s.set_fields(rho)
    o0 = s.observables()
    n = 300
    s.step(n)
    o1 = s.observables()
    M = o0["massA"] + o0["massB"]
    for a, ga in zip("xy", g):
        p0 = o0["momA" + a] + o0["momB" + a]
        p1 = o1["momA" + a] + o1["momB" + a]
        assert abs((p1 - p0) - n * M * ga) < 1e-13 * M, (a, p1 - p0, n * M * ga)


def test_species_momentum_exchange_is_not_conserved(oracle_mod):
    """Sanity check of the previous test's power: each species alone is
    not conserved (the pair forces and u^eq exchange momentum)."""
    rho = W.droplet(36, 30, 8.0, cx=15.3, cy=13.1, seed=12)
    s = oracle_mod.OracleSim(36, 30, tau=(0.6, 1.9))
    s.set_fields(rho)
    o0 = s.observables()
    s.step(50)
    o1 = s.observables()
    assert abs(o1["momAx"] - o0["momAx"]) > 1e-6


@pytest.mark.parametrize("tau", [0.55, 1.0])
def test_single_phase_poiseuille(oracle_mod, tau):
    nx, ny, g = 5, 32, 1e-6
    nu = (tau - 0.5) / 3.0
    y = np.arange(ny)
    ua = g / (2 * nu) * (y + 0.5) * (ny - 0.5 - y)
    rho = np.zeros((2, ny, nx))
    rho[1] = 1.0                       # pure continuous phase B, no A
    u = np.zeros((2, ny, nx))
    u[0] = ua[:, None]
    s = oracle_mod.OracleSim(nx, ny, tau=(1.0, tau), G_AB=0.0, G1=0.0, G2=0.0, g=(g, 0.0), walls=1)
    s.set_fields(rho, u)
    s.step(3000)
    ux = s.fields()["ubar"][0][:, 2]
    assert np.max(np.abs(ux - ua)) / ua.max() < 2e-3
    # flux and relative effective viscosity against the closed-form Q0
    o = s.observables()
    assert abs(o["mu_r"] - 1.0) < 2e-3
    # the parabola starts from rest too (checks the forcing, not only the init)
    s2 = oracle_mod.OracleSim(nx, ny, tau=(1.0, tau), G_AB=0.0, G1=0.0, G2=0.0, g=(g, 0.0), walls=1)
    s2.set_fields(rho)
    s2.step(200)
    assert s2.observables()["Q"] > 0.0


def test_uniform_state_is_steady(oracle_mod):
    """A uniform mixture at rest stays exactly at rest (all stencil sums of a
    constant field vanish)."""
    rho = np.empty((2, 12, 10))
    rho[0], rho[1] = 0.3, 0.7
    s = oracle_mod.OracleSim(10, 12)
    s.set_fields(rho)
    s.step(20)
    fl = s.fields()
    assert np.max(np.abs(fl["ubar"])) < 1e-16
    assert np.max(np.abs(fl["rho"][0] - 0.3)) < 1e-15


def test_threaded_oracle_is_bitwise_single_threaded(oracle_mod):
    """The row loops may run on several OpenMP threads; every node's
    arithmetic is the same on any thread, so the state is bitwise that of one
    thread (walls, body force and ragged sizes included)."""
    rho = W.droplet(45, 37, 9.0, seed=15, periodic=False)
    kw = dict(tau=(0.7, 1.6), g=(2e-5, 0.0), walls=1, wall_mode=0)
    runs = []
    n0 = oracle_mod.set_threads(0)
    try:
        for n in (1, 4):
            oracle_mod.set_threads(n)
            s = oracle_mod.OracleSim(45, 37, **kw)
            s.set_fields(rho)
            s.step(120)
            runs.append(s.get_f())
    finally:
        oracle_mod.set_threads(n0)
    assert np.array_equal(runs[0], runs[1])
