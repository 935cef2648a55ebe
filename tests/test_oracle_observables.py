"""Pins of the oracle's observables against values fixed by construction.

- R_eff, the equimolar radius of species A around the probe (Laplace test of
  Sec. III B): for a sharp disk with exact inside and outside densities the
  excess mass of A over the far field is N_in (rho_in - rho_out), N_in the
  number of nodes in the disk, so R_eff = sqrt(N_in / pi) whatever the two
  densities are; N_in is counted here by brute force over the nodes.
- dp, the Laplace pressure jump: the bulk pressure of Eq. (11) of the inside
  densities minus that of the outside densities.
- umax, the flux Q and the momenta: a uniform mixture moving with a uniform
  velocity u0 exerts no interaction force (every stencil sum of Eqs. 8-9
  cancels), so the barycentric velocity (Eq. 7) is u0 at every node,
  max |u| = |u0| and Q = (1/nx) sum u_x = ny u0_x; with a body force the
  momenta carry the half force of Eq. (6), rho_k (u0 + g/2) per node.
- finite: one non-finite population anywhere clears the flag."""
import math

import numpy as np
import pytest

NX, NY = 64, 60


def _disk_fields(cx, cy, R, inside, outside):
    rho = np.empty((2, NY, NX))
    n_in = 0
    for y in range(NY):
        for x in range(NX):
            dx = abs(x - cx)
            dx = min(dx, NX - dx)
            dy = abs(y - cy)
            dy = min(dy, NY - dy)
            if dx * dx + dy * dy < R * R:
                rho[:, y, x] = inside
                n_in += 1
            else:
                rho[:, y, x] = outside
    return rho, n_in


@pytest.mark.parametrize("cx,cy,R,inside,outside", [
    (31.6, 29.2, 12.3, (1.0, 0.03), (0.03, 1.0)),
    (5.25, 57.5, 10.0, (1.02, 0.01), (0.05, 0.93)),   # disk across the periodic corner
    (40.0, 30.0, 17.0, (0.8, 0.2), (0.1, 0.95)),      # node-centred: boundary ties excluded by '<'
])
def test_equimolar_radius_of_a_sharp_disk(oracle_mod, cx, cy, R, inside, outside):
    rho, n_in = _disk_fields(cx, cy, R, inside, outside)
    s = oracle_mod.OracleSim(NX, NY)
    s.set_fields(rho)
    o = s.observables((cx, cy, R))
    assert abs(o["R_eff"] - math.sqrt(n_in / math.pi)) <= 1e-12 * math.sqrt(n_in / math.pi), (o["R_eff"], n_in)
    dp = (oracle_mod.bulk_pressure(s.params, *inside) - oracle_mod.bulk_pressure(s.params, *outside))
    assert abs(o["dp"] - dp) <= 1e-12 * max(1.0, abs(dp))
    assert abs(o["massA"] - (n_in * inside[0] + (NX * NY - n_in) * outside[0])) <= 1e-12 * o["massA"]


def test_no_probe_gives_nan(oracle_mod):
    rho, _ = _disk_fields(30.0, 30.0, 10.0, (1.0, 0.03), (0.03, 1.0))
    s = oracle_mod.OracleSim(NX, NY)
    s.set_fields(rho)
    o = s.observables((0.0, 0.0, 0.0))
    assert math.isnan(o["dp"]) and math.isnan(o["R_eff"])
    assert math.isnan(o["mu_r"])        # no walls, no body force


@pytest.mark.parametrize("u0", [(0.03, -0.04), (-0.012, 0.005), (0.0, 0.0)])
def test_uniform_motion(oracle_mod, u0):
    rho = np.empty((2, NY, NX))
    rho[0], rho[1] = 0.62, 0.41
    u = np.empty((2, NY, NX))
    u[0], u[1] = u0
    s = oracle_mod.OracleSim(NX, NY, tau=(0.7, 1.3))
    s.set_fields(rho, u)
    o = s.observables()
    speed = math.hypot(*u0)
    assert abs(o["umax"] - speed) <= 1e-14
    assert abs(o["Q"] - NY * u0[0]) <= 1e-13
    n = NX * NY
    for k, r in (("A", 0.62), ("B", 0.41)):
        assert abs(o["mom" + k + "x"] - n * r * u0[0]) <= 1e-13 * n * r   # sum of n rounded terms
        assert abs(o["mom" + k + "y"] - n * r * u0[1]) <= 1e-13 * n * r
    assert o["finite"] == 1.0


def test_momenta_carry_half_the_body_force(oracle_mod):
    g = (2e-4, -6e-5)
    u0 = (0.01, 0.02)
    rho = np.empty((2, NY, NX))
    rho[0], rho[1] = 0.55, 0.47
    u = np.empty((2, NY, NX))
    u[0], u[1] = u0
    s = oracle_mod.OracleSim(NX, NY, g=g)
    s.set_fields(rho, u)
    o = s.observables()
    n = NX * NY
    for k, r in (("A", 0.55), ("B", 0.47)):
        for a in range(2):
            want = n * r * (u0[a] + 0.5 * g[a])
            assert abs(o["mom" + k + "xy"[a]] - want) <= 1e-13 * n * r, (k, a)
    assert abs(o["umax"] - math.hypot(u0[0] + 0.5 * g[0], u0[1] + 0.5 * g[1])) <= 1e-14


@pytest.mark.parametrize("bad", [float("nan"), float("inf"), -float("inf")])
def test_one_non_finite_population_clears_finite(oracle_mod, bad):
    rho, _ = _disk_fields(30.0, 30.0, 10.0, (1.0, 0.03), (0.03, 1.0))
    s = oracle_mod.OracleSim(NX, NY)
    s.set_fields(rho)
    f = s.get_f()
    assert s.observables()["finite"] == 1.0
    f[1, 6, 17, 41] = bad
    s.set_f(f)
    assert s.observables()["finite"] == 0.0
