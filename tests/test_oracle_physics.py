"""Physics pins of the oracle from what the paper states (Secs. III A-C,
Table I, Fig. 2) and from closed forms of the continuum limit.

Runs of a few thousand steps on small lattices; the values printed in the
paper live in tests/golden/paper_values.json with their citations."""
import json
import os

import numpy as np
import pytest

from paper_1806_06943_gb300 import workloads as W

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
C6 = dict(G_AB=3.0, G1=-7.4, G2=6.4)


def _width(prof):
    """Interface width W = (rho_max - rho_min) / (d rho/dx at the mid level),
    by finite difference between the two nodes that bracket the mid level
    (Sec. III B, Fig. 2 caption)."""
    mx, mn = prof.max(), prof.min()
    mid = 0.5 * (mx + mn)
    for x in range(len(prof) - 1):
        if (prof[x] - mid) * (prof[x + 1] - mid) <= 0 and prof[x] != prof[x + 1]:
            return (mx - mn) / abs(prof[x + 1] - prof[x])
    raise AssertionError("no interface")


@pytest.fixture(scope="module")
def flat_equilibrium(oracle_mod):
    s = oracle_mod.OracleSim(64, 5, **C6)
    s.set_fields(W.strip(64, 5, 32, noise=0.0))
    s.step(8000)
    return s.fields()


def test_flat_interface_at_rest_and_symmetric(flat_equilibrium):
    fl = flat_equilibrium
    assert np.max(np.abs(fl["ubar"])) < 1e-8
    rA, rB = fl["rho"][0][2], fl["rho"][1][2]
    # species exchange symmetry of the model with equal couplings
    assert np.max(np.abs(rA - np.roll(rB, 32))) < 1e-12
    # rows are identical (a flat interface stays flat)
    assert np.max(np.abs(fl["rho"][0] - rA[None, :])) < 1e-14


def test_flat_interface_bulk_density_matches_fig2(flat_equilibrium):
    g = GOLD["fig2_interface"]
    rA = flat_equilibrium["rho"][0][2]
    assert abs(rA[32] - g["rho_A_max"]) < 2e-3


def test_flat_interface_width_in_range(flat_equilibrium):
    w = _width(flat_equilibrium["rho"][0][2])
    lo, hi = GOLD["table_I"]["width_bounds"]
    assert lo <= w <= hi


@pytest.mark.parametrize("G1,G2,G_AB", [(c["G1"], c["G2"], gab) for c in GOLD["table_I"]["cases"]
                                        for gab in c["G_AB"]][:6])
def test_table_I_range_ends_give_widths_in_bounds(oracle_mod, G1, G2, G_AB):
    s = oracle_mod.OracleSim(64, 5, G_AB=G_AB, G1=G1, G2=G2)
    s.set_fields(W.strip(64, 5, 32, noise=0.0))
    s.step(6000)
    w = _width(s.fields()["rho"][0][2])
    lo, hi = GOLD["table_I"]["width_bounds"]
    assert lo - 0.5 <= w <= hi + 0.5, w


@pytest.mark.parametrize("tau", [(0.6, 1.5), (0.55, 5.5)])
def test_flat_equilibrium_is_tau_independent(oracle_mod, flat_equilibrium, tau):
    """The equilibrium reached at tau_A = tau_B = 1 stays put when restarted
    at other viscosity ratios (M = 10 and M = 100 here): the Guo forcing
    removes the tau-dependent pressure-tensor terms (Sec. II B, Sec. III C)."""
    rho0 = flat_equilibrium["rho"]
    s = oracle_mod.OracleSim(64, 5, tau=tau, **C6)
    s.set_fields(rho0)
    s.step(3000)
    fl = s.fields()
    assert np.max(np.abs(fl["rho"] - rho0)) < 5e-4
    assert np.max(np.abs(fl["ubar"])) < 2e-4


def test_laplace_law(oracle_mod):
    """Delta p = gamma / R over four radii: linear in 1/R with a small
    intercept, gamma near the printed 0.04 (Sec. III D)."""
    pts = []
    for R, L in [(8, 48), (10, 56), (12, 64), (16, 72)]:
        s = oracle_mod.OracleSim(L, L, **C6)
        s.set_fields(W.droplet(L, L, float(R)))
        s.step(1500)
        o = s.observables((L / 2, L / 2, float(R)))
        pts.append((1.0 / o["R_eff"], o["dp"]))
    x, y = np.array(pts).T
    A = np.vstack([x, np.ones_like(x)]).T
    (gamma, c), *_ = np.linalg.lstsq(A, y, rcond=None)
    fit = A @ np.array([gamma, c])
    r2 = 1 - ((y - fit) ** 2).sum() / ((y - y.mean()) ** 2).sum()
    assert r2 > 0.99
    assert abs(c) < 0.1 * gamma / 16
    gold = GOLD["surface_tension"]
    assert abs(gamma - gold["value"]) < gold["tolerance_rel"] * gold["value"], gamma


@pytest.mark.parametrize("tauB", [0.6667, 1.0, 2.0, 5.5])
def test_layered_poiseuille_core_curvature(oracle_mod, tauB):
    """Two-component Poiseuille flow (Sec. III A, Eq. 19), B in the core,
    A at the walls.  In each bulk layer Eq. (19) is a parabola with
    u'' = -F_b/mu; in the core the curvature must match F_b = rho g with the
    mixture viscosity mu = cs^2 sum_k rho_k (tau_k - 1/2) of the local bulk
    densities (B majority, A minority)."""
    nx, ny = 5, 64
    b, a = ny / 2, ny / 4
    y = np.arange(ny) - (ny - 1) / 2
    tauA = 1.0
    nuA, nuB = (tauA - 0.5) / 3, (tauB - 0.5) / 3
    g = 0.05 / (a * a / (2 * nuB) + (b * b - a * a) / (2 * nuA))
    ua = np.where(np.abs(y) < a, g / (2 * nuB) * (a * a - y * y) + g / (2 * nuA) * (b * b - a * a),
                  g / (2 * nuA) * (b * b - y * y))
    u = np.zeros((2, ny, nx))
    u[0] = ua[:, None]
    s = oracle_mod.OracleSim(nx, ny, tau=(tauA, tauB), g=(g, 0.0), walls=1, wall_mode=0, **C6)
    s.set_fields(W.layered_channel(nx, ny, a), u)
    s.step(20000)
    fl = s.fields()
    ux, r = fl["ubar"][0][:, 2], fl["rho"][:, :, 2]
    core = np.abs(y) < a - 5
    curv = 2 * np.polyfit(y[core], ux[core], 2)[0]
    rb = r[:, core].mean(axis=1)
    mu = (rb[0] * (tauA - 0.5) + rb[1] * (tauB - 0.5)) / 3.0
    pred = -(rb.sum()) * g / mu
    assert abs(curv / pred - 1.0) < 1e-2, (curv, pred)
    if tauB == 1.0:
        # equal viscosities: the whole profile is Eq. (19) up to the
        # diffuse-interface density dip ("small discrepancies near the interface")
        far = np.abs(np.abs(y) - a) > 4
        err = np.sqrt(((ux - ua)[far] ** 2).mean() / (ua[far] ** 2).mean())
        assert err < 0.03, err
        assert abs(ux[ny // 2] - GOLD["poiseuille"]["centreline_velocity"]) < 0.003


def test_pressed_droplets_do_not_coalesce(oracle_mod):
    """Positive disjoining pressure of the two-range model keeps a thin B
    film between two pressed A droplets, while the single-range model
    (G1 = G2 = 0) lets them coalesce (Sec. II C, Sec. III C)."""
    nx, ny, R, gap = 80, 40, 12.0, 2.0
    cx, d = nx / 2, R + gap / 2
    rho = W.droplets(nx, ny, [(cx - d, ny / 2), (cx + d, ny / 2)], [R, R], noise=0.0)
    film = (slice(ny // 2 - 1, ny // 2 + 1), slice(int(cx) - 1, int(cx) + 1))
    two = oracle_mod.OracleSim(nx, ny, **C6)
    two.set_fields(rho)
    two.step(1500)
    one = oracle_mod.OracleSim(nx, ny, G_AB=3.5, G1=0.0, G2=0.0)
    one.set_fields(rho)
    one.step(1500)
    assert two.fields()["rho"][1][film].min() > 0.5
    assert one.fields()["rho"][1][film].min() < 0.1
