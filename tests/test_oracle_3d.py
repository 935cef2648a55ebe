"""Pins of the oracle's 3-D extension (the paper is 2-D; Sec. II A-B carried
to D3Q19 with a 5 x 5 x 5 mid-range stencil).

- Tables: D3Q19 weights sum to 1 with second moment 1/3 and isotropic fourth
  moment; the mid-range weights q(|e|^2) sum to 1, have second moment 1/3
  and fourth moment 4/7 (the 2-D D2Q25 values) and are isotropic to eighth
  order.  The same conditions written for the 5 x 5 plane single out the
  paper's D2Q25 weights (Sec. II B after Eq. 8), which pins the construction.
- Projected onto one axis, both 3-D stencils are the 2-D ones, and so is
  D3Q19 onto D2Q9's axis projection: a flat interface (profile along x)
  evolves in 3-D exactly as in 2-D (to rounding).
- Mass is conserved and total momentum changes by n M g per n steps.
- A spherical drop obeys the 3-D Laplace law dp = 2 gamma / R with the
  tension of the flat interface (within the spread of the 2-D Laplace
  tests)."""
import itertools
from fractions import Fraction

import numpy as np
import pytest

from paper_1806_06943_gb300 import workloads as W

C6 = dict(G_AB=3.0, G1=-7.4, G2=6.4)


def _frac(v):
    return Fraction(v).limit_denominator(100000)


def test_d3q19_and_midrange_tables(oracle_mod):
    t = oracle_mod.tables3()
    w, e, q = t["w"], t["e"], t["q"]
    assert len({tuple(v) for v in e}) == 19 and sorted((v * v).sum() for v in e) == [0] + [1] * 6 + [2] * 12
    assert abs(w.sum() - 1) < 1e-15
    assert abs((w * e[:, 0] ** 2).sum() - 1 / 3) < 1e-15
    assert abs((w * e[:, 0] ** 4).sum() - 3 * (w * e[:, 0] ** 2 * e[:, 1] ** 2).sum()) < 1e-15
    vecs = list(itertools.product(range(-2, 3), repeat=3))
    qf = {k: _frac(q[k]) for k in range(13)}
    M = lambda a, b, c: sum(qf[x * x + y * y + z * z] * Fraction(x) ** a * Fraction(y) ** b * Fraction(z) ** c
                            for x, y, z in vecs)
    assert sum(qf[x * x + y * y + z * z] for x, y, z in vecs) == 1
    assert M(2, 0, 0) == Fraction(1, 3) and M(4, 0, 0) == Fraction(4, 7)
    assert M(4, 0, 0) == 3 * M(2, 2, 0)
    assert M(6, 0, 0) == 15 * M(2, 2, 2) and M(4, 2, 0) == 3 * M(2, 2, 2)
    K8 = M(4, 2, 2) / 3
    assert M(8, 0, 0) == 105 * K8 and M(6, 2, 0) == 15 * K8 and M(4, 4, 0) == 9 * K8
    for a in range(3):      # isotropy: every axis alike
        assert M(*[4 if i == a else 0 for i in range(3)]) == M(4, 0, 0)
    # the projection onto x is the paper's D2Q25 projection
    t2 = oracle_mod.tables()
    for d in range(-2, 3):
        p3 = sum(qf[x * x + y * y + z * z] for x, y, z in vecs if x == d)
        p2 = sum(_frac(t2["p"][j]) for j in range(25) if t2["jx"][j] == d)
        assert p3 == p2, d


def test_isotropy_conditions_single_out_the_paper_d2q25_weights(oracle_mod):
    """Sum 1, second moment 1/3 and isotropy to eighth order over the six
    shells of the 5 x 5 plane determine the weights: the solution is the
    paper's (247/420, 4/63, 4/135, 1/180, 2/945, 1/15120)."""
    sp = pytest.importorskip("sympy")
    vecs = list(itertools.product(range(-2, 3), repeat=2))
    shells = sorted({x * x + y * y for x, y in vecs})
    p = sp.symbols("p0:%d" % len(shells))
    idx = {e2: i for i, e2 in enumerate(shells)}
    M = lambda a, b: sum(p[idx[x * x + y * y]] * sp.Integer(x) ** a * sp.Integer(y) ** b for x, y in vecs)
    eqs = [sum(p[idx[x * x + y * y]] for x, y in vecs) - 1, M(2, 0) - sp.Rational(1, 3), M(4, 0) - 3 * M(2, 2),
           M(6, 0) - 5 * M(4, 2), 15 * M(8, 0) - 105 * M(6, 2), 9 * M(8, 0) - 105 * M(4, 4)]
    sol = sp.solve(eqs, p, dict=True)
    assert len(sol) == 1
    t2 = oracle_mod.tables()
    for j in range(25):
        e2 = int(t2["jx"][j] ** 2 + t2["jy"][j] ** 2)
        assert abs(float(sol[0][p[idx[e2]]]) - t2["p"][j]) < 1e-16


def test_flat_interface_is_the_2d_one(oracle_mod):
    nx = 64
    r2 = W.strip(nx, 5, 32, noise=0.0)
    r3 = np.ascontiguousarray(np.repeat(r2[:, None, :, :], 5, axis=1))
    s2 = oracle_mod.OracleSim(nx, 5, tau=(0.8, 1.3), **C6)
    s2.set_fields(r2)
    s2.step(1000)
    s3 = oracle_mod.OracleSim3(nx, 5, 5, tau=(0.8, 1.3), **C6)
    s3.set_fields(r3)
    s3.step(1000)
    f2, f3 = s2.fields(), s3.fields()
    assert np.max(np.abs(f3["rho"] - f2["rho"][:, None])) < 1e-12
    assert np.max(np.abs(f3["ubar"][0] - f2["ubar"][0][None])) < 1e-12
    assert np.max(np.abs(f3["ubar"][1:])) < 1e-14


def test_mass_and_momentum_budget_3d(oracle_mod):
    n = 12
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    m = (x - 5.3) ** 2 + (y - 6.1) ** 2 + (z - 5.7) ** 2 < 16.0
    rho = np.empty((2, n, n, n))
    rho[0] = np.where(m, 1.0, 0.03)
    rho[1] = np.where(m, 0.03, 1.0)
    g = (2e-6, -1e-6, 3e-6)
    s = oracle_mod.OracleSim3(n, n, n, tau=(0.7, 1.6), g=g, **C6)
    s.set_fields(rho)
    o0 = s.observables()
    s.step(60)
    o1 = s.observables()
    for k in ("massA", "massB"):
        assert abs(o1[k] - o0[k]) < 2e-13 * o0[k]
    M = o0["massA"] + o0["massB"]
    for a, ga in zip("xyz", g):
        dp = (o1["momA" + a] + o1["momB" + a]) - (o0["momA" + a] + o0["momB" + a])
        assert abs(dp - 60 * M * ga) < 1e-13 * M


def test_sphere_obeys_the_3d_laplace_law(oracle_mod):
    flat = oracle_mod.OracleSim(64, 5, **C6)
    flat.set_fields(W.strip(64, 5, 32, noise=0.0))
    flat.step(8000)
    Pt = flat.pressure_tensor()
    gamma = float(((Pt[0][0] + Pt[1][0]) - (Pt[0][1] + Pt[1][1])).sum()) / 5 / 2
    L, R = 32, 8.0
    z, y, x = np.meshgrid(np.arange(L), np.arange(L), np.arange(L), indexing="ij")
    m = (x - L / 2) ** 2 + (y - L / 2) ** 2 + (z - L / 2) ** 2 < R * R
    rho = np.empty((2, L, L, L))
    rho[0] = np.where(m, 1.0, 0.03)
    rho[1] = np.where(m, 0.03, 1.0)
    s = oracle_mod.OracleSim3(L, L, L, **C6)
    s.set_fields(rho)
    s.step(600)
    o = s.observables((L / 2, L / 2, L / 2, R))
    assert o["finite"] == 1.0
    g3 = o["dp"] * o["R_eff"] / 2
    assert abs(g3 / gamma - 1) < 0.12, (g3, gamma)
