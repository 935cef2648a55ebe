"""Pins of the oracle's lattice tables and single-site operators against
closed forms that the paper's lattice choices fix (Sec. II A-B).

A wrong weight, a swapped velocity, a missing 1/2 in the equilibrium or a
dropped Guo term changes one of the moments checked here."""
from fractions import Fraction

import numpy as np
import pytest

pytestmark = pytest.mark.filterwarnings("ignore")


def test_d2q9_moments(oracle_mod):
    t = oracle_mod.tables()
    w, ex, ey = t["w"], t["ex"].astype(float), t["ey"].astype(float)
    # isotropy up to fourth order for D2Q9, cs^2 = 1/3
    assert abs(w.sum() - 1.0) < 1e-15
    assert abs((w * ex).sum()) < 1e-16 and abs((w * ey).sum()) < 1e-16
    assert abs((w * ex * ex).sum() - 1 / 3) < 1e-15
    assert abs((w * ey * ey).sum() - 1 / 3) < 1e-15
    assert abs((w * ex * ey).sum()) < 1e-16
    assert abs((w * ex ** 4).sum() - 1 / 3) < 1e-15
    assert abs((w * ex ** 2 * ey ** 2).sum() - 1 / 9) < 1e-15
    # every velocity appears once, the rest vector first
    vecs = set(zip(t["ex"].tolist(), t["ey"].tolist()))
    assert len(vecs) == 9 and (t["ex"][0], t["ey"][0]) == (0, 0)
    # w depends only on |e|^2 with w(0)=4/9, w(1)=1/9, w(2)=1/36
    for i in range(9):
        e2 = int(ex[i] ** 2 + ey[i] ** 2)
        assert w[i] == {0: 4 / 9, 1: 1 / 9, 2: 1 / 36}[e2]


def test_d2q25_moments_exact(oracle_mod):
    t = oracle_mod.tables()
    p, jx, jy = t["p"], t["jx"], t["jy"]
    vecs = set(zip(jx.tolist(), jy.tolist()))
    assert vecs == {(a, b) for a in range(-2, 3) for b in range(-2, 3)}
    # exact rational moments rebuilt from the float weights (denominators
    # bounded by 15120): sum p = 1, sum p ex^2 = 1/3, 4th order isotropic
    P = [Fraction(float(x)).limit_denominator(20000) for x in p]
    S0 = sum(P)
    S2 = sum(Pi * a * a for Pi, a in zip(P, jx.tolist()))
    S4 = sum(Pi * a ** 4 for Pi, a in zip(P, jx.tolist()))
    S22 = sum(Pi * a * a * b * b for Pi, a, b in zip(P, jx.tolist(), jy.tolist()))
    S1 = sum(Pi * a for Pi, a in zip(P, jx.tolist()))
    assert S0 == 1 and S1 == 0
    assert S2 == Fraction(1, 3)
    assert S4 == Fraction(4, 7) and S22 == Fraction(4, 21) and S4 == 3 * S22
    # the float sums agree to rounding
    assert abs(p.sum() - 1.0) < 1e-15
    assert abs((p * jx * jx).sum() - 1 / 3) < 1e-15


@pytest.mark.parametrize("rho,ux,uy", [(1.0, 0.0, 0.0), (0.73, 0.05, -0.03), (1.04, -0.1, 0.08), (0.008, 0.02, 0.01)])
def test_equilibrium_moments(oracle_mod, rho, ux, uy):
    """sum f^eq = rho, sum f^eq e = rho u, sum f^eq e e = rho cs^2 I + rho u u.
    The last identity fixes the 1/(2 cs^4) factor of the quadratic term."""
    t = oracle_mod.tables()
    ex, ey = t["ex"].astype(float), t["ey"].astype(float)
    f = oracle_mod.equilibrium(rho, ux, uy)
    tol = 1e-15 * max(1.0, rho) * 8
    assert abs(f.sum() - rho) < tol
    assert abs((f * ex).sum() - rho * ux) < tol
    assert abs((f * ey).sum() - rho * uy) < tol
    assert abs((f * ex * ex).sum() - (rho / 3 + rho * ux * ux)) < tol
    assert abs((f * ey * ey).sum() - (rho / 3 + rho * uy * uy)) < tol
    assert abs((f * ex * ey).sum() - rho * ux * uy) < tol


@pytest.mark.parametrize("tau,ux,uy,Fx,Fy", [(1.0, 0.0, 0.0, 1e-3, 0.0), (0.6, 0.03, -0.02, 2e-3, -1e-3),
                                             (5.5, -0.07, 0.04, -4e-4, 3e-3), (2.0, 0.01, 0.09, 0.0, 5e-3)])
def test_guo_moments(oracle_mod, tau, ux, uy, Fx, Fy):
    """Guo forcing moments: sum C = 0, sum C e = (1 - 1/2tau) F,
    sum C e e = (1 - 1/2tau)(u F + F u)."""
    t = oracle_mod.tables()
    ex, ey = t["ex"].astype(float), t["ey"].astype(float)
    C = oracle_mod.guo(tau, ux, uy, Fx, Fy)
    a = 1.0 - 0.5 / tau
    tol = 1e-17 * 50
    assert abs(C.sum()) < tol
    assert abs((C * ex).sum() - a * Fx) < tol
    assert abs((C * ey).sum() - a * Fy) < tol
    assert abs((C * ex * ex).sum() - a * 2 * ux * Fx) < tol
    assert abs((C * ey * ey).sum() - a * 2 * uy * Fy) < tol
    assert abs((C * ex * ey).sum() - a * (ux * Fy + uy * Fx)) < tol


def test_guo_vanishes_at_tau_half(oracle_mod):
    C = oracle_mod.guo(0.5, 0.02, 0.01, 1e-3, 2e-3)
    assert np.all(C == 0.0)


def test_pseudopotential(oracle_mod):
    """psi(rho) = 1 - exp(-rho): psi(0)=0, psi -> 1, psi(1) = 1 - 1/e,
    slope 1 at the origin."""
    assert oracle_mod.psi(0.0) == 0.0
    assert abs(oracle_mod.psi(50.0) - 1.0) < 1e-15
    assert abs(oracle_mod.psi(1.0) - (1.0 - np.exp(-1.0))) < 1e-16
    h = 1e-7
    assert abs(oracle_mod.psi(h) / h - 1.0) < 1e-6
