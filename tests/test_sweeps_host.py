"""Host-side analysis of the physics sweeps, pinned to closed forms: the
finite-difference interface width of the Fig. 2 caption on a tanh profile,
the drop count (periodic in x), the fit of Eq. (20) and the two limits of
the intrinsic viscosity quoted in Sec. III D."""
import numpy as np
import pytest

from paper_1806_06943_gb300 import sweeps as S
from paper_1806_06943_gb300 import workloads as W


@pytest.mark.parametrize("w", [2.5, 4.0, 7.0])
def test_width_of_tanh_profile(w):
    # rho = mid + (d/2) tanh(2 (x - x0) / w), crossing halfway between nodes:
    # the two nodes around it differ by d tanh(1 / w), so W = 1 / tanh(1 / w)
    x = np.arange(200, dtype=np.float64)
    lo, hi = 0.008, 1.041
    prof = 0.5 * (hi + lo) + 0.5 * (hi - lo) * np.tanh(2.0 * (x - 99.5) / w)
    assert S.interface_width(prof) == pytest.approx(1.0 / np.tanh(1.0 / w), rel=1e-9)
    assert S.interface_width(prof) == pytest.approx(w, rel=0.02 + 1.0 / (3 * w * w))


def test_width_of_a_drop_profile_counts_both_interfaces():
    x = np.arange(300, dtype=np.float64)
    prof = 0.5 + 0.5 * (np.tanh((x - 99.5) / 2.0) - np.tanh((x - 199.5) / 2.0))
    assert S.interface_width(prof / prof.max()) == pytest.approx(1.0 / np.tanh(0.25), rel=1e-6)


def test_count_drops_periodic_in_x():
    rho = W.droplets(64, 40, [(10.0, 20.0), (40.0, 20.0)], [6.0, 6.0], seed=1, periodic=False)
    assert S.count_drops(rho[0]) == 2
    wrap = W.droplets(64, 40, [(0.5, 20.0)], [6.0], seed=1, periodic=False)   # split by x = 0
    assert S.count_drops(wrap[0]) == 1
    arr, phi = S.droplet_array(220, 5, 16.7, seed=3)
    assert S.count_drops(arr[0]) == 25 and phi == pytest.approx(25 * np.pi * 16.7 ** 2 / 220 ** 2, rel=0.02)


def test_demt_fit_recovers_eta():
    phi = np.array([0.2, 0.3, 0.45, 0.6])
    eta, r2 = S.demt_fit(phi, (1.0 - phi) ** -0.88)
    assert eta == pytest.approx(0.88, rel=1e-12) and r2 == pytest.approx(1.0)


def test_intrinsic_viscosity_limits():
    assert S.eta_limits(1.0) == pytest.approx((0.0, 1.75))
    d, t = S.eta_limits(1e-12)          # rigid drops (M = mu_B / mu_A -> 0): 2.5 in both
    assert d == pytest.approx(2.5, rel=1e-9) and t == pytest.approx(2.5, rel=1e-9)
    _, t = S.eta_limits(1e12)           # inviscid drops: Taylor's limit is 1
    assert t == pytest.approx(1.0, rel=1e-9)
    d, t = S.eta_limits(0.1)            # drops ten times more viscous than the matrix
    assert 1.0 < d < t < 2.5


def test_forcing_and_viscosity_ratio_readings():
    # F_b = g rho_B^2 L^3 / (8 mu_B^2) with rho_B = 1, nu_B = 1/6: the
    # Poiseuille centreline Reynolds number u_max L / nu_B
    g = S.body_force(37.0, 220)
    umax = g * 220 ** 2 / (8.0 / 6.0)
    assert umax * 220 * 6.0 == pytest.approx(37.0, rel=1e-12)
    assert S.tau_for_ratio(1.0) == 1.0 and S.tau_for_ratio(3.0) == pytest.approx(0.5 + 0.5 / 3.0)


def test_smooth_droplet_profile():
    n, R, w = 128, 30.0, 4.0
    rho = W.smooth_droplet(n, n, R, w, noise=0.0)
    lo, hi = W.MINORITY, W.MAJORITY
    assert np.allclose(rho[0] + rho[1], hi + lo)
    assert rho[0][64, 64] == pytest.approx(hi, abs=1e-12) and rho[0][0, 0] == pytest.approx(lo, abs=1e-12)
    r = np.abs(np.arange(n) - 64.0)
    prof = rho[0][64]
    # the mean density is crossed at r = R, here on a node: the width
    # definition of the Fig. 2 caption then differences that node and the
    # next, rho(R) - rho(R + 1) = (hi - lo) tanh(2 / w) / 2
    assert np.interp(R, r[64:], prof[64:]) == pytest.approx(0.5 * (hi + lo), abs=1e-12)
    assert S.interface_width(prof) == pytest.approx(2.0 / np.tanh(2.0 / w), rel=1e-9)


def test_disjoining_pressure_quadrature_against_a_closed_form(oracle_mod):
    """Eq. (18) for s(h) = a (1/h - 1/H) on h <= H (zero beyond):
    Pi(h) = s/h - a [1/(2h^2) - 1/(2H^2) - (1/h - 1/H)/H], by both the
    oracle's quadrature and the sweep module's, on a fine grid."""
    from paper_1806_06943_gb300 import sweeps
    a, H = 0.3, 40.0
    h = np.linspace(2.0, H, 4001)
    s = a * (1.0 / h - 1.0 / H)
    exact = s / h - a * (0.5 / h ** 2 - 0.5 / H ** 2 - (1.0 / h - 1.0 / H) / H)
    for Pi in (oracle_mod.disjoining_pressure(h, s), sweeps.disjoining_pressure(h, s)):
        assert np.max(np.abs(Pi - exact)) <= 3e-5 * np.max(np.abs(exact))   # trapezoid, dh = 0.0095
    assert np.allclose(oracle_mod.disjoining_pressure(h[::20], s[::20]),
                       sweeps.disjoining_pressure(h[::20], s[::20]), rtol=0, atol=1e-15)


def test_droplet_array_noise_option():
    """The rheology arrays start exactly symmetric with noise=0: two density
    values only, and the 25 cells of the 5 x 5 array (44 x 44 nodes each)
    are identical."""
    from paper_1806_06943_gb300 import sweeps as S
    from paper_1806_06943_gb300 import workloads as W
    rho, phi = S.droplet_array(220, 5, 16.5, seed=W.BASE_SEED + 12, noise=0.0)
    assert set(np.unique(rho[0]).tolist()) == {W.MINORITY, W.MAJORITY}
    cells = [rho[:, 44 * j:44 * j + 44, 44 * i:44 * i + 44] for j in range(5) for i in range(5)]
    assert all(np.array_equal(c, cells[0]) for c in cells)
    assert abs(phi - 0.445) < 0.005
    noisy, _ = S.droplet_array(220, 5, 16.5, seed=W.BASE_SEED + 12)
    assert 0 < np.max(np.abs(noisy - rho)) <= W.NOISE * (1 + 1e-12)
