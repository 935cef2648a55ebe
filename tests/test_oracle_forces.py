"""Pins of the oracle's interaction forces (Eqs. 8-9) against exact lattice
sums on plane waves, and of the bulk equation of state (Eq. 11) against the
forces in the long-wave limit.

For psi(x) = a + b sin(k x + l y) every stencil sum has a closed form:
  sum_i w_i psi(x+e_i) e_ix = b cos(theta) S(k, l),
  S9(k, l)  = (sin k / 9)(2 + cos l)                                  (D2Q9)
  S25(k, l) = 2 sin k (p1 + 2 p2 cos l + 2 p5 cos 2l)
            + 4 sin 2k (p4 + 2 p5 cos l + 2 p8 cos 2l)                 (D2Q25)
(the cosine parts cancel under e -> -e).  Each term is switched on alone so a
wrong sign, weight, belt or operand shows up in exactly one check."""
import math

import numpy as np
import pytest

W1, W2 = 1 / 9, 1 / 36
P1, P2, P4, P5, P8 = 4 / 63, 4 / 135, 1 / 180, 2 / 945, 1 / 15120


def S9(k, l):
    return math.sin(k) / 9.0 * (2.0 + math.cos(l))


def S25(k, l):
    return (2 * math.sin(k) * (P1 + 2 * P2 * math.cos(l) + 2 * P5 * math.cos(2 * l))
            + 4 * math.sin(2 * k) * (P4 + 2 * P5 * math.cos(l) + 2 * P8 * math.cos(2 * l)))


def _wave(nx, ny, mx, my, a, b):
    y, x = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    k, l = 2 * math.pi * mx / nx, 2 * math.pi * my / ny
    th = k * x + l * y
    return a + b * np.sin(th), np.cos(th), k, l


def _forces(oracle_mod, rho, **kw):
    ny, nx = rho.shape[1:]
    s = oracle_mod.OracleSim(nx, ny, **kw)
    s.set_fields(rho)
    return s.fields()["force"]


@pytest.mark.parametrize("mx,my", [(1, 0), (0, 1), (2, 1), (3, -2)])
@pytest.mark.parametrize("term", ["G1", "G2", "GAB"])
def test_plane_wave_forces(oracle_mod, mx, my, term):
    nx, ny = 24, 20
    amps = (0.2, -0.1)
    wA, c, k, l = _wave(nx, ny, mx, my, 0.5, amps[0])
    wB, _, _, _ = _wave(nx, ny, mx, my, 0.3, amps[1])
    if term == "GAB":
        rho = np.stack([wA, wB])                              # densities are the waves
    else:
        rho = np.stack([-np.log1p(-wA), -np.log1p(-wB)])      # psi = 1 - exp(-rho) are the waves
    G = {"G1": 0.0, "G2": 0.0, "G_AB": 0.0}
    coupling = 1.7
    G[{"G1": "G1", "G2": "G2", "GAB": "G_AB"}[term]] = coupling
    F = _forces(oracle_mod, rho, **G)
    psi = 1.0 - np.exp(-rho)
    for kk in range(2):
        if term == "G1":
            ex = -coupling * psi[kk] * amps[kk] * c * S9(k, l)
            ey = -coupling * psi[kk] * amps[kk] * c * S9(l, k)
        elif term == "G2":
            ex = -coupling * psi[kk] * amps[kk] * c * S25(k, l)
            ey = -coupling * psi[kk] * amps[kk] * c * S25(l, k)
        else:
            # Eq. (9): own density times the stencil sum of the OTHER species' density
            ex = -coupling * rho[kk] * amps[1 - kk] * c * S9(k, l)
            ey = -coupling * rho[kk] * amps[1 - kk] * c * S9(l, k)
        assert np.max(np.abs(F[kk, 0] - ex)) < 5e-15, (term, kk, "x")
        assert np.max(np.abs(F[kk, 1] - ey)) < 5e-15, (term, kk, "y")


def test_forces_sum_to_zero_periodic(oracle_mod):
    """Eqs. (8)-(9) are pair forces: on a periodic lattice the competing
    force of each species and the summed repulsion add up to zero."""
    rng = np.random.default_rng(3)
    rho = 0.5 + 0.4 * rng.random((2, 16, 18))
    F = _forces(oracle_mod, rho, G_AB=3.0, G1=-7.4, G2=6.4)
    FA = _forces(oracle_mod, rho, G_AB=0.0, G1=-7.4, G2=6.4)
    scale = np.abs(F).max()
    assert abs(FA[0, 0].sum()) < 1e-13 * scale * F[0, 0].size
    assert abs(FA[1, 1].sum()) < 1e-13 * scale * F[0, 0].size
    assert abs((F[0, 0] + F[1, 0]).sum()) < 1e-13 * scale * F[0, 0].size
    assert abs((F[0, 1] + F[1, 1]).sum()) < 1e-13 * scale * F[0, 0].size


def test_body_force_is_rho_g(oracle_mod):
    rng = np.random.default_rng(4)
    rho = 0.2 + rng.random((2, 8, 10))
    s = oracle_mod.OracleSim(10, 8, G_AB=0.0, G1=0.0, G2=0.0, g=(2e-5, -3e-6))
    s.set_fields(rho)
    fl = s.fields()
    F, r = fl["force"], fl["rho"]          # r = sum_i f^eq(rho), rho up to rounding
    assert np.array_equal(F[:, 0], r * 2e-5)
    assert np.array_equal(F[:, 1], r * -3e-6)
    assert np.allclose(r, rho, rtol=1e-15, atol=0)


@pytest.mark.parametrize("G_AB,G1,G2", [(3.0, -7.4, 6.4), (0.0, -2.0, 0.0), (0.0, 0.0, 1.5), (2.5, 0.0, 0.0)])
def test_long_wave_force_matches_bulk_eos(oracle_mod, G_AB, G1, G2):
    """In the long-wave limit the summed interaction force is minus the
    gradient of the non-ideal part of the bulk pressure, Eq. (11):
    sum_k F_k = -grad[p_b - cs^2 (rho_A + rho_B)] + O(k^2)."""
    nx, ny = 256, 5
    x = np.arange(nx)
    k = 2 * np.pi / nx
    rA = 0.6 + 0.25 * np.sin(k * x)
    rB = 0.4 - 0.15 * np.cos(k * x)
    rho = np.stack([np.tile(rA, (ny, 1)), np.tile(rB, (ny, 1))])
    F = _forces(oracle_mod, rho, G_AB=G_AB, G1=G1, G2=G2)
    Fx = (F[0, 0] + F[1, 0])[2]
    par = oracle_mod.make_params(nx, ny, G_AB=G_AB, G1=G1, G2=G2)
    pnon = np.array([oracle_mod.bulk_pressure(par, a, b) for a, b in zip(rA, rB)]) - (rA + rB) / 3.0
    kk = 2 * np.pi * np.fft.fftfreq(nx)
    dp = np.real(np.fft.ifft(1j * kk * np.fft.fft(pnon)))
    err = np.max(np.abs(Fx + dp)) / np.max(np.abs(dp))
    assert err < 2e-3, err


def test_mirror_walls_equal_reflected_periodic_lattice(oracle_mod):
    """Mirrored ghost rows (neutral walls) are the reflection of the fluid
    about y = -1/2 and y = ny - 1/2: the forces at every fluid row equal those
    of a periodic lattice twice as high holding the reflected field."""
    rng = np.random.default_rng(8)
    nx, ny = 12, 8
    rho = 0.3 + 0.6 * rng.random((2, ny, nx))
    Fw = _forces(oracle_mod, rho, walls=1, wall_mode=0, **dict(G_AB=3.0, G1=-7.4, G2=6.4))
    big = np.concatenate([rho, rho[:, ::-1, :]], axis=1)       # rows ny..2ny-1 reflected
    Fp = _forces(oracle_mod, big, **dict(G_AB=3.0, G1=-7.4, G2=6.4))
    assert np.array_equal(Fw, Fp[:, :, :ny, :])


def test_fixed_walls_equal_periodic_lattice_with_wall_rows(oracle_mod):
    """Fixed ghost rows (non-wetting walls) act like two rows of the wall
    densities on each side of a periodic lattice."""
    rng = np.random.default_rng(9)
    nx, ny = 12, 8
    rho = 0.3 + 0.6 * rng.random((2, ny, nx))
    wall = (0.03, 1.0)
    Fw = _forces(oracle_mod, rho, walls=1, wall_mode=1, wall_rho=wall, **dict(G_AB=3.0, G1=-7.4, G2=6.4))
    pad = np.empty((2, 4, nx))
    pad[0], pad[1] = wall
    big = np.concatenate([rho, pad], axis=1)
    Fp = _forces(oracle_mod, big, **dict(G_AB=3.0, G1=-7.4, G2=6.4))
    # the padded rows hold sum_i f^eq(0.03) rather than 0.03 itself: rounding only
    assert np.max(np.abs(Fw - Fp[:, :, :ny, :])) < 1e-15
