"""The 3-D extension through the C-ABI against the 3-D oracle.

- FP64: populations, densities and velocities within 1e-12 of the oracle
  after 300 steps on a ragged periodic lattice (a drop off the grid, a body
  force, tau_A != tau_B), observables at 1e-12 (sums) / 1e-10 (derived).
- FP32 offsets: densities and velocities within 1e-5 normwise after 300
  steps.
- A flat interface in the 3-D engine equals the 2-D engine's (both FP64) to
  1e-12: projected onto one axis the 3-D stencils are the 2-D ones."""
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


def nrel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def sphere(nx, ny, nz, c, R, seed=5):
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    d2 = 0.0
    for v, cv, n in ((x, c[0], nx), (y, c[1], ny), (z, c[2], nz)):
        d = np.abs(v - cv)
        d2 = d2 + np.minimum(d, n - d) ** 2
    m = d2 < R * R
    rho = np.empty((2, nz, ny, nx))
    rho[0] = np.where(m, 1.0, 0.03)
    rho[1] = np.where(m, 0.03, 1.0)
    rng = np.random.default_rng(seed)
    return rho + 1e-3 * (2 * rng.random(rho.shape) - 1)


@pytest.fixture(scope="module")
def reference(oracle_mod):
    nx, ny, nz = 41, 27, 22
    rho = sphere(nx, ny, nz, (20.3, 13.1, 10.7), 8.0)
    kw = dict(tau=(0.8, 1.3), g=(1e-5, -2e-6, 3e-6), **C6)
    o = oracle_mod.OracleSim3(nx, ny, nz, **kw)
    o.set_fields(rho)
    o.step(300)
    return (nx, ny, nz), rho, kw, o.fields(), o.get_f(), o.observables((20.3, 13.1, 10.7, 8.0))


def run3(lbmod, shape, rho, kw, precision):
    nx, ny, nz = shape
    g = lbmod.Lattice3(nx, ny, nz, precision=precision, **kw)
    g.set_fields(rho)
    g.step(300)
    g.set_probe(20.3, 13.1, 10.7, 8.0)
    return g


def test_fp64_matches_the_oracle(lbmod, reference):
    shape, rho, kw, fo, fpo, oo = reference
    g = run3(lbmod, shape, rho, kw, lbmod.LB_FP64)
    fg = g.fields()
    assert nrel(fg["rho"], fo["rho"]) <= 1e-12
    assert nrel(fg["ubar"], fo["ubar"]) <= 1e-12
    assert nrel(g.get_populations(), fpo) <= 1e-12
    og = g.observables()
    for k in ("massA", "massB"):
        assert abs(og[k] - oo[k]) <= 1e-12 * oo[k]
    M = oo["massA"] + oo["massB"]
    for k in ("momAx", "momAy", "momAz", "momBx", "momBy", "momBz"):
        assert abs(og[k] - oo[k]) <= 1e-12 * M, k
    for k in ("dp", "R_eff", "umax"):
        assert abs(og[k] - oo[k]) <= 1e-10 * abs(oo[k]), k
    assert og["t"] == 300 and og["finite"] == 1.0


def test_fp32_matches_the_oracle(lbmod, reference):
    shape, rho, kw, fo, _, oo = reference
    g = run3(lbmod, shape, rho, kw, lbmod.LB_FP32)
    fg = g.fields()
    er, eu = nrel(fg["rho"], fo["rho"]), nrel(fg["ubar"], fo["ubar"])
    print("3-D FP32: rho %.2e u %.2e" % (er, eu))
    assert er <= 1e-5 and eu <= 1e-5
    og = g.observables()
    for k in ("massA", "massB"):
        assert abs(og[k] - oo[k]) <= 1e-5 * oo[k]
    assert abs(og["dp"] - oo["dp"]) <= 1e-3 * abs(oo["dp"])


def test_flat_interface_equals_the_2d_engine(lbmod):
    nx = 64
    r2 = W.strip(nx, 5, 32, noise=0.0)
    r3 = np.ascontiguousarray(np.repeat(r2[:, None, :, :], 6, axis=1))
    a = lbmod.Lattice(nx, 5, tau=(0.8, 1.3), **C6)
    a.set_fields(r2)
    a.step(500)
    b = lbmod.Lattice3(nx, 5, 6, tau=(0.8, 1.3), **C6)
    b.set_fields(r3)
    b.step(500)
    fa, fb = a.fields(), b.fields()
    assert np.max(np.abs(fb["rho"] - fa["rho"][:, None])) < 1e-12
    assert np.max(np.abs(fb["ubar"][0] - fa["ubar"][0][None])) < 1e-12

