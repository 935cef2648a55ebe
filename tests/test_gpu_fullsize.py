"""Parity at the benchmark's full sizes, in the launch configuration the
benchmark times (tiles of 32 x 8; FP32 one-pass step staged by TMA, FP64
one-pass step): sampled
nodes against the oracle, which advances a 21 x 21 patch of the initial field
around each sampled node.  After two steps a node depends only on nodes
within 6 lattice units, and its diagnostics (forces included) on nodes within
8, so the patch centre sees exactly the full lattice's values.  Plus mass
conservation over 100 steps at full size."""
import numpy as np
import pytest

from paper_1806_06943_gb300 import workloads as W

pytestmark = pytest.mark.gpu

C6 = dict(G_AB=3.0, G1=-7.4, G2=6.4)
HW = 10   # patch half-width


@pytest.fixture(scope="module")
def emulsion4096():
    rho0, _, _, _ = W.random_emulsion(4096, 4096, 0.6, 8.0, 20.0, seed=W.BASE_SEED + 4)
    return rho0


@pytest.fixture(scope="module")
def lbmod():
    from paper_1806_06943_gb300 import build
    build.build()
    from paper_1806_06943_gb300 import lb
    return lb


def bench_mode(lbmod, precision):
    return lbmod.LB_MODE_TMA if precision == lbmod.LB_FP32 else lbmod.LB_MODE_FUSED


def patch(field, cx, cy):
    ny, nx = field.shape[-2:]
    ys = np.arange(cy - HW, cy + HW + 1) % ny
    xs = np.arange(cx - HW, cx + HW + 1) % nx
    return np.ascontiguousarray(field[..., ys[:, None], xs[None, :]])


def check_samples(oracle_mod, rho0, tau, fields, samples, tol_rho, tol_u):
    """Errors are normwise: relative to the lattice's largest value of the
    field (c12 reading), as in the other parity tests."""
    scales = {k: np.max(np.abs(fields[k])) for k in ("rho", "ubar", "mom")}
    for (cx, cy) in samples:
        o = oracle_mod.OracleSim(2 * HW + 1, 2 * HW + 1, tau=tau, **C6)
        o.set_fields(patch(rho0, cx, cy))
        o.step(2)
        fo = o.fields()
        for key, tol in (("rho", tol_rho), ("ubar", tol_u), ("mom", tol_u)):
            ref = fo[key][..., HW, HW]
            got = fields[key][..., cy, cx]
            assert np.max(np.abs(got - ref)) <= tol * scales[key], (key, cx, cy, got, ref)


def sample_nodes(rng, nx, ny, n=12):
    return [(int(rng.integers(0, nx)), int(rng.integers(0, ny))) for _ in range(n)]


@pytest.mark.parametrize("precision,tol_rho,tol_u", [(0, 1e-13, 1e-12), (1, 1e-6, 1e-5)])
def test_dense_emulsion_4096_sampled(lbmod, oracle_mod, emulsion4096, precision, tol_rho, tol_u):
    n = 4096
    rho0 = emulsion4096
    tau = (3.0, 1.0)
    L = lbmod.Lattice(n, n, tau=tau, precision=precision, **C6)
    L.set_config(bench_mode(lbmod, precision), 8)
    L.set_fields(rho0)
    L.step(2)
    f = L.fields()
    rng = np.random.default_rng(7)
    # half of the samples on droplet interfaces, where the stencils matter
    edge = np.argwhere(np.abs(rho0[0] - np.roll(rho0[0], -1, axis=1)) > 0.5)
    picks = [tuple(int(v) for v in edge[i][::-1]) for i in rng.choice(len(edge), 6, replace=False)]
    check_samples(oracle_mod, rho0, tau, f, picks + sample_nodes(rng, n, n, 6), tol_rho, tol_u)


@pytest.mark.parametrize("precision,tol_rho,tol_u", [(0, 1e-13, 1e-12), (1, 1e-6, 1e-5)])
def test_laplace_sweep_24_sampled(lbmod, oracle_mod, precision, tol_rho, tol_u):
    specs = W.laplace_sweep_specs()
    fields0 = [W.droplet(s["nx"], s["ny"], s["R"], seed=W.BASE_SEED + 1 + i) for i, s in enumerate(specs)]
    b = lbmod.Batch([dict(nx=s["nx"], ny=s["ny"], tau=s["tau"]) for s in specs], precision=precision, **C6)
    b.set_config(bench_mode(lbmod, precision), 8)
    for i, r in enumerate(fields0):
        b.set_fields(i, r)
    b.step(2)
    rng = np.random.default_rng(11)
    for i in (0, 7, 13, 23):
        s = specs[i]
        f = b.fields(i)
        cx, cy = s["nx"] // 2, s["ny"] // 2
        ring = [(int(cx + s["R"] * np.cos(a)), int(cy + s["R"] * np.sin(a))) for a in rng.uniform(0, 2 * np.pi, 3)]
        check_samples(oracle_mod, fields0[i], s["tau"], f, ring + sample_nodes(rng, s["nx"], s["ny"], 2),
                      tol_rho, tol_u)


@pytest.mark.parametrize("precision,tol", [(0, 1e-13), (1, 1e-6)])
def test_mass_conserved_at_full_size(lbmod, emulsion4096, precision, tol):
    n = 4096
    rho0 = emulsion4096
    L = lbmod.Lattice(n, n, tau=(3.0, 1.0), precision=precision, **C6)
    L.set_config(bench_mode(lbmod, precision), 8)
    L.set_fields(rho0)
    o0 = L.observables()
    L.step(100)
    o1 = L.observables()
    for k in ("massA", "massB"):
        assert abs(o1[k] - o0[k]) <= tol * o0[k], (k, o0[k], o1[k])
    M = o0["massA"] + o0["massB"]
    for a in ("x", "y"):
        p0, p1 = o0["momA" + a] + o0["momB" + a], o1["momA" + a] + o1["momB" + a]
        assert abs(p1 - p0) <= 10 * tol * M


def test_dense_emulsion_4096_fp32_vs_fp64_2000_steps(lbmod, emulsion4096):
    """The FP32 offset form against the FP64 form (tied to the oracle above)
    on the full 4096^2 emulsion after 2000 steps, normwise per field.

    The emulsion coarsens (13238 drops, moving and merging), and its fine
    detail is sensitive: an FP64 run whose initial densities are perturbed
    once by 1e-7 (relative) moves single interface nodes by up to 1.4e-4
    (rho) and 2.1e-4 (u) after 2000 steps while 99 % of the nodes move by
    3e-7.  FP32 rounds at every step (~6e-8 of each stored offset): its
    error is 7.6e-6 / 5.9e-6 at the 99th percentile and 7.9e-4 / 1.1e-3 at
    the worst interface nodes, 5.5 times the response to the single FP64
    perturbation.  Asserted: the 99th percentile within the 1e-5 of the FP32
    form, the maximum within ten times the FP64 perturbation's (measured in
    the test), the species masses within 1e-7."""
    n = 4096
    out = {}
    pert = emulsion4096 * (1.0 + 1e-7 * W.uniform_noise(78, 0, n, n, 1.0)[None])
    for name, prec, rho0 in (("fp64", lbmod.LB_FP64, emulsion4096), ("fp64_pert", lbmod.LB_FP64, pert),
                             ("fp32", lbmod.LB_FP32, emulsion4096)):
        L = lbmod.Lattice(n, n, tau=(3.0, 1.0), precision=prec, **C6)
        L.set_config(bench_mode(lbmod, prec), 8)
        L.set_fields(rho0)
        L.step(2000)
        f = L.fields()
        out[name] = ({k: f[k] for k in ("rho", "ubar")}, L.observables())
        del f
        L.close()
    (f64, o64), (fpt, _), (f32, o32) = out["fp64"], out["fp64_pert"], out["fp32"]
    for k in ("rho", "ubar"):
        scale = np.max(np.abs(f64[k]))
        d = np.abs(f32[k] - f64[k]) / scale
        dp = np.abs(fpt[k] - f64[k]) / scale
        q99 = np.quantile(d, 0.99)
        print("%s: 99th percentile %.2e, max %.2e (FP64 perturbed by 1e-7: max %.2e)" % (k, q99, d.max(), dp.max()))
        assert q99 <= 1e-5, (k, q99)
        assert d.max() <= 10.0 * dp.max(), (k, d.max(), dp.max())
    for k in ("massA", "massB"):
        assert abs(o32[k] - o64[k]) <= 1e-7 * o64[k], (k, o32[k], o64[k])
