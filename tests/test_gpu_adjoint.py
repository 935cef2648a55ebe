"""The hand-written discrete adjoint (lb_grad) against central finite
differences (h = 1e-4) of the FP64 oracle, for the relative effective
viscosity of a body-forced channel and the Laplace pressure jump of a drop,
through torch.autograd, and on the 512 x 128 channel emulsion over 5000 steps
against finite differences of the FP64 GPU forward.  Tolerance: 1e-4
relative per parameter of (G_AB, G1, G2, tau_A, tau_B), with an absolute
floor of 1e-8 for the finite-difference truncation (h^2 times third
derivatives of order one).

The FP32 forward (offset populations, recomputed in FP32, converted to FP64
populations for the FP64 adjoint) is held to the same 1e-4 against the FP64
gradient and the FP64 finite differences: it differs from them by 2e-5 to
4e-5.  Finite differences of the FP32 forward itself are no reference: its
mu_r carries rounding of ~1e-6 relative, which h = 1e-4 turns into errors of
~1e-2.

One adjoint step on its own (lb_step_vjp): <J v, w> = <v, J^T w> for the
linearised time step J, with J v from central differences of the FP64
forward step, and <w, dStep/dtheta> against central differences in each
parameter."""
import numpy as np
import pytest

from paper_1806_06943_gb300 import workloads as W

pytestmark = pytest.mark.gpu

THETA0 = np.array([3.0, -7.4, 6.4, 1.5, 1.0])


@pytest.fixture(scope="module")
def lbmod():
    from paper_1806_06943_gb300 import build
    build.build()
    from paper_1806_06943_gb300 import lb
    return lb


def oracle_J(oracle_mod, theta, rho, nsteps, objective, probe=None, **kw):
    o = oracle_mod.OracleSim(rho.shape[2], rho.shape[1], G_AB=theta[0], G1=theta[1], G2=theta[2],
                             tau=(theta[3], theta[4]), **kw)
    o.set_fields(rho)
    o.step(nsteps)
    obs = o.observables(probe or (0.0, 0.0, 0.0))
    return obs["mu_r"] if objective == 0 else obs["dp"]


def close(a, b):
    return np.all(np.abs(a - b) <= 1e-4 * np.abs(b) + 1e-8)


def fd_grad(oracle_mod, theta, rho, nsteps, objective, h=1e-4, **kw):
    g = np.zeros(5)
    for a in range(5):
        tp, tm = theta.copy(), theta.copy()
        tp[a] += h
        tm[a] -= h
        g[a] = (oracle_J(oracle_mod, tp, rho, nsteps, objective, **kw)
                - oracle_J(oracle_mod, tm, rho, nsteps, objective, **kw)) / (2 * h)
    return g


def channel_case():
    nx, ny = 32, 20
    rho = W.droplet(nx, ny, 5.0, cx=15.5, cy=9.5, seed=41, periodic=False)
    kw = dict(g=(1e-5, 0.0), walls=1, wall_mode=1, wall_rho=(0.03, 1.0))
    return nx, ny, rho, kw


def test_mu_r_gradient_matches_oracle_fd(lbmod, oracle_mod):
    nx, ny, rho, kw = channel_case()
    nsteps = 120
    L = lbmod.Lattice(nx, ny, G_AB=THETA0[0], G1=THETA0[1], G2=THETA0[2], tau=(THETA0[3], THETA0[4]), **kw)
    L.set_fields(rho)
    J, dJ = L.grad(nsteps, 25, lbmod.LB_OBJ_MU_R)
    J0 = oracle_J(oracle_mod, THETA0, rho, nsteps, 0, **kw)
    assert abs(J - J0) <= 1e-12 * abs(J0)
    g = fd_grad(oracle_mod, THETA0, rho, nsteps, 0, **kw)
    assert close(dJ, g), (dJ, g)
    # the lattice is left where lb_step would leave it
    M = lbmod.Lattice(nx, ny, G_AB=THETA0[0], G1=THETA0[1], G2=THETA0[2], tau=(THETA0[3], THETA0[4]), **kw)
    M.set_fields(rho)
    M.step(nsteps)
    assert L.t == nsteps and np.array_equal(L.get_populations(), M.get_populations())


def test_laplace_gradient_matches_oracle_fd(lbmod, oracle_mod):
    n = 32
    rho = W.droplet(n, n, 8.0, seed=42)
    probe = (n / 2, n / 2, 8.0)
    theta = np.array([3.0, -7.4, 6.4, 1.0, 1.2])
    nsteps = 80
    L = lbmod.Lattice(n, n, G_AB=theta[0], G1=theta[1], G2=theta[2], tau=(theta[3], theta[4]))
    L.set_fields(rho)
    L.set_probe(*probe)
    J, dJ = L.grad(nsteps, 30, lbmod.LB_OBJ_DP)
    assert abs(J - oracle_J(oracle_mod, theta, rho, nsteps, 1, probe=probe)) <= 1e-10 * abs(J)
    g = fd_grad(oracle_mod, theta, rho, nsteps, 1, probe=probe)
    assert close(dJ, g), (dJ, g)


def test_autograd_function(lbmod, oracle_mod):
    torch = pytest.importorskip("torch")
    from paper_1806_06943_gb300.autograd import observable
    nx, ny, rho, kw = channel_case()
    spec = dict(nx=nx, ny=ny, rho=rho, nsteps=60, ckpt_every=16, objective=lbmod.LB_OBJ_MU_R, **kw)
    theta = torch.tensor(THETA0, dtype=torch.float64, requires_grad=True)
    J = observable(theta, spec)
    (2.0 * J).backward()
    g = fd_grad(oracle_mod, THETA0, rho, 60, 0, **kw)
    assert close(theta.grad.numpy(), 2.0 * g)


def test_channel_emulsion_512x128_5000_steps(lbmod):
    """Calibration workload: 512 x 128 channel, hexagonal emulsion at area
    fraction 0.5, 5000 steps, checkpoints every 250; the FP64 adjoint against
    central differences of the FP64 GPU forward (each one tied to the
    oracle's arithmetic) at 1e-4.  The FP32 forward (FP64 adjoint linearised
    at the FP32 trajectory) is held to its observable tolerance: mu_r within
    1e-4 (measured 2e-5) and the gradient within 1e-3 (measured 3.1e-4).  Its
    trajectory carries the FP32 rounding bias of a body-forced flow (c17),
    and the gradient of this dense emulsion is itself sensitive: a 2e-5
    change of the continuous phase's viscosity moves the FP64 gradient by
    1.6e-4."""
    nx, ny = 512, 128
    rho, _, _, _ = W.hex_emulsion(nx, ny, 0.5, R=12.0, spread=2.0, gap=3.0, walls=True, seed=W.BASE_SEED + 3)
    kw = dict(g=(1e-6, 0.0), walls=1, wall_mode=1, wall_rho=(0.03, 1.0))
    theta = np.array([3.0, -7.4, 6.4, 1.0, 1.0])

    def lat(th):
        L = lbmod.Lattice(nx, ny, G_AB=th[0], G1=th[1], G2=th[2], tau=(th[3], th[4]), **kw)
        L.set_fields(rho)
        return L

    J, dJ = lat(theta).grad(5000, 250, lbmod.LB_OBJ_MU_R)
    L32 = lbmod.Lattice(nx, ny, G_AB=theta[0], G1=theta[1], G2=theta[2], tau=(theta[3], theta[4]),
                        precision=lbmod.LB_FP32, **kw)
    L32.set_config(lbmod.LB_MODE_TMA, 8)
    L32.set_fields(rho)
    J32, dJ32 = L32.grad(5000, 250, lbmod.LB_OBJ_MU_R)      # FP32 forward, FP64 adjoint
    assert abs(J32 - J) <= 1e-4 * abs(J)
    assert np.max(np.abs(dJ32 - dJ) / np.abs(dJ)) <= 1e-3, (dJ32, dJ)
    g = np.zeros(5)
    for a in range(5):
        tp, tm = theta.copy(), theta.copy()
        tp[a] += 1e-4
        tm[a] -= 1e-4
        Lp, Lm = lat(tp), lat(tm)
        Lp.step(5000)
        Lm.step(5000)
        g[a] = (Lp.observables()["mu_r"] - Lm.observables()["mu_r"]) / 2e-4
    assert close(dJ, g), (dJ, g)


def test_fp32_forward_gradient(lbmod):
    """FP32 forward, FP64 adjoint: gradient within 1e-4 of the FP64 one, and
    the lattice left where FP32 steps leave it."""
    nx, ny, rho, kw = channel_case()
    th = THETA0
    res = {}
    for prec in (lbmod.LB_FP64, lbmod.LB_FP32):
        L = lbmod.Lattice(nx, ny, G_AB=th[0], G1=th[1], G2=th[2], tau=(th[3], th[4]), precision=prec, **kw)
        L.set_fields(rho)
        res[prec] = L.grad(120, 25, lbmod.LB_OBJ_MU_R)
        M = lbmod.Lattice(nx, ny, G_AB=th[0], G1=th[1], G2=th[2], tau=(th[3], th[4]), precision=prec, **kw)
        M.set_fields(rho)
        M.step(120)
        assert L.t == 120 and np.array_equal(L.get_populations(), M.get_populations())
    (J32, g32), (J64, g64) = res[lbmod.LB_FP32], res[lbmod.LB_FP64]
    assert abs(J32 - J64) <= 1e-5 * abs(J64)
    assert close(g32, g64), (g32, g64)


def test_rejects_unsupported(lbmod):
    L = lbmod.Lattice(16, 16, precision=lbmod.LB_FP32)
    with pytest.raises(lbmod.LBError):   # no probe
        L.grad(10, 5, lbmod.LB_OBJ_DP)
    P = lbmod.Lattice(16, 16)
    with pytest.raises(lbmod.LBError):   # periodic: no mu_r
        P.grad(10, 5, lbmod.LB_OBJ_MU_R)
    with pytest.raises(lbmod.LBError):   # no probe
        P.grad(10, 5, lbmod.LB_OBJ_DP)


@pytest.mark.parametrize("walls", [0, 1])
def test_step_vjp_dot_product(lbmod, walls):
    """The transpose of one linearised time step against the step itself:
    <J v, w> = <v, J^T w> for random v, w (J v by central differences of
    the FP64 forward step, eps = 1e-6), to 1e-7 relative; and the parameter
    part <w, dStep/dtheta> against central differences in G_AB, G1, G2,
    tau_A, tau_B, to 1e-6 relative.  A 20 x 16 drop after 20 steps,
    periodic, and with non-wetting walls and a body force."""
    nx, ny = 20, 16
    kw = dict(tau=(0.9, 1.3), G_AB=3.0, G1=-7.4, G2=6.4)
    if walls:
        kw.update(walls=1, wall_mode=1, wall_rho=(0.03, 1.0), g=(1e-5, 0.0))
    rho = W.droplet(nx, ny, 5.0, seed=7, periodic=not walls)
    L = lbmod.Lattice(nx, ny, **kw)
    L.set_fields(rho)
    L.step(20)
    f0 = L.get_populations()
    rng = np.random.default_rng(3 + walls)
    v = rng.standard_normal(f0.shape) * np.max(np.abs(f0))
    w = rng.standard_normal(f0.shape)

    def step_from(f, **over):
        K = lbmod.Lattice(nx, ny, **{**kw, **over})
        K.set_populations(np.ascontiguousarray(f))
        K.step(1)
        return K.get_populations()

    eps = 1e-6
    Jv = (step_from(f0 + eps * v) - step_from(f0 - eps * v)) / (2 * eps)
    JTw, dth = L.step_vjp(w)
    assert np.array_equal(L.get_populations(), f0)   # the state is left as it was
    lhs, rhs = float(np.sum(Jv * w)), float(np.sum(v * JTw))
    assert abs(lhs - rhs) <= 1e-7 * abs(rhs), (lhs, rhs)
    for i, name in enumerate(("G_AB", "G1", "G2")):
        h = 1e-5 * abs(kw[name])
        d = (step_from(f0, **{name: kw[name] + h}) - step_from(f0, **{name: kw[name] - h})) / (2 * h)
        ref = float(np.sum(w * d))
        assert abs(ref - dth[i]) <= 1e-6 * abs(ref), (name, ref, dth[i])
    for k in (0, 1):
        h = 1e-5
        tp, tm = list(kw["tau"]), list(kw["tau"])
        tp[k] += h
        tm[k] -= h
        d = (step_from(f0, tau=tuple(tp)) - step_from(f0, tau=tuple(tm))) / (2 * h)
        ref = float(np.sum(w * d))
        assert abs(ref - dth[3 + k]) <= 1e-6 * abs(ref), (k, ref, dth[3 + k])


def test_step_vjp_rejects_fp32(lbmod):
    L = lbmod.Lattice(20, 16, precision=lbmod.LB_FP32)
    with pytest.raises(lbmod.LBError) as ei:
        L.step_vjp(np.zeros((2, 9, 16, 20)))
    assert ei.value.code == lbmod.LB_EINVAL
