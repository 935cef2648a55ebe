"""Batched physics sweeps on the GPU engine: the paper's own validation runs,
many lattices per batch.

* Tunable surface tension (Sec. III B, Table I, Fig. 2): for a pair of
  couplings (G1, G2), a scan of G_AB in steps of 0.1; for every G_AB a
  Laplace test over several droplet radii, the interface width W of the
  largest drop measured as the Fig. 2 caption defines it, and the surface
  tension gamma fitted to the Laplace law dp = gamma / R.  Table I reports,
  per case, the G_AB range over which 2 <= W <= 5 and the gamma range over it.
* Emulsion rheology (Sec. III D, Figs. 4b-4d): a regular array of equal
  droplets in an L x L channel with non-wetting walls and a body force; the
  relative effective viscosity mu_r = Q(Phi = 0) / Q(Phi), the ratio of the
  simulated flow rates, against the area fraction Phi, the reduced forcing
  F_b = g L^3 rho_B^2 / (8 mu_B^2) and the viscosity ratio M = mu_B / mu_A,
  and the fit of Eq. (20), mu_r = (1 - Phi)^-[eta] (K = 1), with [eta]
  compared against the Taylor and Douglas limits quoted there.
* Surface tension and disjoining pressure (Secs. II C, III C, Fig. 3): flat
  interfaces and flat films of B between A regions, periodic in x, the
  pressure tensor summed over the lattice by the library's reduction kernel:
  gamma by the integral of Eq. (15), the film tension gamma_f(h) of Eq. (16)
  and the disjoining pressure Pi(h) of Eq. (18); for either forcing of the
  collision (Guo, the method; the velocity shift of the original model).

Every time step runs in the library's kernels (FP32 offset form unless asked
otherwise); this module builds the seeded inputs, reads observables and
densities back, and fits them on the host.
"""
from __future__ import annotations

import math

import numpy as np

from . import lb
from . import workloads as W

ETA_INF = 2.5   # intrinsic viscosity of rigid spheres used by both limits of Sec. III D


# ---- Table I ----------------------------------------------------------------

def interface_width(profile: np.ndarray) -> float:
    """W = (rho_max - rho_min) / |rho(M) - rho(N)| (lattice units), M and N
    the two neighbouring nodes between which the profile crosses the mean
    density (rho_max + rho_min) / 2 (Fig. 2 caption); the mean over every
    crossing of the profile (a drop on a centreline gives two)."""
    p = np.asarray(profile, dtype=np.float64)
    hi, lo = p.max(), p.min()
    mid = 0.5 * (hi + lo)
    s = p - mid
    ws = []
    for i in range(len(p) - 1):
        if s[i] == 0.0 or s[i] * s[i + 1] < 0.0:
            d = abs(p[i + 1] - p[i])
            if d > 0.0:
                ws.append((hi - lo) / d)
    return float(np.mean(ws)) if ws else float("nan")


def laplace_side(R: float) -> int:
    """Square periodic box for a drop of radius R: 8 R rounded up to a
    multiple of 32, at least 128 (as the batched Laplace sweep)."""
    return max(128, int(math.ceil(8.0 * R / 32.0)) * 32)


def tension_scan(G1: float, G2: float, g_ab_values, radii=(12.0, 18.0, 24.0, 42.0), steps: int = 20000,
                 tau=(1.0, 1.0), precision: int = lb.LB_FP32, seed: int = W.BASE_SEED + 11,
                 init_width: float | None = None, noise: float = W.NOISE) -> list[dict]:
    """Laplace tests for every G_AB of g_ab_values at couplings (G1, G2), all
    in one batch; returns per G_AB: W (largest drop), gamma and the R^2 of the
    Laplace fit, and whether every drop stayed finite.  The drops start as
    sharp disks, or with a tanh interface of width init_width, with the
    seeded density noise of amplitude `noise`."""
    g_ab_values = [float(v) for v in g_ab_values]
    specs, fields, probes = [], [], []
    for gab in g_ab_values:
        for R in radii:
            n = laplace_side(R)
            specs.append(dict(nx=n, ny=n, tau=tau, G_AB=gab, G1=G1, G2=G2))
            fields.append(W.droplet(n, n, R, seed=seed, noise=noise) if init_width is None
                          else W.smooth_droplet(n, n, R, init_width, seed=seed, noise=noise))
            probes.append((n / 2, n / 2, R))
    b = lb.Batch(specs, precision=precision)
    try:
        if precision == lb.LB_FP32:
            b.set_config(lb.LB_MODE_TMA, 8)
        else:
            b.set_config(lb.LB_MODE_FUSED, 8)
        for i, (r, p) in enumerate(zip(fields, probes)):
            b.set_fields(i, r)
            b.set_probe(i, *p)
        b.step(steps)
        obs = b.observables(check=False)
        out = []
        nr = len(radii)
        big = int(np.argmax(radii))
        for j, gab in enumerate(g_ab_values):
            o = obs[j * nr:(j + 1) * nr]
            finite = all(x["finite"] == 1.0 for x in o)
            rho_a = b.fields(j * nr + big)["rho"][0]
            n = rho_a.shape[0]
            width = interface_width(rho_a[n // 2]) if finite else float("nan")
            gamma, r2 = float("nan"), float("nan")
            if finite and all(x["R_eff"] > 0 for x in o):
                x = np.array([1.0 / v["R_eff"] for v in o])
                y = np.array([v["dp"] for v in o])
                A = np.vstack([x, np.ones_like(x)]).T
                (gamma, c), *_ = np.linalg.lstsq(A, y, rcond=None)
                f = A @ np.array([gamma, c])
                ss = ((y - y.mean()) ** 2).sum()
                r2 = float(1.0 - ((y - f) ** 2).sum() / ss) if ss > 0 else float("nan")
            out.append(dict(G_AB=gab, W=width, gamma=float(gamma), r2=r2, finite=finite,
                            R_eff=[float(v["R_eff"]) for v in o], dp=[float(v["dp"]) for v in o]))
        return out
    finally:
        b.close()


def width_window(scan: list[dict], lo: float = 2.0, hi: float = 5.0) -> dict:
    """Table I's criterion on a scan in increasing G_AB: the contiguous run
    of G_AB whose width lies in [lo, hi], from the first such value up to the
    last before a width below lo or a run that did not stay finite; with the
    surface tension at its ends.  None where no width is in."""
    start = next((i for i, r in enumerate(scan) if r["finite"] and lo <= r["W"] <= hi), None)
    if start is None:
        return {"G_AB": None, "gamma": None, "W_at_ends": None}
    end = start
    while end + 1 < len(scan) and scan[end + 1]["finite"] and lo <= scan[end + 1]["W"] <= hi:
        end += 1
    first, last = scan[start], scan[end]
    return {"G_AB": (first["G_AB"], last["G_AB"]), "gamma": (first["gamma"], last["gamma"]),
            "W_at_ends": (first["W"], last["W"])}


# ---- Emulsion rheology --------------------------------------------------------

def tau_for_ratio(M: float, tau_c: float = 1.0) -> float:
    """Relaxation time of the droplets for M = mu_B / mu_A at equal densities:
    nu_A = nu_B / M."""
    return 0.5 + (tau_c - 0.5) / M


def body_force(F_bar: float, L: int, tau_c: float = 1.0, rho_b: float = W.MAJORITY) -> float:
    """g from the reduced forcing F_b = g rho_B L^3 rho_B / (8 mu_B^2), read
    with the force density rho_B g of the continuous phase (Sec. III D)."""
    nu = (tau_c - 0.5) / 3.0
    mu = rho_b * nu
    return 8.0 * F_bar * mu * mu / (rho_b * rho_b * L ** 3)


def droplet_array(L: int, n: int, R: float, seed: int, noise: float = W.NOISE) -> tuple[np.ndarray, float]:
    """n x n equal drops on a square lattice of spacing L / n in an L x L
    channel (walls in y), and the achieved area fraction; n = 0 gives the
    droplet-free continuous phase.  noise: amplitude of the seeded uniform
    perturbation of the densities (0: the exact symmetric array)."""
    if n == 0:
        return W.droplets(L, L, [], [], seed=seed, noise=noise, periodic=False), 0.0
    s = L / n
    centres = [((i + 0.5) * s, (j + 0.5) * s) for j in range(n) for i in range(n)]
    rho = W.droplets(L, L, centres, [R] * len(centres), seed=seed, noise=noise, periodic=False)
    phi = float((rho[0] > 0.5 * (W.MAJORITY + W.MINORITY)).mean())
    return rho, phi


def count_drops(rho_a: np.ndarray, threshold: float = 0.5) -> int:
    """Connected regions (4-neighbour) of rho_A > threshold, periodic in x:
    the number of drops, so that coalescence shows."""
    from scipy import ndimage
    lab, n = ndimage.label(rho_a > threshold)
    parent = list(range(n + 1))

    def find(i):
        while parent[i] != i:
            parent[i] = parent[parent[i]]
            i = parent[i]
        return i
    for a, b in zip(lab[:, 0], lab[:, -1]):   # regions that continue across x = 0
        if a and b:
            ra, rb = find(a), find(b)
            if ra != rb:
                parent[ra] = rb
    return len({find(i) for i in range(1, n + 1)})


def rheology(cases: list[dict], L: int = 220, n: int = 5, steps: int = 200000, window: int = 40000,
             sample_every: int = 2000, precision: int = lb.LB_FP32, seed: int = W.BASE_SEED + 12,
             couplings=None, noise: float = W.NOISE) -> list[dict]:
    """mu_r for each case dict(R, M, F_bar) (R = 0: no drops), all in one
    batch: L x L channel, fixed non-wetting wall densities, tau_B = 1.  The
    flow rate Q of every lattice is averaged over the last `window` steps;
    mu_r divides the Q of the droplet-free lattice of the same M and F_bar
    (added where missing) by the case's.  `drops` counts the drops at the
    end (start: n * n), which shows whether they coalesced."""
    couplings = couplings or dict(G_AB=3.0, G1=-7.4, G2=6.4)
    keys = {(c["M"], c["F_bar"]) for c in cases}
    allc = list(cases) + [dict(R=0.0, M=m, F_bar=f) for (m, f) in sorted(keys)
                          if not any(c["R"] == 0.0 and (c["M"], c["F_bar"]) == (m, f) for c in cases)]
    specs, fields, phis = [], [], []
    for c in allc:
        g = body_force(c["F_bar"], L)
        specs.append(dict(nx=L, ny=L, tau=(tau_for_ratio(c["M"]), 1.0), g=(g, 0.0), walls=1, wall_mode=1,
                          wall_rho=(W.MINORITY, W.MAJORITY), **couplings))
        rho, phi = droplet_array(L, n if c["R"] > 0 else 0, c["R"], seed, noise=noise)
        fields.append(rho)
        phis.append(phi)
    b = lb.Batch(specs, precision=precision)
    try:
        b.set_config(lb.LB_MODE_TMA if precision == lb.LB_FP32 else lb.LB_MODE_FUSED, 8)
        for i, r in enumerate(fields):
            b.set_fields(i, r)
        b.step(steps - window)
        qs, fin = [], np.ones(len(allc), dtype=bool)
        for _ in range(window // sample_every):
            b.step(sample_every)
            obs = b.observables(check=False)
            qs.append([o["Q"] for o in obs])
            fin &= np.array([o["finite"] == 1.0 for o in obs])
        q = np.mean(np.array(qs), axis=0)
        drops = [count_drops(b.fields(i)["rho"][0]) if fin[i] and allc[i]["R"] > 0 else 0 for i in range(len(allc))]
        out = []
        for i, c in enumerate(allc):
            ref = next(j for j, d in enumerate(allc) if d["R"] == 0.0 and (d["M"], d["F_bar"]) == (c["M"], c["F_bar"]))
            ok = bool(fin[i] and fin[ref])
            out.append(dict(R=c["R"], M=c["M"], F_bar=c["F_bar"], phi=phis[i], finite=ok, drops=drops[i],
                            Q=float(q[i]) if fin[i] else float("nan"),
                            mu_r=float(q[ref] / q[i]) if ok else float("nan"),
                            Q_spread=float(np.ptp(np.array(qs)[:, i]) / q[i]) if fin[i] else float("nan")))
        return out
    finally:
        b.close()


def demt_fit(phi, mu_r) -> tuple[float, float]:
    """[eta] of Eq. (20) with K = 1, ln mu_r = -[eta] ln(1 - Phi), by least
    squares through the origin; returns ([eta], R^2 of the fit in ln mu_r)."""
    x = -np.log(1.0 - np.asarray(phi, dtype=np.float64))
    y = np.log(np.asarray(mu_r, dtype=np.float64))
    eta = float((x @ y) / (x @ x))
    ss = ((y - y.mean()) ** 2).sum()
    return eta, float(1.0 - ((y - eta * x) ** 2).sum() / ss) if ss > 0 else float("nan")


def eta_limits(M: float) -> tuple[float, float]:
    """Intrinsic viscosity of freely deformable drops (Douglas et al.) and of
    undeformable ones (Taylor) at viscosity ratio M = mu_B / mu_A, with
    [eta]_inf = 2.5, as quoted in Sec. III D: returns (Douglas, Taylor).
    The printed formulas are read with their ratio as drop over matrix
    viscosity, 1 / M here: so both give 2.5 for rigid drops (M -> 0) and
    Taylor's gives 1 for bubbles, as Taylor's result does (at M = 1 either
    reading gives 0 and 1.75)."""
    lam = 1.0 / M
    taylor = (1.0 / lam + ETA_INF) / (1.0 / lam + 1.0)
    douglas = (1.0 - 1.0 / lam) / ((1.0 - 1.0 / lam) / ETA_INF + 1.0 / lam)
    return douglas, taylor


# ---- surface tension and disjoining pressure (Secs. II C, III C) ---------------

FILM_NY = 5      # rows of a flat-interface lattice: the profile varies along x only


def tension_of(sums, ny: int, interfaces: int = 2) -> float:
    """Eq. (15) from the lattice sums of the pressure tensor (kinetic +
    interaction, xx minus yy), per unit length of each of the `interfaces`
    flat interfaces normal to x."""
    pxx = sums[0] + sums[3]
    pyy = sums[1] + sums[4]
    return float(pxx - pyy) / ny / interfaces


def coexistence(G1: float, G2: float, G_AB: float, steps: int = 8000, precision: int = lb.LB_FP64):
    """Bulk densities (majority, minority) of a flat interface equilibrated in
    a 64 x 5 periodic box from the sharp 1.0 / 0.03 strip."""
    L = lb.Lattice(64, FILM_NY, G_AB=G_AB, G1=G1, G2=G2, precision=precision)
    L.set_fields(W.strip(64, FILM_NY, 32, noise=0.0))
    L.step(steps)
    rA = L.fields()["rho"][0][FILM_NY // 2]
    return float(rA.max()), float(rA.min())


def film_scan(G1: float, G2: float, G_AB: float, hs, nx: int = 128, steps: int = 8000, tau=(1.0, 1.0),
              forcing: int = lb.LB_FORCING_GUO, precision: int = lb.LB_FP64) -> dict:
    """Flat films of species B of widths hs between A regions in nx x 5
    periodic boxes, all in one batch, started from sharp steps at the
    coexisting densities of a flat interface, plus the same box at
    h = nx / 2 (two independent interfaces: its gamma_f is 2 gamma).  After
    `steps` steps: gamma_f(h) (Eq. 16, the sum of P_xx - P_yy over the box per
    unit length), s(h) = gamma_f(h) - 2 gamma and Pi(h) (Eq. 18)."""
    hs = [int(h) for h in hs]
    hi, lo = coexistence(G1, G2, G_AB)
    widths = hs + [nx // 2]
    specs = [dict(nx=nx, ny=FILM_NY, tau=tau, G_AB=G_AB, G1=G1, G2=G2, forcing=forcing) for _ in widths]
    b = lb.Batch(specs, precision=precision)
    try:
        b.set_config(lb.LB_MODE_FUSED, 4)
        for i, h in enumerate(widths):
            b.set_fields(i, np.ascontiguousarray(W.strip(nx, FILM_NY, h, noise=0.0, hi=hi, lo=lo)[::-1]))
        b.step(steps)
        gf = [tension_of(b.pressure_tensor(i)[0], FILM_NY, interfaces=1) for i in range(len(widths))]
    finally:
        b.close()
    two_gamma = gf[-1]
    s = np.array(gf[:-1]) - two_gamma
    return {"h": np.array(hs, dtype=np.float64), "gamma_f": np.array(gf[:-1]), "two_gamma": two_gamma,
            "s": s, "Pi": disjoining_pressure(np.array(hs, dtype=np.float64), s), "coexistence": (hi, lo)}


def disjoining_pressure(h: np.ndarray, s: np.ndarray) -> np.ndarray:
    """Pi(h_i) = s_i / h_i - int_{h_i}^inf s(h) / h^2 dh (Eq. 18, with
    Pi(inf) = 0): the integral over the sampled widths by the trapezoid rule,
    nothing beyond the widest film."""
    h = np.asarray(h, dtype=np.float64)
    s = np.asarray(s, dtype=np.float64)
    f = s / h ** 2
    seg = 0.5 * (f[1:] + f[:-1]) * np.diff(h)           # integral over [h_i, h_i+1]
    tail = np.concatenate([np.cumsum(seg[::-1])[::-1], [0.0]])
    return s / h - tail


def flat_tension(G1: float, G2: float, G_AB: float, taus, forcing: int = lb.LB_FORCING_GUO, nx: int = 64,
                 steps: int = 10000, precision: int = lb.LB_FP64) -> list[float]:
    """gamma (Eq. 15) of a flat interface per (tau_A, tau_B) of taus: all in
    one batch, started from the equilibrium of the strip at tau = 1 with Guo
    forcing (so every run starts at rest)."""
    L = lb.Lattice(nx, FILM_NY, G_AB=G_AB, G1=G1, G2=G2, precision=precision)
    L.set_fields(W.strip(nx, FILM_NY, nx // 2, noise=0.0))
    L.step(8000)
    rho0 = L.fields()["rho"]
    L.close()
    specs = [dict(nx=nx, ny=FILM_NY, tau=t, G_AB=G_AB, G1=G1, G2=G2, forcing=forcing) for t in taus]
    b = lb.Batch(specs, precision=precision)
    try:
        b.set_config(lb.LB_MODE_FUSED, 4)
        for i in range(len(specs)):
            b.set_fields(i, rho0)
        b.step(steps)
        return [tension_of(b.pressure_tensor(i)[0], FILM_NY) for i in range(len(specs))]
    finally:
        b.close()
