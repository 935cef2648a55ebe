"""Seeded synthetic initial fields for the binary-mixture lattice Boltzmann
workloads: droplets, flat strips, layered channels and emulsions.

This module only builds input densities (and optional initial velocities) on
the host as float64 numpy arrays laid out [species][ny][nx]; it contains none
of the method's arithmetic.  Both the CUDA path and the CPU checker take their
inputs from here, so the two see bit-identical initial fields.

Noise is a counter-based hash (splitmix64, Steele, Lea & Flood, OOPSLA 2014)
of (seed, species, y, x), so any sub-block of a field can be regenerated
independently of the others.
"""
from __future__ import annotations

import math

import numpy as np

MAJORITY = 1.0
MINORITY = 0.03
NOISE = 1e-3
BASE_SEED = 1806069431

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(z: np.ndarray) -> np.ndarray:
    """splitmix64 output function applied elementwise to uint64 counters."""
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z = z + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform_noise(seed: int, species: int, nx: int, ny: int, amp: float = NOISE) -> np.ndarray:
    """U[-amp, amp) per node, from the hash of (seed, species, y, x)."""
    y, x = np.meshgrid(np.arange(ny, dtype=np.uint64), np.arange(nx, dtype=np.uint64), indexing="ij")
    with np.errstate(over="ignore"):
        key = (np.uint64(seed) * np.uint64(0x100000001B3)) ^ (np.uint64(species) << np.uint64(56))
        ctr = key ^ (y << np.uint64(28)) ^ x
        z = splitmix64(ctr ^ splitmix64(np.uint64(seed)))
    u = (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return amp * (2.0 * u - 1.0)


def disk_mask(nx: int, ny: int, cx: float, cy: float, R: float, periodic: bool = True) -> np.ndarray:
    """Nodes whose centre lies strictly inside the circle (minimum image in x,
    and in y when periodic)."""
    y, x = np.meshgrid(np.arange(ny, dtype=np.float64), np.arange(nx, dtype=np.float64), indexing="ij")
    dx = np.abs(x - cx)
    dx = np.minimum(dx, nx - dx)
    dy = np.abs(y - cy)
    if periodic:
        dy = np.minimum(dy, ny - dy)
    return dx * dx + dy * dy < R * R


def _fill(maskA: np.ndarray, seed: int, hi=MAJORITY, lo=MINORITY, noise=NOISE) -> np.ndarray:
    ny, nx = maskA.shape
    rho = np.empty((2, ny, nx))
    rho[0] = np.where(maskA, hi, lo)
    rho[1] = np.where(maskA, lo, hi)
    if noise:
        rho[0] += uniform_noise(seed, 0, nx, ny, noise)
        rho[1] += uniform_noise(seed, 1, nx, ny, noise)
    return rho


def droplet(nx, ny, R, cx=None, cy=None, seed=BASE_SEED, noise=NOISE, hi=MAJORITY, lo=MINORITY,
            periodic=True) -> np.ndarray:
    """One species-A disk of radius R in species B."""
    cx = nx / 2 if cx is None else cx
    cy = ny / 2 if cy is None else cy
    return _fill(disk_mask(nx, ny, cx, cy, R, periodic), seed, hi, lo, noise)


def smooth_droplet(nx, ny, R, width, cx=None, cy=None, seed=BASE_SEED, noise=NOISE, hi=MAJORITY,
                   lo=MINORITY) -> np.ndarray:
    """One species-A disk of radius R in species B with a tanh interface of
    the given width (rho_A = lo + (hi - lo) (1 - tanh(2 (r - R) / width)) / 2,
    rho_B its mirror), periodic (minimum image)."""
    cx = nx / 2 if cx is None else cx
    cy = ny / 2 if cy is None else cy
    y, x = np.meshgrid(np.arange(ny, dtype=np.float64), np.arange(nx, dtype=np.float64), indexing="ij")
    dx = np.abs(x - cx)
    dx = np.minimum(dx, nx - dx)
    dy = np.abs(y - cy)
    dy = np.minimum(dy, ny - dy)
    a = 0.5 * (1.0 - np.tanh(2.0 * (np.sqrt(dx * dx + dy * dy) - R) / width))
    rho = np.empty((2, ny, nx))
    rho[0] = lo + (hi - lo) * a
    rho[1] = hi + lo - rho[0]
    if noise:
        rho[0] += uniform_noise(seed, 0, nx, ny, noise)
        rho[1] += uniform_noise(seed, 1, nx, ny, noise)
    return rho


def droplets(nx, ny, centres, radii, seed=BASE_SEED, noise=NOISE, hi=MAJORITY, lo=MINORITY,
             periodic=True) -> np.ndarray:
    """Several species-A disks (rasterised per bounding box) in species B."""
    m = np.zeros((ny, nx), dtype=bool)
    for (cx, cy), R in zip(centres, radii):
        r = int(math.ceil(R)) + 1
        ys = np.arange(int(math.floor(cy)) - r, int(math.floor(cy)) + r + 2)
        xs = np.arange(int(math.floor(cx)) - r, int(math.floor(cx)) + r + 2)
        if not periodic:
            ys = ys[(ys >= 0) & (ys < ny)]
        Y, X = np.meshgrid(ys, xs, indexing="ij")
        inside = (X - cx) ** 2 + (Y - cy) ** 2 < R * R
        m[np.mod(Y[inside], ny), np.mod(X[inside], nx)] = True
    return _fill(m, seed, hi, lo, noise)


def strip(nx, ny, width, axis=0, seed=BASE_SEED, noise=NOISE, hi=MAJORITY, lo=MINORITY) -> np.ndarray:
    """A flat slab of species A of the given width, centred, normal to x
    (axis=0) or to y (axis=1)."""
    y, x = np.meshgrid(np.arange(ny, dtype=np.float64), np.arange(nx, dtype=np.float64), indexing="ij")
    c = x if axis == 0 else y
    n = nx if axis == 0 else ny
    m = np.abs(c + 0.5 - n / 2) < width / 2
    return _fill(m, seed, hi, lo, noise)


def layered_channel(nx, ny, a, hi=MAJORITY, lo=MINORITY, noise=0.0, seed=BASE_SEED) -> np.ndarray:
    """Layered channel between walls at y=-1/2 and y=ny-1/2: species B in the
    core |y - yc| < a, species A in the two wall layers."""
    yc = (ny - 1) / 2.0
    y = np.arange(ny, dtype=np.float64)
    core = np.abs(y - yc) < a
    m = np.broadcast_to(~core[:, None], (ny, nx))
    return _fill(np.ascontiguousarray(m), seed, hi, lo, noise)


def hex_emulsion(nx, ny, phi, R=12.0, spread=2.0, gap=3.0, walls=True, seed=BASE_SEED, noise=NOISE):
    """Non-overlapping droplets on a jittered hexagonal lattice, periodic in x
    (and in y unless walls).  Returns (rho, centres, radii, achieved_phi).

    The spacing is chosen for the target area fraction phi at mean radius R;
    each radius is drawn from U[R - spread, R + spread] and clipped so any two
    neighbours keep at least `gap` nodes between them; each centre is jittered
    inside the slack that remains."""
    rng = np.random.default_rng(seed)
    H = ny - 2 * gap if walls else ny
    s = math.sqrt(2.0 * math.pi * R * R / (math.sqrt(3.0) * phi))
    ncol = max(1, int(round(nx / s)))
    sx = nx / ncol
    dy = sx * math.sqrt(3.0) / 2.0
    if walls:
        nrow = max(1, int(math.floor((H - 2 * (R + 0) ) / dy)) + 1)
        span = (nrow - 1) * dy
        y0 = (ny - 1) / 2.0 - span / 2.0
    else:
        nrow = max(2, 2 * int(round(ny / dy / 2)))
        dy = ny / nrow
        y0 = dy / 2
    rmax_pair = (min(sx, math.hypot(sx / 2, dy)) - gap) / 2.0
    centres, radii = [], []
    for j in range(nrow):
        for i in range(ncol):
            r = float(rng.uniform(R - spread, R + spread))
            r = min(r, rmax_pair)
            cx = (i + 0.5 * (j % 2)) * sx + sx / 4
            cy = y0 + j * dy
            if walls:
                lo_y, hi_y = gap - 0.5 + r, ny - 0.5 - gap - r
                if hi_y < lo_y:
                    continue
            slack = max(0.0, rmax_pair - r)
            ang = rng.uniform(0, 2 * math.pi)
            d = rng.uniform(0, slack)
            cx += d * math.cos(ang)
            cy += d * math.sin(ang)
            if walls:
                cy = min(max(cy, lo_y), hi_y)
            centres.append((cx % nx, cy if walls else cy % ny))
            radii.append(r)
    rho = droplets(nx, ny, centres, radii, seed=seed, noise=noise, periodic=not walls)
    achieved = float((rho[0] > 0.5).mean())
    return rho, centres, radii, achieved


def random_emulsion(nx, ny, phi, rmin=8.0, rmax=20.0, gap=2.0, seed=BASE_SEED, noise=NOISE,
                    max_tries=60):
    """Polydisperse periodic emulsion: radii U[rmin, rmax] placed largest
    first by random sequential addition (cell-list overlap test), then a fill
    with rmin droplets until phi or the attempt budget is reached.
    Returns (rho, centres, radii, achieved_phi)."""
    rng = np.random.default_rng(seed)
    area = nx * ny
    target = phi * area
    cell = 2 * rmax + gap
    ncx, ncy = max(1, int(nx // cell)), max(1, int(ny // cell))
    grid: dict = {}
    centres, radii = [], []
    filled = 0.0

    def fits(cx, cy, r):
        gx, gy = int(cx / nx * ncx) % ncx, int(cy / ny * ncy) % ncy
        for ox in (-1, 0, 1):
            for oy in (-1, 0, 1):
                for (qx, qy, qr) in grid.get(((gx + ox) % ncx, (gy + oy) % ncy), ()):
                    ddx = abs(cx - qx); ddx = min(ddx, nx - ddx)
                    ddy = abs(cy - qy); ddy = min(ddy, ny - ddy)
                    if ddx * ddx + ddy * ddy < (r + qr + gap) ** 2:
                        return False
        return True

    def add(cx, cy, r):
        gx, gy = int(cx / nx * ncx) % ncx, int(cy / ny * ncy) % ncy
        grid.setdefault((gx, gy), []).append((cx, cy, r))
        centres.append((cx, cy))
        radii.append(r)

    n_draw = int(target / (math.pi * ((rmin + rmax) / 2) ** 2) * 1.3) + 1
    draws = np.sort(rng.uniform(rmin, rmax, n_draw))[::-1]
    for r in draws:
        if filled >= target:
            break
        for _ in range(max_tries):
            cx, cy = rng.uniform(0, nx), rng.uniform(0, ny)
            if fits(cx, cy, r):
                add(cx, cy, r)
                filled += math.pi * r * r
                break
    misses = 0
    while filled < target and misses < 20 * max_tries:
        cx, cy = rng.uniform(0, nx), rng.uniform(0, ny)
        if fits(cx, cy, rmin):
            add(cx, cy, rmin)
            filled += math.pi * rmin * rmin
            misses = 0
        else:
            misses += 1
    rho = droplets(nx, ny, centres, radii, seed=seed, noise=noise, periodic=True)
    achieved = float((rho[0] > 0.5).mean())
    return rho, centres, radii, achieved


# Named workloads (sizes and recipes of the paper's Sec. III experiments).
def c1_droplet_64():
    """64x64 periodic, one A disk R=12 at the centre, tau_A=tau_B=1."""
    return droplet(64, 64, 12.0, seed=BASE_SEED + 0)


def laplace_sweep_specs():
    """24 periodic lattices: R in {10..45 step 5} x viscosity ratio {1, 3, 10}.
    Side L = clamp(roundup32(8R), 128, 384).  Dispersed tau_d for ratio
    mu_d/mu_c: nu ratio with tau_c = 1 gives tau_d = 0.5 + ratio/2."""
    specs = []
    for ratio in (1.0, 3.0, 10.0):
        tau_d = 0.5 + 0.5 * ratio
        for R in (10, 15, 20, 25, 30, 35, 40, 45):
            L = min(384, max(128, 32 * int(math.ceil(8 * R / 32))))
            specs.append({"nx": L, "ny": L, "R": float(R), "tau": (tau_d, 1.0), "ratio": ratio})
    return specs
