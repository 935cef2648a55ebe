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


def _hex_rows(ny, nrow, R, gap, walls):
    """Row spacing and first row of nrow droplet rows: between the walls the
    rows span the band the drops' centres may occupy, periodic rows are
    evenly spaced."""
    if walls:
        lo_c, hi_c = gap - 0.5 + R, ny - 0.5 - gap - R
        dy = (hi_c - lo_c) / (nrow - 1) if nrow > 1 else 0.0
        return dy, (lo_c if nrow > 1 else (ny - 1) / 2.0)
    dy = ny / nrow
    return dy, dy / 2


def _hex_rmax(nx, ny, nrow, ncol, R, gap, walls):
    """Largest radius two neighbouring sites of the lattice can hold with
    `gap` nodes between them."""
    sx = nx / ncol
    dy, _ = _hex_rows(ny, nrow, R, gap, walls)
    d = sx if nrow == 1 else min(sx, math.hypot(sx / 2, dy))
    if ncol == 1:
        d = dy if nrow > 1 else float(min(nx, ny))
    if not walls and nrow == 2:
        d = min(d, math.hypot(sx / 2, dy))
    return (d - gap) / 2.0


def _hex_layout(nx, ny, nrow, ncol, R, spread, gap, walls, seed):
    """Centres and radii of a jittered hexagonal lattice of nrow x ncol
    droplet sites (see hex_emulsion)."""
    rng = np.random.default_rng(seed)
    sx = nx / ncol
    dy, y0 = _hex_rows(ny, nrow, R, gap, walls)
    rmax_pair = _hex_rmax(nx, ny, nrow, ncol, R, gap, walls)
    centres, radii = [], []
    for j in range(nrow):
        for i in range(ncol):
            r = min(float(rng.uniform(R - spread, R + spread)), rmax_pair)
            cx = (i + 0.5 * (j % 2)) * sx + sx / 4
            cy = y0 + j * dy
            ang = rng.uniform(0, 2 * math.pi)
            d = rng.uniform(0, max(0.0, rmax_pair - r))
            if walls:
                r = min(r, (ny - 2 * gap) / 2.0)
                if j == 0 or j == nrow - 1:
                    r = min(r, R)       # the outer rows sit R + gap from the walls
                lo_y, hi_y = gap - 0.5 + r, ny - 0.5 - gap - r
                if r <= 0 or hi_y < lo_y:
                    continue
            cx += d * math.cos(ang)
            cy += d * math.sin(ang)
            if walls:
                cy = min(max(cy, lo_y), hi_y)
            centres.append((cx % nx, cy if walls else cy % ny))
            radii.append(r)
    return centres, radii


def _clipped_r2(a, b, m):
    """E[min(r, m)^2] for r uniform on [a, b]."""
    if b <= a:
        return min(a, m) ** 2
    if m >= b:
        return (b ** 3 - a ** 3) / (3.0 * (b - a))
    if m <= a:
        return m * m
    return ((m ** 3 - a ** 3) / 3.0 + m * m * (b - m)) / (b - a)


def hex_emulsion(nx, ny, phi, R=12.0, spread=2.0, gap=3.0, walls=True, seed=BASE_SEED, noise=NOISE,
                 min_gap=2.0):
    """Non-overlapping droplets on a jittered hexagonal lattice, periodic in x
    (and in y unless walls), at area fraction phi.  Returns (rho, centres,
    radii, achieved_phi).

    Each radius is drawn from U[R - spread, R + spread] and clipped so that
    any two neighbours keep at least `gap` nodes between them (and the walls
    `gap` nodes from every drop); each centre is jittered inside the slack
    that remains.  Between walls the rows span the band the centres may
    occupy.  The numbers of rows and columns are searched so that the
    rasterised area fraction comes closest to phi, among near ties the lattice
    that clips the fewest radii.  Where even the densest lattice with this gap
    stays more than 0.01 below phi, the gap is narrowed in steps of 0.5 down to
    min_gap."""
    area = float(nx * ny)

    def raster(nr, nc, gp):
        c, r = _hex_layout(nx, ny, nr, nc, R, spread, gp, walls, seed)
        rho = droplets(nx, ny, c, r, seed=seed, noise=noise, periodic=not walls)
        return rho, c, r, float((rho[0] > 0.5).mean())

    best = None
    gp = gap
    while True:
        cands = []
        for nr in range(1, max(2, int(ny / (2.0 * (R - spread) + gp)) + 2)):
            if not walls and nr % 2:
                continue
            for nc in range(1, max(2, int(nx / (2.0 * (R - spread) + gp)) + 2)):
                m = _hex_rmax(nx, ny, nr, nc, R, gp, walls)
                if m < R - spread:
                    continue
                est = math.pi * nr * nc * _clipped_r2(R - spread, R + spread, m) / area
                cands.append((nr, nc, m, est))
        want = phi
        for _ in range(3):      # aim the analytic estimate, correct by the raster's bias
            if not cands:
                break
            near = [c for c in cands if abs(c[3] - want) <= 0.004]
            nr, nc, _, _ = max(near, key=lambda c: c[2]) if near else min(cands, key=lambda c: abs(c[3] - want))
            out = raster(nr, nc, gp)
            if best is None or abs(out[3] - phi) < abs(best[3] - phi):
                best = out
            if abs(out[3] - phi) <= 0.005:
                break
            want += phi - out[3]
        if (best is not None and best[3] >= phi - 0.01) or gp - 0.5 < min_gap - 1e-9:
            if best is None:
                raise ValueError("no droplet fits the lattice")
            return best
        gp -= 0.5


def random_emulsion(nx, ny, phi, rmin=8.0, rmax=20.0, gap=2.0, seed=BASE_SEED, noise=NOISE,
                    max_tries=300):
    """Polydisperse periodic emulsion: radii U[rmin, rmax] placed largest
    first by random sequential addition (up to max_tries uniform candidate
    centres per drop; the first one that keeps `gap` nodes to every placed
    drop wins), then a fill with rmin droplets until phi is reached or
    20 max_tries candidates in a row fail.  The overlap test looks at the
    drops of the 3 x 3 cells of a cell list around each candidate.
    Returns (rho, centres, radii, achieved_phi)."""
    rng = np.random.default_rng(seed)
    area = nx * ny
    target = phi * area
    cell = 2 * rmax + gap
    ncx, ncy = max(1, int(nx // cell)), max(1, int(ny // cell))
    # drops per cell: centres of drops of radius >= rmin keep 2 rmin + gap
    # apart, so a cell holds at most K of them; empty slots sit far away
    K = int((cell / (2 * rmin + gap) + 1.5) ** 2) + 1
    far = 1e30
    slots = np.full((ncy, ncx, K, 3), far)
    slots[..., 2] = 0.0
    count = np.zeros((ncy, ncx), dtype=np.int64)
    centres, radii = [], []
    filled = 0.0
    offs = np.array([-1, 0, 1])

    def first_fit(cand, r):
        """Index of the first candidate centre that fits, or -1 (tested in
        growing chunks: early drops fit at once)."""
        lo = 0
        for hi in (4, 16, 64, len(cand)):
            hi = min(hi, len(cand))
            if hi <= lo:
                continue
            i = fit_chunk(cand[lo:hi], r)
            if i >= 0:
                return lo + i
            lo = hi
        return -1

    def fit_chunk(cand, r):
        gx = (cand[:, 0] / nx * ncx).astype(np.int64) % ncx
        gy = (cand[:, 1] / ny * ncy).astype(np.int64) % ncy
        cy = (gy[:, None, None] + offs[None, :, None]) % ncy
        cx = (gx[:, None, None] + offs[None, None, :]) % ncx
        q = slots[cy, cx].reshape(len(cand), -1, 3)
        dx = np.abs(cand[:, None, 0] - q[..., 0])
        dx = np.minimum(dx, nx - dx)
        dy = np.abs(cand[:, None, 1] - q[..., 1])
        dy = np.minimum(dy, ny - dy)
        ok = (dx * dx + dy * dy >= (r + q[..., 2] + gap) ** 2).all(axis=1)
        idx = np.flatnonzero(ok)
        return int(idx[0]) if idx.size else -1

    def add(x, y, r):
        gx, gy = int(x / nx * ncx) % ncx, int(y / ny * ncy) % ncy
        n = count[gy, gx]
        if n >= K:
            raise RuntimeError("cell list overflow")
        slots[gy, gx, n] = (x, y, r)
        count[gy, gx] = n + 1
        centres.append((float(x), float(y)))
        radii.append(float(r))

    n_draw = int(target / (math.pi * ((rmin + rmax) / 2) ** 2) * 1.3) + 1
    draws = np.sort(rng.uniform(rmin, rmax, n_draw))[::-1]
    for r in draws:
        if filled >= target:
            break
        cand = rng.uniform(0.0, 1.0, (max_tries, 2)) * np.array([nx, ny])
        i = first_fit(cand, r)
        if i >= 0:
            add(cand[i, 0], cand[i, 1], r)
            filled += math.pi * r * r
    misses = 0
    while filled < target and misses < 20 * max_tries:
        cand = rng.uniform(0.0, 1.0, (max_tries, 2)) * np.array([nx, ny])
        i = first_fit(cand, rmin)
        if i >= 0:
            add(cand[i, 0], cand[i, 1], rmin)
            filled += math.pi * rmin * rmin
            misses = 0
        else:
            misses += max_tries
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
