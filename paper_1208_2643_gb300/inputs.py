"""Seeded synthetic initial data for the MPFC solver.

This module holds no part of the solver's arithmetic: it only builds input
fields (the initial-data formulas of Sec. 4 and seeded noise).  Both the CUDA
path's tests/benchmarks and the CPU oracle read their inputs from here, so the
two sides always see bit-identical data.

Arrays are float64, shaped (n, m): row j (y), column i (x); cell centres sit at
x_i = (i + 1/2) h, y_j = (j + 1/2) h (App. A, p_r = (r - 1/2) h with 1-based r).
"""
from __future__ import annotations

import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Counter-based SplitMix64 (Steele, Lea, Flood 2014): the k-th output is the
    SplitMix64 finaliser applied to seed*phi64 + (k+1)*phi64 (mod 2^64)."""
    k = np.arange(offset, offset + count, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) * _GOLDEN + (k + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, count: int, lo: float = -1.0, hi: float = 1.0, offset: int = 0) -> np.ndarray:
    """count doubles uniform in [lo, hi), from the top 53 bits of splitmix64."""
    u = (splitmix64(seed, count, offset) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return lo + (hi - lo) * u


def uniform_at(seed: int, index, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """uniform() evaluated at the given output indices k (any integer array shape): the
    values uniform(seed, count, lo, hi) holds at positions k, bit for bit."""
    k = np.asarray(index, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) * _GOLDEN + (k + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    u = (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return lo + (hi - lo) * u


def noise_at(m: int, mean: float, amp: float, seed: int, rows, cols) -> np.ndarray:
    """The values noise_field(m, n, mean, amp, seed) holds at (rows[j], cols[i]) (any
    n), as a len(rows) x len(cols) array: for patches of fields too large to build on
    the host."""
    idx = np.asarray(rows, dtype=np.int64)[:, None] * m + np.asarray(cols, dtype=np.int64)[None, :]
    return mean + amp * uniform_at(seed, idx)


def _s64(v: int) -> int:
    return v - (1 << 64) if v >= (1 << 63) else v


def noise_field_torch(m: int, n: int, mean: float, amp: float, seed: int, device="cuda", chunk: int = 1 << 25):
    """noise_field() built by torch on `device` (float64, shape (n, m)), bit for bit the
    same values: SplitMix64 in int64 arithmetic (wrapping products, logical shifts as
    arithmetic shifts with the sign bits masked off), the same float64 operations in the
    same order.  For fields too large to build on the host and copy."""
    import torch
    out = torch.empty(n * m, dtype=torch.float64, device=device)
    gold, m1, m2 = _s64(0x9E3779B97F4A7C15), _s64(0xBF58476D1CE4E5B9), _s64(0x94D049BB133111EB)
    base = _s64((seed * 0x9E3779B97F4A7C15) % (1 << 64))

    def lsr(z, sh):
        return (z >> sh) & ((1 << (64 - sh)) - 1)

    for a in range(0, n * m, chunk):
        b = min(a + chunk, n * m)
        k = torch.arange(a + 1, b + 1, dtype=torch.int64, device=device)
        z = k * gold + base
        z = (z ^ lsr(z, 30)) * m1
        z = (z ^ lsr(z, 27)) * m2
        z = z ^ lsr(z, 31)
        u = lsr(z, 11).to(torch.float64) * (1.0 / 9007199254740992.0)
        out[a:b] = (u * 2.0 + (-1.0)) * amp + mean
        del k, z, u
    return out.view(n, m)


def cell_centres(m: int, n: int, h: float):
    x = (np.arange(m) + 0.5) * h
    y = (np.arange(n) + 0.5) * h
    return np.meshgrid(x, y)  # X[j, i], Y[j, i]


def noise_field(m: int, n: int, mean: float, amp: float, seed: int) -> np.ndarray:
    """phi = mean + amp * U(-1, 1), seeded (Sec. 4.4 style random data)."""
    return mean + amp * uniform(seed, m * n).reshape(n, m)


def paper_smooth_field(m: int, n: int, h: float) -> np.ndarray:
    """The smooth initial density of the convergence tests, Sec. 4.1, (4.1), at cell centres."""
    X, Y = cell_centres(m, n, h)
    pi = math.pi
    return (0.07 - 0.02 * np.cos(2 * pi * (X - 12) / 32) * np.sin(2 * pi * (Y - 1) / 32)
            + 0.02 * np.cos(pi * (X + 10) / 32) ** 2 * np.cos(pi * (Y + 3) / 32) ** 2
            - 0.01 * np.sin(4 * pi * X / 32) ** 2 * np.sin(4 * pi * (Y - 6) / 32) ** 2)


def single_mode_amplitude(phi_s: float, eps: float) -> float:
    """A of the one-mode crystal approximation, Sec. 4.6, (4.5)."""
    return 0.8 * phi_s + (4.0 / 15.0) * math.sqrt(max(15.0 * eps - 36.0 * phi_s * phi_s, 0.0))


def crystallite_field(m: int, n: int, h: float, phibar: float, eps: float, count: int = 3,
                      radius_cells: float = 20.0, noise: float = 1e-3, seed: int = 2,
                      edge_cells: float = 0.0) -> np.ndarray:
    """Uniform liquid phibar with `count` hexagonal crystallites (one-mode pattern of
    Sec. 4.6, (4.4), q_t = sqrt(3)/2), each rotated by a random angle in [0, pi/3) inside a
    circular patch of radius radius_cells*h, plus noise*U(-1,1).  The pattern is built for
    |phibar| and mirrored (phi -> -phi is a symmetry of the energy) when phibar < 0.
    edge_cells > 0 gives a tanh edge of that width instead of a sharp one."""
    X, Y = cell_centres(m, n, h)
    Lx, Ly = m * h, n * h
    ps = abs(phibar)
    A = single_mode_amplitude(ps, eps)
    qt = math.sqrt(3.0) / 2.0
    r = uniform(seed, 3 * count, 0.0, 1.0)
    dev = np.zeros((n, m))
    R = radius_cells * h
    for c in range(count):
        cx, cy, th = r[3 * c] * Lx, r[3 * c + 1] * Ly, r[3 * c + 2] * (math.pi / 3.0)
        dx = (X - cx + 0.5 * Lx) % Lx - 0.5 * Lx
        dy = (Y - cy + 0.5 * Ly) % Ly - 0.5 * Ly
        xr = math.cos(th) * dx + math.sin(th) * dy
        yr = -math.sin(th) * dx + math.cos(th) * dy
        pat = A * (np.cos(qt * xr) * np.cos(qt * yr / math.sqrt(3.0)) - 0.5 * np.cos(2 * qt * yr / math.sqrt(3.0)))
        dist = np.sqrt(dx * dx + dy * dy)
        if edge_cells > 0:
            w = 0.5 * (1.0 - np.tanh((dist - R) / (edge_cells * h)))
        else:
            w = (dist <= R).astype(np.float64)
        dev = np.where(w > 0, w * pat, dev)
    phi = ps + dev
    if phibar < 0:
        phi = -phi
    return phi + noise * uniform(seed + 1000003, m * n).reshape(n, m)


def polycrystal_seeds(m: int, n: int, mean: float, count: int, size_cells: int, amp: float,
                      seed: int) -> np.ndarray:
    """Constant density `mean` with `count` small random square perturbations of
    `size_cells` cells (amplitude amp U(-1, 1)) on the bottom rows y = 0, at seeded
    random x positions: the nucleation seeds of the polycrystal run, Sec. 4.5."""
    phi = np.full((n, m), float(mean))
    xs = uniform(seed, count)
    noise = uniform(seed + 1, count * size_cells * size_cells).reshape(count, size_cells, size_cells)
    for k in range(count):
        x0 = int((xs[k] + 1.0) * 0.5 * (m - size_cells))
        phi[0:size_cells, x0:x0 + size_cells] += amp * noise[k]
    return phi


def one_mode_crystal(m: int, n: int, h: float, phi_s: float, eps: float, shift: float = 0.0) -> np.ndarray:
    """The one-mode hexagonal density of Sec. 4.6, (4.4)-(4.5), at cell centres, with its
    x origin moved by `shift` (the shear of the pinned configuration)."""
    X, Y = cell_centres(m, n, h)
    A = single_mode_amplitude(phi_s, eps)
    q = math.sqrt(3.0) / 2.0
    return phi_s + A * (np.cos(q * (X - shift)) * np.cos(q * Y / math.sqrt(3.0))
                        - 0.5 * np.cos(2.0 * q * Y / math.sqrt(3.0)))


def ensemble_instances(count: int = 64, seed: int = 4, rank: int = 0):
    """The batched-ensemble workload: `count` first-order instances with sizes drawn
    uniformly from {128, 256, 512, 1024}^2, epsilon ~ U[0.02, 0.1], beta ~ U[0.5, 1.5],
    mean density ~ U[0.05, 0.1], h = 0.5, s = 0.01, and noise 0.05 U(-1, 1) initial
    data.  Returns a list of dicts: m, n, h, dt, epsilon, beta and phi0."""
    rng = np.random.default_rng(seed)
    sizes = rng.choice([128, 256, 512, 1024], size=count)
    eps, beta = [], []
    for _ in range(count):   # drawn per instance, epsilon then beta
        eps.append(float(rng.uniform(0.02, 0.1)))
        beta.append(float(rng.uniform(0.5, 1.5)))
    mean = rng.uniform(0.05, 0.1, size=count)
    out = []
    for i in range(count):
        m = int(sizes[i])
        out.append(dict(m=m, n=m, h=0.5, dt=0.01, epsilon=eps[i], beta=beta[i],
                        phi0=noise_field(m, m, float(mean[i]), 0.05, 100 + i + 1000 * rank)))
    return out
