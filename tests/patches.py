"""Patches of large seeded fields for the oracle: a cell's neighbourhood cut out as a
small periodic grid with the big grid's red-black colouring, from the generator's
values at those cells (no field of the big size is built on the host)."""
import numpy as np

from paper_1208_2643_gb300 import inputs

PATCH = 16


def patch(m, n, ci, cj, size=PATCH):
    """Rows and columns of the size x size patch around cell (ci, cj) of an m x n
    periodic grid (m, n even), with the grid's colouring ((i + j) parity), and the
    cell's (row, column) in the patch, at least size/2 - 2 cells from the patch's edges."""
    odd = (ci + cj) & 1
    i0, j0 = ci - size // 2, cj - size // 2 - odd
    rows = [(j0 + b) % n for b in range(size)]
    cols = [(i0 + a) % m for a in range(size)]
    return rows, cols, (size // 2 + odd, size // 2)


def at(m, field, rows, cols):
    """Generator field (mean, amplitude, seed) at the patch's cells."""
    return inputs.noise_at(m, *field, rows, cols)


def sample_cells(m, n, count, seed=2024):
    """Corners, edge cells and `count` random cells of an m x n grid."""
    rng = np.random.default_rng(seed)
    fixed = [(0, 0), (m - 1, n - 1), (m - 1, 0), (0, n - 1), (1, n // 2), (m // 2, 1), (m - 2, n - 3),
             (m // 2 + 1, n // 2)]
    return fixed + [(int(i), int(j)) for i, j in zip(rng.integers(0, m, count), rng.integers(0, n, count))]
