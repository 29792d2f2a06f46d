"""Dense-Jacobian Newton solve of N(u) = S on all 3mn unknowns (small grids).

TEST INFRASTRUCTURE ONLY (see the package docstring).

This is the brute-force pin of the multigrid solver: the schemes are uniquely
solvable (Sec. 3.3, second theorem), so the FAS V-cycle must converge to the
same u that plain Newton on the assembled system finds.  It is written in numpy
from the operator definitions of App. B.1/B.2 and shares nothing with the C
oracle: the Laplacian is an assembled sparse-as-dense matrix and the linear
solves use numpy.linalg.solve.
"""
from __future__ import annotations

import numpy as np


def lap_matrix(m, n, h, ny_neumann=False):
    """Matrix of the five-point Delta_h on (n, m) arrays flattened row-major: periodic,
    or (ny_neumann) periodic in x and homogeneous Neumann in y, where a ghost row takes
    the value of the boundary row next to it (App. A, (A.7))."""
    G = m * n
    L = np.zeros((G, G))
    for j in range(n):
        for i in range(m):
            r = j * m + i
            L[r, r] -= 4.0 / h**2
            for (ii, jj) in ((i - 1, j), (i + 1, j), (i, j - 1), (i, j + 1)):
                if ny_neumann:
                    jj = min(max(jj, 0), n - 1)
                L[r, (jj % n) * m + (ii % m)] += 1.0 / h**2
    return L


def _g(scheme, phi, phik):
    if scheme == 1:
        return phi**3
    return 0.25 * (phi**2 + phik**2) * (phi + phik)


def _dg(scheme, phi, phik):
    if scheme == 1:
        return 3.0 * phi**2
    return 0.25 * (3.0 * phi**2 + 2.0 * phi * phik + phik**2)


def newton_solve(scheme, consts, h, S, phik=None, u0=None, tol=1e-14, max_iter=50, ny_neumann=False, W=None):
    """Solves N(u) = S (App. B.1/B.2) by Newton's method with the exact Jacobian.
    W (optional): pinning weight of Sec. 4.6, which adds -W phi to row 2 of N.
    Returns (phi, mu, kappa) as (n, m) arrays and the final max-norm residual."""
    c, gam, theta = consts
    S1, S2, S3 = [np.asarray(x, dtype=np.float64).ravel() for x in S]
    n, m = np.asarray(S[0]).shape
    G = m * n
    L = lap_matrix(m, n, h, ny_neumann)
    pk = np.zeros(G) if phik is None else np.asarray(phik, dtype=np.float64).ravel()
    w = np.zeros(G) if W is None else np.asarray(W, dtype=np.float64).ravel()
    if u0 is None:
        phi, mu, kappa = np.zeros(G), np.zeros(G), np.zeros(G)
    else:
        phi, mu, kappa = [np.asarray(x, dtype=np.float64).ravel().copy() for x in u0]
    I = np.eye(G)
    Z = np.zeros((G, G))
    res = np.inf
    for _ in range(max_iter):
        N1 = phi - c * (L @ mu)
        N2 = mu - _g(scheme, phi, pk) - (gam + w) * phi - L @ kappa
        N3 = kappa - theta * (L @ phi)
        r = np.concatenate([S1 - N1, S2 - N2, S3 - N3])
        res = float(np.max(np.abs(r)))
        if res < tol:
            break
        D = np.diag(gam + w + _dg(scheme, phi, pk))
        J = np.block([[I, -c * L, Z], [-D, I, -L], [-theta * L, Z, I]])
        du = np.linalg.solve(J, r)
        phi, mu, kappa = phi + du[:G], mu + du[G:2 * G], kappa + du[2 * G:]
    shp = (n, m)
    return (phi.reshape(shp), mu.reshape(shp), kappa.reshape(shp)), res
