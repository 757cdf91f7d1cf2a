"""Seeded synthetic target states (the only code shared by the oracle side and the CUDA side).

This module draws inputs; it holds none of the solver's arithmetic.  Every generator returns the
target state y_bar as nodal values on the interior nodes of a uniform grid on the unit box
(lexicographic order, axis 0 fastest), shape (n,) or (nrhs, n).  Each side then forms its own
right-hand side b = M y_bar with its own mass operator.

Recipes (the paper's thermal target, Sec. 6.1, is smooth and analytic; these stand in for it):
  * ``lowest_modes``      sum of the lowest sine modes with N(0,1) coefficients
                          (small 2D correctness case: 4 modes).
  * ``smoothed_noise``    i.i.d. N(0,1) nodal values smoothed by damped Jacobi sweeps
                          (omega = 2/3, zero right-hand side, zero boundary values) with the
                          diagonally scaled Q1 Laplacian stencil (2D: 1 at the centre, -1/8 at the
                          8 neighbours; 3D: 1 at the centre, 0 at faces, -1/16 at edges, -1/32 at
                          vertices), the large 2D workload.
  * ``random_modes_3d``   8 distinct modes drawn from {1..4}^3, N(0,1) coefficients.
  * ``manufactured``      (1 + 4 pi^4 beta) sin(pi x1) sin(pi x2) (...) whose continuum optimal
                          state is the plain sine product.
"""
import itertools

import numpy as np


def interior_coords(dim, nel):
    """Coordinates of the interior nodes, list of dim arrays of length n (axis 0 fastest)."""
    nel = [int(nel)] * dim if np.isscalar(nel) else list(nel)
    axes = [np.arange(1, nel[a]) / nel[a] for a in range(dim)]
    grids = np.meshgrid(*axes[::-1], indexing="ij")  # last axis slowest
    return [g.reshape(-1) for g in grids[::-1]]


def sine_mode(dim, nel, mode):
    x = interior_coords(dim, nel)
    v = np.ones_like(x[0])
    for a in range(dim):
        v = v * np.sin(np.pi * mode[a] * x[a])
    return v


def lowest_mode_list(dim, count):
    """The `count` sine modes with the smallest |j|^2 (ties kept in lexicographic order)."""
    cand = sorted(itertools.product(range(1, count + 2), repeat=dim), key=lambda j: (sum(t * t for t in j), j))
    return [tuple(j) for j in cand[:count]]


def lowest_modes(dim, nel, count=4, seed=0, nrhs=None):
    rng = np.random.default_rng(seed)
    modes = lowest_mode_list(dim, count)
    k = 1 if nrhs is None else nrhs
    vecs = [sine_mode(dim, nel, m) for m in modes]
    out = np.zeros((k, vecs[0].size))
    for r in range(k):
        c = rng.standard_normal(len(modes))
        out[r] = sum(ci * v for ci, v in zip(c, vecs))
    return out[0] if nrhs is None else out


def _smooth_stencil(dim):
    if dim == 2:
        w = np.full((3, 3), -1.0 / 8.0)
        w[1, 1] = 1.0
        return w
    w = np.zeros((3, 3, 3))
    for idx in itertools.product(range(3), repeat=3):
        off = sum(1 for t in idx if t != 1)
        w[idx] = {0: 1.0, 1: 0.0, 2: -1.0 / 16.0, 3: -1.0 / 32.0}[off]
    return w


def smoothed_noise(dim, nel, seed=1, sweeps=3, omega=2.0 / 3.0, nrhs=None):
    nel = [int(nel)] * dim if np.isscalar(nel) else list(nel)
    m = [nel[a] - 1 for a in range(dim)]
    rng = np.random.default_rng(seed)
    k = 1 if nrhs is None else nrhs
    w = _smooth_stencil(dim)
    out = []
    for _ in range(k):
        y = rng.standard_normal(m[::-1])  # array axes: (last, ..., axis 0)
        for _ in range(sweeps):
            pad = np.pad(y, 1)
            ky = np.zeros_like(y)
            for idx in itertools.product(range(3), repeat=dim):
                sl = tuple(slice(idx[t], idx[t] + y.shape[t]) for t in range(dim))
                ky += w[idx] * pad[sl]
            y = y - omega * ky
        out.append(y.reshape(-1))
    out = np.array(out)
    return out[0] if nrhs is None else out


def random_modes_3d(nel, count=8, seed=2, nrhs=None):
    rng = np.random.default_rng(seed)
    allm = list(itertools.product(range(1, 5), repeat=3))
    k = 1 if nrhs is None else nrhs
    out = []
    for _ in range(k):
        pick = rng.choice(len(allm), size=count, replace=False)
        c = rng.standard_normal(count)
        out.append(sum(ci * sine_mode(3, nel, allm[p]) for ci, p in zip(c, pick)))
    out = np.array(out)
    return out[0] if nrhs is None else out


def manufactured(dim, nel, beta):
    """Target whose continuum optimal state is prod_a sin(pi x_a): (I + beta Lap^2) y = y_bar and
    Lap^2 of the sine product is (dim pi^2)^2 times it."""
    return (1.0 + (dim * np.pi ** 2) ** 2 * beta) * sine_mode(dim, nel, (1,) * dim)


def thermal_target(nel):
    """The target temperature of the paper's thermal problem (Sec. 6.1, Eq. ex1target) on all
    (nel+1)^2 nodes of the unit square, boundary included (lexicographic, axis 0 fastest):
    (2 x1 - 1)^2 (2 x2 - 1)^2 on [0, 1/2]^2 and 0 elsewhere.  Its boundary values are the Dirichlet
    data y_c (Eq. ex1boundarycondition)."""
    nel = [int(nel)] * 2 if np.isscalar(nel) else list(nel)
    x0 = np.arange(nel[0] + 1) / nel[0]
    x1 = np.arange(nel[1] + 1) / nel[1]
    X1, X0 = np.meshgrid(x1, x0, indexing="ij")  # array axis 1 = grid axis 0 (fastest)
    y = (2 * X0 - 1) ** 2 * (2 * X1 - 1) ** 2
    y[(X0 > 0.5) | (X1 > 0.5)] = 0.0
    return np.ascontiguousarray(y.reshape(-1))


def harmonic_full(dim, nel, coef=(1.0, 1.0, 2.0, 1.0)):
    """c0 + c1 x1 + c2 x2 + c3 x1 x2 (times 1 + x3 in 3D) on all grid nodes, boundary included: a
    target for which the state equation holds with zero control (Q1 reproduces it, and it is
    harmonic), so the optimal control problem's solution is y = ybar, u = 0, lambda = 0."""
    nel = [int(nel)] * dim if np.isscalar(nel) else list(nel)
    axes = [np.arange(nel[a] + 1) / nel[a] for a in range(dim)]
    grids = np.meshgrid(*axes[::-1], indexing="ij")[::-1]  # grids[a] varies along grid axis a
    c0, c1, c2, c3 = coef
    y = c0 + c1 * grids[0] + c2 * grids[1] + c3 * grids[0] * grids[1]
    if dim == 3:
        y = y * (1.0 + grids[2])
    return np.ascontiguousarray(y.reshape(-1))
