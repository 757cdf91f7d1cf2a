"""Pins of the FP64 CPU oracle against facts fixed outside it (no GPU).

Each test checks the oracle against something it does not compute itself: textbook element
matrices, an independent Kronecker-product assembly, dense brute-force solves of the KKT system
of Sec. 2, closed-form sine modes, the continuum manufactured solution, and the spectral facts
the paper states in Sec. 3.2 and Sec. 4.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1312_5653_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden", "q1_element_unit.txt")


def _golden():
    blocks, cur = {}, None
    for line in open(GOLD):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line[0].isalpha() or line[0].isdigit() and "_" in line:
            cur = line
            blocks[cur] = []
        else:
            blocks[cur].append([float(t) for t in line.split()])
    return {k: np.array(v) for k, v in blocks.items()}


def kron_KM(dim, nel):
    """Independent assembly: Q1 K and M as Kronecker products of the 1D tridiagonal matrices
    K1 = tridiag(-1, 2, -1)/h, M1 = h tridiag(1, 4, 1)/6 (interior nodes, axis 0 fastest)."""
    nel = [nel] * dim if np.isscalar(nel) else nel
    K1, M1 = [], []
    for a in range(dim):
        m, h = nel[a] - 1, 1.0 / nel[a]
        I = np.eye(m)
        E = np.eye(m, k=1) + np.eye(m, k=-1)
        K1.append((2 * I - E) / h)
        M1.append(h * (4 * I + E) / 6)

    def kron_axes(mats):  # mats[a] acts on axis a; axis 0 fastest => rightmost factor
        out = np.array([[1.0]])
        for a in reversed(range(dim)):
            out = np.kron(out, mats[a])
        return out

    K = sum(kron_axes([K1[a] if a == t else M1[a] for a in range(dim)]) for t in range(dim))
    M = kron_axes(M1)
    return K, M


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


# ------------------------------------------------------------------------ element / assembly
def test_element_matrices_match_textbook():
    g = _golden()
    Ke, Me = oracle.element(2, [1.0, 1.0])
    assert np.allclose(Ke * 6, g["2d_stiffness_x6"], atol=1e-13)
    assert np.allclose(Me * 36, g["2d_mass_x36"], atol=1e-13)
    Ke, Me = oracle.element(3, [1.0, 1.0, 1.0])
    ks = g["3d_stiffness_x12_by_hamming_distance"][0]
    ms = g["3d_mass_x216_by_hamming_distance"][0]
    for p in range(8):
        for q in range(8):
            d = bin(p ^ q).count("1")
            assert abs(Ke[p, q] * 12 - ks[d]) < 1e-13
            assert abs(Me[p, q] * 216 - ms[d]) < 1e-13


def test_element_scaling_rectangular():
    # stiffness of a hx x hy rectangle: x-part scales hy/hx, y-part hx/hy; mass scales hx*hy
    Ke1, Me1 = oracle.element(2, [1.0, 1.0])
    Ke, Me = oracle.element(2, [0.5, 2.0])
    assert np.allclose(Me, Me1 * 1.0)
    assert np.allclose(Ke.sum(axis=1), 0.0, atol=1e-13)
    assert abs(Me.sum() - 1.0) < 1e-13


@pytest.mark.parametrize("dim,nel", [(2, 5), (2, (4, 6)), (3, 4), (3, (3, 4, 5))])
def test_assembly_matches_kronecker(dim, nel):
    K, M = oracle.assemble_dense(dim, nel)
    Kk, Mk = kron_KM(dim, nel)
    assert np.abs(K - Kk).max() < 1e-12 * np.abs(Kk).max()
    assert np.abs(M - Mk).max() < 1e-12 * np.abs(Mk).max()
    x = np.random.default_rng(0).standard_normal(K.shape[0])
    Kx, Mx = oracle.apply_KM(dim, nel, x)
    assert rel(Kx, K @ x) < 1e-13 and rel(Mx, M @ x) < 1e-13


@pytest.mark.parametrize("dim,nel", [(2, 7), (3, 5)])
def test_sine_vectors_are_eigenvectors(dim, nel):
    K, M = kron_KM(dim, nel)
    kap, mu = oracle.fd_eigs(dim, nel)
    m = nel - 1
    for idx in [0, 1, m + 2, K.shape[0] - 1]:
        mode, r = [], idx
        for a in range(dim):
            mode.append(r % m + 1)
            r //= m
        v = inputs.sine_mode(dim, nel, mode)
        assert rel(K @ v, kap[idx] * v) < 1e-12
        assert rel(M @ v, mu[idx] * v) < 1e-12


# ------------------------------------------------------------------------ brute force
def dense_kkt(K, M, beta):
    n = K.shape[0]
    Z = np.zeros((n, n))
    return np.block([[M, Z, K], [Z, beta * M, -M], [K, -M, Z]])


@pytest.mark.parametrize("dim,nel,beta", [(2, 6, 1e-4), (2, (5, 7), 1e-2), (3, 4, 1e-6), (2, 8, 1e-8)])
def test_o1_o2_match_dense_brute_force(dim, nel, beta):
    K, M = kron_KM(dim, nel)
    n = K.shape[0]
    rng = np.random.default_rng(3)
    b = rng.standard_normal((2, n))
    S = K @ np.linalg.solve(M, K) + M / beta
    x_ref = np.linalg.solve(S, b.T).T
    assert rel(oracle.schur_solve_kkt(dim, nel, beta, b), x_ref) < 1e-11
    assert rel(oracle.fd_schur_solve(dim, nel, beta, b), x_ref) < 1e-11
    # general KKT right-hand side, dense 3n system by LU with partial pivoting
    ry, ru, rl = rng.standard_normal((3, n))
    sol = np.linalg.solve(dense_kkt(K, M, beta), np.concatenate([ry, ru, rl]))
    for solver in (oracle.kkt_solve, oracle.fd_kkt_solve):
        y, u, l = solver(dim, nel, beta, ry, ru, rl)
        assert rel(np.concatenate([y, u, l]), sol) < 1e-10
    # S y = S x products
    x = rng.standard_normal(n)
    assert rel(oracle.schur_apply(dim, nel, beta, x), S @ x) < 1e-12
    assert rel(oracle.fd_schur_apply(dim, nel, beta, x), S @ x) < 1e-12


def test_kkt_solution_satisfies_range_space_recovery():
    # Sec. 3.1: S l = K y_bar (homogeneous Dirichlet), y = y_bar - M^-1 K l, u = l / beta
    dim, nel, beta = 2, 8, 1e-3
    K, M = kron_KM(dim, nel)
    yb = inputs.smoothed_noise(dim, nel, seed=5)
    y, u, l = oracle.kkt_solve(dim, nel, beta, ry=M @ yb)
    lam = oracle.schur_solve_kkt(dim, nel, beta, K @ yb)
    assert rel(l, lam) < 1e-11
    assert rel(y, yb - np.linalg.solve(M, K @ lam)) < 1e-11
    assert rel(u, lam / beta) < 1e-11
    # x = S^{-1} M y_bar equals beta * y (state elimination of the same system)
    x = oracle.fd_schur_solve(dim, nel, beta, M @ yb)
    assert rel(x, beta * y) < 1e-11


# ------------------------------------------------------------------------ closed forms
@pytest.mark.parametrize("dim,nel,beta,count", [(2, 32, 1e-4, 4), (3, 12, 1e-6, 8)])
def test_closed_form_sine_modes(dim, nel, beta, count):
    """b = M v for a sine vector v gives x = v / ((kappa/mu)^2 + gamma^2) exactly; kappa and mu
    are taken as Rayleigh quotients of the independently assembled matrices."""
    K, M = kron_KM(dim, nel)
    g2 = 1.0 / beta
    for mode in inputs.lowest_mode_list(dim, count):
        v = inputs.sine_mode(dim, nel, mode)
        kap = v @ K @ v / (v @ v)
        mu = v @ M @ v / (v @ v)
        expect = v / ((kap / mu) ** 2 + g2)
        b = M @ v
        assert rel(oracle.fd_schur_solve(dim, nel, beta, b), expect) < 1e-12
        if dim == 2:
            assert rel(oracle.schur_solve_kkt(dim, nel, beta, b), expect) < 1e-11


def test_o1_o2_cross_check_medium():
    rng = np.random.default_rng(11)
    for dim, nel, beta in [(2, 64, 1e-6), (3, 10, 1e-2)]:
        n = oracle.ndof(dim, nel)
        b = rng.standard_normal(n)
        x1 = oracle.schur_solve_kkt(dim, nel, beta, b)
        x2 = oracle.fd_schur_solve(dim, nel, beta, b)
        assert rel(x1, x2) < 1e-11
        assert rel(oracle.schur_apply(dim, nel, beta, x2), b) < 1e-10


@pytest.mark.parametrize("dim", [2, 3])
def test_manufactured_solution_converges_at_second_order(dim):
    beta = 1e-4
    sizes = [8, 16, 32, 64] if dim == 2 else [4, 8, 16]
    errs = []
    for N in sizes:
        yb = inputs.manufactured(dim, N, beta)
        b = oracle.apply_M(dim, N, yb)
        y = oracle.fd_schur_solve(dim, N, beta, b) / beta
        exact = inputs.sine_mode(dim, N, (1,) * dim)
        errs.append(np.abs(y - exact).max())
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 1.85) and np.all(rates < 2.15), rates


# ------------------------------------------------------------------------ paper identities
@pytest.mark.parametrize("beta", [1e-2, 1e-4, 1e-8])
def test_complex_factorisation_is_exact(beta):
    """Sec. 4: S = (K + M/(i sqrt beta)) M^-1 (K - M/(i sqrt beta)); the factors commute."""
    K, M = kron_KM(2, 6)
    g = 1.0 / np.sqrt(beta)
    S = K @ np.linalg.solve(M, K) + M / beta
    A = K + 1j * g * M
    Ab = K - 1j * g * M
    paper = (K + M / (1j * np.sqrt(beta))) @ np.linalg.solve(M, K - M / (1j * np.sqrt(beta)))
    assert np.linalg.norm(paper - S) / np.linalg.norm(S) < 1e-13
    assert np.linalg.norm(A @ np.linalg.solve(M, Ab) - S) / np.linalg.norm(S) < 1e-13
    assert np.abs(S - S.T).max() < 1e-12 * np.abs(S).max()


@pytest.mark.parametrize("dim,nel,beta", [(2, 7, 1e-4), (3, 4, 1e-2), (2, 9, 1e-8)])
def test_real_input_shortcut(dim, nel, beta):
    """A - conj(A) = 2 i gamma M gives S^-1 = (conj(A)^-1 - A^-1)/(2 i gamma), so for real b
    S^-1 b = -Im(A^-1 b)/gamma; the two-factor solve conj(A)^-1 M A^-1 b is real."""
    K, M = kron_KM(dim, nel)
    g = 1.0 / np.sqrt(beta)
    b = np.random.default_rng(1).standard_normal(K.shape[0])
    S = K @ np.linalg.solve(M, K) + M / beta
    x = np.linalg.solve(S, b)
    A = K + 1j * g * M
    z = np.linalg.solve(A, b)
    assert rel(-z.imag / g, x) < 1e-10
    two = np.linalg.solve(A.conj(), M @ z)
    assert np.abs(two.imag).max() < 1e-10 * np.abs(two).max()
    assert rel(two.real, x) < 1e-10
    zc = np.linalg.solve(A.conj(), b)
    assert rel(zc, z.conj()) < 1e-13
    # the oracle's complex solve agrees with the dense one, for both signs
    assert rel(oracle.fd_complex_solve(dim, nel, g, b), z) < 1e-12
    assert rel(oracle.fd_complex_solve(dim, nel, g, b, sgn=-1), zc) < 1e-12
    bc = b + 1j * np.random.default_rng(2).standard_normal(b.size)
    assert rel(oracle.fd_complex_solve(dim, nel, g, bc), np.linalg.solve(A, bc)) < 1e-12


def test_pearson_wathen_bounds():
    """Sec. 3.2: S_p = (K + M/sqrt(beta)) M^-1 (K + M/sqrt(beta)) = S + 2 K/sqrt(beta) and the
    eigenvalues of S_p^-1 S lie in [1/2, 1]."""
    for beta in [1e-1, 1e-4, 1e-8]:
        K, M = kron_KM(2, 6)
        g = 1.0 / np.sqrt(beta)
        S = K @ np.linalg.solve(M, K) + M / beta
        Sp = (K + g * M) @ np.linalg.solve(M, K + g * M)
        assert np.linalg.norm(Sp - (S + 2 * g * K)) / np.linalg.norm(Sp) < 1e-13
        ev = np.linalg.eigvals(np.linalg.solve(Sp, S)).real
        assert ev.min() >= 0.5 - 1e-10 and ev.max() <= 1 + 1e-10


def test_mgw_preconditioner_three_eigenvalues():
    """Sec. 3.2: P_mgw = diag(M, beta M, S) gives P^-1 A with eigenvalues in {1, (1 +- sqrt 5)/2}."""
    K, M = kron_KM(2, 5)
    beta = 1e-3
    n = K.shape[0]
    S = K @ np.linalg.solve(M, K) + M / beta
    A = dense_kkt(K, M, beta)
    Z = np.zeros((n, n))
    P = np.block([[M, Z, Z], [Z, beta * M, Z], [Z, Z, S]])
    ev = np.linalg.eigvals(np.linalg.solve(P, A))
    targets = np.array([1.0, (1 + 5 ** 0.5) / 2, (1 - 5 ** 0.5) / 2])
    dist = np.abs(ev[:, None] - targets[None, :]).min(axis=1)
    assert dist.max() < 1e-8


def test_fd_threads_do_not_change_results():
    """The OpenMP split of the O2 sine transforms gives bitwise the same x for 1 and 4 threads."""
    b = np.random.default_rng(11).standard_normal((2, 63 * 47))
    prev = oracle.set_threads(0)  # the count in effect, unchanged
    try:
        oracle.set_threads(1)
        x1 = oracle.fd_schur_solve(2, (64, 48), 1e-4, b)
        oracle.set_threads(4)
        x4 = oracle.fd_schur_solve(2, (64, 48), 1e-4, b)
    finally:
        oracle.set_threads(prev)
    assert np.array_equal(x1, x4)


# ------------------------------------------------------------ Dirichlet data, S_p (Sec. 3.2, 6.1)
def _full_kron_K(dim, nel):
    """Independent assembly of the stiffness on ALL grid nodes (Neumann, boundary included) as
    Kronecker products of 1D matrices whose end rows have one element: K1 = (1/h) tridiag(-1, 2, -1)
    with 1/h at both ends."""
    nel = [nel] * dim if np.isscalar(nel) else nel
    K1, M1 = [], []
    for a in range(dim):
        m, h = nel[a] + 1, 1.0 / nel[a]
        E = np.eye(m, k=1) + np.eye(m, k=-1)
        d = np.full(m, 2.0)
        d[0] = d[-1] = 1.0
        K1.append((np.diag(d) - E) / h)
        M1.append(h * (np.diag(2 * d) + E) / 6)

    def kron_axes(mats):
        out = np.array([[1.0]])
        for a in reversed(range(dim)):
            out = np.kron(out, mats[a])
        return out

    return sum(kron_axes([K1[a] if a == t else M1[a] for a in range(dim)]) for t in range(dim))


@pytest.mark.parametrize("dim,nel", [(2, 7), (2, (6, 9)), (3, 4), (3, (3, 5, 4))])
def test_full_stiffness_against_kronecker_assembly(dim, nel):
    """K y + K_c y_c (Sec. 2) equals the interior rows of an independently assembled full-grid
    stiffness applied to the full vector; harmonic (bi/trilinear) data give zero."""
    Kf = _full_kron_K(dim, nel)
    inner = oracle.interior_index(dim, nel)
    y = np.random.default_rng(3).standard_normal(oracle.nfull(dim, nel))
    assert rel(oracle.full_stiffness(dim, nel, y), (Kf @ y)[inner]) < 1e-13
    assert np.abs(oracle.full_stiffness(dim, nel, inputs.harmonic_full(dim, nel))).max() < 1e-12
    # zero boundary data: the interior operator K of the homogeneous problem
    yz = np.zeros_like(y)
    yz[inner] = y[inner]
    Kx, _ = oracle.apply_KM(dim, nel, y[inner])
    assert rel(oracle.full_stiffness(dim, nel, yz), Kx) < 1e-13


def test_control_solve_harmonic_target_is_exact():
    """If ybar is harmonic and its boundary values are y_c, y = ybar satisfies the state equation
    with u = 0 at zero cost: the solution is (ybar, 0, 0)."""
    for dim, nel in [(2, 12), (3, 6)]:
        yf = inputs.harmonic_full(dim, nel)
        yb = oracle.interior_of(dim, nel, yf)
        for fd in (False, True):
            y, u, l = oracle.control_solve(dim, nel, 1e-4, yf, fd=fd)
            assert rel(y, yb) < 1e-12
            assert np.linalg.norm(u) < 1e-10 * np.linalg.norm(yb) and np.linalg.norm(l) < 1e-14 * np.linalg.norm(yb)


@pytest.mark.parametrize("beta", [2e-2, 2e-5, 2e-8])
def test_control_solve_thermal_target(beta):
    """Sec. 6.1: the paper's target and boundary data.  O1 (banded KKT) and O2 (sine basis) agree;
    the solution satisfies the constraint K y + K_c y_c = M u, u = lambda / beta, and
    S lambda = K ybar + K_c y_c (Eq. schurcomplementsystem) against a dense S."""
    N = 16
    yf = inputs.thermal_target(N)
    y1, u1, l1 = oracle.control_solve(2, N, beta, yf)
    y2, u2, l2 = oracle.control_solve(2, N, beta, yf, fd=True)
    assert rel(y2, y1) < 1e-11 and rel(u2, u1) < 1e-11 and rel(l2, l1) < 1e-11
    K, M = kron_KM(2, N)
    kc = oracle.boundary_coupling(2, N, yf)
    assert np.linalg.norm(K @ y1 + kc - M @ u1) < 1e-10 * np.linalg.norm(K @ y1)
    assert rel(u1, l1 / beta) < 1e-12
    S = K @ np.linalg.solve(M, K) + M / beta
    yb = oracle.interior_of(2, N, yf)
    assert rel(S @ l1, K @ yb + kc) < 1e-9


def test_thermal_target_values():
    """Eq. ex1target on a 4 x 4 grid: (2x - 1)^2 (2y - 1)^2 on [0, 1/2]^2, 0 elsewhere."""
    t = inputs.thermal_target(4).reshape(5, 5)  # [x2 index, x1 index]
    assert t[0, 0] == 1.0 and t[0, 1] == 0.25 and t[1, 1] == 0.0625 and t[2, 2] == 0.0
    assert t[0, 3] == 0.0 and t[3, 0] == 0.0 and t[1, 0] == 0.25


@pytest.mark.parametrize("dim,nel", [(2, 6), (3, 4)])
def test_pw_solve_against_dense(dim, nel):
    """O2's S_p^{-1} b (Sec. 3.2, Eq. pearsonapproximation) against a dense (K + gM) M^-1 (K + gM)."""
    beta = 1e-3
    K, M = kron_KM(dim, nel)
    g = 1.0 / np.sqrt(beta)
    Sp = (K + g * M) @ np.linalg.solve(M, K + g * M)
    b = np.random.default_rng(4).standard_normal((2, K.shape[0]))
    assert rel(oracle.fd_pw_solve(dim, nel, beta, b), np.linalg.solve(Sp, b.T).T) < 1e-12
