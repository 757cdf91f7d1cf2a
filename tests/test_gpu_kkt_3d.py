"""GPU parity of the full-space path (Sec. 3.2: KKT operator, P_mgw preconditioner, MINRES) and
of 3D solves (8^3-element subdomains, the block-level kernels) against the FP64 CPU oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle
from paper_1312_5653_gb300 import inputs
from paper_1312_5653_gb300 import schur as S

DEV = "cuda:0"


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


def gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(DEV)


@pytest.mark.parametrize("prec", [S.SCHUR_FP64, S.SCHUR_MIXED])
def test_kkt_apply_and_preconditioner(prec):
    dim, N, P, beta = 2, 32, 4, 1e-4
    n = (N - 1) ** 2
    rng = np.random.default_rng(4)
    sol = S.Solver(dim, N, beta, nsub=P, precision=prec)
    v = rng.standard_normal((2, 3 * n))
    r = sol.schur_kkt_apply(gpu(v)).cpu().numpy()
    for c in range(2):
        y, u, l = v[c, :n], v[c, n:2 * n], v[c, 2 * n:]
        Ky, My = oracle.apply_KM(dim, N, y)
        Ku, Mu = oracle.apply_KM(dim, N, u)
        Kl, Ml = oracle.apply_KM(dim, N, l)
        ref = np.concatenate([My + Kl, beta * Mu - Ml, Ky - Mu])
        assert rel(r[c], ref) < 1e-13
    z = sol.schur_kkt_precond_apply(gpu(v)).cpu().numpy()
    for c in range(2):
        zy, zu, zl = z[c, :n], z[c, n:2 * n], z[c, 2 * n:]
        assert rel(oracle.apply_M(dim, N, zy), v[c, :n]) < 1e-11          # M z_y = r_y
        assert rel(beta * oracle.apply_M(dim, N, zu), v[c, n:2 * n]) < 1e-11  # beta M z_u = r_u
        assert rel(zl, oracle.fd_schur_solve(dim, N, beta, v[c, 2 * n:])) < (1e-10 if prec == S.SCHUR_FP64 else 1e-8)
    sol.close()


@pytest.mark.parametrize("beta", [1e-4, 1e-8])
def test_kkt_minres_multi_rhs(beta):
    """Full-space form: MINRES with P_mgw on (M y_bar, 0, 0) for several targets at once; the
    preconditioned operator has three eigenvalues, so a handful of iterations suffice."""
    dim, N, P = 2, 64, 8
    n = (N - 1) ** 2
    yb = inputs.smoothed_noise(dim, N, seed=10, nrhs=4)
    ry = oracle.apply_M(dim, N, yb)
    rhs = np.zeros((4, 3 * n))
    rhs[:, :n] = ry
    y, u, l = oracle.fd_kkt_solve(dim, N, beta, ry=ry)
    ref = np.concatenate([y, u, l], axis=1)
    sol = S.Solver(dim, N, beta, nsub=P, precision=S.SCHUR_MIXED)
    x, it = sol.schur_kkt_minres(gpu(rhs), tol=1e-10, max_it=40)
    x = x.cpu().numpy()
    for c in range(4):
        assert rel(x[c], ref[c]) < 1e-8, (c, it)
    assert it <= 12, it
    sol.close()


@pytest.mark.parametrize("prec", [S.SCHUR_FP64, S.SCHUR_MIXED])
def test_3d_eight_cubed_subdomains(prec):
    """3D, 32^3 Q1 elements, 4^3 subdomains of 8^3 (the subdomain shape of the large 3D case),
    beta = 1e-6, target = 8 random sine modes."""
    dim, N, P, beta = 3, 32, 4, 1e-6
    yb = inputs.random_modes_3d(N, count=8, seed=2)
    b = oracle.apply_M(dim, N, yb)
    xref = oracle.fd_schur_solve(dim, N, beta, b)
    sol = S.Solver(dim, N, beta, nsub=P, precision=prec)
    x = sol.schur_solve(gpu(b)).cpu().numpy()
    print("3d", prec, sol.last_stats, rel(x, xref))
    assert rel(x, xref) <= (1e-10 if prec == S.SCHUR_FP64 else 1e-8)
    sol.close()


def test_3d_large_mixed_precision():
    """128^3 Q1 elements (2,048,383 dofs), 16^3 subdomains of 8^3, beta = 1e-6, mixed precision
    with FP64 refinement; the refinement stops at ||b - A z|| / ||b|| <= 1e-10 and the result is
    compared with the fast-diagonalisation oracle and its true residual ||b - S x|| / ||b||."""
    dim, N, P, beta = 3, 128, 16, 1e-6
    yb = inputs.random_modes_3d(N, count=8, seed=2)
    b = oracle.apply_M(dim, N, yb)
    xref = oracle.fd_schur_solve(dim, N, beta, b)
    sol = S.Solver(dim, N, beta, nsub=P, precision=S.SCHUR_MIXED, tol=1e-10)
    x = sol.schur_solve(gpu(b)).cpu().numpy()
    st = sol.last_stats
    res = np.linalg.norm(b - oracle.fd_schur_apply(dim, N, beta, x)) / np.linalg.norm(b)
    # kappa(S) * eps bounds the real residual of any FP64 x: the oracle's own solution reaches
    # about 1e-10 here, so the GPU result is held to a small multiple of that
    res_ref = np.linalg.norm(b - oracle.fd_schur_apply(dim, N, beta, xref)) / np.linalg.norm(b)
    print("3d large", st, "relerr", rel(x, xref), "S-residual", res, "oracle S-residual", res_ref)
    assert rel(x, xref) <= 1e-8
    assert st["rel_residual"] <= 1e-10
    assert res <= max(4 * res_ref, 1e-10)
    sol.close()
