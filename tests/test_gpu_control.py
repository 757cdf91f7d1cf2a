"""GPU parity of the two further forms of the paper's method.

1. The Pearson-Wathen approximation S_p = (K + gamma M) M^-1 (K + gamma M) (Sec. 3.2, Eq.
   pearsonapproximation) inverted through the real factor K + gamma M (factor SCHUR_FACTOR_PW):
   schur_solve against the oracle's sine-basis S_p^-1, and MINRES on the KKT system with P_mgw built
   on S_p against the oracle's KKT solution (the preconditioner changes the iteration count only).
2. The range-space method with Dirichlet data (the thermal problem of Sec. 6.1):
   schur_control_solve's (y, u, lambda) against the oracle's banded KKT solve with right-hand side
   (M ybar, 0, -K_c y_c), the relative constraint violation of Eq. relativeconstraintviolation, and a
   harmonic target whose exact solution is (ybar, 0, 0).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle
from paper_1312_5653_gb300 import inputs
from paper_1312_5653_gb300 import schur as S

TOL = {S.SCHUR_FP64: 1e-10, S.SCHUR_MIXED: 1e-8}


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.mark.parametrize("prec", [S.SCHUR_FP64, S.SCHUR_MIXED])
@pytest.mark.parametrize("dim,N,P,beta", [(2, 64, 4, 1e-4), (2, 64, 4, 1e-8), (3, 16, 2, 1e-6)])
def test_pw_schur_solve_matches_oracle(prec, dim, N, P, beta):
    n = oracle.ndof(dim, N)
    bh = np.random.default_rng(12).standard_normal((2, n))
    sol = S.Solver(dim, N, beta, nsub=P, precision=prec, tol=1e-12, factor=S.SCHUR_FACTOR_PW)
    x = sol.schur_solve(torch.from_numpy(bh).cuda()).cpu().numpy()
    st = sol.last_stats
    sol.close()
    ref = oracle.fd_pw_solve(dim, N, beta, bh)
    assert rel(x, ref) <= TOL[prec], (rel(x, ref), st)


def test_pw_factor_is_the_real_shifted_operator():
    """schur_complex_solve with the S_p factor solves (K + gamma M) z = b: real z, checked against a
    dense solve."""
    dim, N, beta = 2, 16, 1e-3
    K, M = oracle.assemble_dense(dim, N)
    g = 1.0 / np.sqrt(beta)
    b = np.random.default_rng(2).standard_normal(K.shape[0])
    sol = S.Solver(dim, N, beta, nsub=2, factor=S.SCHUR_FACTOR_PW)
    z = sol.schur_complex_solve(torch.from_numpy(b).cuda()).cpu().numpy()
    sol.close()
    ref = np.linalg.solve(K + g * M, b)
    assert rel(z.real, ref) <= 1e-11 and np.abs(z.imag).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("beta", [1e-4, 1e-8])
def test_kkt_minres_with_pw_preconditioner(beta):
    dim, N, P = 2, 64, 4
    n = oracle.ndof(dim, N)
    yb = inputs.smoothed_noise(dim, N, seed=30, nrhs=2)
    ry = oracle.apply_M(dim, N, yb)
    rhs = np.zeros((2, 3 * n))
    rhs[:, :n] = ry
    y, u, l = oracle.fd_kkt_solve(dim, N, beta, ry=ry)
    ref = np.concatenate([y, u, l], axis=1)
    its = {}
    for factor in (S.SCHUR_FACTOR_EXACT, S.SCHUR_FACTOR_PW):
        sol = S.Solver(dim, N, beta, nsub=P, precision=S.SCHUR_MIXED, tol=1e-11, factor=factor)
        x, it = sol.schur_kkt_minres(torch.from_numpy(rhs).cuda(), tol=1e-10, max_it=80)
        sol.close()
        xh = x.cpu().numpy()
        for c in range(2):
            assert rel(xh[c], ref[c]) <= 1e-8, (factor, c, rel(xh[c], ref[c]))
        its[factor] = it
    # exact Schur block: at most a handful of MINRES steps (three distinct eigenvalues); S_p: the
    # spectrum of S_p^-1 S lies in [1/2, 1], so more steps but a bounded number
    assert its[S.SCHUR_FACTOR_EXACT] <= 6 and its[S.SCHUR_FACTOR_EXACT] < its[S.SCHUR_FACTOR_PW] <= 40, its


@pytest.mark.parametrize("prec", [S.SCHUR_FP64, S.SCHUR_MIXED])
@pytest.mark.parametrize("beta", [2e-2, 2e-4, 2e-6, 2e-8])
def test_thermal_control_solve_matches_oracle(prec, beta):
    N, P = 64, 4
    yf = inputs.thermal_target(N)
    yref, uref, lref = oracle.control_solve(2, N, beta, yf)
    sol = S.Solver(2, N, beta, nsub=P, precision=prec, tol=1e-12)
    y, u, lam, viol = sol.schur_control_solve(torch.from_numpy(yf).cuda())
    sol.close()
    y, u, lam = y.cpu().numpy(), u.cpu().numpy(), lam.cpu().numpy()
    assert rel(y, yref) <= TOL[prec] and rel(u, uref) <= TOL[prec] and rel(lam, lref) <= TOL[prec], \
        (rel(y, yref), rel(u, uref), rel(lam, lref))
    # the state equation K y + K_c y_c = M u holds to the solve's accuracy
    assert viol[0] <= 1e-8, viol
    # against the oracle's own violation of the same metric
    K, M = oracle.assemble_dense(2, N)
    kc = oracle.boundary_coupling(2, N, yf)
    v_or = np.linalg.norm(K @ yref + kc - M @ uref) / np.linalg.norm(K @ yref)
    assert v_or <= 1e-10


def test_thermal_control_solve_harmonic_target_and_multi_rhs():
    """Column 0: a harmonic target with its own boundary values (exact solution ybar, 0, 0);
    column 1: the paper's target.  Both in one call (nrhs = 2)."""
    N, P, beta = 32, 4, 1e-4
    yf = np.stack([inputs.harmonic_full(2, N), inputs.thermal_target(N)])
    sol = S.Solver(2, N, beta, nsub=P, tol=1e-12)
    y, u, lam, viol = sol.schur_control_solve(torch.from_numpy(yf).cuda())
    sol.close()
    y, u = y.cpu().numpy(), u.cpu().numpy()
    yb0 = oracle.interior_of(2, N, yf[0])
    assert rel(y[0], yb0) <= 1e-12 and np.abs(u[0]).max() <= 1e-9 * np.abs(yb0).max()
    yref, uref, _ = oracle.control_solve(2, N, beta, yf[1])
    assert rel(y[1], yref) <= 1e-10 and rel(u[1], uref) <= 1e-10
    assert viol[1] <= 1e-8


def test_control_solve_rejects_pw_factor_and_short_ld():
    N = 16
    sol = S.Solver(2, N, 1e-4, nsub=2, factor=S.SCHUR_FACTOR_PW)
    with pytest.raises(S.SchurError):
        sol.schur_control_solve(torch.from_numpy(inputs.thermal_target(N)).cuda())
    sol.close()
    sol = S.Solver(2, N, 1e-4, nsub=2)
    short = torch.zeros(oracle.ndof(2, N), dtype=torch.float64, device="cuda")  # n < (N+1)^2 entries
    with pytest.raises(S.SchurError):
        sol.schur_control_solve(short)
    sol.close()
