"""GPU parity of the factored Schur solve against the FP64 CPU oracle (all through the C-ABI).

Tolerances (stated by the method's target): FP64 path relative error <= 1e-10, mixed-precision
path (complex FP32 FETI-DP with FP64 refinement) <= 1e-8, both against the oracle's x = S^{-1} b.
Internal steps (local operators, coarse matrix) are compared with dense definitions on tiny meshes.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle
from paper_1312_5653_gb300 import inputs
from paper_1312_5653_gb300 import schur as S

from dense_ref import dense_feti_dp, local_operators

DEV = "cuda:0"
TOL = {S.SCHUR_FP64: 1e-10, S.SCHUR_MIXED: 1e-8}
PRECS = [S.SCHUR_FP64, S.SCHUR_MIXED]


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


def gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(DEV)


# 2D layer sizes b = s + 1 of 5, 9, 14, 17 and 32 cover the exact (9, 17) and padded (8, 16, 32)
# register-tile widths of the column-per-thread formation kernel.  3D subdomains of 2^3, 4^3 and
# 8^3 elements (layers of 9, 25 and 81 nodes; 8^3 is the size of the 128^3 workload) run the
# tensor-core formation: one, three and four column tiles, ragged last tiles and chunks.
@pytest.mark.parametrize("dim,N,P,beta", [(2, 8, 2, 1e-4), (2, 12, 3, 1e-2), (3, 6, 3, 1e-6), (2, 16, 2, 1e-6),
                                          (2, 26, 2, 1e-3), (2, 32, 2, 1e-4), (2, 62, 2, 1e-2), (3, 12, 3, 1e-4),
                                          (3, 16, 2, 1e-6)])
@pytest.mark.parametrize("prec", PRECS)
def test_local_operators_match_dense_definitions(dim, N, P, beta, prec):
    sol = S.Solver(dim, N, beta, nsub=P, precision=prec)
    tol = 1e-11 if prec == S.SCHUR_FP64 else 2e-5
    for sd in range(P ** dim):
        F, Frc, Sd = local_operators(dim, N, P, beta, sd)
        for which, ref in ((0, F), (1, Frc), (2, Sd)):
            got = sol.schur_debug_operator(which, sd)
            assert np.abs(got - ref).max() <= tol * np.abs(ref).max(), (sd, which)
    _, _, _, _, Kcc = dense_feti_dp(dim, N, P, beta, np.zeros((N - 1) ** dim))
    got = sol.schur_debug_operator(3)
    assert np.abs(got - Kcc).max() <= tol * np.abs(Kcc).max()
    inv = sol.schur_debug_operator(4)
    assert np.abs(inv @ Kcc - np.eye(Kcc.shape[0])).max() <= (1e-10 if prec == S.SCHUR_FP64 else 1e-5)
    sol.close()


# Coarse grids of 17 x 17 (five reduction levels, odd counts), 9 x 9, 15 x 15 and 5 x 5 x 5 (3D
# layers of 25): the cyclic-reduction inverse against the assembled coarse matrix.
@pytest.mark.parametrize("dim,N,P,beta", [(2, 36, 18, 1e-3), (2, 40, 10, 1e-6), (2, 64, 16, 1e-2), (3, 12, 6, 1e-4)])
@pytest.mark.parametrize("prec", PRECS)
def test_coarse_inverse_multilevel(dim, N, P, beta, prec):
    sol = S.Solver(dim, N, beta, nsub=P, precision=prec)
    K = sol.schur_debug_operator(3)
    inv = sol.schur_debug_operator(4)
    nc = (P - 1) ** dim
    assert K.shape == (nc, nc) and inv.shape == (nc, nc)
    # the mixed form assembles the coarse matrix from FP32 local operators: symmetric to FP32 rounding
    assert np.abs(K - K.T).max() <= (1e-12 if prec == S.SCHUR_FP64 else 1e-6) * np.abs(K).max()
    ref = np.linalg.inv(K)
    err = np.abs(inv - ref).max() / np.abs(ref).max()
    # FP32: unit roundoff 6e-8 times the growth of the reduction on these coarse grids
    assert err <= (1e-11 if prec == S.SCHUR_FP64 else 1e-4), err
    sol.close()


@pytest.mark.parametrize("dim,N,P,beta", [(2, 12, 3, 1e-2), (2, 16, 4, 1e-8), (3, 6, 3, 1e-6), (3, 8, 2, 1e-4)])
@pytest.mark.parametrize("prec", PRECS)
def test_complex_factor_solve(dim, N, P, beta, prec):
    rng = np.random.default_rng(5)
    n = (N - 1) ** dim
    b = rng.standard_normal(n)
    sol = S.Solver(dim, N, beta, nsub=P, precision=prec)
    z = sol.schur_complex_solve(gpu(b)).cpu().numpy()
    zref = oracle.fd_complex_solve(dim, N, 1.0 / np.sqrt(beta), b)
    assert rel(z, zref) <= (1e-11 if prec == S.SCHUR_FP64 else 1e-9)
    # complex right-hand side (the refinement solves with complex residuals)
    bi = rng.standard_normal(n)
    z = sol.schur_complex_solve(gpu(b), gpu(bi)).cpu().numpy()
    assert rel(z, oracle.fd_complex_solve(dim, N, 1.0 / np.sqrt(beta), b + 1j * bi)) <= 1e-9
    sol.close()


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("local_mode", [S.SCHUR_LOCAL_PER_SUBDOMAIN, S.SCHUR_LOCAL_SHARED])
def test_small_2d_lowest_modes(prec, local_mode):
    """32 x 32 Q1 elements, 4 x 4 subdomains of 8 x 8, beta = 1e-4, target = 4 lowest sine modes."""
    dim, N, P, beta = 2, 32, 4, 1e-4
    yb = inputs.lowest_modes(dim, N, count=4, seed=0)
    b = oracle.apply_M(dim, N, yb)
    xref = oracle.schur_solve_kkt(dim, N, beta, b)
    assert rel(xref, oracle.fd_schur_solve(dim, N, beta, b)) < 1e-12
    sol = S.Solver(dim, N, beta, nsub=P, precision=prec, local_mode=local_mode)
    x = sol.schur_solve(gpu(b)).cpu().numpy()
    assert rel(x, xref) <= TOL[prec], sol.last_stats
    # host-buffer entry point gives the same result
    xh = sol.schur_solve_host(b)
    assert rel(xh, xref) <= TOL[prec]
    sol.close()


@pytest.mark.parametrize("prec", PRECS)
def test_multi_rhs_chunks_and_zero(prec):
    dim, N, P, beta = 2, 24, 3, 1e-6
    n = (N - 1) ** 2
    ybs = inputs.smoothed_noise(dim, N, seed=3, nrhs=17)
    b = oracle.apply_M(dim, N, ybs)
    b[5] = 0.0  # a zero right-hand side gives x = 0
    xref = oracle.fd_schur_solve(dim, N, beta, b)
    sol = S.Solver(dim, N, beta, nsub=P, precision=prec)
    x = sol.schur_solve(gpu(b)).cpu().numpy()
    for r in range(17):
        if r == 5:
            assert np.abs(x[r]).max() == 0.0
        else:
            assert rel(x[r], xref[r]) <= TOL[prec], r
    # the same columns solved alone agree (columns are independent)
    x3 = sol.schur_solve(gpu(b[:3])).cpu().numpy()
    assert rel(x3, x[:3]) <= TOL[prec]
    # nrhs = 0 is a no-op
    e = torch.zeros((0, n), dtype=torch.float64, device=DEV)
    sol.schur_solve(e, torch.zeros_like(e))
    sol.close()


# 3D cases of the tensor-core formation: a single 8^3 subdomain (every face Dirichlet), two 8^3
# subdomains, and boxes of 6 x 4 x 8 elements (layers of 35 nodes, nine layers).
@pytest.mark.parametrize("nel,nsub", [((12, 8), (3, 2)), ((8, 8), (2, 1)), ((6, 6), (1, 1)), ((6, 8, 4), (3, 2, 2)),
                                      ((20, 20), (10, 10)), ((24, 16), (2, 2)), ((8, 8, 8), (1, 1, 1)),
                                      ((16, 8, 8), (2, 1, 1)), ((12, 8, 16), (2, 2, 2))])
@pytest.mark.parametrize("prec", PRECS)
def test_ragged_and_degenerate_partitions(nel, nsub, prec):
    """Anisotropic grids, no primal corners (nsub = 1 on an axis), a single subdomain (no
    multipliers), and 2-element subdomains (the smallest allowed)."""
    dim = len(nel)
    beta = 1e-3
    rng = np.random.default_rng(9)
    n = int(np.prod([e - 1 for e in nel]))
    b = rng.standard_normal(n)
    xref = oracle.fd_schur_solve(dim, list(nel), beta, b)
    sol = S.Solver(dim, list(nel), beta, nsub=list(nsub), precision=prec)
    x = sol.schur_solve(gpu(b)).cpu().numpy()
    assert rel(x, xref) <= TOL[prec], sol.last_stats
    sol.close()


def test_invalid_arguments_are_rejected():
    with pytest.raises(S.SchurError) as e:
        S.Solver(2, 30, 1e-4, nsub=4)  # 30 % 4 != 0
    assert e.value.code == S.SCHUR_EINVAL
    with pytest.raises(S.SchurError):
        S.Solver(2, 32, -1.0, nsub=4)
    with pytest.raises(S.SchurError):
        S.Solver(2, 32, 1e-4, nsub=32)  # one element per subdomain: below the 2-element minimum
    with pytest.raises(S.SchurError) as e:
        S.Solver(3, 16, 1e-4, nsub=2, precision=S.SCHUR_MIXED, tc_split=2)  # 0, 1 or 3 only
    assert e.value.code == S.SCHUR_EINVAL


@pytest.mark.parametrize("split", [1, 3])
def test_3d_tensor_core_split(split):
    """3D, 16^3 Q1 elements in 2^3 subdomains of 8^3: the local operators formed from one TF32
    product (tc_split = 1, TF32 rounding of the layer operands) or from the three-term split
    (FP32 accuracy); the FP64 refinement reaches the mixed-precision target either way."""
    dim, N, P, beta = 3, 16, 2, 1e-6
    yb = inputs.random_modes_3d(N, count=8, seed=2)
    b = oracle.apply_M(dim, N, yb)
    xref = oracle.fd_schur_solve(dim, N, beta, b)
    sol = S.Solver(dim, N, beta, nsub=P, precision=S.SCHUR_MIXED, tc_split=split)
    F, _, _ = local_operators(dim, N, P, beta, 0)
    got = sol.schur_debug_operator(0, 0)
    err = np.abs(got - F).max() / np.abs(F).max()
    # three products keep FP32 accuracy; one TF32 product has 10-bit operands
    assert err <= (2e-5 if split == 3 else 2e-2), err
    x = sol.schur_solve(gpu(b)).cpu().numpy()
    print("split", split, "F err", err, sol.last_stats)
    assert rel(x, xref) <= TOL[S.SCHUR_MIXED], sol.last_stats
    sol.close()


@pytest.mark.parametrize("beta", [1e-2, 1e-4, 1e-6, 1e-8])
@pytest.mark.parametrize("prec", PRECS)
def test_large_2d_beta_sweep(beta, prec):
    """1024 x 1024 Q1 elements, 64 x 64 subdomains of 16 x 16, smoothed-noise target: the
    workload the benchmark times, compared entry by entry with the fast-diagonalisation oracle."""
    dim, N, P = 2, 1024, 64
    yb = inputs.smoothed_noise(dim, N, seed=1)
    b = oracle.apply_M(dim, N, yb)
    xref = oracle.fd_schur_solve(dim, N, beta, b)
    sol = S.Solver(dim, N, beta, nsub=P, precision=prec)
    x = sol.schur_solve(gpu(b)).cpu().numpy()
    print("beta", beta, "prec", prec, sol.last_stats, "relerr", rel(x, xref))
    assert rel(x, xref) <= TOL[prec], sol.last_stats
    sol.close()
