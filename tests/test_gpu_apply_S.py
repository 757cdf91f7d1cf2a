"""GPU parity of the FP64 Schur complement apply y = S x (Sec. 3.1: S = K M^-1 K + M / beta).

schur_apply_S runs K and M as matrix-free Q1 stencils and M^-1 as a fixed-degree Chebyshev
iteration; the oracle computes the same product two independent ways: O1 by a banded Cholesky
factorisation of the element-loop-assembled M (``oracle.schur_apply``) and O2 by the sine-basis
diagonalisation of K and M (``oracle.fd_schur_apply``).  Both oracle functions are pinned in
tests/test_oracle.py (dense definition, sine eigenpairs).  The two oracle routes agree to ~1e-13,
the Chebyshev degree is chosen for 1e-15, so 1e-12 relative is the bar here.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle
from paper_1312_5653_gb300 import schur as S

TOL = 1e-12


def _inputs(n, nrhs, ld, seed):
    """nrhs seeded N(0,1) columns of length n in an (nrhs, ld) array; the tail [n, ld) is NaN so a
    read beyond n shows up in the result."""
    rng = np.random.default_rng(seed)
    x = np.full((nrhs, ld), np.nan)
    x[:, :n] = rng.standard_normal((nrhs, n))
    return x


@pytest.mark.parametrize("dim,nel,nsub", [(2, 64, 4), (2, (48, 32), (3, 2)), (3, 16, 2), (3, (12, 8, 16), (3, 2, 4))])
@pytest.mark.parametrize("beta", [1e-2, 1e-8])
@pytest.mark.parametrize("nrhs,pad", [(1, 0), (3, 5)])
def test_apply_S_matches_oracle(dim, nel, nsub, beta, nrhs, pad):
    n = oracle.ndof(dim, nel)
    ld = n + pad
    xh = _inputs(n, nrhs, ld, seed=31 + nrhs)
    x = torch.from_numpy(xh).cuda()
    y = torch.full_like(x, 7.0)  # entries beyond n must stay untouched
    sol = S.Solver(dim, nel, beta, nsub=nsub)
    sol.schur_apply_S(x, y)
    torch.cuda.synchronize()
    sol.close()
    yh = y.cpu().numpy()
    assert np.all(yh[:, n:] == 7.0)
    ref1 = oracle.schur_apply(dim, nel, beta, xh[:, :n])
    ref2 = oracle.fd_schur_apply(dim, nel, beta, xh[:, :n])
    for c in range(nrhs):
        e1 = np.linalg.norm(yh[c, :n] - ref1[c]) / np.linalg.norm(ref1[c])
        e2 = np.linalg.norm(yh[c, :n] - ref2[c]) / np.linalg.norm(ref2[c])
        assert e1 <= TOL and e2 <= TOL, (c, e1, e2)


def test_apply_S_inverts_schur_solve():
    """S (S^-1 b) = b: the apply and the FETI-DP solve agree with each other as well as with the oracle."""
    dim, N, beta = 2, 64, 1e-4
    n = oracle.ndof(dim, N)
    b = torch.from_numpy(_inputs(n, 2, n, seed=5)).cuda()
    sol = S.Solver(dim, N, beta, nsub=4, tol=1e-13)
    x = sol.schur_solve(b)
    y = sol.schur_apply_S(x)
    torch.cuda.synchronize()
    sol.close()
    err = (torch.linalg.norm(y - b) / torch.linalg.norm(b)).item()
    # x carries the solve's error; S amplifies its high-frequency part by up to ~||conj(A) M^-1|| / gamma
    # (about 1e3 at 64^2, beta = 1e-4), so a 1e-13 complex residual allows ~1e-10 here
    assert err <= 1e-9, err
