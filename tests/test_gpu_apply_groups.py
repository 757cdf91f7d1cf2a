"""GPU parity of the local apply paths for one right-hand side and for groups of subdomains.

With SCHUR_LOCAL_SHARED every subdomain of one boundary type uses the same stored F, S and Frc;
the dual operator then applies each staged operator to a group of up to eight subdomains at once.
Per subdomain (the default) a single right-hand side takes the packed-operator kernel that walks
the column and the row of the upper triangle.  Both must give the oracle's x = S^{-1} b
(FP64 1e-10, mixed 1e-8), with and without the augmented coarse problem (Frc with corner and face
columns), for one and two right-hand sides, on 16^2 and 8^2 subdomains (60 and 28 interface nodes).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle
from paper_1312_5653_gb300 import inputs
from paper_1312_5653_gb300 import schur as S

DEV = "cuda:0"
TOL = {S.SCHUR_FP64: 1e-10, S.SCHUR_MIXED: 1e-8}


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


def gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(DEV)


@pytest.mark.parametrize("N,P", [(128, 8), (96, 12)])
@pytest.mark.parametrize("prec", [S.SCHUR_FP64, S.SCHUR_MIXED])
@pytest.mark.parametrize("augment", [0, 1])
@pytest.mark.parametrize("nrhs", [1, 2])
def test_shared_groups_and_single_rhs_match_oracle(N, P, prec, augment, nrhs):
    dim, beta = 2, 1e-4
    yb = inputs.smoothed_noise(dim, N, seed=11, nrhs=nrhs)
    b = oracle.apply_M(dim, N, yb)
    xref = oracle.fd_schur_solve(dim, N, beta, b)
    xs = {}
    for mode in (S.SCHUR_LOCAL_PER_SUBDOMAIN, S.SCHUR_LOCAL_SHARED):
        sol = S.Solver(dim, N, beta, nsub=P, precision=prec, local_mode=mode, augment=augment)
        x = sol.schur_solve(gpu(b)).cpu().numpy()
        assert rel(x, xref) <= TOL[prec], (mode, sol.last_stats)
        xs[mode] = x
        sol.close()
    # both storage modes solve the same problem
    assert rel(xs[S.SCHUR_LOCAL_SHARED], xs[S.SCHUR_LOCAL_PER_SUBDOMAIN]) <= 2 * TOL[prec]
