"""GPU pin of the batched block LDL^T factorisation: ||L D L^T - A|| / ||A|| on the local matrix.

The library factors each subdomain's remainder matrix on the full local grid of (s+1)^d nodes,
layer by layer along the last axis, with the removed nodes (the 2^d subdomain vertices, which are
primal, and the nodes on global Dirichlet faces) as identity rows and columns.  It stores the layer
pivot inverses D_K^{-1}.  With the layer couplings A_{K,K-1} of A, the block factor is
L_{K,K-1} = A_{K,K-1} D_{K-1}^{-1}, so L D L^T has the off-diagonal blocks of A and the diagonal
blocks D_K + A_{K,K-1} D_{K-1}^{-1} A_{K-1,K}.  The test rebuilds A from the oracle's Q1 element
matrices and the subdomain's position alone (no library maps), takes the exported D_K^{-1}, and
checks the reconstruction for a corner, an edge and an interior subdomain.  Tolerances: FP64
1e-12, FP32 (mixed form) 2e-5, relative in the Frobenius norm.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1312_5653_gb300 import schur as S

from dense_ref import local_neumann

TOL = {S.SCHUR_FP64: 1e-12, S.SCHUR_MIXED: 2e-5}


def padded_local_matrix(dim, N, P, beta, sd):
    """A = K + i gamma M of subdomain sd with its removed nodes replaced by identity rows/columns."""
    s = N // P
    A, loc = local_neumann(dim, N, P, beta)
    pos = [(sd // P ** a) % P for a in range(dim)]
    removed = []
    for i, c in enumerate(loc):
        vertex = all(c[a] in (0, s) for a in range(dim))
        dirichlet = any((pos[a] == 0 and c[a] == 0) or (pos[a] == P - 1 and c[a] == s) for a in range(dim))
        if vertex or dirichlet:
            removed.append(i)
    A = A.copy()
    A[removed, :] = 0.0
    A[:, removed] = 0.0
    A[removed, removed] = 1.0
    return A


def reconstruct(A, Dinv):
    L, b = Dinv.shape[0], Dinv.shape[1]
    blk = lambda K, J: A[K * b:(K + 1) * b, J * b:(J + 1) * b]
    R = np.zeros_like(A)
    for K in range(L):
        D = np.linalg.inv(Dinv[K])
        if K > 0:
            D = D + blk(K, K - 1) @ Dinv[K - 1] @ blk(K - 1, K)
            R[K * b:(K + 1) * b, (K - 1) * b:K * b] = blk(K, K - 1)
            R[(K - 1) * b:K * b, K * b:(K + 1) * b] = blk(K - 1, K)
        R[K * b:(K + 1) * b, K * b:(K + 1) * b] = D
    return R


@pytest.mark.parametrize("dim,N,P,beta", [(2, 32, 4, 1e-4), (2, 48, 3, 1e-8), (2, 64, 4, 1e-2), (3, 12, 3, 1e-6),
                                          (3, 16, 2, 1e-4)])
@pytest.mark.parametrize("prec", [S.SCHUR_FP64, S.SCHUR_MIXED])
def test_layer_factor_reconstructs_local_matrix(dim, N, P, beta, prec):
    sol = S.Solver(dim, N, beta, nsub=P, precision=prec)
    nsd = P ** dim
    for sd in sorted({0, 1, nsd // 2, nsd - 1}):
        Dinv = sol.schur_debug_operator(6, sd)
        A = padded_local_matrix(dim, N, P, beta, sd)
        assert Dinv.shape[0] * Dinv.shape[1] == A.shape[0]
        err = np.linalg.norm(reconstruct(A, Dinv) - A) / np.linalg.norm(A)
        assert err <= TOL[prec], (sd, err)
    sol.close()
