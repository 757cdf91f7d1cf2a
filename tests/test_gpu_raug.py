"""GPU parity of the augmented coarse problem (Sec. 5: FETI-DP augmented by the edge-based
translational mode, the paper's RAUG; for the scalar problem one zero-average-jump constraint per
pair of face-adjacent subdomains).

The augmentation changes the dual operator and the coarse problem but not the solution: the
augmented GPU solve must reproduce the oracle (O1/O2) in both precisions.  Its internal pieces are
compared with the dense definitional reference (tests/dense_ref.py): the coupling columns
[F_rc, F Q_s] of a subdomain and the inverse of the assembled augmented coarse matrix
[[K_cc, -X^T], [-X, -Y]].  The augmentation must not increase the Krylov iteration count where the
corner-only coarse space is weakest (large beta)."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle
from paper_1312_5653_gb300 import inputs
from paper_1312_5653_gb300 import schur as S

import dense_ref as D

TOL = {S.SCHUR_FP64: 1e-10, S.SCHUR_MIXED: 1e-8}


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def lib_face_index(dim, P):
    """The library's face numbering: faces normal to axis 0, then 1 (then 2), each lexicographic
    over the lower subdomain's coordinates (axis a ranging over P - 1 values)."""
    idx, k = {}, 0
    for a in range(dim):
        ext = [P - 1 if b == a else P for b in range(dim)]
        for flat in range(int(np.prod(ext))):
            S_ = [(flat // int(np.prod(ext[:b]))) % ext[b] for b in range(dim)]
            lo = sum(S_[b] * P ** b for b in range(dim))
            idx[(lo, lo + P ** a)] = k
            k += 1
    return idx


@pytest.mark.parametrize("prec", [S.SCHUR_FP64, S.SCHUR_MIXED])
@pytest.mark.parametrize("dim,N,P", [(2, 64, 4), (2, 128, 8), (3, 16, 2), (3, 32, 4)])
@pytest.mark.parametrize("beta", [1e-2, 1e-4, 1e-6, 1e-8])
def test_augmented_solve_matches_oracle(prec, dim, N, P, beta):
    yb = inputs.smoothed_noise(dim, N, seed=7, nrhs=2) if dim == 2 else inputs.random_modes_3d(N, count=8, seed=7, nrhs=2)
    b = oracle.apply_M(dim, N, yb)
    ref = oracle.fd_schur_solve(dim, N, beta, b)
    sol = S.Solver(dim, N, beta, nsub=P, precision=prec, tol=1e-12, augment=1)
    x = sol.schur_solve(torch.from_numpy(b).cuda()).cpu().numpy()
    info = sol.info()
    sol.close()
    faces = dim * (P - 1) * P ** (dim - 1)
    assert info["n_coarse"] == (P - 1) ** dim + faces
    assert rel(x, ref) <= TOL[prec], rel(x, ref)


def test_augmented_coarse_pieces_match_dense_reference():
    """2D 12 x 12 elements, 3 x 3 subdomains: the coupling columns [F_rc, F Q_s] of the middle
    subdomain and the inverse of the augmented coarse matrix against the dense definitions."""
    dim, N, P, beta = 2, 12, 3, 1e-3
    sol = S.Solver(dim, N, beta, nsub=P, augment=1)
    info = sol.info()
    nD = info["n_delta"]
    sd = 4  # the middle subdomain: all four faces have neighbours
    Phi = np.zeros((nD, 8, 2))
    rc = S.load().schur_debug_operator(sol.ctx, 5, sd, Phi.ctypes.data_as(ctypes.c_void_p), Phi.size // 2)
    assert rc == S.SCHUR_OK, S.last_error()
    Phi = Phi[..., 0] + 1j * Phi[..., 1]
    Kinv = sol.schur_debug_operator(4)
    sol.close()
    F, Frc, _ = D.local_operators(dim, N, P, beta, sd)
    # Q_s: slot j on local face f = 2a + side, sign +1 on the high side
    s = N // P
    loc = D._local_nodes(dim, s)
    slots = S.schur_partition_export(dim, N, P, 1)
    Qs = np.zeros((nD, 2 * dim))
    for j, node in enumerate(slots):
        l = loc[int(node)]
        for a in range(dim):
            if l[a] == 0:
                Qs[j, 2 * a] = -1.0
            if l[a] == s:
                Qs[j, 2 * a + 1] = 1.0
    assert rel(Phi[:, :4], Frc) < 1e-11
    assert rel(Phi[:, 4:], F @ Qs) < 1e-11
    # the dense augmented coarse matrix, faces in the library's order
    cap = {}
    orig = np.block

    def grab(x):
        r = orig(x)
        cap["K"] = r
        return r

    n = (N - 1) ** dim
    np.block = grab
    try:
        D.dense_feti_dp(dim, N, P, beta, np.ones(n), aug=True)
    finally:
        np.block = orig
    Kd = cap["K"]
    nco = (P - 1) ** dim
    info_p = S.schur_partition(dim, N, P)
    lam = S.schur_partition_export(dim, N, P, 0).reshape(-1, 2)
    _, pairs = D.face_pairs(dim, P, lam, info_p["n_delta"])
    order = lib_face_index(dim, P)
    perm = np.arange(Kd.shape[0])
    for k, pr in enumerate(pairs):
        perm[nco + order[pr]] = nco + k
    Kd = Kd[np.ix_(perm, perm)]
    assert Kinv.shape == Kd.shape
    assert rel(Kinv, np.linalg.inv(Kd)) < 1e-10


@pytest.mark.parametrize("beta", [1e-2, 1e-4])
def test_augmentation_reduces_iterations(beta):
    """2D 256 x 256 elements, 8 x 8 subdomains of 32 x 32 (H/h = 32): one FP64 FETI-DP solve to
    1e-10 with and without the face-average augmentation."""
    dim, N, P = 2, 256, 8
    b = oracle.apply_M(dim, N, inputs.smoothed_noise(dim, N, seed=3))
    its = {}
    for aug in (0, 1):
        sol = S.Solver(dim, N, beta, nsub=P, tol=1e-3, inner_tol=1e-10, max_refine=1, augment=aug)
        sol.schur_solve(torch.from_numpy(b).cuda())
        its[aug] = sol.last_stats["iters_first"]
        sol.close()
    assert its[1] < its[0], its


def test_augmented_coarse_size_limit():
    with pytest.raises(S.SchurError):
        S.Solver(2, 256, 1e-4, nsub=64, augment=1)  # 63^2 + 2 * 63 * 64 > 4096 coarse unknowns
    with pytest.raises(S.SchurError):
        S.Solver(2, 64, 1e-4, nsub=4, augment=2)


@pytest.mark.parametrize("prec", [S.SCHUR_FP64, S.SCHUR_MIXED])
def test_augmented_1024_all_betas(prec):
    """2D 1024^2 Q1 elements in 16 x 16 subdomains of 64^2 (H/h = 64, the paper's ratio; 705 coarse
    unknowns with the augmentation): all four betas of the 1024^2 workload against the oracle."""
    N, P = 1024, 16
    b = oracle.apply_M(2, N, inputs.smoothed_noise(2, N, seed=1))
    bd = torch.from_numpy(b).cuda()
    oracle.set_threads(0)
    for beta in (1e-2, 1e-4, 1e-6, 1e-8):
        sol = S.Solver(2, N, beta, nsub=P, precision=prec, tol=1e-12, augment=1)
        x = sol.schur_solve(bd).cpu().numpy()
        sol.close()
        ref = oracle.fd_schur_solve(2, N, beta, b)
        assert rel(x, ref) <= TOL[prec], (beta, rel(x, ref))


def test_augmented_128cube_mixed():
    """3D 128^3 Q1 elements in 8^3 subdomains of 16^3 (1687 coarse unknowns with the augmentation),
    mixed precision refined to 1e-10, against the oracle."""
    N, P, beta = 128, 8, 1e-6
    b = oracle.apply_M(3, N, inputs.random_modes_3d(N, count=8, seed=2))
    sol = S.Solver(3, N, beta, nsub=P, precision=S.SCHUR_MIXED, tol=1e-10, augment=1)
    x = sol.schur_solve(torch.from_numpy(b).cuda()).cpu().numpy()
    sol.close()
    ref = oracle.fd_schur_solve(3, N, beta, b)
    assert rel(x, ref) <= 1e-8, rel(x, ref)
