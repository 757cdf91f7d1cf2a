"""The allocation-free entry point schur_apply_S_static against schur_apply_S and the oracle.

schur_apply_S_static serves callers that cannot allocate device memory (no schur_ctx, work
vectors in a fixed device array inside the library).  It must give the same y = S x as the
context-based schur_apply_S, call after call, although every call reuses the same array; both
are also compared with the oracle's S x (Sec. 3.1, S = K M^-1 K + M / beta), computed by a banded
Cholesky factorisation of M (O1) and by sine-basis diagonalisation (O2)."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle
from paper_1312_5653_gb300 import inputs
from paper_1312_5653_gb300 import schur as S


def _static_apply(lib, mesh, beta, x, y):
    nrhs, ld = (1, x.numel()) if x.dim() == 1 else x.shape
    return lib.schur_apply_S_static(ctypes.byref(mesh), beta, ctypes.c_void_p(x.data_ptr()),
                                    ctypes.c_void_p(y.data_ptr()), nrhs, ld,
                                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("dim,N,beta", [(2, 64, 1e-4), (2, 64, 1e-2), (2, 64, 1e-8), (3, 16, 1e-6)])
def test_static_apply_matches_context_apply_twice(dim, N, beta):
    lib = S.load()
    mesh = S.make_mesh(dim, N)
    n = (N - 1) ** dim
    sol = S.Solver(dim, N, beta, nsub=4)
    for call in range(2):  # two calls in a row: the shared array is reused
        xh = inputs.smoothed_noise(dim, N, seed=20 + call, nrhs=2)
        x = torch.from_numpy(xh).cuda()
        ref = sol.schur_apply_S(x)
        y = torch.full_like(x, float("nan"))
        assert _static_apply(lib, mesh, beta, x, y) == S.SCHUR_OK, S.last_error()
        torch.cuda.synchronize()
        err = (torch.linalg.norm(y - ref) / torch.linalg.norm(ref)).item()
        assert err <= 1e-12, (call, err)
        yh = y.cpu().numpy()
        for ref_o in (oracle.schur_apply(dim, N, beta, xh), oracle.fd_schur_apply(dim, N, beta, xh)):
            e_o = np.linalg.norm(yh - ref_o) / np.linalg.norm(ref_o)
            assert e_o <= 1e-12, (call, e_o)
    sol.close()


def test_static_apply_leading_dimension_and_padding():
    """ld > n with three columns: only the first n entries of each column are read and written."""
    lib = S.load()
    dim, N, beta = 3, (12, 8, 16), 1e-8
    mesh = S.make_mesh(dim, N)
    n = oracle.ndof(dim, N)
    ld = n + 3
    xh = np.full((3, ld), np.nan)
    xh[:, :n] = np.random.default_rng(8).standard_normal((3, n))
    x = torch.from_numpy(xh).cuda()
    y = torch.full_like(x, 5.0)
    assert _static_apply(lib, mesh, beta, x, y) == S.SCHUR_OK, S.last_error()
    torch.cuda.synchronize()
    yh = y.cpu().numpy()
    assert np.all(yh[:, n:] == 5.0)
    ref = oracle.fd_schur_apply(dim, N, beta, xh[:, :n])
    assert np.linalg.norm(yh[:, :n] - ref) / np.linalg.norm(ref) <= 1e-12


def test_static_apply_rejects_meshes_beyond_its_array():
    lib = S.load()
    big = S.make_mesh(2, 1026)  # 1025^2 > 2^20 interior nodes
    x = torch.zeros(1025 * 1025, dtype=torch.float64, device="cuda")
    assert _static_apply(lib, big, 1e-4, x, x.clone()) == S.SCHUR_EINVAL
    assert "2^20" in S.last_error()
    assert _static_apply(lib, S.make_mesh(2, 64), -1.0, x[:63 * 63], x[:63 * 63].clone()) == S.SCHUR_EINVAL
    # per-axis counts whose product overflows a 64-bit integer are refused before any multiply
    huge = S.make_mesh(3, [1 << 30, 1 << 30, 1 << 30])
    assert _static_apply(lib, huge, 1e-4, x, x.clone()) == S.SCHUR_EINVAL
    # y overlapping x is refused (y = K w is written before M x / beta is added)
    assert _static_apply(lib, S.make_mesh(2, 64), 1e-4, x[:63 * 63], x[10:10 + 63 * 63]) == S.SCHUR_EINVAL
