"""The allocation-free entry point schur_apply_S_static against schur_apply_S.

schur_apply_S_static serves callers that cannot allocate device memory (no schur_ctx, work
vectors in a fixed device array inside the library).  It must give the same y = S x as the
context-based schur_apply_S, call after call, although every call reuses the same array."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1312_5653_gb300 import inputs
from paper_1312_5653_gb300 import schur as S


def _static_apply(lib, mesh, beta, x, y):
    nrhs, ld = (1, x.numel()) if x.dim() == 1 else x.shape
    return lib.schur_apply_S_static(ctypes.byref(mesh), beta, ctypes.c_void_p(x.data_ptr()),
                                    ctypes.c_void_p(y.data_ptr()), nrhs, ld,
                                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("dim,N,beta", [(2, 64, 1e-4), (3, 16, 1e-6)])
def test_static_apply_matches_context_apply_twice(dim, N, beta):
    lib = S.load()
    mesh = S.make_mesh(dim, N)
    n = (N - 1) ** dim
    sol = S.Solver(dim, N, beta, nsub=4)
    for call in range(2):  # two calls in a row: the shared array is reused
        x = torch.from_numpy(inputs.smoothed_noise(dim, N, seed=20 + call, nrhs=2)).cuda()
        ref = sol.schur_apply_S(x)
        y = torch.full_like(x, float("nan"))
        assert _static_apply(lib, mesh, beta, x, y) == S.SCHUR_OK, S.last_error()
        torch.cuda.synchronize()
        err = (torch.linalg.norm(y - ref) / torch.linalg.norm(ref)).item()
        assert err <= 1e-12, (call, err)
    sol.close()


def test_static_apply_rejects_meshes_beyond_its_array():
    lib = S.load()
    big = S.make_mesh(2, 1026)  # 1025^2 > 2^20 interior nodes
    x = torch.zeros(1025 * 1025, dtype=torch.float64, device="cuda")
    assert _static_apply(lib, big, 1e-4, x, x.clone()) == S.SCHUR_EINVAL
    assert _static_apply(lib, S.make_mesh(2, 64), -1.0, x[:63 * 63], x[:63 * 63].clone()) == S.SCHUR_EINVAL
