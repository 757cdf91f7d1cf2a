"""Host logic of the FETI-DP partition (no GPU): counts, jump-operator structure, and a dense
definitional FETI-DP solve (Sec. 5) built on the library's exported maps, checked against the
oracle's complex solve.  Also checks that the C-ABI library loads and exports every symbol that
include/schur.h declares."""
import os
import re

import numpy as np
import pytest

import oracle
from paper_1312_5653_gb300 import schur as S

from dense_ref import _local_nodes, dense_feti_dp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_library_exports_every_declared_symbol():
    hdr = open(os.path.join(ROOT, "include", "schur.h")).read()
    declared = sorted(set(re.findall(r"\b(schur_[a-z_]+)\s*\(", hdr)))
    lib = S.load()
    missing = [d for d in declared if not hasattr(lib, d)]
    assert not missing, missing
    assert set(declared) <= set(S.EXPORTS) | {"schur_ndof"}


def closed_form_counts(dim, N, P):
    s = N // P
    n = (N - 1) ** dim
    if dim == 2:
        nlam = 2 * (P - 1) * (N - 1 - (P - 1))
        nD = 4 * (s - 1)
    else:
        nlam = 3 * (P - 1) * P * P * (s - 1) ** 2 + 6 * 3 * (P - 1) ** 2 * P * (s - 1)
        nD = 6 * (s - 1) ** 2 + 12 * (s - 1)
    return dict(n=n, n_lambda=nlam, n_coarse=(P - 1) ** dim, n_delta=nD, n_local=(s + 1) ** dim, n_sub=P ** dim)


@pytest.mark.parametrize("dim,N,P", [(2, 32, 4), (2, 1024, 64), (2, 512, 32), (3, 128, 16), (3, 12, 3)])
def test_partition_counts(dim, N, P):
    info = S.schur_partition(dim, N, P)
    for k, v in closed_form_counts(dim, N, P).items():
        assert info[k] == v, (k, info[k], v)
    shared = S.schur_partition(dim, N, P, S.SCHUR_LOCAL_SHARED)
    assert shared["n_classes"] == min(3, P) ** dim


@pytest.mark.parametrize("dim,N,P", [(2, 8, 2), (2, 12, 3), (3, 6, 3), (3, 4, 2)])
def test_jump_operator_structure(dim, N, P):
    s = N // P
    lam = S.schur_partition_export(dim, N, P, 0).reshape(-1, 2)
    slots = S.schur_partition_export(dim, N, P, 1)
    info = S.schur_partition(dim, N, P)
    nD = info["n_delta"]
    loc = _local_nodes(dim, s)
    seen = set()
    mult = {}
    for a, b in lam:
        sa, ja = divmod(int(a), nD)
        sb, jb = divmod(int(b), nD)
        assert sa < sb
        Sa = [(sa // P ** t) % P for t in range(dim)]
        Sb = [(sb // P ** t) % P for t in range(dim)]
        Ga = tuple(Sa[t] * s + loc[slots[ja]][t] for t in range(dim))
        Gb = tuple(Sb[t] * s + loc[slots[jb]][t] for t in range(dim))
        assert Ga == Gb and all(0 < g < N for g in Ga)
        assert (sa, sb, Ga) not in seen
        seen.add((sa, sb, Ga))
        mult.setdefault(Ga, set()).update([sa, sb])
    for G, subs in mult.items():
        m = len(subs)
        on = sum(1 for g in G if g % s == 0)
        assert m == 2 ** on
        assert sum(1 for k in seen if k[2] == G) == m * (m - 1) // 2


@pytest.mark.parametrize("dim,N,P,beta", [(2, 8, 2, 1e-4), (2, 12, 3, 1e-2), (2, 12, 4, 1e-8), (3, 6, 3, 1e-6),
                                          (3, 4, 2, 1e-2)])
def test_dense_feti_dp_reproduces_oracle(dim, N, P, beta):
    rng = np.random.default_rng(7)
    n = (N - 1) ** dim
    b = rng.standard_normal(n)
    z, F, d, lamv, _ = dense_feti_dp(dim, N, P, beta, b)
    zref = oracle.fd_complex_solve(dim, N, 1.0 / np.sqrt(beta), b)
    assert np.linalg.norm(z - zref) / np.linalg.norm(zref) < 1e-10
    # the dual system is consistent (redundant multipliers in 3D make F singular)
    assert np.linalg.norm(F @ lamv - d) <= 1e-10 * np.linalg.norm(d)
    # complex symmetric, not Hermitian
    assert np.abs(F - F.T).max() < 1e-10 * np.abs(F).max()


def test_setup_rejects_bad_arguments_before_touching_the_device():
    """Invalid meshes, beta or options return SCHUR_EINVAL without any CUDA call (NULL stream)."""
    import ctypes
    lib = S.load()

    def setup(dim, nel, beta, **kw):
        ctx = ctypes.c_void_p()
        rc = lib.schur_setup(ctypes.byref(S.make_mesh(dim, nel)), beta, ctypes.byref(S.default_opts(**kw)), None,
                             ctypes.byref(ctx))
        assert not ctx.value
        return rc

    assert setup(2, 30, 1e-4, nsub=4) == S.SCHUR_EINVAL        # nel not a multiple of nsub
    assert setup(2, 32, 0.0, nsub=4) == S.SCHUR_EINVAL         # beta must be positive
    assert setup(2, 32, float("nan"), nsub=4) == S.SCHUR_EINVAL
    assert setup(2, 32, 1e-4, nsub=32) == S.SCHUR_EINVAL       # one element per subdomain
    bad = S.make_mesh(3, 32)
    bad.dim = 4
    ctx = ctypes.c_void_p()
    assert lib.schur_setup(ctypes.byref(bad), 1e-4, ctypes.byref(S.default_opts()), None,
                           ctypes.byref(ctx)) == S.SCHUR_EINVAL
    assert setup(2, 32, 1e-4, nsub=4, precision=7) == S.SCHUR_EINVAL
    assert setup(2, 32, 1e-4, nsub=4, max_iter=0) == S.SCHUR_EINVAL
    assert setup(2, 32, 1e-4, nsub=4, max_iter=512) == S.SCHUR_EINVAL
    assert S.last_error()
    assert S.schur_ndof(3, [3, 4, 5]) == 2 * 3 * 4
