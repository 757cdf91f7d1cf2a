"""Reference oracle (FP64, CPU) for the factored Schur complement solve.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The product library
(``paper_1312_5653_gb300``) never imports, links or runs it, and the two share no code.

The arithmetic lives in ``oracle.c`` (plain single-threaded C).  This module only marshals numpy
arrays through ctypes.  Every function works on real FP64 vectors over the n interior nodes of a
uniform Q1 grid on the unit box (lexicographic order, axis 0 fastest), column-major for several
right-hand sides.  ``beta`` is the paper's regularisation phi and gamma = 1/sqrt(beta).

Paper passages (arXiv 1312.5653): Sec. 2 (discretisation and the KKT system), Sec. 3.1 (the
negative Schur complement S = K M^-1 K + M/beta and the recovery of y, u), Sec. 3.2 (the
block-diagonal preconditioner P_mgw and the Pearson-Wathen approximation S_p), Sec. 4 (the
factorisation S = (K + M/(i sqrt beta)) M^-1 (K - M/(i sqrt beta))).
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force=False):
    """Compile oracle.c into liboracle.so next to it (plain gcc, no architecture flags)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "oracle.h"))):
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        I = ctypes.c_int
        D = ctypes.c_double
        lib.or_ndof.restype = ctypes.c_long
        lib.or_ndof.argtypes = [I, P]
        lib.or_bandwidth.argtypes = [I, P]
        lib.or_element.argtypes = [I, P, P, P]
        lib.or_assemble.argtypes = [I, P, P, P]
        lib.or_apply_KM.argtypes = [I, P, I, P, P, P]
        lib.or_kkt_solve.argtypes = [I, P, D, I, P, P, P, P, P, P]
        lib.or_schur_solve_kkt.argtypes = [I, P, D, I, P, P]
        lib.or_schur_apply.argtypes = [I, P, D, I, P, P]
        lib.or_fd_schur_solve.argtypes = [I, P, D, I, P, P]
        lib.or_fd_schur_apply.argtypes = [I, P, D, I, P, P]
        lib.or_fd_complex_solve.argtypes = [I, P, D, I, I, P, P, P, P]
        lib.or_fd_kkt_solve.argtypes = [I, P, D, I, P, P, P, P, P, P]
        lib.or_fd_eigs.argtypes = [I, P, P, P]
        _lib = lib
    return _lib


def _nel(dim, nel):
    if np.isscalar(nel):
        nel = [int(nel)] * dim
    a = np.zeros(3, dtype=np.int32)
    a[:dim] = nel
    return a


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _vec(x, n):
    """Return (C-contiguous FP64 array of shape (nrhs, n), squeeze flag)."""
    x = np.asarray(x, dtype=np.float64)
    squeeze = x.ndim == 1
    x = np.ascontiguousarray(x.reshape(-1, n))
    return x, squeeze


def _check(rc, what):
    if rc != 0:
        raise RuntimeError("oracle %s failed with code %d" % (what, rc))


def ndof(dim, nel):
    return int(_load().or_ndof(dim, _p(_nel(dim, nel))))


def element(dim, h):
    """Q1 element stiffness and mass (2-point Gauss), element nodes lexicographic."""
    nn = 1 << dim
    hh = np.ones(3)
    hh[:dim] = h
    Ke = np.zeros((nn, nn))
    Me = np.zeros((nn, nn))
    _check(_load().or_element(dim, _p(hh), _p(Ke), _p(Me)), "element")
    return Ke, Me


def assemble_dense(dim, nel):
    """Dense K, M (only for small meshes) from the oracle's banded element-loop assembly."""
    lib = _load()
    ne = _nel(dim, nel)
    n = ndof(dim, nel)
    w = lib.or_bandwidth(dim, _p(ne))
    Kb = np.zeros((n, w + 1))
    Mb = np.zeros((n, w + 1))
    _check(lib.or_assemble(dim, _p(ne), _p(Kb), _p(Mb)), "assemble")
    K = np.zeros((n, n))
    M = np.zeros((n, n))
    for i in range(n):
        for k in range(min(w, i) + 1):
            K[i, i - k] = K[i - k, i] = Kb[i, k]
            M[i, i - k] = M[i - k, i] = Mb[i, k]
    return K, M


def apply_KM(dim, nel, x):
    """(K x, M x)."""
    n = ndof(dim, nel)
    xx, sq = _vec(x, n)
    Kx = np.zeros_like(xx)
    Mx = np.zeros_like(xx)
    _check(_load().or_apply_KM(dim, _p(_nel(dim, nel)), xx.shape[0], _p(xx), _p(Kx), _p(Mx)), "apply_KM")
    return (Kx[0], Mx[0]) if sq else (Kx, Mx)


def apply_M(dim, nel, x):
    n = ndof(dim, nel)
    xx, sq = _vec(x, n)
    Mx = np.zeros_like(xx)
    _check(_load().or_apply_KM(dim, _p(_nel(dim, nel)), xx.shape[0], _p(xx), None, _p(Mx)), "apply_M")
    return Mx[0] if sq else Mx


def kkt_solve(dim, nel, beta, ry=None, ru=None, rl=None):
    """O1: solve the KKT system of Sec. 2 for (y, u, lambda)."""
    n = ndof(dim, nel)
    given = [r for r in (ry, ru, rl) if r is not None]
    nrhs = _vec(given[0], n)[0].shape[0] if given else 1
    sq = np.asarray(given[0]).ndim == 1 if given else True
    arrs = [None if r is None else _vec(r, n)[0] for r in (ry, ru, rl)]
    y = np.zeros((nrhs, n)); u = np.zeros((nrhs, n)); l = np.zeros((nrhs, n))
    _check(_load().or_kkt_solve(dim, _p(_nel(dim, nel)), float(beta), nrhs, _p(arrs[0]), _p(arrs[1]),
                                _p(arrs[2]), _p(y), _p(u), _p(l)), "kkt_solve")
    return (y[0], u[0], l[0]) if sq else (y, u, l)


def schur_solve_kkt(dim, nel, beta, b):
    """O1: x = S^{-1} b (the multiplier block of the KKT solve with right-hand side (0, 0, -b))."""
    n = ndof(dim, nel)
    bb, sq = _vec(b, n)
    x = np.zeros_like(bb)
    _check(_load().or_schur_solve_kkt(dim, _p(_nel(dim, nel)), float(beta), bb.shape[0], _p(bb), _p(x)),
           "schur_solve_kkt")
    return x[0] if sq else x


def schur_apply(dim, nel, beta, x):
    """y = S x = K M^{-1} K x + M x / beta (banded Cholesky of M)."""
    n = ndof(dim, nel)
    xx, sq = _vec(x, n)
    y = np.zeros_like(xx)
    _check(_load().or_schur_apply(dim, _p(_nel(dim, nel)), float(beta), xx.shape[0], _p(xx), _p(y)),
           "schur_apply")
    return y[0] if sq else y


def fd_schur_solve(dim, nel, beta, b):
    """O2: x = S^{-1} b by fast diagonalisation."""
    n = ndof(dim, nel)
    bb, sq = _vec(b, n)
    x = np.zeros_like(bb)
    _check(_load().or_fd_schur_solve(dim, _p(_nel(dim, nel)), float(beta), bb.shape[0], _p(bb), _p(x)),
           "fd_schur_solve")
    return x[0] if sq else x


def fd_schur_apply(dim, nel, beta, x):
    n = ndof(dim, nel)
    xx, sq = _vec(x, n)
    y = np.zeros_like(xx)
    _check(_load().or_fd_schur_apply(dim, _p(_nel(dim, nel)), float(beta), xx.shape[0], _p(xx), _p(y)),
           "fd_schur_apply")
    return y[0] if sq else y


def fd_complex_solve(dim, nel, gamma, b, sgn=1):
    """O2: z = (K + i*sgn*gamma*M)^{-1} b for real or complex b."""
    n = ndof(dim, nel)
    b = np.asarray(b)
    bre, sq = _vec(b.real, n)
    bim = _vec(b.imag, n)[0] if np.iscomplexobj(b) else None
    zre = np.zeros_like(bre)
    zim = np.zeros_like(bre)
    _check(_load().or_fd_complex_solve(dim, _p(_nel(dim, nel)), float(gamma), int(sgn), bre.shape[0], _p(bre),
                                       _p(bim), _p(zre), _p(zim)), "fd_complex_solve")
    z = zre + 1j * zim
    return z[0] if sq else z


def fd_kkt_solve(dim, nel, beta, ry=None, ru=None, rl=None):
    """O2: KKT solve mode by mode."""
    n = ndof(dim, nel)
    given = [r for r in (ry, ru, rl) if r is not None]
    nrhs = _vec(given[0], n)[0].shape[0] if given else 1
    sq = np.asarray(given[0]).ndim == 1 if given else True
    arrs = [None if r is None else _vec(r, n)[0] for r in (ry, ru, rl)]
    y = np.zeros((nrhs, n)); u = np.zeros((nrhs, n)); l = np.zeros((nrhs, n))
    _check(_load().or_fd_kkt_solve(dim, _p(_nel(dim, nel)), float(beta), nrhs, _p(arrs[0]), _p(arrs[1]),
                                   _p(arrs[2]), _p(y), _p(u), _p(l)), "fd_kkt_solve")
    return (y[0], u[0], l[0]) if sq else (y, u, l)


def fd_eigs(dim, nel):
    """(kappa, mu): K and M eigenvalues of each sine vector, index order = node order."""
    n = ndof(dim, nel)
    k = np.zeros(n)
    m = np.zeros(n)
    _check(_load().or_fd_eigs(dim, _p(_nel(dim, nel)), _p(k), _p(m)), "fd_eigs")
    return k, m
