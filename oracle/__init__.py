"""Reference oracle (FP64, CPU) for the factored Schur complement solve.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The product library
(``paper_1312_5653_gb300``) never imports, links or runs it, and the two share no code.

The arithmetic lives in ``oracle.c`` (plain C; only the independent lines of the O2 sine transforms
are shared out over OpenMP threads, see ``set_threads``).  This module only marshals numpy arrays
through ctypes.  Every function works on real FP64 vectors over the n interior nodes of a
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
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
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
        lib.or_full_stiffness.argtypes = [I, P, I, P, P]
        lib.or_fd_pw_solve.argtypes = [I, P, D, I, P, P]
        lib.or_set_threads.argtypes = [I]
        lib.or_set_threads.restype = I
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


def set_threads(nthreads):
    """Threads of the O2 sine transforms (OpenMP); returns the count in effect.  The results are
    the same for every count (each transform line is computed by one thread, in the same order)."""
    return int(_load().or_set_threads(int(nthreads)))


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


def fd_pw_solve(dim, nel, beta, b):
    """O2: x = S_p^{-1} b for the Pearson-Wathen S_p = (K + M/sqrt(beta)) M^-1 (K + M/sqrt(beta))
    (Sec. 3.2) by fast diagonalisation."""
    n = ndof(dim, nel)
    bb, sq = _vec(b, n)
    x = np.zeros_like(bb)
    _check(_load().or_fd_pw_solve(dim, _p(_nel(dim, nel)), float(beta), bb.shape[0], _p(bb), _p(x)), "fd_pw_solve")
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


def nfull(dim, nel):
    """Grid nodes of the whole mesh, boundary included: prod(nel[a] + 1)."""
    ne = _nel(dim, nel)
    return int(np.prod(ne[:dim].astype(np.int64) + 1))


def interior_of(dim, nel, yfull):
    """The interior-node values (length n, oracle order) of full-grid vectors (..., nfull)."""
    ne = _nel(dim, nel)[:dim]
    yf = np.asarray(yfull, dtype=np.float64)
    shp = tuple(int(e) + 1 for e in ne[::-1])  # C order: last axis fastest = grid axis 0
    a = yf.reshape(yf.shape[:-1] + shp)
    sl = (Ellipsis,) + tuple(slice(1, -1) for _ in range(dim))
    return a[sl].reshape(yf.shape[:-1] + (-1,))


def full_stiffness(dim, nel, yfull):
    """K y_int + K_c y_c on the interior nodes for full-grid vectors (Sec. 2, element loop)."""
    n, nf = ndof(dim, nel), nfull(dim, nel)
    yy, sq = _vec(yfull, nf)
    out = np.zeros((yy.shape[0], n))
    _check(_load().or_full_stiffness(dim, _p(_nel(dim, nel)), yy.shape[0], _p(yy), _p(out)), "full_stiffness")
    return out[0] if sq else out


def boundary_coupling(dim, nel, yfull):
    """K_c y_c alone: the full-grid vector with its interior values set to zero."""
    yb = np.array(yfull, dtype=np.float64, copy=True)
    n, nf = ndof(dim, nel), nfull(dim, nel)
    flat = yb.reshape(-1, nf)
    mask = np.ones(nf, dtype=bool)
    mask[interior_index(dim, nel)] = False
    flat[:, ~mask] = 0.0
    return full_stiffness(dim, nel, yb)


def interior_index(dim, nel):
    """Positions of the interior nodes (oracle order) within the full-grid vector."""
    ne = _nel(dim, nel)[:dim]
    idx = np.arange(nfull(dim, nel)).reshape(tuple(int(e) + 1 for e in ne[::-1]))
    sl = tuple(slice(1, -1) for _ in range(dim))
    return idx[sl].reshape(-1)


def control_solve(dim, nel, beta, yfull, fd=False):
    """The range-space problem of Sec. 3.1 with Dirichlet data y_c = the boundary values of yfull
    (the thermal problem of Sec. 6.1): the KKT system of Sec. 2 with right-hand side
    (M ybar, 0, -K_c y_c), solved by O1 (banded KKT factorisation) or, with fd=True, by O2
    (sine basis).  Returns (y, u, lambda) on the interior nodes."""
    yb = interior_of(dim, nel, yfull)
    ry = apply_M(dim, nel, yb)
    rl = -boundary_coupling(dim, nel, yfull)
    return (fd_kkt_solve if fd else kkt_solve)(dim, nel, beta, ry=ry, rl=rl)
