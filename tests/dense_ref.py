"""Dense, definitional FETI-DP reference (Sec. 5) for tiny meshes, built on the library's
exported partition maps and the oracle's element matrices.  Test infrastructure only."""
import numpy as np

import oracle
from paper_1312_5653_gb300 import schur as S


def _local_nodes(dim, s):
    ext = [s + 1] * dim
    return [tuple((p // int(np.prod(ext[:a]))) % ext[a] for a in range(dim)) for p in range(int(np.prod(ext)))]



def local_neumann(dim, N, P, beta):
    """Subdomain Neumann matrix K + i gamma M on the (s+1)^dim local grid (oracle element loop)."""
    s = N // P
    g = 1.0 / np.sqrt(beta)
    Ke, Me = oracle.element(dim, [1.0 / N] * dim)
    Ae = Ke + 1j * g * Me
    loc = _local_nodes(dim, s)
    idx = {c: i for i, c in enumerate(loc)}
    A = np.zeros((len(loc), len(loc)), dtype=complex)
    for e in [tuple((k // s ** a) % s for a in range(dim)) for k in range(s ** dim)]:
        nodes = [idx[tuple(e[a] + ((q >> a) & 1) for a in range(dim))] for q in range(1 << dim)]
        for p in range(1 << dim):
            for q in range(1 << dim):
                A[nodes[p], nodes[q]] += Ae[p, q]
    return A, loc


def local_operators(dim, N, P, beta, sd):
    """(F, Frc, S) of subdomain sd, indexed by the library's interface slots (rows/columns of
    Dirichlet slots zero) and local corners (columns of Dirichlet corners zero)."""
    s = N // P
    A, loc = local_neumann(dim, N, P, beta)
    slots = S.schur_partition_export(dim, N, P, 1)
    nD = len(slots)
    Sc = [(sd // P ** t) % P for t in range(dim)]
    G = [tuple(Sc[a] * s + c[a] for a in range(dim)) for c in loc]
    dirich = [any(x in (0, N) for x in GG) for GG in G]
    vert = [i for i, c in enumerate(loc) if all(x in (0, s) for x in c)]
    corner_of = {i: sum((1 << a) for a in range(dim) if loc[i][a] == s) for i in vert}
    r = [i for i in range(len(loc)) if not dirich[i] and i not in vert]
    rpos = {i: k for k, i in enumerate(r)}
    Ainv = np.linalg.inv(A[np.ix_(r, r)])
    cset = [i for i in vert if not dirich[i]]
    X = Ainv @ A[np.ix_(r, cset)]
    F = np.zeros((nD, nD), complex)
    Frc = np.zeros((nD, 1 << dim), complex)
    interior = [i for i, c in enumerate(loc) if all(0 < x < s for x in c)]
    Aii_inv = np.linalg.inv(A[np.ix_(interior, interior)])
    sl = [int(p) for p in slots]
    Sfull = A[np.ix_(sl, sl)] - A[np.ix_(sl, interior)] @ Aii_inv @ A[np.ix_(interior, sl)]
    Sd = np.zeros((nD, nD), complex)
    act = [not dirich[p] for p in sl]
    for j, pj in enumerate(sl):
        if not act[j]:
            continue
        for k, pk in enumerate(sl):
            if act[k]:
                F[j, k] = Ainv[rpos[pj], rpos[pk]]
                Sd[j, k] = Sfull[j, k]
        for kc, ic in enumerate(cset):
            Frc[j, corner_of[ic]] = X[rpos[pj], kc]
    return F, Frc, Sd


def face_pairs(dim, P, lam, nD):
    """Q of the augmented coarse problem (Sec. 5, augmentation by the edge-based translational mode):
    one column per pair of face-adjacent subdomains, ones on the multipliers between that pair.
    Returns (Q, list of pairs)."""
    pairs, col = [], {}
    Q = np.zeros((len(lam), 0))
    entries = []
    for li, (a, bb) in enumerate(lam):
        sa, sb = int(a) // nD, int(bb) // nD
        ca = [(sa // P ** t) % P for t in range(dim)]
        cb = [(sb // P ** t) % P for t in range(dim)]
        if sum(abs(x - y) for x, y in zip(ca, cb)) != 1:
            continue  # 3D diagonal pairs along subdomain edge lines: not a face
        key = (min(sa, sb), max(sa, sb))
        if key not in col:
            col[key] = len(pairs)
            pairs.append(key)
        entries.append((li, col[key]))
    Q = np.zeros((len(lam), len(pairs)))
    for li, c in entries:
        Q[li, c] = 1.0
    return Q, pairs


def dense_feti_dp(dim, N, P, beta, b, aug=False):
    """Plain dense FETI-DP for (K + i gamma M) z = b following Sec. 5: corners primal, remainder
    matrices A_rr, jump operator B from the exported maps, coarse matrix, dual problem solved
    exactly, primal recovery by averaging the subdomain copies.  aug=True augments the coarse
    problem with the constraints Q^T B u = 0 (zero average jump across every subdomain face, enforced
    by coarse unknowns mu): coarse matrix [[K_cc, -X^T], [-X, -Y]] with X = Q^T F_rc, Y = Q^T F_rr Q,
    coupling Phi = [F_rc, F_rr Q], right-hand side [f_c; -Q^T d_r], multipliers lambda + Q mu."""
    s = N // P
    A, loc = local_neumann(dim, N, P, beta)
    nl = len(loc)
    info = S.schur_partition(dim, N, P)
    nD, nlam, nco, nsd = info["n_delta"], info["n_lambda"], info["n_coarse"], info["n_sub"]
    lam = S.schur_partition_export(dim, N, P, 0).reshape(-1, 2)
    slots = S.schur_partition_export(dim, N, P, 1)
    corners = S.schur_partition_export(dim, N, P, 2).reshape(nsd, 1 << dim)
    n = (N - 1) ** dim
    gid = lambda G: sum((G[a] - 1) * (N - 1) ** a for a in range(dim))
    vert = [i for i, c in enumerate(loc) if all(x in (0, s) for x in c)]
    corner_of = {i: sum((1 << a) for a in range(dim) if loc[i][a] == s) for i in vert}
    subs = []
    for sd in range(nsd):
        Sc = [(sd // P ** t) % P for t in range(dim)]
        G = [tuple(Sc[a] * s + c[a] for a in range(dim)) for c in loc]
        dirich = [any(x in (0, N) for x in GG) for GG in G]
        r = [i for i in range(nl) if not dirich[i] and i not in vert]
        cset = [i for i in vert if not dirich[i]]
        mult = {}
        for i in r:
            on = sum(1 for a in range(dim) if loc[i][a] in (0, s))
            mult[i] = 2 ** on if on else 1
        fr = np.array([b[gid(G[i])] / mult[i] for i in r], dtype=complex)
        Arr = A[np.ix_(r, r)]
        Arc = A[np.ix_(r, cset)]
        Acc = A[np.ix_(cset, cset)]
        Br = np.zeros((nlam, len(r)))
        rpos = {i: k for k, i in enumerate(r)}
        Bc = np.zeros((len(cset), nco))
        for k, i in enumerate(cset):
            Bc[k, corners[sd, corner_of[i]]] = 1
        subs.append(dict(G=G, r=r, c=cset, fr=fr, Arr=Arr, Arc=Arc, Acc=Acc, Br=Br, Bc=Bc, rpos=rpos))
    for li, (a, bb) in enumerate(lam):
        for code, sign in ((a, 1.0), (bb, -1.0)):
            sd, j = divmod(int(code), nD)
            subs[sd]["Br"][li, subs[sd]["rpos"][int(slots[j])]] = sign
    Frr = np.zeros((nlam, nlam), complex)
    Frc = np.zeros((nlam, nco), complex)
    Kcc = np.zeros((nco, nco), complex)
    dr = np.zeros(nlam, complex)
    fc = np.zeros(nco, complex)
    cdone = set()
    for sd, sub in enumerate(subs):
        Ainv = np.linalg.inv(sub["Arr"])
        Br, Bc = sub["Br"], sub["Bc"]
        Frr += Br @ Ainv @ Br.T
        Frc += Br @ Ainv @ sub["Arc"] @ Bc
        Kcc += Bc.T @ (sub["Acc"] - sub["Arc"].T @ Ainv @ sub["Arc"]) @ Bc
        dr += Br @ Ainv @ sub["fr"]
        fc -= Bc.T @ (sub["Arc"].T @ Ainv @ sub["fr"])
        for k, i in enumerate(sub["c"]):
            ci = int(np.argmax(Bc[k]))
            if ci not in cdone:
                fc[ci] += b[gid(sub["G"][i])]
                cdone.add(ci)
    if aug:
        Q, _ = face_pairs(dim, P, lam, nD)
        X = Q.T @ Frc
        Y = Q.T @ Frr @ Q
        Kaug = np.block([[Kcc, -X.T], [-X, -Y]])
        Phi = np.concatenate([Frc, Frr @ Q], axis=1)
        rhs0 = np.concatenate([fc, -Q.T @ dr])
        Ka_inv = np.linalg.inv(Kaug)
        F = Frr + Phi @ Ka_inv @ Phi.T
        d = dr - Phi @ Ka_inv @ rhs0
        lam0 = np.linalg.lstsq(F, d, rcond=None)[0]
        w = Ka_inv @ (rhs0 + Phi.T @ lam0)
        uc = w[:nco]
        lamv = lam0 + Q @ w[nco:]
    else:
        Kinv = np.linalg.inv(Kcc) if nco else np.zeros((0, 0))
        F = Frr + Frc @ Kinv @ Frc.T
        d = dr - Frc @ Kinv @ fc
        lamv = np.linalg.lstsq(F, d, rcond=None)[0]
        uc = Kinv @ (fc + Frc.T @ lamv)
    z = np.zeros(n, complex)
    cnt = np.zeros(n)
    for sub in subs:
        ur = np.linalg.solve(sub["Arr"], sub["fr"] - sub["Br"].T @ lamv - sub["Arc"] @ (sub["Bc"] @ uc))
        for k, i in enumerate(sub["r"]):
            z[gid(sub["G"][i])] += ur[k]
            cnt[gid(sub["G"][i])] += 1
        for k, i in enumerate(sub["c"]):
            z[gid(sub["G"][i])] += (sub["Bc"] @ uc)[k]
            cnt[gid(sub["G"][i])] += 1
    return z / cnt, F, d, lamv, Kcc


