"""Serving: continuous batching of mixed meshes, dimensions and beta through schur_server; every
result equals the same request solved alone (and the oracle) within the solver tolerance; the
memory budget admits, evicts and rejects."""
import random
import threading
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle
from paper_1312_5653_gb300 import inputs
from paper_1312_5653_gb300 import schur as S


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


KEYS = [(2, 64, 1e-2), (2, 128, 1e-5), (2, 256, 1e-8), (3, 32, 1e-4), (2, 64, 1e-8)]


def make_rhs(dim, N, nrhs, seed):
    yb = inputs.smoothed_noise(dim, N, seed=seed, nrhs=nrhs)
    return oracle.apply_M(dim, N, yb)


def test_mixed_stream_matches_solo_and_oracle():
    rng = random.Random(0)
    reqs = []
    for i in range(30):
        dim, N, beta = KEYS[rng.randrange(len(KEYS))]
        reqs.append((dim, N, beta, make_rhs(dim, N, rng.randint(1, 4), 100 + i)))
    srv = S.Server(budget_bytes=16 << 30, workers=4, precision=S.SCHUR_MIXED, tol=1e-10)
    tickets = [None] * len(reqs)

    def producer(idx):
        for i in idx:
            time.sleep(rng.random() * 0.003)
            dim, N, beta, b = reqs[i]
            tickets[i] = srv.submit(dim, N, beta, b)

    try:
        threads = [threading.Thread(target=producer, args=(list(range(k, len(reqs), 3)),)) for k in range(3)]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        results = [srv.wait(t) for t in tickets]
        info = srv.info()
    finally:
        srv.close()
    assert info["completed"] == len(reqs)
    lat = [st["ms_solve"] for _, st in results]
    print("served", len(reqs), "p50 %.1f ms p99 %.1f ms" % (np.percentile(lat, 50), np.percentile(lat, 99)), info)
    solo = {}
    for (dim, N, beta, b), (x, st) in zip(reqs, results):
        assert st["status"] == 0
        xref = oracle.fd_schur_solve(dim, N, beta, b)
        assert rel(x, xref) <= 1e-8
        key = (dim, N, beta)
        if key not in solo:
            solo[key] = S.Solver(dim, N, beta, nsub=N // (16 if dim == 2 else 8), precision=S.SCHUR_MIXED, tol=1e-10)
        xs = solo[key].schur_solve(torch.from_numpy(np.ascontiguousarray(b)).cuda()).cpu().numpy()
        assert rel(x, xs) <= 1e-8
    for s in solo.values():
        s.close()


def _reservation_of_one_key():
    """Bytes the server reserves for one 256^2 context (its own admission estimate)."""
    srv = S.Server(budget_bytes=8 << 30, workers=1, precision=S.SCHUR_MIXED, tol=1e-10)
    try:
        b = make_rhs(2, 256, 1, 6)
        srv.wait(srv.submit(2, 256, 1e-3, b))
        info = srv.info()
        assert info["cached_contexts"] == 1
        return info["bytes_reserved"]
    finally:
        srv.close()


def test_budget_admission_eviction_and_rejection():
    one_key = _reservation_of_one_key()
    assert one_key > 0
    # room for one 256^2 context, not two: the second key must evict the first
    srv = S.Server(budget_bytes=one_key * 3 // 2, workers=2, precision=S.SCHUR_MIXED, tol=1e-10)
    try:
        _budget_body(srv)
    finally:
        srv.close()


def _budget_body(srv):
    b1 = make_rhs(2, 256, 1, 7)
    b2 = make_rhs(2, 256, 1, 8)
    t1 = srv.submit(2, 256, 1e-3, b1)
    t2 = srv.submit(2, 256, 1e-6, b2)  # a second key: admitted after the first is evicted
    x1, _ = srv.wait(t1)
    x2, _ = srv.wait(t2)
    assert rel(x1, oracle.fd_schur_solve(2, 256, 1e-3, b1)) <= 1e-8
    assert rel(x2, oracle.fd_schur_solve(2, 256, 1e-6, b2)) <= 1e-8
    assert srv.info()["cached_contexts"] == 1
    # a mesh whose estimate exceeds the whole budget is refused at submission
    with pytest.raises(S.SchurError) as e:
        srv.submit(2, 1024, 1e-3, np.zeros(1023 * 1023))
    assert e.value.code == S.SCHUR_EBUSY
