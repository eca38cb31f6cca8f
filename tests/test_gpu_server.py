"""GPU tests of the continuous-batching server (ls_server_*).

Requests of uneven size and method are submitted from two host threads while
earlier ones are running; each result must meet its tolerance (checked with
the oracle's FP64 residual), match the oracle's solution within
cond(A) * rtol, and be bitwise identical to the same system solved alone
(the engine's per-system arithmetic does not depend on the mix).  A budget
that holds only a few requests must still serve them all; a request larger
than the budget is refused; unknown tickets are argument errors; stopping
with work in flight returns without hanging and cancels what is left.
"""
import threading
import time

import numpy as np
import pytest
import torch

from paper_1511_07207_gb300 import binding as B
from paper_1511_07207_gb300 import inputs

pytestmark = pytest.mark.gpu


def _request(spec, gpu, rtol):
    A = spec.matrix()
    Xs = spec.solution()
    Bm = A @ Xs
    Ad = torch.from_numpy(A).to(gpu)                       # borrowed by the server
    Bh = np.asfortranarray(Bm)                             # copied at submit
    Xh = np.zeros((spec.n, spec.nrhs), order="F")          # written at completion
    method = B.LS_METHOD_CG if spec.kind == "spd" else B.LS_METHOD_GMRES
    sysd = B.make_system(method, Ad, Bh, Xh, B.make_opts(rtol=rtol, restart=30))
    return dict(A=A, B=Bm, Ad=Ad, Bh=Bh, X=Xh, sys=sysd, spec=spec, rtol=rtol)


def _wait(srv, tickets, timeout=120.0):
    infos = {}
    t0 = time.time()
    while len(infos) < len(tickets):
        for t in tickets:
            if t in infos:
                continue
            st, done, info = B.ls_server_poll(srv, t)
            assert st == B.LS_OK
            if done:
                infos[t] = info
        assert time.time() - t0 < timeout, "server did not finish"
        time.sleep(0.002)
    return infos


def _specs(k, seed):
    r = np.random.default_rng(seed)
    out = []
    for i in range(k):
        n = int(np.exp(r.uniform(np.log(32), np.log(700))))
        out.append(inputs.SystemSpec(n, "spd" if i % 2 == 0 else "nonsym",
                                     int(r.integers(1, 9)), 500 + seed * 100 + i))
    return out


def test_server_serves_mixed_requests(ctx, gpu, oracle):
    srv = B.ls_server_start(ctx, hbm_budget_bytes=1 << 30, max_slots=8, step_iters=4)
    try:
        reqs = [_request(sp, gpu, 1e-10 if i % 3 else 1e-6) for i, sp in enumerate(_specs(24, 1))]
        tickets = [None] * len(reqs)

        def submit(idx):
            for i in idx:
                st, t = B.ls_server_submit(srv, reqs[i]["sys"])
                assert st == B.LS_OK
                tickets[i] = t
                time.sleep(0.001)

        th = [threading.Thread(target=submit, args=(range(k, len(reqs), 2),)) for k in (0, 1)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        infos = _wait(srv, tickets)
    finally:
        assert B.ls_server_stop(srv) == B.LS_OK
    for rq, t in zip(reqs, tickets):
        info = infos[t]
        assert info["status"] == B.LS_OK, (rq["spec"], info)
        assert info["time_ms"] > 0
        A, Bm, X, rtol = rq["A"], rq["B"], rq["X"], rq["rtol"]
        for j in range(Bm.shape[1]):
            rel = np.linalg.norm(oracle.residual(A, Bm[:, j], X[:, j])) / np.linalg.norm(Bm[:, j])
            assert rel <= rtol * 1.0000001
        if rq["rtol"] == 1e-10:
            ref = (oracle.cg if rq["spec"].kind == "spd" else oracle.gmres)(A, Bm[:, 0], rtol=1e-12)
            s = np.linalg.svd(A, compute_uv=False)
            assert np.linalg.norm(X[:, 0] - ref["x"]) <= 4 * s[0] / s[-1] * 1e-10 * np.linalg.norm(ref["x"])
    # alone == in the mix, bitwise, for every request
    for rq in reqs:
        Xd = torch.zeros((rq["spec"].n, rq["spec"].nrhs), dtype=torch.float64, device=gpu).T.contiguous().T
        one = B.make_system(rq["sys"].method, rq["Ad"], torch.from_numpy(rq["Bh"]).to(gpu).T.contiguous().T,
                            Xd, B.make_opts(rtol=rq["rtol"], restart=30))
        st, _ = B.ls_batch_solve(ctx, [one])
        assert st == B.LS_OK
        assert np.array_equal(Xd.cpu().numpy(), rq["X"]), rq["spec"]


@pytest.mark.parametrize("merge", [1, 0])
def test_server_shared_matrices(ctx, gpu, oracle, merge):
    """Requests that share a device matrix (merged into one slot as extra
    right-hand-side columns when merge_rhs is on) each meet their tolerance and
    agree with the oracle's solution within cond(A) * rtol."""
    mats = []
    for k, kind in enumerate(("spd", "nonsym", "spd")):
        sp = inputs.SystemSpec(300 + 97 * k, kind, 1, 900 + k)
        A = sp.matrix()
        mats.append((sp, A, torch.from_numpy(A).to(gpu)))
    r = np.random.default_rng(5)
    reqs = []
    for i in range(18):
        sp, A, Ad = mats[i % 3]
        s = int(r.integers(1, 6))
        Xs = r.uniform(-1, 1, (sp.n, s))
        Bm = A @ Xs
        rtol = 1e-10 if i % 2 else 1e-6
        Xh = np.zeros((sp.n, s), order="F")
        Bh = np.asfortranarray(Bm)            # must stay alive until submit has copied it
        method = B.LS_METHOD_CG if sp.kind == "spd" else B.LS_METHOD_GMRES
        sysd = B.make_system(method, Ad, Bh, Xh, B.make_opts(rtol=rtol, restart=30))
        reqs.append(dict(A=A, B=Bm, Bh=Bh, X=Xh, sys=sysd, rtol=rtol, kind=sp.kind))
    srv = B.ls_server_start(ctx, hbm_budget_bytes=1 << 30, max_slots=4, step_iters=4, merge_rhs=merge)
    try:
        tickets = []
        for rq in reqs:                       # a burst: the queue fills before admission
            st, t = B.ls_server_submit(srv, rq["sys"])
            assert st == B.LS_OK
            tickets.append(t)
        infos = _wait(srv, tickets)
    finally:
        assert B.ls_server_stop(srv) == B.LS_OK
    for rq, t in zip(reqs, tickets):
        assert infos[t]["status"] == B.LS_OK
        A, Bm, X = rq["A"], rq["B"], rq["X"]
        for j in range(Bm.shape[1]):
            rel = np.linalg.norm(oracle.residual(A, Bm[:, j], X[:, j])) / np.linalg.norm(Bm[:, j])
            assert rel <= rq["rtol"] * 1.0000001
        assert infos[t]["rel_res"] <= rq["rtol"]


def test_server_budget_and_errors(ctx, gpu):
    specs = _specs(10, 2)
    reqs = [_request(sp, gpu, 1e-10) for sp in specs]
    # a budget that holds about two of the largest requests at a time
    srv = B.ls_server_start(ctx, hbm_budget_bytes=8 << 20, max_slots=4, step_iters=2)
    try:
        tickets = []
        for rq in reqs:
            st, t = B.ls_server_submit(srv, rq["sys"])
            assert st == B.LS_OK
            tickets.append(t)
        infos = _wait(srv, tickets)
        assert all(infos[t]["status"] == B.LS_OK for t in tickets)
        # collected tickets and tickets never issued are argument errors
        assert B.ls_server_poll(srv, tickets[0])[0] == B.LS_ERR_ARG
        assert B.ls_server_poll(srv, 10 ** 9)[0] == B.LS_ERR_ARG
        # larger than the whole budget
        big = _request(inputs.SystemSpec(2500, "spd", 32, 9), gpu, 1e-10)
        st, _ = B.ls_server_submit(srv, big["sys"])
        assert st == B.LS_ERR_NOMEM
        bad = B.make_system(B.LS_METHOD_GMRES, reqs[0]["Ad"], reqs[0]["Bh"], reqs[0]["X"],
                            B.make_opts(restart=64))
        assert B.ls_server_submit(srv, bad)[0] == B.LS_ERR_ARG
    finally:
        assert B.ls_server_stop(srv) == B.LS_OK


def test_server_stop_with_work_in_flight(ctx, gpu):
    srv = B.ls_server_start(ctx, hbm_budget_bytes=256 << 20, max_slots=2, step_iters=1)
    reqs = [_request(sp, gpu, 1e-12) for sp in _specs(8, 3)]
    tickets = []
    for rq in reqs:
        st, t = B.ls_server_submit(srv, rq["sys"])
        assert st == B.LS_OK
        tickets.append(t)
    t0 = time.time()
    assert B.ls_server_stop(srv) == B.LS_OK
    assert time.time() - t0 < 30
