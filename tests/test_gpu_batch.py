"""GPU parity of ls_batch_solve with the oracle.

Every right-hand side column of every system is an independent solve of
A x = b_j; the batched engine refines in FP64 around FP32 inner CG (SPD) or
GMRES(m) (nonsymmetric) steps.  Each column must reach the FP64 tolerance
(true relative residual computed by the oracle) and agree with the oracle's
FP64 solution within cond(A) * rtol.  A system solved alone and inside a
batch must give bitwise identical results (its arithmetic does not depend
on the other systems).
"""
import numpy as np
import pytest
import torch

from paper_1511_07207_gb300 import binding as B
from paper_1511_07207_gb300 import inputs

pytestmark = pytest.mark.gpu


def _systems(specs, gpu, on_device=True, rtol=1e-10, restart=30):
    arrays, systems = [], []
    for sp in specs:
        A = sp.matrix()
        Xs = sp.solution()
        Bm = A @ Xs
        if on_device:
            Ad = torch.from_numpy(A).to(gpu)
            Bd = torch.from_numpy(np.asfortranarray(Bm)).to(gpu).T.contiguous().T   # column-major
            Xd = torch.zeros((sp.n, sp.nrhs), dtype=torch.float64, device=gpu).T.contiguous().T
        else:
            Ad, Bd = A, np.asfortranarray(Bm)
            Xd = np.zeros((sp.n, sp.nrhs), order="F")
        method = B.LS_METHOD_CG if sp.kind == "spd" else B.LS_METHOD_GMRES
        o = B.make_opts(rtol=rtol, restart=restart)
        systems.append(B.make_system(method, Ad, Bd, Xd, o))
        arrays.append((A, Bm, Xs, Ad, Bd, Xd))
    return arrays, systems


def _x(Xd):
    return Xd.cpu().numpy() if hasattr(Xd, "cpu") else Xd


def _check(oracle, arrays, specs, infos, rtol=1e-10):
    for (A, Bm, Xs, _, _, Xd), sp, info in zip(arrays, specs, infos):
        X = _x(Xd)
        assert info["status"] == B.LS_OK, (sp, info)
        for j in range(sp.nrhs):
            b = Bm[:, j]
            nb = np.linalg.norm(b)
            rel = np.linalg.norm(oracle.residual(A, b, X[:, j])) / nb
            assert rel <= rtol * 1.0000001, (sp.n, j, rel)
            if sp.kind == "spd":
                ref = oracle.cg(A, b, rtol=1e-12)
            else:
                ref = oracle.gmres(A, b, m=30, rtol=1e-12)
            s = np.linalg.svd(A, compute_uv=False)
            kap = s[0] / s[-1]
            err = np.linalg.norm(X[:, j] - ref["x"]) / np.linalg.norm(ref["x"])
            assert err <= 4 * kap * rtol, (sp.n, j, err)
        assert info["true_rel_res"] <= rtol * 1.0000001


SMALL = [inputs.SystemSpec(n, kind, s, seed)
         for (n, kind, s, seed) in [(1, "spd", 1, 1), (5, "nonsym", 2, 2), (64, "spd", 3, 3),
                                    (100, "nonsym", 1, 4), (257, "spd", 32, 5),
                                    (257, "nonsym", 8, 6), (600, "spd", 5, 7),
                                    (513, "nonsym", 32, 8), (129, "spd", 4, 9), (33, "nonsym", 7, 10)]]


def test_batch_matches_oracle(ctx, gpu, oracle):
    arrays, systems = _systems(SMALL, gpu)
    st, infos = B.ls_batch_solve(ctx, systems)
    assert st == B.LS_OK
    _check(oracle, arrays, SMALL, infos)
    assert infos[0]["launches"] > 0


def test_batch_host_buffers(ctx, gpu, oracle):
    specs = SMALL[:5]
    arrays, systems = _systems(specs, gpu, on_device=False)
    st, infos = B.ls_batch_solve(ctx, systems)
    assert st == B.LS_OK
    _check(oracle, arrays, specs, infos)


def test_alone_equals_in_mix(ctx, gpu):
    specs = SMALL
    arrays, systems = _systems(specs, gpu)
    st, _ = B.ls_batch_solve(ctx, systems)
    assert st == B.LS_OK
    for k in (2, 5, 7):
        a1, s1 = _systems([specs[k]], gpu)
        st, _ = B.ls_batch_solve(ctx, s1)
        assert st == B.LS_OK
        assert np.array_equal(_x(a1[0][5]), _x(arrays[k][5])), specs[k]


def test_batch_config_reduced(ctx, gpu, oracle):
    """The 512-system workload at reduced size: 48 systems, n log-uniform in
    [64, 512], half SPD, 1..32 right-hand sides."""
    specs = inputs.batch_specs(48, seed=1, lo=64, hi=512, max_rhs=32)
    arrays, systems = _systems(specs, gpu)
    st, infos = B.ls_batch_solve(ctx, systems)
    assert st == B.LS_OK
    _check(oracle, arrays[:8], specs[:8], infos[:8])
    for (A, Bm, _, _, _, Xd), info in zip(arrays, infos):
        X = _x(Xd)
        R = Bm - A @ X
        assert np.all(np.linalg.norm(R, axis=0) <= 1.0000001e-10 * np.linalg.norm(Bm, axis=0))


def test_batch_edge_cases(ctx, gpu):
    n = 40
    A = inputs.spd_matrix(n, 0.1, seed=3)
    Bm = np.zeros((n, 2), order="F")
    Bm[:, 1] = A @ inputs.solution(n, seed=3)
    Ad = torch.from_numpy(A).to(gpu)
    Bd = torch.from_numpy(Bm).to(gpu).T.contiguous().T
    Xd = torch.full((n, 2), 7.0, dtype=torch.float64, device=gpu).T.contiguous().T
    st, infos = B.ls_batch_solve(ctx, [B.make_system(B.LS_METHOD_CG, Ad, Bd, Xd)])
    assert st == B.LS_OK
    X = Xd.cpu().numpy()
    assert not X[:, 0].any()                             # b = 0 column -> x = 0
    assert np.linalg.norm(A @ X[:, 1] - Bm[:, 1]) <= 1e-10 * np.linalg.norm(Bm[:, 1])
    # argument checks
    big = torch.zeros((B.LS_BATCH_MAX_N + 1, 1), dtype=torch.float64, device=gpu)
    s = B.make_system(B.LS_METHOD_CG, Ad, Bd, Xd)
    s.n = B.LS_BATCH_MAX_N + 1
    assert B.ls_batch_solve(ctx, [s])[0] == B.LS_ERR_ARG
    s = B.make_system(B.LS_METHOD_GMRES, Ad, Bd, Xd, B.make_opts(restart=33))
    assert B.ls_batch_solve(ctx, [s])[0] == B.LS_ERR_ARG
    s = B.make_system(B.LS_METHOD_CG, Ad, Bd, Xd)
    s.nrhs = 33
    assert B.ls_batch_solve(ctx, [s])[0] == B.LS_ERR_ARG
    del big
    # NaN in one system does not poison the others
    Bn = Bm.copy(order="F")
    Bn[3, 1] = np.nan
    Bnd = torch.from_numpy(Bn).to(gpu).T.contiguous().T
    X2 = torch.zeros((n, 2), dtype=torch.float64, device=gpu).T.contiguous().T
    X3 = torch.zeros((n, 2), dtype=torch.float64, device=gpu).T.contiguous().T
    st, infos = B.ls_batch_solve(ctx, [B.make_system(B.LS_METHOD_CG, Ad, Bnd, X2),
                                       B.make_system(B.LS_METHOD_CG, Ad, Bd, X3)])
    assert infos[0]["status"] == B.LS_ERR_NAN and infos[1]["status"] == B.LS_OK
    assert st == B.LS_ERR_NAN


def test_tensor_core_products_match_fp32_pipe(ctx, gpu, oracle, monkeypatch):
    """The inner block products of systems with 9-32 right-hand sides run on
    the tensor cores (three TF32 products of a head/tail split, about FP32
    accuracy); LS_ENGINE_TC=0 runs them on the FP32 pipe instead.  Both reach
    the FP64 tolerance against the oracle, the solutions agree within the
    residual bound, and they are not bitwise equal (the tensor-core path ran)."""
    specs = [inputs.SystemSpec(n, kind, s, seed)
             for (n, kind, s, seed) in [(300, "spd", 16, 21), (700, "nonsym", 32, 22),
                                        (1025, "spd", 32, 23), (513, "nonsym", 12, 24),
                                        (2048, "spd", 20, 25), (97, "spd", 3, 26)]]
    results = {}
    for mode in ("3", "0"):
        monkeypatch.setenv("LS_ENGINE_TC", mode)
        arrays, systems = _systems(specs, gpu)
        st, infos = B.ls_batch_solve(ctx, systems)
        assert st == B.LS_OK
        _check(oracle, arrays[:3], specs[:3], infos[:3])
        for (A, Bm, _, _, _, Xd), info in zip(arrays, infos):
            assert info["status"] == B.LS_OK
            X = _x(Xd)
            assert np.all(np.linalg.norm(Bm - A @ X, axis=0) <= 1.0000001e-10 * np.linalg.norm(Bm, axis=0))
        results[mode] = [_x(a[5]) for a in arrays]
    monkeypatch.delenv("LS_ENGINE_TC")
    differs = False
    for (A, Bm, _, _, _, _), sp, Xt, Xf in zip(arrays, specs, results["3"], results["0"]):
        inv = 1.0 / np.linalg.svd(A, compute_uv=False)[-1]
        bound = inv * (np.linalg.norm(Bm - A @ Xt, axis=0) + np.linalg.norm(Bm - A @ Xf, axis=0))
        assert np.all(np.max(np.abs(Xt - Xf), axis=0) <= bound + 1e-300), sp
        if sp.nrhs > 8 and not np.array_equal(Xt, Xf):
            differs = True
    assert differs

