"""GPU parity at the workloads the method is measured on, through the C ABI.

* Fixed step counts: after k steps of CG or GMRES the GPU iterate is the
  oracle's up to rounding, compared element by element.  Tolerance (first
  order in the rounding): each step perturbs the iterate by at most kappa
  times the relative error of one product, about sqrt(n) 2^-48 (A is carried
  to 2^-48 by the FP32 pair, sums round at 2^-53), so after k steps
  |x_gpu - x_oracle|_max <= k kappa sqrt(n) 2^-48 |x_oracle|_max.
* Converged solves: x_gpu - x_oracle = A^-1 (r_oracle - r_gpu), so
  |x_gpu - x_oracle|_max <= ||x_gpu - x_oracle||_2
                         <= ||A^-1||_2 (||r_gpu||_2 + ||r_oracle||_2),
  with both true residuals computed by the oracle in FP64.  The same bound
  with the rounding of b = A x* (|db| <= gamma_n |A||x*|) holds against x*.
  ||A^-1||_2: exact (numpy) for small n; for the n = 16384 families
  1 / sigma_min from the recipe: the SPD matrix G G^T/n + sigma I has
  lambda_min >= sigma minus its formation rounding (gamma_n 0.64 n ~ 2e-8,
  far below sigma / 100); 2 I + G/(2 sqrt n) has
  sigma_min >= 2 - ||G||_2 / (2 sqrt n) and ||G||_2 <= 2 sqrt n + t except
  with probability exp(-t^2 / 2) (Gaussian concentration); t = 8 is used.
* Accuracy gate at n = 16384: solved to rtol 1e-12, the error against x*
  and against the oracle's x (also solved to 1e-12) is at most 1e-8.

The n = 16384 cases build the 2 GiB matrices on the device from the seeded
recipe, copy them to the host for the oracle (OpenMP over the host cores),
and take about a minute.
"""
import math
import os

import numpy as np
import pytest
import torch

from paper_1511_07207_gb300 import binding as B
from paper_1511_07207_gb300 import inputs

pytestmark = pytest.mark.gpu

NT = os.cpu_count() or 1
U48 = 2.0 ** -48


def _cg(ctx, gpu, Ad, b, **kw):
    bd = torch.from_numpy(b).to(gpu)
    xd = torch.zeros(len(b), dtype=torch.float64, device=gpu)
    st, info = B.ls_cg_solve(ctx, Ad, bd, xd, B.make_opts(**kw))
    return st, info, xd.cpu().numpy()


def _gmres(ctx, gpu, Ad, b, **kw):
    bd = torch.from_numpy(b).to(gpu)
    xd = torch.zeros(len(b), dtype=torch.float64, device=gpu)
    st, info = B.ls_gmres_solve(ctx, Ad, bd, xd, B.make_opts(**kw))
    return st, info, xd.cpu().numpy()


def _fixed_tol(k, kappa, n, xref):
    return k * kappa * math.sqrt(n) * U48 * np.max(np.abs(xref))


# ---------------------------------------------------------------------------
# fixed step counts, element by element
# ---------------------------------------------------------------------------
# the three product paths: FP32 pair in one fused kernel (A in shared memory),
# FP32 pair in the general path, native FP64
MODES = {"fused": dict(f64_matvec=0, fused=1), "general": dict(f64_matvec=0, fused=0),
         "native": dict(f64_matvec=1)}


@pytest.mark.parametrize("mode", sorted(MODES))
@pytest.mark.parametrize("n", [777, 1000])
def test_cg_fixed_count_elementwise(ctx, gpu, oracle, n, mode):
    A = inputs.spd_matrix(n, 0.1, seed=5 + n)
    b = A @ inputs.solution(n, seed=6 + n)
    ev = np.linalg.eigvalsh(A)
    kappa = ev[-1] / ev[0]
    Ad = torch.from_numpy(A).to(gpu)
    for k in (1, 2, 5, 20):
        st, info, x = _cg(ctx, gpu, Ad, b, rtol=1e-300, max_iter=k, **MODES[mode])
        ref = oracle.cg(A, b, rtol=1e-300, max_iter=k)
        assert st == B.LS_NOT_CONVERGED == ref["status"]
        assert info["iters"] == ref["iters"] == k
        assert np.max(np.abs(x - ref["x"])) <= _fixed_tol(k, kappa, n, ref["x"]), k


@pytest.mark.parametrize("mode", sorted(MODES))
@pytest.mark.parametrize("n,m", [(777, 30), (1000, 50)])
def test_gmres_fixed_count_elementwise(ctx, gpu, oracle, n, m, mode):
    """k < m: the k-th iterate of the first cycle; k > m: across a restart.
    The restart family (1.1 I + G / sqrt n) keeps the residual far from
    convergence for 20 steps."""
    A = inputs.restart_matrix(n, seed=7 + n)
    b = A @ inputs.solution(n, seed=8 + n)
    s = np.linalg.svd(A, compute_uv=False)
    kappa = s[0] / s[-1]
    Ad = torch.from_numpy(A).to(gpu)
    for k in (1, 2, 5, 20, m + 3):
        st, info, x = _gmres(ctx, gpu, Ad, b, restart=m, rtol=1e-300, max_iter=k, **MODES[mode])
        ref = oracle.gmres(A, b, m=m, rtol=1e-300, max_iter=k)
        assert st == B.LS_NOT_CONVERGED == ref["status"]
        assert info["iters"] == ref["iters"] == k
        assert np.max(np.abs(x - ref["x"])) <= _fixed_tol(k, kappa, n, ref["x"]), k


# ---------------------------------------------------------------------------
# n = 512, seed 0: the small configuration exactly
# ---------------------------------------------------------------------------
def _converged_bounds(oracle, A, b, xs, x, xref, inv_norm, nthreads=1):
    rg = np.linalg.norm(oracle.residual(A, b, x, nthreads=nthreads))
    ro = np.linalg.norm(oracle.residual(A, b, xref, nthreads=nthreads))
    n = len(b)
    gam = n * 2.0 ** -53 / (1 - n * 2.0 ** -53)
    db = gam * np.linalg.norm(np.abs(A) @ np.abs(xs)) if n <= 4096 else None
    return rg, ro, inv_norm * (rg + ro), (inv_norm * (rg + db) if db is not None else None)


@pytest.mark.parametrize("fused", [0, 1])
def test_small_config_seed0(ctx, gpu, oracle, fused):
    n = 512
    # CG on G G^T / n + 0.1 I, seed 0
    A = inputs.spd_matrix(n, 0.1, seed=0)
    xs = inputs.solution(n, seed=0)
    b = A @ xs
    st, info, x = _cg(ctx, gpu, torch.from_numpy(A).to(gpu), b, rtol=1e-10, fused=fused)
    ref = oracle.cg(A, b, rtol=1e-10)
    assert st == B.LS_OK == ref["status"]
    inv = 1.0 / np.linalg.eigvalsh(A)[0]
    rg, ro, bx, bs = _converged_bounds(oracle, A, b, xs, x, ref["x"], inv)
    assert rg <= 1e-10 * np.linalg.norm(b)
    assert np.max(np.abs(x - ref["x"])) <= bx
    assert np.linalg.norm(x - xs) <= bs
    assert abs(info["iters"] - ref["iters"]) <= 1
    # GMRES(30) on 2 I + G / (2 sqrt n), seed 0
    A = inputs.nonsym_matrix(n, seed=0)
    xs = inputs.solution(n, seed=0)
    b = A @ xs
    st, info, x = _gmres(ctx, gpu, torch.from_numpy(A).to(gpu), b, restart=30, rtol=1e-10, fused=fused)
    ref = oracle.gmres(A, b, m=30, rtol=1e-10)
    assert st == B.LS_OK == ref["status"]
    inv = 1.0 / np.linalg.svd(A, compute_uv=False)[-1]
    rg, ro, bx, bs = _converged_bounds(oracle, A, b, xs, x, ref["x"], inv)
    assert rg <= 1e-10 * np.linalg.norm(b)
    assert np.max(np.abs(x - ref["x"])) <= bx
    assert np.linalg.norm(x - xs) <= bs
    assert abs(info["iters"] - ref["iters"]) <= 1


# ---------------------------------------------------------------------------
# n = 16384: the headline systems against full oracle solves
# ---------------------------------------------------------------------------
N2 = 16384
SIGMA2 = 1e-3


@pytest.fixture(scope="module")
def spd16k(gpu):
    Ad = inputs.spd_matrix(N2, SIGMA2, seed=0, device=gpu)
    xs = inputs.solution(N2, seed=0)
    b = (Ad @ torch.from_numpy(xs).to(gpu)).cpu().numpy()
    A = Ad.cpu().numpy()
    yield Ad, A, b, xs
    del Ad
    torch.cuda.empty_cache()


@pytest.fixture(scope="module")
def nonsym16k(gpu):
    Ad = inputs.nonsym_matrix(N2, seed=1, device=gpu)
    xs = inputs.solution(N2, seed=1)
    b = (Ad @ torch.from_numpy(xs).to(gpu)).cpu().numpy()
    A = Ad.cpu().numpy()
    yield Ad, A, b, xs
    del Ad
    torch.cuda.empty_cache()


_ORACLE = {}


def _oracle_solve(oracle, key, A, b, rtol):
    """Full oracle solve at n = 16384, once per (system, rtol) in this module."""
    if (key, rtol) not in _ORACLE:
        _ORACLE[(key, rtol)] = (oracle.cg(A, b, rtol=rtol, nthreads=NT) if key == "spd"
                                else oracle.gmres(A, b, m=50, rtol=rtol, nthreads=NT))
    return _ORACLE[(key, rtol)]


def _inv_spd():
    return 1.0 / (0.99 * SIGMA2)


def _inv_nonsym(n):
    return 1.0 / (2.0 - (2.0 * math.sqrt(n) + 8.0) / (2.0 * math.sqrt(n)))


@pytest.mark.parametrize("f64_matvec", [0, 1])
def test_n16384_cg_matches_full_oracle_solve(ctx, gpu, oracle, spd16k, f64_matvec):
    Ad, A, b, xs = spd16k
    st, info, x = _cg(ctx, gpu, Ad, b, rtol=1e-10, f64_matvec=f64_matvec)
    ref = _oracle_solve(oracle, "spd", A, b, 1e-10)
    assert st == B.LS_OK == ref["status"]
    rg, ro, bx, _ = _converged_bounds(oracle, A, b, xs, x, ref["x"], _inv_spd(), nthreads=NT)
    nb = np.linalg.norm(b)
    assert rg <= 1e-10 * nb and ro <= 1e-10 * nb
    assert np.max(np.abs(x - ref["x"])) <= bx
    # normwise: kappa (rel_res_gpu + rel_res_oracle), kappa <= (4 + sigma) / sigma
    kappa = (4 + SIGMA2) / SIGMA2
    assert np.linalg.norm(x - ref["x"]) <= kappa * (rg + ro) / nb * np.linalg.norm(ref["x"])
    assert abs(info["iters"] - ref["iters"]) <= 2 + ref["iters"] // 50


def test_n16384_gmres_matches_full_oracle_solve(ctx, gpu, oracle, nonsym16k):
    Ad, A, b, xs = nonsym16k
    for f64_matvec in (0, 1):
        st, info, x = _gmres(ctx, gpu, Ad, b, restart=50, rtol=1e-10, f64_matvec=f64_matvec)
        ref = _oracle_solve(oracle, "nonsym", A, b, 1e-10)
        assert st == B.LS_OK == ref["status"]
        rg, ro, bx, _ = _converged_bounds(oracle, A, b, xs, x, ref["x"], _inv_nonsym(N2), nthreads=NT)
        nb = np.linalg.norm(b)
        assert rg <= 1e-10 * nb and ro <= 1e-10 * nb
        assert np.max(np.abs(x - ref["x"])) <= bx
        assert abs(info["iters"] - ref["iters"]) <= 1


def test_n16384_accuracy_gate(ctx, gpu, oracle, spd16k, nonsym16k):
    """rtol 1e-12: error <= 1e-8 against x* and against the oracle's x."""
    Ad, A, b, xs = spd16k
    st, info, x = _cg(ctx, gpu, Ad, b, rtol=1e-12)
    ref = _oracle_solve(oracle, "spd", A, b, 1e-12)
    assert st == B.LS_OK == ref["status"]
    assert np.linalg.norm(x - xs) <= 1e-8 * np.linalg.norm(xs)
    assert np.linalg.norm(x - ref["x"]) <= 1e-8 * np.linalg.norm(ref["x"])
    Ad, A, b, xs = nonsym16k
    st, info, x = _gmres(ctx, gpu, Ad, b, restart=50, rtol=1e-12)
    ref = _oracle_solve(oracle, "nonsym", A, b, 1e-12)
    assert st == B.LS_OK == ref["status"]
    assert np.linalg.norm(x - xs) <= 1e-8 * np.linalg.norm(xs)
    assert np.linalg.norm(x - ref["x"]) <= 1e-8 * np.linalg.norm(ref["x"])


# ---------------------------------------------------------------------------
# the batched workload at full size: systems with n in [1024, 2048], 32 columns
# ---------------------------------------------------------------------------
def test_batch_full_size_systems(ctx, gpu, oracle):
    """Twelve systems of the 512-system workload's largest sizes, each with 32
    right-hand sides, solved in one batch; every column against the oracle's
    FP64 solve with the residual bound above."""
    r = inputs.rng(12, 3)
    ns = inputs.log_uniform_int(r, 1024, 2048, 12)
    specs = [inputs.SystemSpec(int(ns[i]), "spd" if i % 2 == 0 else "nonsym", 32, 9000 + i)
             for i in range(12)]
    arrays, systems = [], []
    for sp in specs:
        A = sp.matrix()
        Xs = sp.solution()
        Bm = A @ Xs
        Ad = torch.from_numpy(A).to(gpu)
        Bd = torch.from_numpy(np.asfortranarray(Bm)).to(gpu).T.contiguous().T
        Xd = torch.zeros((sp.n, sp.nrhs), dtype=torch.float64, device=gpu).T.contiguous().T
        method = B.LS_METHOD_CG if sp.kind == "spd" else B.LS_METHOD_GMRES
        systems.append(B.make_system(method, Ad, Bd, Xd, B.make_opts(rtol=1e-10, restart=30)))
        arrays.append((A, Bm, Xs, Ad, Bd, Xd))
    st, infos = B.ls_batch_solve(ctx, systems)
    assert st == B.LS_OK
    for (A, Bm, Xs, _, _, Xd), sp, info in zip(arrays, specs, infos):
        assert info["status"] == B.LS_OK, (sp, info)
        X = Xd.cpu().numpy()
        sv = np.linalg.svd(A, compute_uv=False)
        inv = 1.0 / sv[-1]
        for j in range(sp.nrhs):
            b = Bm[:, j]
            ref = (oracle.cg(A, b, rtol=1e-10, nthreads=NT) if sp.kind == "spd"
                   else oracle.gmres(A, b, m=30, rtol=1e-10, nthreads=NT))
            rg, ro, bx, bs = _converged_bounds(oracle, A, b, Xs[:, j], X[:, j], ref["x"], inv, nthreads=NT)
            assert rg <= 1.0000001e-10 * np.linalg.norm(b), (sp.n, j)
            assert np.max(np.abs(X[:, j] - ref["x"])) <= bx, (sp.n, j)
            assert np.linalg.norm(X[:, j] - Xs[:, j]) <= bs, (sp.n, j)
