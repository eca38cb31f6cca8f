"""Seeded synthetic inputs for the dense Krylov solvers.

This module holds only the input recipes; it contains none of the solver
arithmetic and imports nothing from the library or the oracle, so both sides
can be fed the same bits.  The paper leaves its test matrices unspecified
(section "Results" only gives the sizes), so the families below are the
standard well-posed dense test sets:

* SPD:          A = G G^T / n + sigma I, G with i.i.d. N(0, 1) entries.
                The spectrum lies in about [sigma, 4 + sigma]
                (Marchenko-Pastur), so cond(A) ~ 4 / sigma: about 40 for
                sigma = 0.1 and about 4e3 for sigma = 1e-3.  The matrix is
                made exactly symmetric by mirroring its upper triangle.
* nonsymmetric: A = 2 I + G / (2 sqrt(n)); its eigenvalues fill a disk of
                radius about 1/2 around 2 (circular law).
* restart:      A = 1.1 I + G / sqrt(n); eigenvalues fill the unit disk
                around 1.1, so GMRES converges slowly and restarts matter.
* x* ~ U[-1, 1] and b = A x*.

Random numbers come from numpy's Philox counter-based generator keyed by
(seed, stream id), so every matrix, solution and right-hand side is
reproducible on any host.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# stream ids that separate the random draws of one seed
_S_G, _S_X, _S_MISC = 1, 2, 3


def rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=(int(seed) << 8) + int(stream)))


def gaussian(n: int, seed: int, cols: int | None = None) -> np.ndarray:
    """G (n x cols, default square) with i.i.d. N(0, 1) FP64 entries."""
    return rng(seed, _S_G).standard_normal((n, n if cols is None else cols))


def spd_matrix(n: int, sigma: float, seed: int, device=None):
    """A = G G^T / n + sigma I, exactly symmetric.

    With ``device`` (a torch device) the product is formed there with torch
    and a torch tensor is returned; otherwise numpy on the host.
    """
    G = gaussian(n, seed)
    if device is not None:
        import torch
        Gt = torch.from_numpy(G).to(device)
        del G
        A = Gt @ Gt.T
        del Gt
        A.div_(n)
        A = torch.triu(A) + torch.triu(A, 1).T
        A.diagonal().add_(sigma)
        return A
    A = (G @ G.T) / n
    A = np.triu(A) + np.triu(A, 1).T
    A[np.diag_indices(n)] += sigma
    return A


def nonsym_matrix(n: int, seed: int, shift: float = 2.0, scale: float = 0.5, device=None):
    """A = shift I + scale G / sqrt(n)  (default 2 I + G / (2 sqrt(n)))."""
    G = gaussian(n, seed)
    A = G * (scale / math.sqrt(n))
    A[np.diag_indices(n)] += shift
    if device is not None:
        import torch
        return torch.from_numpy(A).to(device)
    return A


def restart_matrix(n: int, seed: int, device=None):
    """A = 1.1 I + G / sqrt(n): slow GMRES convergence, exercises restarts."""
    return nonsym_matrix(n, seed, shift=1.1, scale=1.0, device=device)


def solution(n: int, seed: int, nrhs: int | None = None) -> np.ndarray:
    """x* with i.i.d. U[-1, 1] entries (n, or n x nrhs column-major-ready)."""
    r = rng(seed, _S_X)
    if nrhs is None:
        return r.uniform(-1.0, 1.0, n)
    return r.uniform(-1.0, 1.0, (n, nrhs))


def rhs(A, xstar):
    """b = A x* in FP64 (numpy or torch, following A)."""
    return A @ xstar


def distinct_eig_spd(n: int, eigs, seed: int) -> np.ndarray:
    """Q diag(lambda) Q^T with the given eigenvalues repeated to length n."""
    Q, _ = np.linalg.qr(gaussian(n, seed))
    lam = np.resize(np.asarray(eigs, dtype=np.float64), n)
    A = (Q * lam) @ Q.T
    return np.triu(A) + np.triu(A, 1).T


# ---------------------------------------------------------------------------
# workload descriptors
# ---------------------------------------------------------------------------

def log_uniform_int(r: np.random.Generator, lo: int, hi: int, size: int) -> np.ndarray:
    """n = round(exp(U(ln lo, ln hi)))."""
    return np.rint(np.exp(r.uniform(math.log(lo), math.log(hi), size))).astype(np.int64)


@dataclass
class SystemSpec:
    """One dense system of a batch: kind 'spd' (CG) or 'nonsym' (GMRES)."""
    n: int
    kind: str
    nrhs: int
    seed: int
    rtol: float = 1e-10

    def matrix(self, device=None):
        if self.kind == "spd":
            return spd_matrix(self.n, 0.1, self.seed, device=device)
        return nonsym_matrix(self.n, self.seed, device=device)

    def solution(self):
        return solution(self.n, self.seed, self.nrhs)


def batch_specs(count: int = 512, seed: int = 0, lo: int = 64, hi: int = 2048,
                max_rhs: int = 32) -> list[SystemSpec]:
    """Independent systems: n log-uniform in [lo, hi], half SPD and half
    nonsymmetric (alternating), 1..max_rhs right-hand sides each."""
    r = rng(seed, _S_MISC)
    ns = log_uniform_int(r, lo, hi, count)
    ks = r.integers(1, max_rhs + 1, count)
    return [SystemSpec(int(ns[i]), "spd" if i % 2 == 0 else "nonsym", int(ks[i]),
                       seed * 100003 + i + 1) for i in range(count)]


@dataclass
class Request:
    """One served solve: arrival time (s), the system, and its tolerance."""
    t_arrival: float
    spec: SystemSpec
    precision: str = "f64"          # 'bf16' for the 1e-6 requests


def serve_requests(rate: float = 2000.0, duration: float = 60.0, seed: int = 0,
                   lo: int = 128, hi: int = 8192, max_rhs: int = 8,
                   pool: int = 64) -> tuple[list[Request], list[SystemSpec]]:
    """Poisson arrivals; each request draws a matrix from a pre-generated pool
    of ``pool`` matrices per kind (n log-uniform in [lo, hi]) and asks for
    rtol 1e-6 (BF16 refined) or 1e-10 (FP64) with probability 1/2, with
    1..max_rhs right-hand sides."""
    r = rng(seed, _S_MISC + 1)
    ns = log_uniform_int(r, lo, hi, 2 * pool)
    pool_specs = [SystemSpec(int(ns[i]), "spd" if i < pool else "nonsym", 1,
                             seed * 7919 + 1000 + i) for i in range(2 * pool)]
    reqs: list[Request] = []
    t = 0.0
    while True:
        t += r.exponential(1.0 / rate)
        if t >= duration:
            break
        j = int(r.integers(0, 2 * pool))
        tight = bool(r.integers(0, 2))
        base = pool_specs[j]
        spec = SystemSpec(base.n, base.kind, int(r.integers(1, max_rhs + 1)),
                          base.seed, 1e-10 if tight else 1e-6)
        reqs.append(Request(t, spec, "f64" if tight else "bf16"))
    return reqs, pool_specs
