"""The tile-shape autotuner on the GPU: ls_autotune times the candidates of
the batched engine (task widths 256 / 512 / 1024 columns, tensor-core or
FP32-pipe products), writes a cache that ls_tune_load reads back, and the
engine then uses the tuned shapes.  Every tile shape is a valid way of
computing the same block products, so a batch solved with the tuned, the
default and a forced alternative shape reaches the FP64 tolerance in each
case and agrees with the oracle within the residual bound; with a fixed
cache the results are bitwise reproducible."""
import json

import numpy as np
import pytest
import torch

from paper_1511_07207_gb300 import binding as B
from paper_1511_07207_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _defaults_after(lslib):
    yield
    B.ls_tune_reset()


def _batch(gpu, specs):
    arrays, systems = [], []
    for sp in specs:
        A = sp.matrix()
        Bm = A @ sp.solution()
        Ad = torch.from_numpy(A).to(gpu)
        Bd = torch.from_numpy(np.asfortranarray(Bm)).to(gpu).T.contiguous().T
        Xd = torch.zeros((sp.n, sp.nrhs), dtype=torch.float64, device=gpu).T.contiguous().T
        method = B.LS_METHOD_CG if sp.kind == "spd" else B.LS_METHOD_GMRES
        systems.append(B.make_system(method, Ad, Bd, Xd, B.make_opts(rtol=1e-10, restart=30)))
        arrays.append((A, Bm, Xd))
    return arrays, systems


SPECS = [inputs.SystemSpec(n, kind, s, seed) for (n, kind, s, seed) in
         [(1100, "spd", 32, 41), (900, "nonsym", 20, 42), (1700, "spd", 12, 43), (600, "spd", 5, 44)]]


def _solve_and_check(ctx, gpu, oracle):
    arrays, systems = _batch(gpu, SPECS)
    st, infos = B.ls_batch_solve(ctx, systems)
    assert st == B.LS_OK
    out = []
    for (A, Bm, Xd), sp, info in zip(arrays, SPECS, infos):
        assert info["status"] == B.LS_OK, sp
        X = Xd.cpu().numpy()
        R = Bm - A @ X
        assert np.all(np.linalg.norm(R, axis=0) <= 1.0000001e-10 * np.linalg.norm(Bm, axis=0)), sp
        inv = 1.0 / np.linalg.svd(A, compute_uv=False)[-1]
        for j in (0, sp.nrhs - 1):
            ref = (oracle.cg(A, Bm[:, j], rtol=1e-10) if sp.kind == "spd"
                   else oracle.gmres(A, Bm[:, j], m=30, rtol=1e-10))
            bound = inv * (np.linalg.norm(R[:, j]) + np.linalg.norm(oracle.residual(A, Bm[:, j], ref["x"])))
            assert np.max(np.abs(X[:, j] - ref["x"])) <= bound, (sp, j)
        out.append(X)
    return out


def test_autotune_writes_a_cache_the_engine_uses(ctx, gpu, oracle, tmp_path):
    path = str(tmp_path / "tune.json")
    assert B.ls_autotune(ctx, path, B.LS_TUNE_QUICK) == B.LS_OK
    doc = json.load(open(path))
    sms = torch.cuda.get_device_properties(gpu).multi_processor_count
    assert doc["format"] == "ls-tune-1" and doc["sms"] == sms
    keys = {(e["bucket"], e["sp"]) for e in doc["entries"]}
    assert keys == {(9, 16), (9, 32), (10, 16), (10, 32)}
    for e in doc["entries"]:
        assert e["ks32"] in (256, 512, 1024) and e["tc"] in (0, 1) and e["ms"] > 0
        n = 3 << (e["bucket"] - 1)
        assert B.ls_tune_lookup(n, e["sp"], sms) == (B.LS_OK, e["ks32"], e["tc"])
    tuned = _solve_and_check(ctx, gpu, oracle)
    again = _solve_and_check(ctx, gpu, oracle)
    assert all(np.array_equal(a, b) for a, b in zip(tuned, again))
    # reading the file back gives the same choices and the same bits
    B.ls_tune_reset()
    assert B.ls_tune_load(path) == B.LS_OK
    assert all(np.array_equal(a, b) for a, b in zip(tuned, _solve_and_check(ctx, gpu, oracle)))
    # the defaults are valid too
    B.ls_tune_reset()
    _solve_and_check(ctx, gpu, oracle)


def test_forced_alternative_shapes_reach_the_tolerance(ctx, gpu, oracle, tmp_path):
    sms = torch.cuda.get_device_properties(gpu).multi_processor_count
    entries = [{"bucket": b, "sp": sp, "ks32": ks, "tc": tc, "ms": 1.0}
               for b, ks in ((9, 256), (10, 1024)) for sp, tc in ((8, 0), (16, 0), (32, 1))]
    path = tmp_path / "forced.json"
    path.write_text(json.dumps({"format": "ls-tune-1", "sms": sms, "precision": "fp32", "entries": entries}))
    assert B.ls_tune_load(str(path)) == B.LS_OK
    assert B.ls_tune_lookup(1100, 32, sms) == (B.LS_OK, 1024, 1)
    _solve_and_check(ctx, gpu, oracle)
