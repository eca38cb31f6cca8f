"""Host-loop mode (LS_HOSTLOOP=1: every solver loop driven from the host with
the same kernels and arguments, the mode the ncu captures use) gives results
bit-identical to graph mode for every solver.  The mode is read once per
process, so the host-loop side runs in a child process."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import json, sys
import numpy as np, torch
sys.path.insert(0, %r)
from paper_1511_07207_gb300 import binding as B, inputs
dev = torch.device("cuda:0")
ctx = B.ls_create(0, torch.cuda.current_stream(dev))
n, s = 300, 3
out = {}
Aspd = inputs.spd_matrix(n, 0.1, seed=1)
Ans = inputs.nonsym_matrix(n, seed=2)
for name, A, fn, kw in (("cg", Aspd, B.ls_cg_solve, {}), ("gmres", Ans, B.ls_gmres_solve, {"restart": 8}),
                        ("bicgstab", Ans, B.ls_bicgstab_solve, {}), ("jacobi", Ans, B.ls_jacobi_solve, {}),
                        ("gauss_seidel", Ans, B.ls_gauss_seidel_solve, {})):
    b = torch.from_numpy(A @ inputs.solution(n, seed=3)).to(dev)
    x = torch.zeros(n, dtype=torch.float64, device=dev)
    st, info = fn(ctx, torch.from_numpy(A).to(dev), b, x, B.make_opts(rtol=1e-10, **kw))
    out[name] = [st, info["iters"], x.cpu().numpy().tolist()]
for name, A, fn, kw in (("block_cg", Aspd, B.ls_block_cg_solve, {}),
                        ("block_gmres", Ans, B.ls_block_gmres_solve, {"restart": 4})):
    Bm = A @ inputs.solution(n, seed=4, nrhs=s)
    Bd = torch.from_numpy(Bm.T.copy()).to(dev).t()
    X = torch.zeros((s, n), dtype=torch.float64, device=dev).t()
    st, info = fn(ctx, torch.from_numpy(A).to(dev), Bd, X, B.make_opts(rtol=1e-10, **kw))
    out[name] = [st, info["iters"], X.cpu().numpy().tolist()]
B.ls_destroy(ctx)
print("RESULT " + json.dumps(out))
'''


def _run(hostloop):
    env = dict(os.environ)
    env.pop("LS_HOSTLOOP", None)
    if hostloop:
        env["LS_HOSTLOOP"] = "1"
    p = subprocess.run([sys.executable, "-c", CHILD % ROOT], env=env, capture_output=True, text=True,
                       timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    line = [l for l in p.stdout.splitlines() if l.startswith("RESULT ")][-1]
    return json.loads(line[len("RESULT "):])


def test_hostloop_matches_graph_mode():
    graph, host = _run(False), _run(True)
    assert graph.keys() == host.keys()
    for name in graph:
        sg, ig, xg = graph[name]
        sh, ih, xh = host[name]
        assert sg == sh == 0, name
        assert ig == ih, name
        assert np.array_equal(np.array(xg), np.array(xh)), name
