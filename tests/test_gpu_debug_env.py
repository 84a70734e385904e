"""FEI_DEBUG=1 in the environment: every launch of the library is followed
by a wait on its stream and an error check (skipped while a plan captures
its CUDA graph).  The same calls must succeed and give the same results,
bit for bit, as without it.  The variable is read once per process, so
each setting runs in a child process."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import hashlib
import numpy as np
import torch
from paper_1310_1194_gb300 import api, inputs
torch.cuda.set_stream(torch.cuda.Stream())
digests = []
def add(*ts):
    h = hashlib.sha256()
    for t in ts:
        h.update(t.detach().cpu().numpy().tobytes())
    digests.append(h.hexdigest()[:16])
w = inputs.workload("mixed", n_max=300)
g = [torch.from_numpy(np.ascontiguousarray(w[k])).cuda() for k in ("geom", "K", "b", "c", "f")]
deg = torch.from_numpy(np.ascontiguousarray(w["degree"])).to(torch.int32).cuda()
A, b, st, lay = api.fei_integrate(*g, degree=deg, precision="tc_f16x3")
add(A, b, st)
plan = api.Plan(max_elem=300, precision="tc_f16x3")
A2, b2, st2, _ = plan.execute(*g, degree=deg, layout=lay)
plan.execute(*g, degree=deg, layout=lay, out=(A2, b2, st2))  # graph replay
add(A2, b2, st2)
w4 = inputs.workload("p4", n_max=50)
g4 = [torch.from_numpy(np.ascontiguousarray(w4[k])).cuda() for k in ("geom", "K", "b", "c", "f")]
A4, b4, st4, _ = api.fei_integrate(*g4, p=4, precision="fp32")
add(A4, b4)
gA = torch.ones_like(A4, dtype=torch.float64)
gb = torch.ones_like(b4, dtype=torch.float64)
add(*api.fei_integrate_backward(*g4, gA, gb, p=4, precision="fp64"))
l2g, nd = inputs.dof_map(w)
asm = api.Assembly(l2g, nd, degree=w["degree"])
add(*asm.integrate_assemble(*g, precision="fp64", degree=deg))
torch.cuda.synchronize()
print("DIGEST", " ".join(digests))
'''


def run(debug):
    env = dict(os.environ)
    env.pop("FEI_DEBUG", None)
    if debug:
        env["FEI_DEBUG"] = "1"
    env["PYTHONPATH"] = ROOT + os.pathsep + env.get("PYTHONPATH", "")
    r = subprocess.run([sys.executable, "-c", SCRIPT], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    return [x for x in r.stdout.splitlines() if x.startswith("DIGEST")][0]


def test_debug_mode_same_results():
    parts = ("integrate", "plan", "uniform", "adjoint", "assembly")
    on, off = run(True).split()[1:], run(False).split()[1:]
    assert dict(zip(parts, on)) == dict(zip(parts, off))
