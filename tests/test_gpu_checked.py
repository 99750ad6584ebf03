"""The checked build (libdq_checked.so, -DDQ_CHECKED) on the GPU.

In that build every device rank used to gather x is compared with the sector dimension, and an
out-of-range rank raises the sector's error word instead of reading outside x. Valid operators
must therefore run with a clean error word and match the oracle to the same tolerances as the
normal build; this is checked in a fresh process (the binding picks the library when it is imported) on every
kernel family that gathers through a device rank: the general products (Q = 2 and Q = 4, FP64 and
FP32, several right-hand sides), the batched product, the term gradients and the batched rank.
"""

import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import numpy as np, torch
from paper_2407_14591_gb300 import binding as b, workloads as wl
from oracle import OracleSector, matvec as o_matvec
assert b.LIB_PATH.endswith("libdq_checked.so"), b.LIB_PATH
rng = np.random.default_rng(5)
cases = []
J = rng.uniform(0.5, 1.5, 14); h = rng.uniform(-3, 3, 14)
cases.append((14, 2, 7, 3, wl.heisenberg_terms(wl.chain_bonds(14), J, 1.0) + wl.field_terms(h), 3))
bh = [("HOP", i, j, 1.0) for i, j in wl.chain_bonds(10)] + [("U", i, -1, float(u)) for i, u in enumerate(rng.uniform(2, 6, 10))]
cases.append((10, 4, 12, 2, bh, 2))  # two right-hand sides: the general boson kernel
cases.append((10, 4, 12, 2, bh, 1))  # one: the boson panel kernel
for L, Q, N, n_sub, terms, nrhs in cases:
    s = b.make_sector(L, Q, N, n_sub); t = b.make_terms(s, terms)
    o = OracleSector(L, Q, N, partition=s.partition)
    x = rng.uniform(-1, 1, (o.dim, nrhs)).squeeze()
    ref = o_matvec(o, terms, x)
    for dt, tol in ((torch.float64, 1e-12), (torch.float32, 1e-5)):
        y = b.matvec(s, t, torch.from_numpy(x).to("cuda", dt)).double().cpu().numpy()
        assert np.linalg.norm(y - ref) <= tol * np.linalg.norm(ref), (L, Q, dt)
    s.check_device()
# batched product
LN = [(10, 5), (12, 6)]
secs = [b.make_sector(L, 2, N, 0) for L, N in LN]
tl = [wl.heisenberg_terms(wl.chain_bonds(L), 1.0, 1.0) + wl.field_terms(rng.uniform(-5, 5, L)) for L, _ in LN]
terms = [b.make_terms(s, t) for s, t in zip(secs, tl)]
xs = [torch.from_numpy(rng.uniform(-1, 1, (s.dim, 2))).cuda() for s in secs]
ys = [torch.empty_like(x) for x in xs]
b.make_batch(secs, terms, 2, torch.float64).matvec(xs, ys)
torch.cuda.synchronize()
for (L, N), s, tt, x, y in zip(LN, secs, tl, xs, ys):
    ref = o_matvec(OracleSector(L, 2, N, partition=s.partition), tt, x.cpu().numpy())
    assert np.max(np.abs(y.cpu().numpy() - ref)) <= 1e-12 * np.max(np.abs(ref))
    s.check_device()
# term gradients (each g_q = <dy, T_q x> against the oracle's T_q x) and batched rank
s = b.make_sector(14, 2, 7, 3)
o = OracleSector(14, 2, 7, partition=s.partition)
tl = wl.heisenberg_terms(wl.chain_bonds(14), 1.0, 1.0)
xn, dn = rng.uniform(-1, 1, o.dim), rng.uniform(-1, 1, o.dim)
g = b.term_grads(s, tl, torch.from_numpy(xn).cuda(), torch.from_numpy(dn).cuda()).cpu().numpy()
gref = np.array([dn @ o_matvec(o, [(k, i, j, 1.0)], xn) for k, i, j, _ in tl])
assert np.max(np.abs(g - gref)) <= 1e-12 * np.max(np.abs(gref))
idx = torch.arange(s.dim, device="cuda")
assert torch.equal(s.index_of_batch(s.state_at_batch(idx)), idx)
s.check_device()
print("CHECKED-OK")
"""


def test_checked_build_runs_clean_and_matches():
    from paper_2407_14591_gb300 import build

    build.build(checked=True)
    env = dict(os.environ, DQ_CHECKED="1", PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    res = subprocess.run([sys.executable, "-c", SCRIPT], cwd=ROOT, env=env, capture_output=True, text=True,
                         timeout=900)
    assert res.returncode == 0 and "CHECKED-OK" in res.stdout, res.stdout[-2000:] + res.stderr[-4000:]
