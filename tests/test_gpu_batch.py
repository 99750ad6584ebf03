"""The batched product (many Q = 2 sectors, several right-hand sides, one launch) on the GPU.

Checked against the oracle on small disordered chains and lattices, against the single-sector
product on the 64-chain workload, across every launch shape of the autotuner, and when replayed
from a captured CUDA graph.
"""

import numpy as np
import pytest
import torch

from oracle import OracleSector, matvec as o_matvec
from paper_2407_14591_gb300 import binding as b
from paper_2407_14591_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
DEV = "cuda"


def small_items(seed=0):
    rng = np.random.default_rng(seed)
    items = []
    for L, N in [(10, 5), (11, 4), (12, 6), (13, 5), (14, 7), (17, 8)]:
        h = rng.uniform(-5, 5, L)
        terms = wl.heisenberg_terms(wl.chain_bonds(L), 1.0, 1.0) + wl.field_terms(h)
        items.append((L, N, terms))
    nn, nnn = wl.square_bonds(4, 3)
    items.append((12, 5, wl.heisenberg_terms(nn, 1.0) + wl.heisenberg_terms(nnn, 0.5)))
    return items


@pytest.mark.parametrize("nrhs", [1, 3, 8])
def test_batch_small_vs_oracle_every_mapping(nrhs):
    """Every candidate of the autotuner (both row mappings, every launch shape) against the
    oracle; all candidates give bitwise the same y (one thread per row, fixed summation order)."""
    items = small_items(nrhs)
    secs = [b.make_sector(L, 2, N, 0) for L, N, _ in items]
    terms = [b.make_terms(s, t) for s, (_, _, t) in zip(secs, items)]
    rng = np.random.default_rng(100 + nrhs)
    xs = [rng.uniform(-1, 1, (s.dim, nrhs)) for s in secs]
    oracles = [OracleSector(L, 2, N, partition=s.partition) for s, (L, N, _) in zip(secs, items)]
    for dtype in (torch.float64, torch.float32):
        batch = b.make_batch(secs, terms, nrhs, dtype)
        xt = [torch.from_numpy(x).to(DEV, dtype).contiguous() for x in xs]
        refs = [o_matvec(o, t, x.double().cpu().numpy()) for o, (_, _, t), x in zip(oracles, items, xt)]
        first = None
        for shape in range(batch.n_shapes()):
            batch.set_shape(shape)
            yt = [torch.full_like(x, float("nan")) for x in xt]
            batch.matvec(xt, yt)
            torch.cuda.synchronize()
            for ref, y in zip(refs, yt):
                got = y.double().cpu().numpy()
                if dtype == torch.float64:
                    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref)), shape
                else:
                    assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref), shape
            if first is None:
                first = yt
            else:
                assert all(torch.equal(a, c) for a, c in zip(first, yt)), shape


@pytest.fixture(scope="module")
def workload4():
    ws = wl.batched_chains(64, 8)
    secs = [b.make_sector(w.L, 2, w.N, 0) for w in ws]
    terms = [b.make_terms(s, w.terms) for s, w in zip(secs, ws)]
    xs = wl.batched_vectors([s.dim for s in secs], 8)
    return ws, secs, terms, xs


def test_workload4_batch_equals_single_sector_products(workload4):
    ws, secs, terms, xs = workload4
    assert len(secs) == 64 and all(16 <= w.L <= 26 for w in ws)
    batch = b.make_batch(secs, terms, 8, torch.float64)
    xt = [torch.from_numpy(x).to(DEV) for x in xs]
    yt = [torch.empty_like(x) for x in xt]
    batch.matvec(xt, yt)
    torch.cuda.synchronize()
    for s, t, x, y in zip(secs, terms, xt, yt):
        ref = b.matvec(s, t, x)
        torch.cuda.synchronize()
        assert torch.max(torch.abs(y - ref)).item() <= 1e-12 * torch.max(torch.abs(ref)).item()
    # oracle on the smallest sector of the draw
    k = int(np.argmin([s.dim for s in secs]))
    o = OracleSector(ws[k].L, 2, ws[k].N, partition=secs[k].partition)
    ref = o_matvec(o, ws[k].terms, xs[k])
    got = yt[k].cpu().numpy()
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_workload4_tune_and_graph_replay(workload4):
    ws, secs, terms, xs = workload4
    batch = b.make_batch(secs, terms, 8, torch.float32)
    xt = [torch.from_numpy(x).to(DEV, torch.float32) for x in xs]
    y0 = [torch.empty_like(x) for x in xt]
    batch.matvec(xt, y0)
    torch.cuda.synchronize()
    choice = batch.tune(xt, [torch.empty_like(x) for x in xt])
    assert 0 <= choice < batch.n_shapes()
    y1 = [torch.empty_like(x) for x in xt]
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        batch.matvec(xt, y1)  # warm-up on the capture stream
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    for y in y1:
        y.zero_()
    with torch.cuda.graph(g):
        batch.matvec(xt, y1)
    g.replay()
    torch.cuda.synchronize()
    # rows are computed by one thread each in a fixed order: every launch shape gives the same bits
    for a, c in zip(y0, y1):
        assert torch.equal(a, c)


@pytest.mark.slow
def test_workload4_largest_sectors_against_oracle_rows(workload4):
    """The four largest sectors of the 64-chain draw, in the batched launch: oracle rows (gather
    reading, FP64) on the first and last 4096 rows and 2^16 random rows of each, for all eight
    right-hand sides, with FP64 and FP32 vectors (FP32 against the oracle applied to the rounded x)."""
    from oracle import matvec_rows as o_matvec_rows

    ws, secs, terms, xs = workload4
    order = np.argsort([s.dim for s in secs])[::-1][:4]
    outs = {}
    for dtype in (torch.float64, torch.float32):
        batch = b.make_batch(secs, terms, 8, dtype)
        xt = [torch.from_numpy(x).to(DEV, dtype) for x in xs]
        ys = []
        for shape in (1, 7):  # one candidate of each row mapping (block-stride rows, warp walk)
            batch.set_shape(shape)
            yt = [torch.empty_like(x) for x in xt]
            batch.matvec(xt, yt)
            torch.cuda.synchronize()
            ys.append([yt[k] for k in order])
        assert all(torch.equal(a, c) for a, c in zip(*ys))
        outs[dtype] = [(xt[k].double().cpu().numpy(), ys[0][q]) for q, k in enumerate(order)]
        del batch
    for q, k in enumerate(order):
        w, s = ws[k], secs[k]
        o = OracleSector(w.L, 2, w.N, partition=s.partition)
        rng = np.random.default_rng(int(k))
        rows = np.unique(np.concatenate([np.arange(4096), rng.choice(s.dim, 1 << 16, replace=False),
                                         np.arange(s.dim - 4096, s.dim)]))
        for dtype in (torch.float64, torch.float32):
            xin, y = outs[dtype][q]
            ref = o_matvec_rows(o, w.terms, xin, rows)
            got = y[torch.from_numpy(rows).to(DEV)].double().cpu().numpy()
            if dtype == torch.float64:
                assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref)), (k, w.L, w.N)
            else:
                assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref), (k, w.L, w.N)
        del o
