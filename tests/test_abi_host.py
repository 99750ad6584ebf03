"""The C-ABI library on the host (CPU only, no kernel launches).

Checks that libdq.so loads and exports every function declared in include/dq.h, that the host
sector builder (Eq. (dim), Eq. (offset), Eq. (stride), local tables from Alg. 1) and the host
forms of get_index / increment / get_state (Alg. 2-4) agree bit-exactly with the oracle's sorted
list, and that invalid arguments are rejected with the documented status codes. Without a CUDA
device the sector keeps host tables only and every device call fails loudly.
"""

import ctypes
import os
import re

import numpy as np
import pytest

from oracle import OracleSector, sector_dim
from paper_2407_14591_gb300 import binding as b
from paper_2407_14591_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(dq_\w+)\s*\(", text)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    names = declared_functions()
    assert "dq_matvec" in names and "dq_make_sector" in names
    lib = ctypes.CDLL(b.LIB_PATH)
    for name in names:
        assert hasattr(lib, name), name
    assert set(b.EXPORTED) <= set(names)


CASES = [(9, 2, 4, 3), (10, 2, 5, 2), (12, 2, 6, 5), (11, 2, 4, 11), (8, 3, 7, 3), (7, 4, 9, 2), (9, 3, 5, 4),
         (6, 5, 10, 3), (5, 16, 20, 2), (12, 2, 0, 3), (12, 2, 12, 2), (11, 4, 11, 2), (16, 2, 8, 1), (13, 3, 11, 0),
         (64, 2, 2, 4), (64, 2, 3, 3), (32, 4, 3, 3),
         (70, 2, 2, 5), (33, 4, 3, 3), (128, 2, 2, 8), (100, 2, 2, 0), (42, 8, 2, 0)]  # two-word states


@pytest.mark.parametrize("L,Q,N,n_sub", CASES)
def test_host_rank_unrank_increment_match_oracle(L, Q, N, n_sub):
    s = b.make_sector(L, Q, N, n_sub)
    o = OracleSector(L, Q, N, partition=s.partition)
    assert s.dim == o.dim == sector_dim(L, Q, N)
    rows = range(o.dim) if o.dim <= 3000 else np.random.default_rng(L * Q + N).choice(o.dim, 3000, replace=False)
    for r in rows:
        w = int(o.basis[r])
        assert s.state_at(int(r)) == w
        assert s.index_of(w) == r
        assert s.next_state(w) == int(o.basis[(r + 1) % o.dim])


def test_partition_and_default_n_sub():
    assert b.make_sector(30, 2, 15, 2).partition == [15, 15]
    assert b.make_sector(30, 2, 15, 3).partition == [10, 10, 10]
    assert b.make_sector(30, 2, 15, 5).partition == [6] * 5
    assert b.make_sector(17, 2, 8, 0).partition == [9, 8]  # ceil(17/16) = 2, longer part first
    assert b.make_sector(14, 4, 14, 0).partition == [7, 7]
    assert b.make_sector(16, 2, 8, 0).partition == [16]


def test_workload_dimensions():
    assert b.make_sector(20, 2, 10, 2).dim == 184_756
    assert b.make_sector(30, 2, 15, 2).dim == 155_117_520
    assert b.make_sector(14, 4, 14, 2).dim == 6_472_168
    assert b.make_sector(24, 2, 12, 2).dim == 2_704_156
    assert b.make_sector(64, 2, 32, 4).dim == sector_dim(64, 2, 32)


def test_argument_errors():
    for args in [(0, 2, 0, 1), (10, 1, 3, 1), (10, 17, 3, 1), (129, 2, 3, 9), (65, 4, 3, 5), (10, 2, 11, 2),
                 (10, 2, -1, 2), (10, 2, 5, 11), (10, 2, 5, -1), (128, 2, 2, 65)]:
        with pytest.raises(b.DQError) as e:
            b.make_sector(*args)
        assert e.value.code == b.DQ_EINVAL
    with pytest.raises(b.DQError) as e:
        b.make_sector(60, 2, 30, 1)  # one subsystem of 60 bits has no table
    assert e.value.code == b.DQ_ERANGE
    s = b.make_sector(10, 3, 7, 2)
    with pytest.raises(b.DQError) as e:
        s.state_at(s.dim)
    assert e.value.code == b.DQ_EINDEX
    for bad in (0, 0b11 << 4, 1 << 20, 0b01_01_01_01_01_01_01 | (0b11 << 18)):
        with pytest.raises(b.DQError) as e:
            s.index_of(bad)
        assert e.value.code == b.DQ_ESTATE
    with pytest.raises(b.DQError) as e:
        s.next_state(0)
    assert e.value.code == b.DQ_ESTATE


def test_terms_validation():
    s2 = b.make_sector(8, 2, 4, 2)
    s4 = b.make_sector(6, 4, 6, 2)
    b.make_terms(s2, wl.heisenberg_terms(wl.chain_bonds(8), 1.0) + [("HOP", 0, 3, 1.0), ("U", 2, -1, 1.0)])
    b.make_terms(s4, [("HOP", 0, 1, 1.0), ("U", 2, -1, 4.0), ("NN", 1, 2, 0.5), ("N", 0, -1, 1.0)])
    for terms, sec in [([("XY", 0, 0, 1.0)], s2), ([("ZZ", 0, 8, 1.0)], s2), ([("Z", -1, 0, 1.0)], s2),
                       ([("XY", 0, 1, 1.0)], s4), ([(9, 0, 1, 1.0)], s2), ([("HOP", 1, 1, 1.0)], s4),
                       ([("N", 0, -1, float("nan"))], s2)]:
        with pytest.raises(b.DQError) as e:
            b.make_terms(sec, terms)
        assert e.value.code == b.DQ_EINVAL


def test_device_calls_fail_loudly_without_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    s = b.make_sector(8, 2, 4, 2)
    t = b.make_terms(s, wl.heisenberg_terms(wl.chain_bonds(8), 1.0))
    lib = b.lib()
    x = ctypes.c_void_p(0x1000)
    y = ctypes.c_void_p(0x100000)
    rc = lib.dq_matvec(s.handle, t.handle, x, y, b.DQ_F64, 1, None)
    assert rc == b.DQ_ECUDA and b"no CUDA device" in lib.dq_last_error()
    rc = lib.dq_state_at_batch(s.handle, x, y, 4, None)
    assert rc == b.DQ_ECUDA


def test_timing_hooks_without_products():
    """dq_timing_*: enabling clears the record; with no product call nothing is timed or counted."""
    b.timing_enable(True)
    assert b.timing_read() == (0.0, 0, 0)
    b.timing_enable(False)
    assert b.timing_read() == (0.0, 0, 0)


def test_two_word_forms():
    """States wider than 64 bits: the one-word functions refuse the sector (DQ_EINVAL) and the
    two-word ones serve it; on a one-word sector the two-word forms equal the one-word ones."""
    lib = b.lib()
    w = b.make_sector(70, 2, 2, 5)
    out = ctypes.c_uint64()
    assert lib.dq_state_at(w.handle, ctypes.c_uint64(0), ctypes.byref(out)) == b.DQ_EINVAL
    assert b"two-word" in lib.dq_last_error()
    assert lib.dq_index_of(w.handle, ctypes.c_uint64(3), ctypes.byref(out)) == b.DQ_EINVAL
    assert lib.dq_state_at_batch(w.handle, ctypes.c_void_p(16), ctypes.c_void_p(32), 1, None) == b.DQ_EINVAL
    top = (1 << 69) | (1 << 68)  # both particles on the first two sites: the last state
    assert w.index_of(top) == w.dim - 1 and w.state_at(w.dim - 1) == top
    assert w.next_state(top) == w.state_at(0) == 0b11
    with pytest.raises(b.DQError) as e:
        w.index_of((1 << 70) | 1)
    assert e.value.code == b.DQ_ESTATE
    n = b.make_sector(20, 2, 10, 2)
    st2 = (ctypes.c_uint64 * 2)()
    for i in (0, 17, n.dim - 1):
        assert lib.dq_state_at2(n.handle, ctypes.c_uint64(i), st2) == b.DQ_OK
        assert st2[1] == 0 and st2[0] == n.state_at(i)
        assert lib.dq_index_of2(n.handle, st2, ctypes.byref(out)) == b.DQ_OK and out.value == i


def test_cluster_terms_host_side():
    """App. C clusters: every term lies inside one cluster of at most m sites, the clusters cover
    the lattice, and invalid cluster sizes are refused."""
    L = 30
    terms = wl.heisenberg_terms(wl.chain_bonds(L), 1.0) + wl.field_terms(np.linspace(-1, 1, L))
    s = b.make_sector(L, 2, 15, 2)
    t = b.make_cluster_terms(s, terms, 11)
    assert t.path == "cluster"
    clusters, entries = t.clusters()
    assert all(len(c) <= 11 for c in clusters) and 3 <= len(clusters) <= 4
    assert sorted(set(x for c in clusters for x in c)) == list(range(L))
    for kind, i, j, _ in terms:
        sites = {i} if j < 0 else {i, j}
        assert any(sites <= set(c) for c in clusters)
    assert entries >= len(clusters)  # at least the diagonal of every cluster
    for m in (1, 13):
        with pytest.raises(b.DQError) as e:
            b.make_cluster_terms(s, terms, m)
        assert e.value.code == b.DQ_EINVAL
    s4 = b.make_sector(8, 4, 8, 2)
    with pytest.raises(b.DQError):
        b.make_cluster_terms(s4, [("HOP", 0, 1, 1.0)], 7)  # 7 sites of 2 bits > 12 bits
    t4 = b.make_cluster_terms(s4, [("HOP", i, (i + 1) % 8, 1.0) for i in range(8)], 6)
    assert all(len(c) <= 6 for c in t4.clusters()[0])
