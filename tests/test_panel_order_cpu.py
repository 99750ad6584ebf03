"""The ordering facts the panel products rest on, checked on the oracle's canonical order (CPU).

The canonical order sorts by the key (n_0, sigma0, ..., n_{K-1}, sigma_{K-1}) (Sec. 3.1-3.2), so
fixing the leading subsystems' entries leaves a contiguous range of indices. The panel kernels use
two consequences, both checked here on the oracle's explicit sorted list (which shares nothing
with the library):
- the rows that share the pattern of all subsystems but the last two form one contiguous range of
  D_Q(L_tail, n_tail) rows, and the sequence of tail patterns in it depends only on the tail's
  particle number n_tail (the tail form of the panel kernel tabulates it once per n_tail);
- with two subsystems, the rows of one P_0 pattern are contiguous and ordered by P_1's own
  lexicographic order (Lin's two tables, Sec. 3.3), for any Q (the boson panel kernel).
"""

import numpy as np
import pytest

from oracle import OracleSector, sector_dim


def tail_runs(o, tail_sites):
    """Group the canonical basis by the word above the low tail bits; returns, per group in
    order of appearance, (first index, prefix word, tail words)."""
    tb = o.nb * tail_sites
    words = np.array([int(w) for w in o.basis], dtype=object)
    prefix = [w >> tb for w in words]
    tails = [w & ((1 << tb) - 1) for w in words]
    runs = []
    for i, p in enumerate(prefix):
        if runs and runs[-1][1] == p:
            runs[-1][2].append(tails[i])
        else:
            runs.append((i, p, [tails[i]]))
    return runs


def digit_sum(w, nb, sites):
    return sum((w >> (nb * k)) & ((1 << nb) - 1) for k in range(sites))


@pytest.mark.parametrize("L,Q,N,n_sub", [(12, 2, 6, 4), (15, 2, 7, 5), (13, 2, 5, 3), (12, 2, 12, 6), (12, 2, 1, 4),
                                         (9, 3, 8, 3), (8, 4, 9, 4)])
def test_prefix_blocks_are_contiguous_with_one_tail_order_per_particle_number(L, Q, N, n_sub):
    o = OracleSector(L, Q, N, n_sub=n_sub)
    part = o.partition
    tail = part[-2] + part[-1]
    runs = tail_runs(o, tail)
    # every prefix appears in exactly one run: the rows sharing it are contiguous
    assert len({p for _, p, _ in runs}) == len(runs)
    order_of = {}
    for start, p, tails in runs:
        n_tail = N - digit_sum(p, o.nb, L - tail)
        assert all(digit_sum(t, o.nb, tail) == n_tail for t in tails)
        assert len(tails) == sector_dim(tail, Q, n_tail)
        # the same tail order behind every prefix with this tail particle number
        assert order_of.setdefault(n_tail, tails) == tails
    # and that order is the two-subsystem canonical order of the tail on its own
    for n_tail, tails in order_of.items():
        ot = OracleSector(tail, Q, n_tail, partition=part[-2:])
        assert [int(w) for w in ot.basis] == tails


@pytest.mark.parametrize("L,Q,N", [(8, 4, 8), (7, 4, 10), (8, 3, 6), (6, 8, 9), (8, 4, 0), (8, 4, 24)])
def test_two_subsystem_panels_follow_the_last_subsystems_own_order(L, Q, N):
    o = OracleSector(L, Q, N, n_sub=2)
    L1 = o.partition[1]
    runs = tail_runs(o, L1)
    assert len({p for _, p, _ in runs}) == len(runs)
    for _, p, tails in runs:
        assert tails == sorted(tails)  # P_1's lexicographic order inside its block
        n1 = N - digit_sum(p, o.nb, L - L1)
        assert len(tails) == sector_dim(L1, Q, n1)
