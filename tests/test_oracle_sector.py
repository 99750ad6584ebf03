"""Pins for the oracle's sector machinery (CPU only).

Each check ties the oracle to something other than itself: Eq. (dim) (the oracle uses the App. A
polynomial instead), brute-force enumeration with itertools, the worked example and Table 1 of
Sec. 3.1, Cover's example of Sec. 3.4, the on-the-fly limit Eq. (N=L), and the general
offset/stride recipe Eq. (index), (ck), (offset), (stride) written out here from Sec. 3.2.
"""

import itertools
from math import comb

import numpy as np
import pytest

from conftest import read_golden
from oracle import OracleSector, cover_index, enumerate_lex, most_equal_partition, sector_dim
from oracle.sector import composite_key, subsystem_fields


def dim_closed_form(L, Q, n):
    """Eq. (dim): sum_k (-1)^k C(L,k) C(L-1+n-Qk, L-1)."""
    if L == 0:
        return 1 if n == 0 else 0
    return sum((-1) ** k * comb(L, k) * comb(L - 1 + n - Q * k, L - 1) for k in range(n // Q + 1))


def test_dim_matches_eq_dim():
    for Q in range(2, 7):
        for L in range(1, 16):
            for n in range(0, (Q - 1) * L + 1):
                assert sector_dim(L, Q, n) == dim_closed_form(L, Q, n), (L, Q, n)


def test_dim_binomial_q2_and_out_of_range():
    for L in range(0, 31):
        for n in range(0, L + 1):
            assert sector_dim(L, 2, n) == comb(L, n)
    assert sector_dim(5, 3, 11) == 0 and sector_dim(5, 3, -1) == 0


def test_dim_brute_force_and_printed_values():
    for Q in (2, 3, 4):
        for L in range(1, 8):
            counts = {}
            for w in itertools.product(range(Q), repeat=L):
                counts[sum(w)] = counts.get(sum(w), 0) + 1
            for n, c in counts.items():
                assert sector_dim(L, Q, n) == c
    assert sector_dim(9, 2, 4) == 126  # Sec. 3.1, Fig. 3
    # the five workloads' sector dimensions
    assert sector_dim(20, 2, 10) == 184_756
    assert sector_dim(30, 2, 15) == 155_117_520
    assert sector_dim(14, 4, 14) == 6_472_168 == dim_closed_form(14, 4, 14)
    assert sector_dim(24, 2, 12) == 2_704_156


@pytest.mark.parametrize("L,Q,N", [(6, 2, 3), (5, 3, 4), (4, 4, 5), (7, 2, 0), (7, 2, 7), (3, 5, 6)])
def test_enumerate_lex_is_itertools_order(L, Q, N):
    nb = (Q - 1).bit_length()
    ref = []
    for w in itertools.product(range(Q), repeat=L):  # itertools.product is lexicographic
        if sum(w) == N:
            v = 0
            for d in w:
                v = (v << nb) | d
            ref.append(v)
    got = enumerate_lex(L, Q, N)
    assert got.tolist() == ref


def test_partition_rule():
    assert most_equal_partition(9, 3) == [3, 3, 3]
    assert most_equal_partition(30, 2) == [15, 15]
    assert most_equal_partition(30, 3) == [10, 10, 10]
    assert most_equal_partition(30, 5) == [6, 6, 6, 6, 6]
    assert most_equal_partition(17, 2) == [9, 8]
    assert most_equal_partition(11, 4) == [3, 3, 3, 2]
    # default n_sub = ceil(Nbits L / 16), Eq. (Nopt_from_L)
    assert len(most_equal_partition(14, 0, Q=4)) == 2
    assert len(most_equal_partition(16, 0)) == 1 and len(most_equal_partition(17, 0)) == 2
    assert len(most_equal_partition(24, 0)) == 2 and len(most_equal_partition(33, 0)) == 3


def _bits(s):
    return int(s, 2)


def test_worked_example_and_table1():
    g = {}
    table1 = []
    for row in read_golden("worked_example_L9_N4.txt"):
        if row[0] == "table1":
            table1.append((row[1], int(row[2])))
        else:
            g[row[0]] = row[1:]
    L, Q, N = int(g["L"][0]), int(g["Q"][0]), int(g["N"][0])
    part = [int(v) for v in g["partition"]]
    sec = OracleSector(L, Q, N, partition=part)
    assert sec.dim == int(g["dim"][0])
    word = _bits("".join(g["state"]))
    assert sec.index_of(word) == int(g["index"][0])
    assert sec.state_at(int(g["index"][0])) == word
    # Table 1
    for pat, idx in table1:
        assert sec.local_index(_bits(pat), 3) == idx
    assert [sec.local_index(_bits(p), 3) for p in g["state"]] == [int(v) for v in g["local_index"]]
    # offsets and strides read off the sorted basis, as the figure captions describe them
    fields = subsystem_fields(sec.basis, L, Q, part)
    nA, sA = fields[0]
    nB, sB = fields[1]
    offA, offB, offC = (int(v) for v in g["offset"])
    strA, strB, strC = (int(v) for v in g["stride"])
    # offset_A: first global index whose A state has n_A = 1
    assert int(np.argmax(nA == 1)) == offA
    # stride_A: number of global states per A state inside the n_A = 1 layer
    assert int(np.sum(sA == _bits("001"))) == strA
    # c_A and c_A + c_B: where the prefixes |010> and |010>|101> start
    start_A = int(np.argmax(sA == _bits("010")))
    start_AB = int(np.argmax((sA == _bits("010")) & (sB == _bits("101"))))
    assert [start_A, start_AB] == [int(v) for v in g["prefix_start"]]
    cA, cB, cC = (int(v) for v in g["c"])
    assert start_A == cA and start_AB == cA + cB and int(g["index"][0]) == cA + cB + cC
    # offset_B inside the A = |010> layer: first state with n_B = 2, counted from the layer start
    layer = sA == _bits("010")
    assert int(np.argmax(layer & (nB == 2))) - start_A == offB
    # stride_B: states per B state with n_B = 2 inside that layer; last subsystem: 1
    assert int(np.sum(layer & (sB == _bits("011")))) == strB
    assert offC == 0 and strC == 1


def test_cover_example():
    rows = read_golden("cover_example.txt")
    S = None
    for row in rows:
        if row[0] == "S":
            S = [tuple(int(c) for c in w.split(",")) for w in row[1:]]
    for row in rows:
        if row[0] == "count":
            prefix = tuple(int(c) for c in row[1].split(","))
            assert sum(1 for s in S if s[: len(prefix)] == prefix) == int(row[2])
        if row[0] == "index":
            x = tuple(int(c) for c in row[1].split(","))
            assert cover_index(x, S) == int(row[2])
    assert [cover_index(s, S) for s in S] == list(range(len(S)))


def _key_tuples(sec):
    fields = subsystem_fields(sec.basis, sec.L, sec.Q, sec.partition)
    return [tuple((int(n[r]), int(s[r])) for n, s in fields) for r in range(sec.dim)]


@pytest.mark.parametrize("L,Q,N,part", [(9, 2, 4, [3, 3, 3]), (5, 3, 4, [2, 2, 1]), (6, 4, 7, [2, 2, 2]),
                                        (8, 2, 3, [3, 3, 2]), (7, 3, 6, [4, 3])])
def test_canonical_index_is_cover_index_over_subsystem_letters(L, Q, N, part):
    """Sec. 3.4: with letters (n_k, sigma^(k)) ordered by particle number then locally, Cover's
    formula gives the canonical index."""
    sec = OracleSector(L, Q, N, partition=part)
    S = _key_tuples(sec)
    for r in range(sec.dim):
        assert cover_index(S[r], S) == r


def _dq(l, Q, m):
    return sector_dim(l, Q, m) if m >= 0 else 0


def recipe_index(word, L, Q, N, part):
    """Eq. (index) with Eq. (ck), (offset), (stride) written out from Sec. 3.2 (test-side).

    Gamma_k is the length of the complement after P_k; the local index is the lexicographic
    rank inside the subsystem's own particle-number sector (Table 1)."""
    nb = (Q - 1).bit_length()
    digs = [(word >> (nb * (L - 1 - i))) & ((1 << nb) - 1) for i in range(L)]
    idx, lam, start = 0, 0, 0
    for k, Lk in enumerate(part):
        sub = digs[start:start + Lk]
        start += Lk
        gamma = L - start
        nk = sum(sub)
        nlow = max(0, N - lam - (Q - 1) * gamma)
        offset = sum(_dq(Lk, Q, m) * _dq(gamma, Q, N - lam - m) for m in range(nlow, nk))
        stride = _dq(gamma, Q, N - lam - nk)
        # local index: count lexicographically smaller patterns with the same digit sum
        local = 0
        acc = 0
        for pos, d in enumerate(sub):
            for q in range(d):
                local += _dq(Lk - 1 - pos, Q, nk - acc - q)
            acc += d
        idx += offset + stride * local
        lam += nk
    return idx


@pytest.mark.parametrize("L,Q,N,n_sub", [(9, 2, 4, 3), (10, 2, 5, 2), (10, 2, 4, 3), (8, 3, 7, 3),
                                          (7, 4, 9, 2), (9, 3, 5, 4), (6, 5, 10, 3), (11, 2, 5, 11),
                                          (8, 2, 4, 1), (12, 2, 6, 5)])
def test_oracle_order_matches_offset_stride_recipe(L, Q, N, n_sub):
    sec = OracleSector(L, Q, N, n_sub=n_sub)
    got = [recipe_index(int(w), L, Q, N, sec.partition) for w in sec.basis]
    assert got == list(range(sec.dim))


@pytest.mark.parametrize("L,Q,N", [(10, 2, 4), (6, 3, 5), (5, 4, 7)])
def test_limits_reduce_to_lexicographic(L, Q, N):
    """n_sub = 1 and n_sub = L both give plain lexicographic order (Sec. 3.3, 3.4)."""
    lex = enumerate_lex(L, Q, N)
    for n_sub in (1, L):
        sec = OracleSector(L, Q, N, n_sub=n_sub)
        assert np.array_equal(sec.basis, lex)


def on_the_fly_index(word, L, Q, N):
    """Eq. (N=L): contribution of site i is sum_{k < q_i} D_Q(L-1-i, N - lambda_i - k)."""
    nb = (Q - 1).bit_length()
    idx, lam = 0, 0
    for i in range(L):
        q = (word >> (nb * (L - 1 - i))) & ((1 << nb) - 1)
        for k in range(q):
            idx += _dq(L - 1 - i, Q, N - lam - k)
        lam += q
    return idx


@pytest.mark.parametrize("L,Q,N", [(12, 2, 5), (7, 3, 6), (6, 4, 8)])
def test_on_the_fly_limit(L, Q, N):
    sec = OracleSector(L, Q, N, n_sub=L)
    assert [on_the_fly_index(int(w), L, Q, N) for w in sec.basis] == list(range(sec.dim))


def test_two_subsystem_lin_table():
    """Sec. 3.3 (N = 2): index = T0[s0] + T1[s1] with T0 = c_0 and T1 the bare local index."""
    L, Q, N = 10, 2, 5
    sec = OracleSector(L, Q, N, n_sub=2)
    L0, L1 = sec.partition
    T0, T1 = {}, {}
    for r, w in enumerate(sec.basis.tolist()):
        s0, s1 = w >> L1, w & ((1 << L1) - 1)
        T1.setdefault(s1, sec.local_index(s1, L1))
        T0.setdefault(s0, r - T1[s1])
        assert T0[s0] == r - T1[s1]


def test_rank_unrank_increment_and_errors():
    sec = OracleSector(12, 3, 9, n_sub=3)
    idx = sec.index_of_many(sec.basis)
    assert np.array_equal(idx, np.arange(sec.dim))
    for r in (0, 1, sec.dim // 2, sec.dim - 2):
        assert sec.next_state(sec.state_at(r)) == sec.state_at(r + 1)
    assert sec.next_state(sec.state_at(sec.dim - 1)) == sec.state_at(0)  # wrap (Alg. 3)
    with pytest.raises(IndexError):
        sec.state_at(sec.dim)
    bad_digit = 0b11 << 2  # a digit equal to 3 >= Q
    with pytest.raises(ValueError):
        sec.index_of(bad_digit)
    with pytest.raises(ValueError):
        sec.index_of(0)  # wrong particle number
    with pytest.raises(ValueError):
        sec.index_of(int(sec.basis[0]) | (1 << 40))  # bits above L * Nbits


def test_composite_key_is_tuple_order():
    sec = OracleSector(9, 3, 7, partition=[4, 3, 2])
    words = enumerate_lex(9, 3, 7)
    keys = composite_key(words, 9, 3, [4, 3, 2])
    fields = subsystem_fields(words, 9, 3, [4, 3, 2])
    tuples = [tuple(v for n, s in fields for v in (int(n[r]), int(s[r]))) for r in range(len(words))]
    assert np.argsort(keys, kind="stable").tolist() == sorted(range(len(words)), key=lambda r: tuples[r])
    assert np.array_equal(sec.basis, words[np.argsort(keys, kind="stable")])


@pytest.mark.parametrize("L,Q,N,part", [(64, 2, 2, [16, 16, 16, 16]), (64, 2, 3, [32, 32]), (32, 4, 3, [11, 11, 10])])
def test_full_width_words_sort_by_the_key_tuple(L, Q, N, part):
    """Sectors whose words use all 64 bits (the sort key then needs more than 64 bits): the
    canonical order equals Python's sort of the words by the tuple (n_0, sigma^(0), n_1, ...)
    built digit by digit, and rank(unrank(i)) = i."""
    o = OracleSector(L, Q, N, partition=part)
    nb = (Q - 1).bit_length()

    def digits(w):
        return [(w >> (nb * (L - 1 - i))) & ((1 << nb) - 1) for i in range(L)]

    def key(w):
        d, out, s = digits(w), [], 0
        for Lk in part:
            sub = d[s:s + Lk]
            out.append(sum(sub))
            out.append(tuple(sub))
            s += Lk
        return tuple(out)

    words = sorted((int(w) for w in o.basis), key=key)
    assert [int(w) for w in o.basis] == words
    assert all(sum(digits(w)) == N for w in words[:50])
    idx = np.arange(0, o.dim, max(1, o.dim // 500))
    assert np.array_equal(o.index_of_many(o.basis[idx]), idx)


# ---------------------------------------------------------------- words wider than 64 bits ---

def _q2_words_brute(L, N):
    from itertools import combinations
    return sorted(sum(1 << (L - 1 - i) for i in c) for c in combinations(range(L), N))


def _q4_words_brute(L, N):
    """All digit strings over {0..3} with digit sum N <= 3 (N particles placed on sites with
    repetition), as Python integers, sorted."""
    from itertools import combinations_with_replacement
    return sorted({sum(1 << (2 * (L - 1 - i)) for i in c) for c in combinations_with_replacement(range(L), N)})


@pytest.mark.parametrize("L,Q,N", [(70, 2, 2), (100, 2, 3), (128, 2, 2), (33, 4, 3), (64, 4, 2)])
def test_wide_words_enumeration_matches_brute_force(L, Q, N):
    """Words of more than 64 bits are exact integers; lexicographic enumeration equals the sorted
    brute-force list of all digit strings with digit sum N, and the dimension is Eq. (dim)'s."""
    words = [int(w) for w in enumerate_lex(L, Q, N)]
    ref = _q2_words_brute(L, N) if Q == 2 else _q4_words_brute(L, N)
    assert words == ref
    assert len(words) == sector_dim(L, Q, N) == dim_closed_form(L, Q, N)


@pytest.mark.parametrize("L,Q,N,n_sub", [(70, 2, 2, 3), (66, 2, 2, 5), (33, 4, 3, 3), (128, 2, 2, 8)])
def test_wide_words_order_matches_offset_stride_recipe(L, Q, N, n_sub):
    """The canonical order of two-word states equals Eq. (index) written out in this test (on
    every state, or every 5th for the largest case), and rank(unrank(i)) = i through the binary
    search."""
    sec = OracleSector(L, Q, N, n_sub=n_sub)
    assert sec.wide
    pick = range(0, sec.dim, 5 if sec.dim > 5000 else 1)
    got = [recipe_index(int(sec.basis[r]), L, Q, N, sec.partition) for r in pick]
    assert got == list(pick)
    idx = np.arange(0, sec.dim, max(1, sec.dim // 300))
    assert np.array_equal(sec.index_of_many(sec.basis[idx]), idx)
    assert sec.next_state(int(sec.basis[-1])) == int(sec.basis[0])


def test_wide_words_cover_index_over_subsystem_letters():
    """Sec. 3.4 on a sector of 66-bit words: Cover's index over the letters (n_k, sigma^(k)) is
    the canonical index (checked on a sample of states)."""
    sec = OracleSector(66, 2, 2, partition=[22, 22, 22])
    S = _key_tuples(sec)
    for r in list(range(0, sec.dim, 97)) + [sec.dim - 1]:
        assert cover_index(S[r], S) == r


def test_wide_words_validity():
    sec = OracleSector(70, 2, 2, n_sub=3)
    good = (1 << 69) | 1
    assert sec.is_valid([good]).all()
    assert not sec.is_valid([(1 << 70) | 1]).any()  # a bit above L * Nbits
    assert not sec.is_valid([(1 << 69) | 3]).any()  # three particles
    assert sec.state_at(sec.index_of(good)) == good
