"""Oracle for the particle-number sector: dimension, enumeration, canonical order, rank/unrank.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``): plain, slow, obviously correct, FP64 and
exact integers throughout; it shares no code with the CUDA path.

Conventions (written from the paper):

* A basis state of L sites with local dimension Q is a digit string (sigma_0, ..., sigma_{L-1}),
  sigma_i in {0..Q-1}; its particle number is the digit sum (Sec. 2.1, Eq. (nup)).
* It is stored in one integer word with Nbits = ceil(log2 Q) bits per site, site 0 in the most
  significant digit (Sec. 4.2, the |3;2;1;0> -> 11100100 = 228 example). With this layout the
  integer order of the words is the lexicographic order of the digit strings. Words of up to 64
  bits are numpy uint64; wider words (L * Nbits up to 128; the paper's state class holds as many
  words as the sites need, Sec. 4.1) are exact Python integers in object arrays (small sectors).
* The lattice is split into n_sub consecutive subsystems P_0 .. P_{n_sub-1} (Sec. 3).
* Canonical order (Sec. 3.1 and Sec. 3.2): P_{n_sub-1} varies fastest; each subsystem's states are
  ordered first by their own particle number n_k, then by a local order inside that sector. The
  paper leaves the local order free; Table 1 orders it lexicographically (001, 010, 100 and
  011, 101, 110), and that is the order used here. So the canonical order is the sort of the
  sector's states by the key (n_0, sigma^(0), n_1, sigma^(1), ..., n_{K-1}, sigma^(K-1)), each
  sigma^(k) compared as a digit string with its first site most significant.

The oracle realises that definition literally: it enumerates the whole sector in lexicographic
order, sorts it by the key, ranks by binary search in the sorted keys and unranks by indexing.
It never uses offsets, strides or Eq. (dim).
"""

from __future__ import annotations

import math

import numpy as np

__all__ = [
    "nbits_for",
    "sector_dim",
    "most_equal_partition",
    "enumerate_lex",
    "canonical_basis",
    "cover_index",
    "OracleSector",
]


def nbits_for(Q: int) -> int:
    """Bits per site, Nbits = ceil(log2 Q) (Sec. 4.2)."""
    if Q < 2:
        raise ValueError("Q must be >= 2")
    return (Q - 1).bit_length()


def sector_dim(L: int, Q: int, N: int) -> int:
    """D_Q(L, N) as the coefficient of x^N in (1 + x + ... + x^(Q-1))^L (App. A).

    Computed by multiplying the polynomial out with exact Python integers; Eq. (dim) (the
    alternating binomial sum) is deliberately not used here.
    """
    if L < 0 or Q < 2:
        raise ValueError("need L >= 0 and Q >= 2")
    poly = [1]
    for _ in range(L):
        nxt = [0] * (len(poly) + Q - 1)
        for p, c in enumerate(poly):
            if c:
                for q in range(Q):
                    nxt[p + q] += c
        poly = nxt
    return poly[N] if 0 <= N < len(poly) else 0


def most_equal_partition(L: int, n_sub: int, Q: int = 2) -> list[int]:
    """Most-equal split of L sites into n_sub consecutive parts (Sec. 4.3).

    Parts have length ceil(L/n_sub) or floor(L/n_sub); the paper does not say which parts are
    the longer ones, and this reading puts the (L mod n_sub) longer parts first. n_sub = 0 asks
    for the paper's default number of subsystems ceil(Nbits * L / 16) (Eq. (Nopt_from_L)).
    """
    if n_sub == 0:
        n_sub = max(1, math.ceil(nbits_for(Q) * L / 16))
    if not 1 <= n_sub <= L:
        raise ValueError("need 1 <= n_sub <= L")
    base, extra = divmod(L, n_sub)
    return [base + 1 if k < extra else base for k in range(n_sub)]


def _site_shift(L: int, nb: int, i: int) -> int:
    """Bit position of site i's digit (site 0 most significant)."""
    return nb * (L - 1 - i)


def _int_of(words: np.ndarray, v: int):
    """v as an operand for the word array: np.uint64 for uint64 words, a Python int for
    exact-integer (object) words."""
    return int(v) if words.dtype == object else np.uint64(v)


def site_digit(words: np.ndarray, L: int, Q: int, i: int) -> np.ndarray:
    """Digit of site i for every word (vectorised)."""
    nb = nbits_for(Q)
    return ((words >> _int_of(words, _site_shift(L, nb, i))) & _int_of(words, (1 << nb) - 1)).astype(np.int64)


def enumerate_lex(L: int, Q: int, N: int) -> np.ndarray:
    """All digit strings of length L over {0..Q-1} with digit sum N, in lexicographic order.

    Plain lexicographic counting: the strings are grown site by site from site 0, each prefix
    being followed by its extensions with digit 0, 1, ..., Q-1 in that order, and prefixes that
    can no longer reach the sum N are dropped. Returned as packed words (site 0 most
    significant), ascending.
    """
    nb = nbits_for(Q)
    if L * nb > 128:
        raise ValueError("L * Nbits must be <= 128")
    wide = L * nb > 64
    dt = object if wide else np.uint64
    if not 0 <= N <= (Q - 1) * L:
        return np.zeros(0, dtype=dt)
    words = np.zeros(1, dtype=dt)
    if wide:
        words[0] = 0
    sums = np.zeros(1, dtype=np.int64)
    digits = np.array([int(d) for d in range(Q)], dtype=object) if wide else np.arange(Q, dtype=np.uint64)
    shift = int(nb) if wide else np.uint64(nb)
    for i in range(L):
        remaining = L - 1 - i
        words = ((words[:, None] << shift) | digits[None, :]).ravel()
        sums = (sums[:, None] + np.arange(Q, dtype=np.int64)[None, :]).ravel()
        keep = (sums <= N) & (sums + (Q - 1) * remaining >= N)
        words, sums = words[keep], sums[keep]
    assert np.all(sums == N)
    return words


def _subsystem_starts(part: list[int]) -> list[int]:
    starts, s = [], 0
    for Lk in part:
        starts.append(s)
        s += Lk
    return starts


def subsystem_fields(words: np.ndarray, L: int, Q: int, part: list[int]):
    """For each subsystem k: (n_k, sigma^(k)) for every word.

    sigma^(k) is the integer of P_k's digits with its first site most significant, so integer
    order equals the lexicographic order of P_k's digit string.
    """
    nb = nbits_for(Q)
    out = []
    for k, (s, Lk) in enumerate(zip(_subsystem_starts(part), part)):
        low_shift = nb * (L - s - Lk)
        sig = (words >> _int_of(words, low_shift)) & _int_of(words, (1 << (nb * Lk)) - 1)
        n_k = np.zeros(words.shape, dtype=np.int64)
        for i in range(s, s + Lk):
            n_k += site_digit(words, L, Q, i)
        out.append((n_k, sig))
    return out


def composite_key(words: np.ndarray, L: int, Q: int, part: list[int]) -> np.ndarray:
    """Pack the sort key (n_0, sigma^(0), ..., n_{K-1}, sigma^(K-1)) into one integer per word.

    Each n_k gets bit_length((Q-1) L_k) bits and each sigma^(k) Nbits L_k bits, most significant
    field first, so integer order of the packed key is the tuple order. The key is a uint64 when
    it fits in 64 bits; otherwise (words of up to 64 bits plus the n_k fields) it is an array of
    exact Python integers, which sort and binary-search the same way (small sectors only).
    """
    nb = nbits_for(Q)
    widths = []
    for Lk in part:
        widths.append(((Q - 1) * Lk).bit_length())
        widths.append(nb * Lk)
    if sum(widths) > 64:
        key = np.zeros(words.shape, dtype=object)
        for (n_k, sig), (wn, ws) in zip(subsystem_fields(words, L, Q, part), zip(widths[0::2], widths[1::2])):
            key = (key << wn) | np.array([int(v) for v in n_k.ravel()], dtype=object).reshape(words.shape)
            key = (key << ws) | np.array([int(v) for v in sig.ravel()], dtype=object).reshape(words.shape)
        return key
    key = np.zeros(words.shape, dtype=np.uint64)
    for (n_k, sig), (wn, ws) in zip(subsystem_fields(words, L, Q, part), zip(widths[0::2], widths[1::2])):
        key = (key << np.uint64(wn)) | n_k.astype(np.uint64)
        key = (key << np.uint64(ws)) | sig.astype(np.uint64)
    return key


def canonical_basis(L: int, Q: int, N: int, part: list[int]):
    """The sector in canonical order: (sorted words, their packed keys).

    Lexicographic enumeration followed by a stable sort on the subsystem key (Sec. 3.1-3.2).
    """
    words = enumerate_lex(L, Q, N)
    keys = composite_key(words, L, Q, part)
    order = np.argsort(keys, kind="stable")
    return words[order], keys[order]


def cover_index(x, S) -> int:
    """Cover's enumerative index of word x in the set S (Sec. 3.4, Eq. (cover)).

    index(x) = sum_k sum_{l < x_k} n_S(x_0, ..., x_{k-1}, l), where n_S(prefix) counts the
    elements of S that start with prefix. Letters may be any mutually comparable values (ints,
    or tuples such as (n_k, sigma^(k))). Pure Python, for small sets only.
    """
    x = tuple(x)
    S = [tuple(s) for s in S]
    total = 0
    for k in range(len(x)):
        prefix = x[:k]
        total += sum(1 for s in S if s[:k] == prefix and s[k] < x[k])
    return total


class OracleSector:
    """One particle-number sector in canonical order, held as an explicit sorted list."""

    def __init__(self, L: int, Q: int, N: int, n_sub: int = 0, partition: list[int] | None = None):
        nb = nbits_for(Q)
        if L < 1 or L * nb > 128:
            raise ValueError("need 1 <= L and L * Nbits <= 128")
        if not 0 <= N <= (Q - 1) * L:
            raise ValueError("need 0 <= N <= (Q-1) L")
        self.L, self.Q, self.N, self.nb = L, Q, N, nb
        self.partition = list(partition) if partition is not None else most_equal_partition(L, n_sub, Q)
        if sum(self.partition) != L or min(self.partition) < 1:
            raise ValueError("partition must cover the L sites with non-empty parts")
        self.basis, self.keys = canonical_basis(L, Q, N, self.partition)

    @classmethod
    def from_arrays(cls, L: int, Q: int, N: int, partition: list[int], basis: np.ndarray, keys: np.ndarray):
        """The same sector from the canonical basis and keys of an instance built earlier (for
        example in another process, shared through shared memory): nothing is enumerated again."""
        self = cls.__new__(cls)
        self.L, self.Q, self.N, self.nb = L, Q, N, nbits_for(Q)
        self.partition = list(partition)
        self.basis, self.keys = basis, keys
        return self

    @property
    def dim(self) -> int:
        return int(self.basis.shape[0])

    def digits(self, words: np.ndarray | None = None) -> np.ndarray:
        """(n, L) array of site digits (small sectors only)."""
        w = self.basis if words is None else self.words_array(words)
        return np.stack([site_digit(w, self.L, self.Q, i) for i in range(self.L)], axis=1)

    @property
    def wide(self) -> bool:
        """Words are wider than 64 bits (exact Python integers)."""
        return self.L * self.nb > 64

    def words_array(self, words) -> np.ndarray:
        """Words as this sector stores them (uint64, or Python integers when wide)."""
        if self.wide:
            return np.array([int(v) for v in np.asarray(words, dtype=object).ravel()], dtype=object).reshape(
                np.shape(words))
        return np.asarray(words, dtype=np.uint64)

    def is_valid(self, words: np.ndarray) -> np.ndarray:
        """Word is a state of this sector: no bits above L*Nbits, digits < Q, digit sum N."""
        w = self.words_array(words)
        ok = np.ones(w.shape, dtype=bool)
        if self.L * self.nb < 64:
            ok &= (w >> np.uint64(self.L * self.nb)) == 0
        elif self.wide:
            ok &= (w >> (self.L * self.nb)) == 0
        tot = np.zeros(w.shape, dtype=np.int64)
        for i in range(self.L):
            d = site_digit(w, self.L, self.Q, i)
            ok &= d < self.Q
            tot += d
        return ok & (tot == self.N)

    def state_at(self, index: int) -> int:
        """Function (iii) of Sec. 2.2: the state with a given canonical index."""
        if not 0 <= index < self.dim:
            raise IndexError("index out of range")
        return int(self.basis[index])

    def index_of_many(self, words: np.ndarray) -> np.ndarray:
        """Function (i) of Sec. 2.2 for many states: binary search of their keys."""
        w = self.words_array(words)
        if not np.all(self.is_valid(w)):
            raise ValueError("state not in this sector")
        k = composite_key(w, self.L, self.Q, self.partition)
        pos = np.searchsorted(self.keys, k)
        assert np.all(pos < self.dim) and np.all(self.keys[pos] == k)
        return pos.astype(np.int64)

    def index_of(self, word: int) -> int:
        return int(self.index_of_many(self.words_array([word]))[0])

    def next_state(self, word: int) -> int:
        """Function (ii) of Sec. 2.2: the next state in canonical order; the last wraps to the
        first (minimal) state, as Alg. 3 returns the minimal state for a maximal input."""
        return int(self.basis[(self.index_of(word) + 1) % self.dim])

    def local_index(self, pattern: int, Lk: int) -> int:
        """Index of a P_k digit pattern inside its own particle-number sector, local order
        lexicographic (Table 1): the number of Lk-site patterns with the same digit sum that
        compare lower."""
        nb = self.nb
        digs = [(pattern >> (nb * (Lk - 1 - s))) & ((1 << nb) - 1) for s in range(Lk)]
        n = sum(digs)
        same = enumerate_lex(Lk, self.Q, n)
        return int(np.searchsorted(same, np.uint64(pattern)))
