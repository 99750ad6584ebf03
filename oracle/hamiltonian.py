"""Oracle for the operator terms and the product y = H x on one sector.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``). FP64 throughout.

Terms are tuples ``(kind, i, j, coef)`` with ``kind`` a string; single-site kinds ignore ``j``.
The operator conventions follow the paper's example Hamiltonian (App. D: spin-1/2 chain,
H = sum_k 1/2 (S+_k S-_{k+1} + S-_k S+_{k+1}) + Sz_k Sz_{k+1} + h_k Sz_k) with a particle being
an up spin, and the standard Bose-Hubbard form for bosons (the paper only says the method
applies to bosons, Sec. 5):

=========  =====================================================  ==========================
kind       operator                                               Q
=========  =====================================================  ==========================
``XY``     coef * 1/2 (S+_i S-_j + S-_i S+_j)                     2
``ZZ``     coef * Sz_i Sz_j,  Sz = sigma - 1/2                    2
``Z``      coef * Sz_i                                            2
``HOP``    -coef * (b+_i b_j + b+_j b_i), b+|Q-1> = 0             any
``NN``     coef * n_i n_j                                         any
``N``      coef * n_i                                             any
``U``      coef / 2 * n_i (n_i - 1)                               any
=========  =====================================================  ==========================

``matvec`` is the column (scatter) form y_k = sum_j <k|H|j> x_j: every term is applied to every
basis state |sigma_j>, the resulting state is ranked by binary search, and amp * x_j is added at
that row (the matrix-free product of Sec. 2.2 and Sec. 4.4, done term by term).
"""

from __future__ import annotations

import numpy as np

from .sector import OracleSector, nbits_for, site_digit

__all__ = ["KINDS", "check_terms", "diagonal", "matvec", "matvec_rows"]

KINDS = ("XY", "ZZ", "Z", "HOP", "NN", "N", "U")
_PAIR = {"XY", "ZZ", "HOP", "NN"}
_SPIN = {"XY", "ZZ", "Z"}


def check_terms(sector: OracleSector, terms) -> list[tuple[str, int, int, float]]:
    out = []
    for t in terms:
        kind, i, j, c = t[0], int(t[1]), int(t[2]), float(t[3])
        if kind not in KINDS:
            raise ValueError(f"unknown term kind {kind!r}")
        if kind in _SPIN and sector.Q != 2:
            raise ValueError("spin-1/2 terms need Q = 2")
        if not 0 <= i < sector.L:
            raise ValueError("site out of range")
        if kind in _PAIR:
            if not 0 <= j < sector.L or i == j:
                raise ValueError("pair term needs two distinct sites in range")
        out.append((kind, i, j, c))
    return out


def _bit(sector: OracleSector, i: int):
    """Integer value of one particle on site i (lowest bit of its digit): np.uint64, or a Python
    int for words wider than 64 bits."""
    if sector.wide:
        return 1 << (sector.nb * (sector.L - 1 - i))
    return np.uint64(1) << np.uint64(sector.nb * (sector.L - 1 - i))


def _diag_term(sector: OracleSector, kind: str, i: int, j: int, c: float, words) -> np.ndarray:
    di = site_digit(words, sector.L, sector.Q, i).astype(np.float64)
    if kind == "ZZ":
        dj = site_digit(words, sector.L, sector.Q, j).astype(np.float64)
        return c * (di - 0.5) * (dj - 0.5)
    if kind == "Z":
        return c * (di - 0.5)
    if kind == "NN":
        dj = site_digit(words, sector.L, sector.Q, j).astype(np.float64)
        return c * di * dj
    if kind == "N":
        return c * di
    if kind == "U":
        return 0.5 * c * di * (di - 1.0)
    raise AssertionError(kind)


def diagonal(sector: OracleSector, terms, words=None) -> np.ndarray:
    """<sigma|H|sigma> for each word (default: the whole basis)."""
    terms = check_terms(sector, terms)
    w = sector.basis if words is None else sector.words_array(words)
    d = np.zeros(w.shape, dtype=np.float64)
    for kind, i, j, c in terms:
        if kind in ("ZZ", "Z", "NN", "N", "U"):
            d += _diag_term(sector, kind, i, j, c, w)
    return d


def _offdiag_images(sector: OracleSector, kind: str, i: int, j: int, c: float, words):
    """For an off-diagonal term, the states it produces from ``words``.

    Yields (source positions, produced words, amplitudes): term|words[pos]> = amp |produced>.
    """
    if kind == "XY":
        di = site_digit(words, sector.L, sector.Q, i)
        dj = site_digit(words, sector.L, sector.Q, j)
        pos = np.nonzero(di != dj)[0]
        flip = _bit(sector, i) | _bit(sector, j)
        yield pos, words[pos] ^ flip, np.full(pos.shape, 0.5 * c)
    elif kind == "HOP":
        for a, b in ((i, j), (j, i)):  # b+_a b_b, then its Hermitian conjugate
            da = site_digit(words, sector.L, sector.Q, a)
            db = site_digit(words, sector.L, sector.Q, b)
            pos = np.nonzero((da < sector.Q - 1) & (db > 0))[0]
            new = words[pos] + _bit(sector, a) - _bit(sector, b)
            amp = -c * np.sqrt((da[pos] + 1).astype(np.float64) * db[pos].astype(np.float64))
            yield pos, new, amp
    else:
        raise AssertionError(kind)


def matvec(sector: OracleSector, terms, x: np.ndarray) -> np.ndarray:
    """y = H x in the column (scatter) form, FP64. x has shape (D,) or (D, nrhs)."""
    terms = check_terms(sector, terms)
    x = np.asarray(x, dtype=np.float64)
    if x.shape[0] != sector.dim:
        raise ValueError("x has the wrong length")
    xs = x.reshape(sector.dim, -1)
    y = np.zeros_like(xs)
    words = sector.basis
    for kind, i, j, c in terms:
        if kind in ("XY", "HOP"):
            for pos, new, amp in _offdiag_images(sector, kind, i, j, c, words):
                rows = sector.index_of_many(new)
                np.add.at(y, rows, amp[:, None] * xs[pos])
        else:
            y += _diag_term(sector, kind, i, j, c, words)[:, None] * xs
    return y.reshape(x.shape)


def matvec_rows(sector: OracleSector, terms, x: np.ndarray, rows: np.ndarray) -> np.ndarray:
    """y[rows] of y = H x, computed row by row (gather reading of the same sum).

    Every term here is real and Hermitian, so <r|H|j> = <j|H|r>: applying each term to the row
    state |sigma_r> lists exactly the columns j with a nonzero <r|H|j> and their values. Used
    for sectors too large for ``matvec`` to sweep.
    """
    terms = check_terms(sector, terms)
    x = np.asarray(x, dtype=np.float64)
    rows = np.asarray(rows, dtype=np.int64)
    xs = x.reshape(sector.dim, -1)
    words = sector.basis[rows]
    out = np.zeros((rows.shape[0], xs.shape[1]), dtype=np.float64)
    for kind, i, j, c in terms:
        if kind in ("XY", "HOP"):
            for pos, new, amp in _offdiag_images(sector, kind, i, j, c, words):
                cols = sector.index_of_many(new)
                np.add.at(out, pos, amp[:, None] * xs[cols])
        else:
            out += _diag_term(sector, kind, i, j, c, words)[:, None] * xs[rows]
    return out.reshape((rows.shape[0],) + x.shape[1:])
