"""Plain CPU oracle for the U(1)-sector matrix-free product (test infrastructure).

This package is TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it. The product path
(the C-ABI library and its Python binding) never imports, calls or links anything here, and
this package imports nothing from the product.

It is written from the paper's definitions, not from its divide-and-conquer machinery:

* ``sector``      -- sector dimension (App. A polynomial coefficient), lexicographic
                     enumeration of the sector, the canonical order as a sort by subsystem key
                     (Sec. 3.1-3.2, Table 1), rank by binary search, unrank by array access,
                     Cover's enumerative index (Sec. 3.4, Eq. (cover)).
* ``hamiltonian`` -- the operator terms and the column (scatter) form of y = H x, plus a
                     sampled-row (gather) form for sectors too large to sweep.
* ``lanczos``     -- FP64 Lanczos with full re-orthogonalisation and a tridiagonal solve.

Every function says which passage of the paper it follows. All floating point is FP64.
"""

from .sector import (  # noqa: F401
    OracleSector,
    canonical_basis,
    cover_index,
    enumerate_lex,
    most_equal_partition,
    nbits_for,
    sector_dim,
)
from .hamiltonian import matvec, matvec_rows, diagonal  # noqa: F401
from .lanczos import lanczos  # noqa: F401
