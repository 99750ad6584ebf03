"""Thin ctypes binding of ``libdq.so`` (the C-ABI declared in ``include/dq.h``).

Argument marshalling only: every step of the basis machinery and of the product runs in the
library (host sector builder in C++, kernels in CUDA). The names follow the C-ABI without the
``dq_`` prefix. Importing this module loads the library and raises if it has not been built;
there is no fallback.

Vectors are torch tensors on the CUDA device that was current when the sector was made,
float64 or float32, contiguous, shape (D,) or (D, nrhs). Calls run on torch's current stream.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# DQ_CHECKED=1 selects the checked build (device rank results compared with D; see build.py)
LIB_PATH = os.path.join(_HERE, "libdq_checked.so" if os.environ.get("DQ_CHECKED") == "1" else "libdq.so")

DQ_OK, DQ_EINVAL, DQ_ERANGE, DQ_EINDEX, DQ_ESTATE, DQ_ENOMEM, DQ_ECUDA, DQ_EDEVICE = 0, -1, -2, -3, -4, -5, -6, -7
DQ_F64, DQ_F32 = 0, 1
DQ_LZ_DOUBLE_SINGLE = 16
KINDS = {"XY": 0, "ZZ": 1, "Z": 2, "HOP": 3, "NN": 4, "N": 5, "U": 6}

EXPORTED = (
    "dq_last_error", "dq_make_sector", "dq_free_sector", "dq_sector_dim", "dq_sector_partition",
    "dq_state_at", "dq_index_of", "dq_next_state", "dq_state_at_batch", "dq_index_of_batch",
    "dq_state_at2", "dq_index_of2", "dq_next_state2", "dq_state_at_batch2", "dq_index_of_batch2",
    "dq_check_device", "dq_make_terms", "dq_terms_path", "dq_free_terms", "dq_matvec", "dq_matvec_noalloc",
    "dq_lanczos", "dq_make_cluster_terms", "dq_cluster_info", "dq_batch_make", "dq_batch_matvec", "dq_batch_tune", "dq_batch_shape", "dq_batch_free", "dq_term_grads",
    "dq_timing_enable", "dq_timing_read",
)


class DQError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class _Term(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("i", ctypes.c_int), ("j", ctypes.c_int), ("coef", ctypes.c_double)]


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is not built; run `python -m paper_2407_14591_gb300.build`")
    lib = ctypes.CDLL(LIB_PATH)
    vp, u64, i32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int
    P = ctypes.POINTER
    sig = {
        "dq_last_error": (ctypes.c_char_p, []),
        "dq_make_sector": (i32, [i32, i32, i32, i32, P(vp)]),
        "dq_free_sector": (None, [vp]),
        "dq_sector_dim": (i32, [vp, P(u64)]),
        "dq_sector_partition": (i32, [vp, P(i32), P(i32)]),
        "dq_state_at": (i32, [vp, u64, P(u64)]),
        "dq_index_of": (i32, [vp, u64, P(u64)]),
        "dq_next_state": (i32, [vp, u64, P(u64)]),
        "dq_state_at_batch": (i32, [vp, vp, vp, u64, vp]),
        "dq_index_of_batch": (i32, [vp, vp, vp, u64, vp]),
        "dq_state_at2": (i32, [vp, u64, P(u64)]),
        "dq_index_of2": (i32, [vp, P(u64), P(u64)]),
        "dq_next_state2": (i32, [vp, P(u64), P(u64)]),
        "dq_state_at_batch2": (i32, [vp, vp, vp, u64, vp]),
        "dq_index_of_batch2": (i32, [vp, vp, vp, u64, vp]),
        "dq_check_device": (i32, [vp, vp]),
        "dq_make_terms": (i32, [vp, P(_Term), i32, P(vp)]),
        "dq_free_terms": (None, [vp]),
        "dq_make_cluster_terms": (i32, [vp, P(_Term), i32, i32, P(vp)]),
        "dq_cluster_info": (i32, [vp, P(i32), P(i32), P(i32)]),
        "dq_terms_path": (i32, [vp, P(i32)]),
        "dq_matvec": (i32, [vp, vp, vp, vp, i32, i32, vp]),
        "dq_matvec_noalloc": (i32, [vp, vp, vp, vp, i32, vp]),
        "dq_batch_make": (i32, [i32, P(vp), P(vp), i32, i32, P(vp)]),
        "dq_batch_matvec": (i32, [vp, P(vp), P(vp), vp]),
        "dq_batch_tune": (i32, [vp, P(vp), P(vp), vp, P(i32)]),
        "dq_batch_free": (None, [vp]),
        "dq_batch_shape": (i32, [vp, i32, P(i32)]),
        "dq_term_grads": (i32, [vp, P(_Term), i32, vp, vp, i32, i32, vp, vp]),
        "dq_lanczos": (i32, [vp, vp, vp, i32, i32, i32, P(ctypes.c_double), P(ctypes.c_double),
                             P(ctypes.c_double), P(i32), vp, vp]),
        "dq_timing_enable": (i32, [i32]),
        "dq_timing_read": (i32, [P(ctypes.c_double), P(ctypes.c_longlong), P(ctypes.c_longlong)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()


def lib() -> ctypes.CDLL:
    return _lib


def _check(rc: int):
    if rc != DQ_OK:
        raise DQError(rc, _lib.dq_last_error().decode())


def _stream_handle(stream=None):
    import torch

    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


class Sector:
    """A particle-number sector (L, Q, N) split into n_sub subsystems (0 = paper default)."""

    def __init__(self, L: int, Q: int, N: int, n_sub: int = 0):
        h = ctypes.c_void_p()
        _check(_lib.dq_make_sector(L, Q, N, n_sub, ctypes.byref(h)))
        self._h = h
        self.L, self.Q, self.N = L, Q, N
        D = ctypes.c_uint64()
        _check(_lib.dq_sector_dim(h, ctypes.byref(D)))
        self.dim = int(D.value)
        n = ctypes.c_int()
        parts = (ctypes.c_int * 64)()
        _check(_lib.dq_sector_partition(h, ctypes.byref(n), parts))
        self.partition = [int(parts[k]) for k in range(n.value)]
        self.n_sub = n.value

    @property
    def handle(self):
        return self._h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            _lib.dq_free_sector(h)
            self._h = None

    @property
    def wide(self) -> bool:
        """States take two words (L * Nbits > 64)."""
        return self.L * (self.Q - 1).bit_length() > 64

    def state_at(self, index: int) -> int:
        """Function (iii) on the host; the state as a Python int (two-word form when wide)."""
        if self.wide:
            out = (ctypes.c_uint64 * 2)()
            _check(_lib.dq_state_at2(self._h, ctypes.c_uint64(index), out))
            return int(out[0]) | (int(out[1]) << 64)
        out = ctypes.c_uint64()
        _check(_lib.dq_state_at(self._h, ctypes.c_uint64(index), ctypes.byref(out)))
        return int(out.value)

    def index_of(self, state: int) -> int:
        out = ctypes.c_uint64()
        if self.wide:
            w = (ctypes.c_uint64 * 2)(state & (2 ** 64 - 1), state >> 64)
            _check(_lib.dq_index_of2(self._h, w, ctypes.byref(out)))
        else:
            _check(_lib.dq_index_of(self._h, ctypes.c_uint64(state), ctypes.byref(out)))
        return int(out.value)

    def next_state(self, state: int) -> int:
        if self.wide:
            w = (ctypes.c_uint64 * 2)(state & (2 ** 64 - 1), state >> 64)
            out = (ctypes.c_uint64 * 2)()
            _check(_lib.dq_next_state2(self._h, w, out))
            return int(out[0]) | (int(out[1]) << 64)
        out = ctypes.c_uint64()
        _check(_lib.dq_next_state(self._h, ctypes.c_uint64(state), ctypes.byref(out)))
        return int(out.value)

    def state_at_batch2(self, index, out=None):
        """Two-word batched function (iii): returns an int64 CUDA tensor of shape (n, 2), column 0
        the low word and column 1 the high word of each state."""
        import torch

        idx = index.contiguous()
        out = torch.empty((idx.numel(), 2), dtype=torch.int64, device=idx.device) if out is None else out
        _check(_lib.dq_state_at_batch2(self._h, ctypes.c_void_p(idx.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                       idx.numel(), _stream_handle()))
        return out

    def index_of_batch2(self, states, out=None):
        """Two-word batched function (i): states is an int64 CUDA tensor of shape (n, 2)."""
        import torch

        st = states.contiguous()
        n = st.shape[0]
        out = torch.empty(n, dtype=torch.int64, device=st.device) if out is None else out
        _check(_lib.dq_index_of_batch2(self._h, ctypes.c_void_p(st.data_ptr()), ctypes.c_void_p(out.data_ptr()), n,
                                       _stream_handle()))
        return out

    def state_at_batch(self, index, out=None):
        """Batched function (iii) on the device; index: int64/uint64 CUDA tensor."""
        import torch

        idx = index.contiguous()
        out = torch.empty_like(idx) if out is None else out
        _check(_lib.dq_state_at_batch(self._h, ctypes.c_void_p(idx.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                      idx.numel(), _stream_handle()))
        return out

    def index_of_batch(self, states, out=None):
        """Batched function (i) on the device; states: int64/uint64 CUDA tensor of words."""
        import torch

        st = states.contiguous()
        out = torch.empty_like(st) if out is None else out
        _check(_lib.dq_index_of_batch(self._h, ctypes.c_void_p(st.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                      st.numel(), _stream_handle()))
        return out

    def check_device(self):
        _check(_lib.dq_check_device(self._h, _stream_handle()))


def make_sector(L: int, Q: int, N: int, n_sub: int = 0) -> Sector:
    return Sector(L, Q, N, n_sub)


def sector_dim(sector: Sector) -> int:
    return sector.dim


def state_at(sector: Sector, index: int) -> int:
    return sector.state_at(index)


def index_of(sector: Sector, state: int) -> int:
    return sector.index_of(state)


def next_state(sector: Sector, state: int) -> int:
    return sector.next_state(state)


class Terms:
    """Operator terms compiled for one sector; ``terms`` is a list of (kind, i, j, coef). With
    ``cluster_sites`` the cluster-merged form of App. C (dq_make_cluster_terms)."""

    def __init__(self, sector: Sector, terms, cluster_sites: int | None = None):
        arr = (_Term * max(1, len(terms)))()
        for q, (kind, i, j, c) in enumerate(terms):
            k = KINDS[kind] if isinstance(kind, str) else int(kind)
            arr[q] = _Term(k, int(i), int(j), float(c))
        h = ctypes.c_void_p()
        if cluster_sites is None:
            _check(_lib.dq_make_terms(sector.handle, arr, len(terms), ctypes.byref(h)))
        else:
            _check(_lib.dq_make_cluster_terms(sector.handle, arr, len(terms), int(cluster_sites), ctypes.byref(h)))
        self._h = h
        self.sector = sector  # keeps the sector alive while the terms exist

    def clusters(self):
        """(list of site lists, largest number of entries a row meets) of cluster-merged terms."""
        n = ctypes.c_int()
        _check(_lib.dq_cluster_info(self._h, ctypes.byref(n), None, None))
        sites = (ctypes.c_int * (12 * max(1, n.value)))()
        ent = ctypes.c_int()
        _check(_lib.dq_cluster_info(self._h, ctypes.byref(n), sites, ctypes.byref(ent)))
        return [[v for v in sites[12 * c:12 * c + 12] if v >= 0] for c in range(n.value)], ent.value

    @property
    def handle(self):
        return self._h

    @property
    def path(self) -> str:
        """'panel', 'panel_pb', 'panel_w', 'panel_q', 'general' or 'cluster': the product kernel used
        for one right-hand side."""
        v = ctypes.c_int()
        _check(_lib.dq_terms_path(self._h, ctypes.byref(v)))
        return {1: "panel", 2: "cluster", 3: "panel_pb", 4: "panel_w", 5: "panel_q"}.get(v.value, "general")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            _lib.dq_free_terms(h)
            self._h = None


def make_terms(sector: Sector, terms) -> Terms:
    return Terms(sector, terms)


def make_cluster_terms(sector: Sector, terms, cluster_sites: int) -> Terms:
    return Terms(sector, terms, cluster_sites)


def _dtype_code(t) -> int:
    import torch

    if t.dtype == torch.float64:
        return DQ_F64
    if t.dtype == torch.float32:
        return DQ_F32
    raise TypeError("vectors must be float64 or float32")


def _check_vec(sector: Sector, t, name: str):
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if t.shape[0] != sector.dim or t.dim() not in (1, 2):
        raise ValueError(f"{name} must have shape (D,) or (D, nrhs) with D = {sector.dim}")


def matvec(sector: Sector, terms: Terms, x, y=None):
    """y = H x on torch's current stream; returns y (allocated if not given)."""
    import torch

    _check_vec(sector, x, "x")
    if y is None:
        y = torch.empty_like(x)
    _check_vec(sector, y, "y")
    if y.dtype != x.dtype or y.shape != x.shape:
        raise ValueError("x and y must have the same dtype and shape")
    nrhs = 1 if x.dim() == 1 else x.shape[1]
    _check(_lib.dq_matvec(sector.handle, terms.handle, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                          _dtype_code(x), nrhs, _stream_handle()))
    return y


def matvec_noalloc(sector: Sector, terms: Terms, x, y):
    """y = H x through the allocation-free entry point (panel path, D below its static limit).

    y must be given: this call allocates nothing, on the device or through torch."""
    _check_vec(sector, x, "x")
    _check_vec(sector, y, "y")
    if x.dim() != 1 or y.dtype != x.dtype or y.shape != x.shape:
        raise ValueError("x and y must be single vectors of the same dtype")
    _check(_lib.dq_matvec_noalloc(sector.handle, terms.handle, ctypes.c_void_p(x.data_ptr()),
                                  ctypes.c_void_p(y.data_ptr()), _dtype_code(x), _stream_handle()))
    return y


class Batch:
    """One launch over many Q = 2 sectors (each with its terms), nrhs right-hand sides each."""

    def __init__(self, sectors, terms, nrhs: int, dtype):
        import torch

        n = len(sectors)
        self.sectors, self.terms, self.nrhs = list(sectors), list(terms), nrhs
        self.dtype = dtype
        code = DQ_F64 if dtype == torch.float64 else DQ_F32
        sv = (ctypes.c_void_p * n)(*[s.handle.value for s in sectors])
        tv = (ctypes.c_void_p * n)(*[t.handle.value for t in terms])
        h = ctypes.c_void_p()
        _check(_lib.dq_batch_make(n, sv, tv, nrhs, code, ctypes.byref(h)))
        self._h = h
        self.choice = None

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            _lib.dq_batch_free(h)
            self._h = None

    def _ptrs(self, xs, ys):
        for s, x, y in zip(self.sectors, xs, ys):
            for t, name in ((x, "x"), (y, "y")):
                _check_vec(s, t, name)
                if t.dtype != self.dtype or t.numel() != s.dim * self.nrhs:
                    raise ValueError(f"{name} must hold D * nrhs elements of the batch dtype")
        n = len(self.sectors)
        return ((ctypes.c_void_p * n)(*[x.data_ptr() for x in xs]), (ctypes.c_void_p * n)(*[y.data_ptr() for y in ys]))

    def matvec(self, xs, ys):
        xp, yp = self._ptrs(xs, ys)
        _check(_lib.dq_batch_matvec(self._h, xp, yp, _stream_handle()))
        return ys

    def n_shapes(self) -> int:
        n = ctypes.c_int()
        _check(_lib.dq_batch_shape(self._h, -1, ctypes.byref(n)))
        return n.value

    def set_shape(self, shape: int):
        """Use candidate `shape` (mapping and launch shape) for later products."""
        _check(_lib.dq_batch_shape(self._h, int(shape), None))
        self.choice = int(shape)

    def tune(self, xs, ys) -> int:
        xp, yp = self._ptrs(xs, ys)
        c = ctypes.c_int()
        _check(_lib.dq_batch_tune(self._h, xp, yp, _stream_handle(), ctypes.byref(c)))
        self.choice = c.value
        return c.value


def term_grads(sector: Sector, terms, x, dy):
    """g_q = sum_i sum_r dy[i, r] (T_q x)[i, r] for each (kind, i, j[, coef]) in ``terms``;
    returns a float64 CUDA tensor of len(terms)."""
    import torch

    _check_vec(sector, x, "x")
    _check_vec(sector, dy, "dy")
    if dy.dtype != x.dtype or dy.shape != x.shape:
        raise ValueError("x and dy must have the same dtype and shape")
    arr = (_Term * max(1, len(terms)))()
    for q, t in enumerate(terms):
        kind, i, j = t[0], t[1], t[2]
        arr[q] = _Term(KINDS[kind] if isinstance(kind, str) else int(kind), int(i), int(j), 0.0)
    out = torch.empty(max(1, len(terms)), dtype=torch.float64, device=x.device)
    nrhs = 1 if x.dim() == 1 else x.shape[1]
    _check(_lib.dq_term_grads(sector.handle, arr, len(terms), ctypes.c_void_p(x.data_ptr()),
                              ctypes.c_void_p(dy.data_ptr()), _dtype_code(x), nrhs, ctypes.c_void_p(out.data_ptr()),
                              _stream_handle()))
    return out[: len(terms)]


def make_batch(sectors, terms, nrhs: int, dtype) -> Batch:
    return Batch(sectors, terms, nrhs, dtype)


def lanczos(sector: Sector, terms: Terms, v0, steps: int, reorth=True, want_vector: bool = False,
            double_single: bool = False) -> dict:
    """Ground-state energy by Lanczos (synchronous). ``reorth``: False/0 none, True/1 full
    re-orthogonalisation (second Gram-Schmidt pass when needed), 2 (second pass always).
    ``double_single``: the passes over the basis in double-single arithmetic instead of FP64.
    Returns E0, alpha, beta, steps_done and, with ``want_vector``, the Ritz vector of E0 as
    ``psi`` (a CUDA tensor like v0)."""
    import torch

    _check_vec(sector, v0, "v0")
    if v0.dim() != 1:
        raise ValueError("v0 must be one vector")
    E0 = ctypes.c_double()
    alpha = (ctypes.c_double * max(1, steps))()
    beta = (ctypes.c_double * max(1, steps))()
    done = ctypes.c_int()
    psi = torch.empty_like(v0) if want_vector else None
    _check(_lib.dq_lanczos(sector.handle, terms.handle, ctypes.c_void_p(v0.data_ptr()), steps, _dtype_code(v0),
                           int(reorth) | (DQ_LZ_DOUBLE_SINGLE if double_single else 0), ctypes.byref(E0), alpha,
                           beta, ctypes.byref(done),
                           ctypes.c_void_p(psi.data_ptr() if psi is not None else 0), _stream_handle()))
    m = done.value
    out = {"E0": E0.value, "alpha": np.array(alpha[:m]), "beta": np.array(beta[:m]), "steps_done": m}
    if psi is not None:
        out["psi"] = psi
    return out


def timing_enable(on: bool = True):
    """Turn the main-kernel timing hooks on (clearing the record) or off."""
    _check(_lib.dq_timing_enable(1 if on else 0))


def timing_read():
    """(main-kernel milliseconds, product calls, kernels launched) since the last timing_enable(True)."""
    ms, n, k = ctypes.c_double(), ctypes.c_longlong(), ctypes.c_longlong()
    _check(_lib.dq_timing_read(ctypes.byref(ms), ctypes.byref(n), ctypes.byref(k)))
    return ms.value, n.value, k.value
