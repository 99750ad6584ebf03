"""The allocation-free product entry point, dq_matvec_noalloc (GPU only).

It serves callers that may not allocate device memory while they run; its scratch is a static
device array. This file is collected last on purpose: if it fails, a run that stops at the first
failure has already run every other test. It passes alone in a fresh process as well, since its
first call on the device performs the one-time set-up itself.
"""

import ctypes

import numpy as np
import pytest
import torch

from paper_2407_14591_gb300 import binding as b
from paper_2407_14591_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("lat,path", [((5, 4), "panel_w"), ((11, 2), "panel")])
def test_noalloc_matches_matvec_on_two_calls(lat, path):
    """Two calls in a row, each against dq_matvec on the same input (FP64 bar 1e-12, FP32 1e-5),
    on both panel paths (D = 184,756 and 705,432)."""
    L = lat[0] * lat[1]
    s = b.make_sector(L, 2, L // 2, 2)
    nn, nnn = wl.square_bonds(*lat)
    t = b.make_terms(s, wl.heisenberg_terms(nn, 1.0) + wl.heisenberg_terms(nnn, 0.5))
    assert t.path == path
    lib = b.lib()
    rng = np.random.default_rng(20240719)
    for call in range(2):
        x = torch.from_numpy(rng.uniform(-1, 1, s.dim) * (10.0 ** (3 * call))).to("cuda")
        ref = b.matvec(s, t, x, torch.empty_like(x))
        out = torch.full_like(x, float("nan"))
        rc = lib.dq_matvec_noalloc(s.handle, t.handle, ctypes.c_void_p(x.data_ptr()),
                                   ctypes.c_void_p(out.data_ptr()), b.DQ_F64, _stream())
        assert rc == b.DQ_OK, lib.dq_last_error()
        torch.cuda.synchronize()
        s.check_device()
        r, o = ref.cpu().numpy(), out.cpu().numpy()
        assert np.max(np.abs(o - r)) <= 1e-12 * np.max(np.abs(r)), call
    x32 = torch.from_numpy(rng.uniform(-1, 1, s.dim).astype(np.float32)).to("cuda")
    ref32 = b.matvec(s, t, x32, torch.empty_like(x32))
    out32 = b.matvec_noalloc(s, t, x32, torch.empty_like(x32))
    torch.cuda.synchronize()
    assert torch.linalg.norm(out32.double() - ref32.double()) <= 1e-5 * torch.linalg.norm(ref32.double())


def test_noalloc_boson_panel_path():
    """The boson panel path (Q = 4, two subsystems; D = 44,803) against dq_matvec, FP64 and FP32."""
    rng = np.random.default_rng(4)
    L = 10
    terms = [("HOP", i, j, 1.0) for i, j in wl.chain_bonds(L)] + [("U", i, -1, float(u)) for i, u in
                                                                   enumerate(rng.uniform(2, 6, L))]
    s = b.make_sector(L, 4, L, 2)
    t = b.make_terms(s, terms)
    assert t.path == "panel_q"
    for dt, tol in ((torch.float64, 1e-12), (torch.float32, 1e-5)):
        x = torch.from_numpy(rng.uniform(-1, 1, s.dim)).to("cuda", dt)
        ref = b.matvec(s, t, x, torch.empty_like(x))
        out = b.matvec_noalloc(s, t, x, torch.full_like(x, float("nan")))
        torch.cuda.synchronize()
        s.check_device()
        assert torch.max(torch.abs(out.double() - ref.double())).item() <= tol * torch.max(torch.abs(ref.double())).item()


def test_noalloc_rejects_too_large_and_off_path():
    s = b.make_sector(26, 2, 13, 2)  # D = 10,400,600 > 8,388,568 (FP64 limit)
    t = b.make_terms(s, wl.heisenberg_terms(wl.chain_bonds(26), 1.0))
    assert t.path == "panel"
    lib = b.lib()
    dummy = ctypes.c_void_p(0x1000)
    rc = lib.dq_matvec_noalloc(s.handle, t.handle, dummy, ctypes.c_void_p(0x10000000000), b.DQ_F64, _stream())
    assert rc == b.DQ_ERANGE
    assert b"8388568" in lib.dq_last_error()
    # per-bond couplings with three subsystems: the general kernel, which the call does not serve
    # (checked before the call: the call must return before it could launch anything)
    s2 = b.make_sector(12, 2, 6, 3)
    t2 = b.make_terms(s2, wl.heisenberg_terms(wl.chain_bonds(12), np.linspace(0.5, 1.5, 12)))
    assert t2.path == "general"
    rc = lib.dq_matvec_noalloc(s2.handle, t2.handle, dummy, ctypes.c_void_p(0x10000000000), b.DQ_F64, _stream())
    assert rc == b.DQ_EINVAL


def test_noalloc_call_takes_no_device_memory():
    """After one call has done the per-device set-up, a call on a fresh sector and terms leaves the
    device's free memory unchanged: the call itself allocates nothing."""
    nn, nnn = wl.square_bonds(4, 4)
    terms = wl.heisenberg_terms(nn, 1.0) + wl.heisenberg_terms(nnn, 0.5)
    s0 = b.make_sector(16, 2, 8, 2)
    t0 = b.make_terms(s0, terms)
    x0 = torch.rand(s0.dim, dtype=torch.float64, device="cuda")
    b.matvec_noalloc(s0, t0, x0, torch.empty_like(x0))  # set-up (and kernel load) on this device
    s = b.make_sector(16, 2, 7, 2)
    t = b.make_terms(s, terms)
    assert t.path == "panel_w"
    x = torch.rand(s.dim, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    ref = b.matvec(s, t, x, torch.empty_like(x))
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    b.matvec_noalloc(s, t, x, y)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.max(torch.abs(y - ref)).item() <= 1e-12 * torch.max(torch.abs(ref)).item()
