"""The allocation-free parameter-shift entry point against the regular one.

sv_grad_param_shift_noalloc is for callers that cannot let the library call
cudaMalloc (device memory owned by another allocator, or a running loop that
must not hit cudaMalloc's implicit synchronisation).  It keeps its plan and
scratch in one fixed device array shared by every call, which still holds
the previous call's contents when the next call starts; so each problem is
run twice in a row, and two different problems follow each other.  This
file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu

TOL = {"c64": (1e-5, 1e-4), "c128": (1e-12, 1e-12)}


def _close(a, b, tol):
    a, b = np.asarray(a), np.asarray(b)
    assert np.max(np.abs(a - b)) <= tol * max(1.0, float(np.max(np.abs(b))))


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_noalloc_matches_regular_entry_point(dtype):
    import torch
    import paper_2406_03466_gb300 as sv
    lib = sv.library()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    tol_e, tol_g = TOL[dtype]
    for w in (wl.mcvqe(8, 4), wl.qcl(6, 2, 7), wl.vqe_random_pauli(4, 2, 10)):
        prob = sv.Problem.from_spec(w, dtype)
        theta = torch.as_tensor(w.theta, dtype=torch.float64, device="cuda")
        l0, e0, g0 = sv.sv_grad_param_shift(prob, theta)
        for _ in range(2):
            e = torch.full((w.n_instances,), np.nan, dtype=torch.float64, device="cuda")
            l = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
            g = torch.full((w.n_params,), np.nan, dtype=torch.float64, device="cuda")
            st = lib.sv_grad_param_shift_noalloc(
                ctypes.byref(prob.struct), ctypes.c_void_p(theta.data_ptr()),
                ctypes.c_void_p(e.data_ptr()), ctypes.c_void_p(l.data_ptr()),
                ctypes.c_void_p(g.data_ptr()), stream)
            assert st == sv.SV_OK, sv.sv_last_error()
            torch.cuda.synchronize()
            _close(e.cpu().numpy(), e0.cpu().numpy(), tol_e)
            _close(l.cpu().numpy(), l0.cpu().numpy(), tol_e)
            _close(g.cpu().numpy(), g0.cpu().numpy()[: w.n_params], tol_g)


def test_noalloc_rejects_problems_beyond_its_array():
    import torch
    import paper_2406_03466_gb300 as sv
    w = wl.qcl(6, 30, 2000)   # (2P + 1) I doubles = 17 MB > 8 MiB
    prob = sv.Problem.from_spec(w, "c64")
    theta = torch.as_tensor(w.theta, dtype=torch.float64, device="cuda")
    g = torch.empty(w.n_params, dtype=torch.float64, device="cuda")
    st = sv.library().sv_grad_param_shift_noalloc(
        ctypes.byref(prob.struct), ctypes.c_void_p(theta.data_ptr()), None, None,
        ctypes.c_void_p(g.data_ptr()), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == sv.SV_ERR_UNSUPPORTED
    assert "at most" in sv.sv_last_error()
