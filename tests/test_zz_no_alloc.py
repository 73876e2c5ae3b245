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


def test_noalloc_rejects_capture_and_large_states():
    """A capturing stream is refused (the call uploads a host-side plan that a
    graph replay would read after it is freed), and so is a problem above the
    on-chip engine's qubit limit; neither enqueues any work."""
    import torch
    import paper_2406_03466_gb300 as sv
    lib = sv.library()
    w = wl.mcvqe(8, 4)
    prob = sv.Problem.from_spec(w, "c64")
    theta = torch.as_tensor(w.theta, dtype=torch.float64, device="cuda")
    g = torch.empty(w.n_params, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        graph.capture_begin()
        try:
            st = lib.sv_grad_param_shift_noalloc(
                ctypes.byref(prob.struct), ctypes.c_void_p(theta.data_ptr()), None, None,
                ctypes.c_void_p(g.data_ptr()), ctypes.c_void_p(side.cuda_stream))
            msg = sv.sv_last_error()
        finally:
            graph.capture_end()
    del graph
    torch.cuda.synchronize()
    assert st == sv.SV_ERR_UNSUPPORTED
    assert "captured" in msg

    big = wl.mcvqe(16, 1, n_refs=1)
    prob16 = sv.Problem.from_spec(big, "c64")
    th16 = torch.as_tensor(big.theta, dtype=torch.float64, device="cuda")
    g16 = torch.empty(big.n_params, dtype=torch.float64, device="cuda")
    st = lib.sv_grad_param_shift_noalloc(
        ctypes.byref(prob16.struct), ctypes.c_void_p(th16.data_ptr()), None, None,
        ctypes.c_void_p(g16.data_ptr()), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == sv.SV_ERR_UNSUPPORTED
    assert "at most 13 qubits" in sv.sv_last_error()


_FRESH = r"""
import ctypes, sys
sys.path.insert(0, sys.argv[1])
import numpy as np
import torch
import paper_2406_03466_gb300 as sv
import workloads as wl
torch.cuda.set_device(0)
lib = sv.library()
stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
cases = []
for w in (wl.mcvqe(8, 4), wl.qcl(6, 2, 7), wl.vqe_random_pauli(4, 2, 10)):
    prob = sv.Problem.from_spec(w, "c64")
    theta = torch.as_tensor(w.theta, dtype=torch.float64, device="cuda")
    out = [torch.empty(n, dtype=torch.float64, device="cuda") for n in (w.n_instances, 1, w.n_params)]
    cases.append((prob, theta, out))
torch.cuda.synchronize()
def run_all():
    for prob, theta, (e, l, g) in cases:
        st = lib.sv_grad_param_shift_noalloc(
            ctypes.byref(prob.struct), ctypes.c_void_p(theta.data_ptr()),
            ctypes.c_void_p(e.data_ptr()), ctypes.c_void_p(l.data_ptr()),
            ctypes.c_void_p(g.data_ptr()), stream)
        assert st == sv.SV_OK, sv.sv_last_error()
    torch.cuda.synchronize()
run_all()          # the very first library calls of this process
free0 = torch.cuda.mem_get_info()[0]
for _ in range(3):
    run_all()
free1 = torch.cuda.mem_get_info()[0]
assert free1 == free0, (free0, free1)
assert all(np.isfinite(c[2][2].cpu().numpy()).all() for c in cases)
print("NOALLOC_FRESH_OK", free0, free1)
"""


def test_noalloc_allocates_nothing_in_a_fresh_process():
    """In a new process whose first library calls are allocation-free ones,
    the device's free memory does not move across repeated calls (modules
    load eagerly, so kernel loading cannot be mistaken for an allocation)."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, CUDA_MODULE_LOADING="EAGER")
    r = subprocess.run([sys.executable, "-c", _FRESH, root], capture_output=True, text=True,
                       env=env, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "NOALLOC_FRESH_OK" in r.stdout
