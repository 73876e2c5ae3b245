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
import paper_2406_03466_gb300 as sv
import workloads as wl
rt = ctypes.CDLL("libcudart.so.13")   # the CUDA runtime libsv.so is linked against
assert rt.cudaSetDevice(0) == 0 and rt.cudaFree(None) == 0


class Dev:
    # a float64 device array made with cudaMalloc (no torch in this process)
    def __init__(self, a):
        a = np.ascontiguousarray(a, dtype=np.float64)
        self.shape = a.shape
        self.p = ctypes.c_void_p()
        assert rt.cudaMalloc(ctypes.byref(self.p), ctypes.c_size_t(max(8, a.nbytes))) == 0
        if a.size:
            assert rt.cudaMemcpy(self.p, a.ctypes.data_as(ctypes.c_void_p),
                                 ctypes.c_size_t(a.nbytes), 1) == 0

    def data_ptr(self):
        return self.p.value


def free_bytes():
    f, t = ctypes.c_size_t(), ctypes.c_size_t()
    assert rt.cudaDeviceSynchronize() == 0 and rt.cudaMemGetInfo(ctypes.byref(f), ctypes.byref(t)) == 0
    return f.value


def cases(seed):
    out = []
    for w in (wl.mcvqe(8, 4, seed=seed), wl.qcl(6, 2, 7, seed=seed),
              wl.vqe_random_pauli(4, 2, 10, seed=seed)):
        d = 0 if w.inputs is None else int(np.asarray(w.inputs).shape[1])
        circ = sv.Circuit(w.n_qubits, w.gates, w.n_params, d)
        obs = sv.PauliSum(w.n_qubits, w.pauli_letters, w.pauli_coeffs)
        dev = lambda a: None if a is None else Dev(a)  # noqa: E731
        prob = sv.Problem(circ, obs, w.refs, "c64", inputs=dev(w.inputs), cost=w.cost,
                          weights=dev(w.weights), targets=dev(w.targets))
        outs = [Dev(np.zeros(k)) for k in (w.n_instances, 1, w.n_params)]
        out.append((prob, Dev(w.theta), outs, [w, prob.inputs, prob.weights, prob.targets]))
    return out


def run(cs):
    for prob, th, outs, _ in cs:
        st = sv.library().sv_grad_param_shift_noalloc(
            ctypes.byref(prob.struct), th.p, outs[0].p, outs[1].p, outs[2].p, None)
        assert st == sv.SV_OK, sv.sv_last_error()
    assert rt.cudaDeviceSynchronize() == 0


first, later = cases(0), cases(1)   # the same shapes (same kernels), other values
run(first)          # the very first library calls of this process
free0 = free_bytes()
for _ in range(3):
    run(later)
    run(first)
free1 = free_bytes()
assert free1 == free0, (free0, free1)
g = np.zeros(later[0][3][0].n_params)
assert rt.cudaMemcpy(g.ctypes.data_as(ctypes.c_void_p), later[0][2][2].p,
                     ctypes.c_size_t(g.nbytes), 2) == 0
assert np.isfinite(g).all() and np.abs(g).max() > 0
print("NOALLOC_FRESH_OK", free0, free1)
"""


def test_noalloc_allocates_nothing_in_a_fresh_process():
    """In a new process without torch whose first library calls are
    allocation-free ones, the device's free memory does not move across
    repeated calls on problems the library has not seen before (modules
    load eagerly at context creation, so kernel loading cannot be mistaken
    for an allocation; a library cache keyed on the problem would have to
    allocate for the new problems)."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, CUDA_MODULE_LOADING="EAGER")
    r = subprocess.run([sys.executable, "-c", _FRESH, root], capture_output=True, text=True,
                       env=env, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "NOALLOC_FRESH_OK" in r.stdout
