"""The C ABI without a GPU: argument checks run before any device work and
report SV_ERR_ARG with a message; well-formed calls on a machine without a
GPU fail with SV_ERR_CUDA instead of computing anywhere else (there is no CPU
fallback).  Runs only where CUDA is unavailable."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
sv = pytest.importorskip("paper_2406_03466_gb300")
import workloads as wl  # noqa: E402

pytestmark = pytest.mark.skipif(torch.cuda.is_available(), reason="checks the no-GPU behaviour")

SV_OK, SV_ERR_ARG, SV_ERR_CUDA = 0, 1, 3


def _grad(prob, theta):
    out = [torch.zeros(max(1, k), dtype=torch.float64) for k in (prob.n_instances, 1,
                                                                  prob.n_params)]
    L = sv.library()
    st = L.sv_grad_param_shift(ctypes.byref(prob.struct), ctypes.c_void_p(theta.data_ptr()),
                               *[ctypes.c_void_p(t.data_ptr()) for t in out], None)
    return st, L.sv_last_error().decode()


def _problem(w):
    return sv.Problem.from_spec(w, "c64", device="cpu")


def test_bad_arguments_are_rejected_before_device_work():
    w = wl.mcvqe(6, 2)
    th = torch.as_tensor(w.theta, dtype=torch.float64)
    prob = _problem(w)
    prob.struct.n_instances = 0
    st, msg = _grad(prob, th)
    assert st == SV_ERR_ARG and "n_instances" in msg
    prob = _problem(w)
    keep = int(prob._refs[0])
    prob._refs[0] = 1 << 6  # a basis index of 7 qubits (the struct points at this array)
    st, msg = _grad(prob, th)
    prob._refs[0] = keep  # the array may be the workload's own
    assert st == SV_ERR_ARG and "reference" in msg
    prob = _problem(w)
    prob.struct.dtype = 7
    st, msg = _grad(prob, th)
    assert st == SV_ERR_ARG and "dtype" in msg
    prob = _problem(w)
    prob.struct.cost = 9
    st, msg = _grad(prob, th)
    assert st == SV_ERR_ARG and "cost" in msg


def test_no_cpu_fallback():
    w = wl.mcvqe(6, 2)
    th = torch.as_tensor(w.theta, dtype=torch.float64)
    st, msg = _grad(_problem(w), th)
    assert st == SV_ERR_CUDA, (st, msg)
