"""Batched state-vector gradients on one GB300 GPU: Python binding of libsv.so.

A thin ctypes layer over the C ABI in ``include/sv.h``.  It only marshals
arguments: gate lists become ``sv_gate`` arrays, Pauli rows become X/Z bit
masks, torch tensors become device pointers and streams.  Every step of the
computation (state preparation, gate application, expectation values,
parameter-shift and adjoint gradients) runs in the library's CUDA kernels.
PyTorch provides device memory and streams.

There is no CPU fallback: importing this package fails if ``libsv.so`` has
not been built (``python paper_2406_03466_gb300/build.py``).
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libsv.so")

SV_OK, SV_ERR_ARG, SV_ERR_OOM, SV_ERR_CUDA, SV_ERR_TIMEOUT, SV_ERR_UNSUPPORTED = range(6)
SV_C64, SV_C128 = 0, 1
SV_COST_LINEAR, SV_COST_MSE = 0, 1
GATE_CODES = {"RX": 0, "RY": 1, "RZ": 2, "CNOT": 3, "X": 4, "H": 5, "CZ": 6,
              "ENC_RY_ASIN": 7, "ENC_RZ_ACOS_SQ": 8}


class SvError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        detail = _lib.sv_last_error().decode() if _lib is not None else ""
        msg = _lib.sv_status_string(status).decode() if _lib is not None else str(status)
        super().__init__(f"{where}: {msg} ({detail})")


# ------------------------------------------------------------------ ABI types

class sv_gate(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int32), ("target", ctypes.c_int32), ("control", ctypes.c_int32),
                ("param", ctypes.c_int32), ("angle", ctypes.c_double)]


class sv_circuit(ctypes.Structure):
    _fields_ = [("n_qubits", ctypes.c_int32), ("n_gates", ctypes.c_int32),
                ("n_params", ctypes.c_int32), ("input_dim", ctypes.c_int32),
                ("gates", ctypes.POINTER(sv_gate))]


class sv_pauli_sum(ctypes.Structure):
    _fields_ = [("n_qubits", ctypes.c_int32), ("n_terms", ctypes.c_int32),
                ("x_mask", ctypes.POINTER(ctypes.c_uint64)),
                ("z_mask", ctypes.POINTER(ctypes.c_uint64)),
                ("coeff", ctypes.POINTER(ctypes.c_double))]


class sv_plan_opts(ctypes.Structure):
    _fields_ = [("reg_bits", ctypes.c_int32), ("threads_per_block", ctypes.c_int32),
                ("no_fusion", ctypes.c_int32), ("epilogue", ctypes.c_int32),
                ("tile_bits", ctypes.c_int32), ("coalesce_bits", ctypes.c_int32),
                ("no_relabel", ctypes.c_int32), ("tensor_blocks", ctypes.c_int32)]


class sv_slot(ctypes.Structure):
    _fields_ = [("circuit", ctypes.c_int32), ("theta_row", ctypes.c_int32),
                ("shift_param", ctypes.c_int32), ("input_row", ctypes.c_int32),
                ("ref", ctypes.c_int64), ("shift", ctypes.c_double)]


class sv_problem(ctypes.Structure):
    _fields_ = [("dtype", ctypes.c_int32), ("circuit", ctypes.POINTER(sv_circuit)),
                ("observable", ctypes.POINTER(sv_pauli_sum)), ("n_instances", ctypes.c_int32),
                ("refs", ctypes.POINTER(ctypes.c_int64)), ("inputs", ctypes.c_void_p),
                ("input_stride", ctypes.c_int32), ("cost", ctypes.c_int32),
                ("weights", ctypes.c_void_p), ("targets", ctypes.c_void_p),
                ("opts", ctypes.POINTER(sv_plan_opts))]


EXPORTED = ("sv_alloc", "sv_free", "sv_state_info", "sv_apply_circuit_batch",
            "sv_expect_pauli_sum", "sv_energies", "sv_param_shift_energies", "sv_grad_param_shift", "sv_grad_adjoint",
            "sv_grad_param_shift_plain", "sv_grad_param_shift_noalloc", "sv_autotune",
            "sv_tuned_shape", "sv_tuned_tile", "sv_plan_info", "sv_h_plan_info", "sv_phase_timing",
            "sv_grad_adjoint_multi", "sv_grad_ddcl", "sv_grad_ddcl_param_shift",
            "sv_grad_param_shift_host", "sv_grad_adjoint_host", "sv_param_shift_energies_range", "sv_sample",
            "sv_param_shift_combine",
            "sv_last_phase_ms", "sv_last_adjoint_info", "sv_status_string",
            "sv_last_error",
            "sv_sync_status", "sv_shutdown", "sv_version")


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is not built; run `python paper_2406_03466_gb300/build.py` "
                          "(requires nvcc). There is no CPU fallback.")
    lib = ctypes.CDLL(LIB_PATH)
    V, I32, P = ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER
    lib.sv_alloc.argtypes = [P(V), I32, I32, I32, V, ctypes.c_size_t, V]
    lib.sv_free.argtypes = [V]
    lib.sv_state_info.argtypes = [V, P(V), P(I32), P(I32), P(I32)]
    lib.sv_apply_circuit_batch.argtypes = [V, P(sv_circuit), I32, P(sv_slot), I32, V, I32, V, I32,
                                           P(sv_plan_opts), V]
    lib.sv_expect_pauli_sum.argtypes = [V, P(sv_pauli_sum), I32, V, V]
    lib.sv_energies.argtypes = [P(sv_problem), V, V, V, V]
    lib.sv_param_shift_energies.argtypes = [P(sv_problem), V, V, V]
    lib.sv_grad_param_shift.argtypes = [P(sv_problem), V, V, V, V, V]
    lib.sv_grad_param_shift_host.argtypes = [P(sv_problem), V, V, V, V, V]
    lib.sv_grad_adjoint.argtypes = [P(sv_problem), V, V, V, V, V, I32, V]
    lib.sv_grad_adjoint_host.argtypes = [P(sv_problem), V, V, V, V, I32, V]
    lib.sv_grad_adjoint_multi.argtypes = [P(sv_problem), I32, P(V), P(V), P(V), P(V), V]
    lib.sv_grad_ddcl.argtypes = [P(sv_problem), V, V, V, V, V]
    lib.sv_grad_ddcl_param_shift.argtypes = [P(sv_problem), V, V, V, V, V]
    lib.sv_sample.argtypes = [V, I32, V, ctypes.c_int64, V, V, V]
    lib.sv_param_shift_energies_range.argtypes = [P(sv_problem), V, I32, I32, V, V]
    lib.sv_param_shift_combine.argtypes = [P(sv_problem), V, V, V, V, V]
    lib.sv_grad_param_shift_plain.argtypes = [P(sv_problem), V, V, V, V, V]
    lib.sv_grad_param_shift_noalloc.argtypes = [P(sv_problem), V, V, V, V, V]
    lib.sv_autotune.argtypes = [P(sv_problem), V, I32, V]
    lib.sv_plan_info.argtypes = [P(sv_circuit), I32, P(sv_plan_opts)] + [P(I32)] * 5
    lib.sv_tuned_shape.argtypes = [P(sv_problem), I32, P(I32), P(I32), P(ctypes.c_float)]
    lib.sv_tuned_tile.argtypes = [P(sv_problem), I32, P(I32), P(I32), P(I32), P(ctypes.c_float)]
    lib.sv_debug_wait_expiry.argtypes = [I32, V]
    lib.sv_debug_wait_expiry.restype = I32
    lib.sv_h_plan_info.argtypes = [P(sv_pauli_sum), I32, P(I32), P(I32)]
    lib.sv_phase_timing.argtypes = [I32]
    lib.sv_last_phase_ms.argtypes = [P(ctypes.c_float)] * 3
    lib.sv_last_adjoint_info.argtypes = [P(ctypes.c_int32), P(ctypes.c_int64)]
    lib.sv_status_string.argtypes = [I32]
    lib.sv_status_string.restype = ctypes.c_char_p
    lib.sv_last_error.restype = ctypes.c_char_p
    lib.sv_sync_status.argtypes = [V]
    lib.sv_version.restype = I32
    for name in EXPORTED:
        if name not in ("sv_status_string", "sv_last_error", "sv_version"):
            getattr(lib, name).restype = I32
    return lib


_lib = None
_lib = _load()


def _check(status, where):
    if status != SV_OK:
        raise SvError(status, where)


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _dtype_code(dtype) -> int:
    if dtype in (SV_C64, "c64", "complex64"):
        return SV_C64
    if dtype in (SV_C128, "c128", "complex128"):
        return SV_C128
    raise ValueError(f"dtype {dtype!r}")


# ---------------------------------------------------------------- marshalling

class Circuit:
    """A gate list marshalled into an ``sv_circuit``.

    ``gates`` holds objects with ``op`` (name or code), ``target``, ``control``,
    ``param`` and ``angle`` attributes, or 5-tuples in that order.
    """

    def __init__(self, n_qubits: int, gates: Sequence, n_params: int, input_dim: int = 0):
        arr = (sv_gate * max(1, len(gates)))()
        for i, g in enumerate(gates):
            if isinstance(g, tuple):
                op, target, control, param, angle = g
            else:
                op, target, control, param, angle = g.op, g.target, g.control, g.param, g.angle
            arr[i] = sv_gate(GATE_CODES[op] if isinstance(op, str) else int(op), int(target),
                             int(control), int(param), float(angle))
        self._arr = arr
        self.n_qubits, self.n_params, self.input_dim = n_qubits, n_params, input_dim
        self.struct = sv_circuit(n_qubits, len(gates), n_params, input_dim,
                                 ctypes.cast(arr, ctypes.POINTER(sv_gate)))


class PauliSum:
    """Pauli rows (0=I, 1=X, 2=Y, 3=Z per qubit) and coefficients as X/Z masks."""

    def __init__(self, n_qubits: int, letters, coeffs):
        letters = np.asarray(letters, dtype=np.int64).reshape(-1, n_qubits)
        bits = np.uint64(1) << np.arange(n_qubits, dtype=np.uint64)
        xm = (((letters == 1) | (letters == 2)) * bits).sum(axis=1).astype(np.uint64)
        zm = (((letters == 3) | (letters == 2)) * bits).sum(axis=1).astype(np.uint64)
        self._x = np.ascontiguousarray(xm, dtype=np.uint64)
        self._z = np.ascontiguousarray(zm, dtype=np.uint64)
        self._c = np.ascontiguousarray(coeffs, dtype=np.float64)
        U64 = ctypes.POINTER(ctypes.c_uint64)
        self.n_qubits = n_qubits
        self.struct = sv_pauli_sum(n_qubits, len(self._c),
                                   self._x.ctypes.data_as(U64), self._z.ctypes.data_as(U64),
                                   self._c.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))


def plan_opts(reg_bits=0, threads_per_block=0, no_fusion=False, epilogue=0,
              tile_bits=0, coalesce_bits=0, no_relabel=False,
              tensor_blocks=False) -> sv_plan_opts:
    o = sv_plan_opts()
    o.reg_bits, o.threads_per_block = int(reg_bits), int(threads_per_block)
    o.no_fusion, o.epilogue, o.tile_bits = int(bool(no_fusion)), int(epilogue), int(tile_bits)
    o.coalesce_bits, o.no_relabel = int(coalesce_bits), int(bool(no_relabel))
    o.tensor_blocks = int(bool(tensor_blocks))
    return o


class Problem:
    """An ``sv_problem``: circuit, observable, instances and cost.

    ``inputs``/``weights``/``targets`` are float64 CUDA tensors (or None).
    """

    def __init__(self, circuit: Circuit, observable: PauliSum, refs, dtype="c64",
                 inputs=None, cost="linear", weights=None, targets=None,
                 opts: Optional[sv_plan_opts] = None):
        self.circuit, self.observable, self.opts = circuit, observable, opts
        self._refs = np.ascontiguousarray(refs, dtype=np.int64)
        self.inputs, self.weights, self.targets = inputs, weights, targets
        self.n_instances = len(self._refs)
        self.dtype = _dtype_code(dtype)
        self.cost = SV_COST_MSE if cost == "mse" else SV_COST_LINEAR
        self.struct = sv_problem(
            self.dtype, ctypes.pointer(circuit.struct), ctypes.pointer(observable.struct),
            self.n_instances, self._refs.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
            _ptr(inputs), 0 if inputs is None else int(inputs.shape[1]), self.cost,
            _ptr(weights), _ptr(targets), None if opts is None else ctypes.pointer(opts))

    @property
    def n_params(self) -> int:
        return self.circuit.n_params

    @classmethod
    def from_spec(cls, spec, dtype="c64", device="cuda", opts=None):
        """Marshal any object with the workload attributes (n_qubits, gates,
        n_params, pauli_letters, pauli_coeffs, refs, inputs, weights, targets, cost)."""
        import torch
        d = 0 if spec.inputs is None else int(np.asarray(spec.inputs).shape[1])
        circ = Circuit(spec.n_qubits, spec.gates, spec.n_params, d)
        obs = PauliSum(spec.n_qubits, spec.pauli_letters, spec.pauli_coeffs)

        def dev(a):
            return None if a is None else torch.as_tensor(np.asarray(a, dtype=np.float64),
                                                          device=device).contiguous()
        return cls(circ, obs, spec.refs, dtype, inputs=dev(spec.inputs), cost=spec.cost,
                   weights=dev(spec.weights), targets=dev(spec.targets), opts=opts)


# ------------------------------------------------------------------- states

class StateBatch:
    """``sv_state`` over a torch-owned buffer of shape (batch, 2^n), complex."""

    def __init__(self, n_qubits: int, batch: int, dtype="c64", device="cuda", stream=None):
        import torch
        code = _dtype_code(dtype)
        tdt = torch.complex64 if code == SV_C64 else torch.complex128
        self.tensor = torch.empty((batch, 1 << n_qubits), dtype=tdt, device=device)
        h = ctypes.c_void_p()
        nbytes = self.tensor.numel() * self.tensor.element_size()
        _check(_lib.sv_alloc(ctypes.byref(h), n_qubits, batch, code, _ptr(self.tensor), nbytes,
                             _stream(stream)), "sv_alloc")
        self.handle = h
        self.n_qubits, self.batch, self.dtype = n_qubits, batch, code

    def free(self):
        if self.handle:
            _lib.sv_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def sv_alloc(n_qubits: int, batch: int, dtype="c64", device="cuda", stream=None) -> StateBatch:
    return StateBatch(n_qubits, batch, dtype, device, stream)


def sv_free(state: StateBatch) -> None:
    state.free()


def make_slots(rows) -> ctypes.Array:
    """rows: iterables (circuit, theta_row, shift_param, input_row, ref, shift)."""
    rows = list(rows)
    arr = (sv_slot * max(1, len(rows)))()
    for i, (c, tr, sp, ir, ref, sh) in enumerate(rows):
        arr[i] = sv_slot(int(c), int(tr), int(sp), int(ir), int(ref), float(sh))
    return arr, len(rows)


def sv_apply_circuit_batch(state: StateBatch, circuits: Sequence[Circuit], slots, theta,
                           inputs=None, opts: Optional[sv_plan_opts] = None, stream=None):
    """slots: the (array, count) pair of ``make_slots``; theta: float64 CUDA
    tensor (rows, P); inputs: float64 CUDA tensor (rows, D) or None."""
    arr, count = slots
    circ_arr = (sv_circuit * len(circuits))(*[c.struct for c in circuits])
    th_stride = int(theta.shape[-1]) if theta is not None and theta.dim() > 1 else (
        0 if theta is None else int(theta.numel()))
    in_stride = 0 if inputs is None else int(inputs.shape[-1])
    _check(_lib.sv_apply_circuit_batch(state.handle, circ_arr, len(circuits), arr, count,
                                       _ptr(theta), th_stride, _ptr(inputs), in_stride,
                                       None if opts is None else ctypes.byref(opts),
                                       _stream(stream)), "sv_apply_circuit_batch")


def sv_expect_pauli_sum(state: StateBatch, h: PauliSum, n_rows: Optional[int] = None, out=None,
                        stream=None):
    import torch
    rows = state.batch if n_rows is None else n_rows
    if out is None:
        out = torch.empty(rows, dtype=torch.float64, device=state.tensor.device)
    _check(_lib.sv_expect_pauli_sum(state.handle, ctypes.byref(h.struct), rows, _ptr(out),
                                    _stream(stream)), "sv_expect_pauli_sum")
    return out


def _outputs(problem: Problem, device, energy_out, loss_out, grad_out):
    import torch
    f = dict(dtype=torch.float64, device=device)
    if energy_out is None:
        energy_out = torch.empty(problem.n_instances, **f)
    if loss_out is None:
        loss_out = torch.empty(1, **f)
    if grad_out is None:
        grad_out = torch.empty(max(1, problem.n_params), **f)
    return energy_out, loss_out, grad_out


def sv_energies(problem: Problem, theta, energy_out=None, loss_out=None, stream=None):
    """(loss[1], energies[I]) of every instance in one batched launch."""
    e, l, _ = _outputs(problem, theta.device, energy_out, loss_out, None)
    _check(_lib.sv_energies(ctypes.byref(problem.struct), _ptr(theta), _ptr(e), _ptr(l),
                            _stream(stream)), "sv_energies")
    return l, e


def sv_param_shift_energies(problem: Problem, theta, out=None, stream=None):
    """Energies of the whole parameter-shift batch, [(2P + 1) I], one launch."""
    import torch
    if out is None:
        out = torch.empty((2 * problem.n_params + 1) * problem.n_instances, dtype=torch.float64,
                          device=theta.device)
    _check(_lib.sv_param_shift_energies(ctypes.byref(problem.struct), _ptr(theta), _ptr(out),
                                        _stream(stream)), "sv_param_shift_energies")
    return out


def sv_grad_param_shift(problem: Problem, theta, energy_out=None, loss_out=None, grad_out=None,
                        stream=None):
    """(loss[1], energies[I], grad[P]) by the batched parameter-shift rule."""
    e, l, g = _outputs(problem, theta.device, energy_out, loss_out, grad_out)
    _check(_lib.sv_grad_param_shift(ctypes.byref(problem.struct), _ptr(theta), _ptr(e), _ptr(l),
                                    _ptr(g), _stream(stream)), "sv_grad_param_shift")
    return l, e, g


def sv_grad_param_shift_host(problem: Problem, theta, energy_out=None, loss_out=None,
                             grad_out=None, stream=None):
    """sv_grad_param_shift with host (CPU) float64 tensors in and out; returns
    once the results are in host memory.  (loss[1], energies[I], grad[P])."""
    import torch
    for t in (theta, energy_out, loss_out, grad_out):
        if t is not None and (t.device.type != "cpu" or t.dtype != torch.float64
                              or not t.is_contiguous()):
            raise ValueError("sv_grad_param_shift_host takes contiguous float64 CPU tensors")
    e, l, g = _outputs(problem, torch.device("cpu"), energy_out, loss_out, grad_out)
    _check(_lib.sv_grad_param_shift_host(ctypes.byref(problem.struct), _ptr(theta), _ptr(e),
                                         _ptr(l), _ptr(g), _stream(stream)),
           "sv_grad_param_shift_host")
    return l, e, g


def sv_grad_adjoint(problem: Problem, theta, weights=None, energy_out=None, loss_out=None,
                    grad_out=None, checkpoint_every: int = 0, stream=None):
    """(loss[1], energies[I], grad[P]) by the adjoint reverse sweep.  ``weights``
    (float64 CUDA tensor [I]) replaces dL/dE_i of the problem's cost."""
    e, l, g = _outputs(problem, theta.device, energy_out, loss_out, grad_out)
    _check(_lib.sv_grad_adjoint(ctypes.byref(problem.struct), _ptr(theta), _ptr(weights),
                                _ptr(e), _ptr(l), _ptr(g), int(checkpoint_every),
                                _stream(stream)), "sv_grad_adjoint")
    return l, e, g


def sv_grad_adjoint_host(problem: Problem, theta, energy_out=None, loss_out=None,
                         grad_out=None, checkpoint_every: int = 0, stream=None):
    """sv_grad_adjoint with host (CPU) float64 tensors in and out and the
    problem's own cost; returns once the results are in host memory.
    (loss[1], energies[I], grad[P])."""
    import torch
    for t in (theta, energy_out, loss_out, grad_out):
        if t is not None and (t.device.type != "cpu" or t.dtype != torch.float64
                              or not t.is_contiguous()):
            raise ValueError("sv_grad_adjoint_host takes contiguous float64 CPU tensors")
    e, l, g = _outputs(problem, torch.device("cpu"), energy_out, loss_out, grad_out)
    _check(_lib.sv_grad_adjoint_host(ctypes.byref(problem.struct), _ptr(theta), _ptr(e), _ptr(l),
                                     _ptr(g), int(checkpoint_every), _stream(stream)),
           "sv_grad_adjoint_host")
    return l, e, g


def sv_grad_adjoint_multi(problems, thetas, outputs=None, stream=None):
    """Adjoint gradients of several tile-path problems of different qubit counts
    and depths at once (replayed as one CUDA graph after the first call).
    Returns [(loss[1], energies[I], grad[P])] per problem; ``outputs`` (the
    same list, preallocated) keeps the graph's output pointers fixed."""
    n = len(problems)
    if outputs is None:
        outputs = [(l, e, g) for e, l, g in
                   (_outputs(p, th.device, None, None, None) for p, th in zip(problems, thetas))]
    arr = (sv_problem * n)(*[p.struct for p in problems])
    ptrs = lambda xs: (ctypes.c_void_p * n)(*[_ptr(x) for x in xs])  # noqa: E731
    _check(_lib.sv_grad_adjoint_multi(arr, n, ptrs(thetas), ptrs([o[1] for o in outputs]),
                                      ptrs([o[0] for o in outputs]), ptrs([o[2] for o in outputs]),
                                      _stream(stream)), "sv_grad_adjoint_multi")
    return outputs


def sv_sample(state, row: int, uniforms, counts: bool = False, stream=None):
    """Shots of one state row (Z basis): (samples int64 [S], counts int64 [2^n] or
    None) for the caller's uniforms (float64 CUDA tensor [S] in [0, 1))."""
    import torch
    n = state.n_qubits
    samples = torch.empty(max(1, uniforms.numel()), dtype=torch.int64, device=uniforms.device)
    cnt = torch.empty(1 << n, dtype=torch.int64, device=uniforms.device) if counts else None
    _check(_lib.sv_sample(state.handle, int(row), _ptr(uniforms), int(uniforms.numel()),
                          _ptr(samples), _ptr(cnt), _stream(stream)), "sv_sample")
    return samples[: uniforms.numel()], cnt


def bitstring_counts(samples):
    """The counts map of a shot list, flattened to arrays on the device:
    (distinct basis indices, their counts), indices ascending."""
    import torch
    return torch.unique(samples, sorted=True, return_counts=True)


def sv_param_shift_energies_range(problem: Problem, theta, slot_begin: int, n_slots: int,
                                  out=None, stream=None):
    """Energies of parameter-shift slots [slot_begin, slot_begin + n_slots)."""
    import torch
    if out is None:
        out = torch.empty(max(1, n_slots), dtype=torch.float64, device=theta.device)
    _check(_lib.sv_param_shift_energies_range(ctypes.byref(problem.struct), _ptr(theta),
                                              int(slot_begin), int(n_slots), _ptr(out),
                                              _stream(stream)), "sv_param_shift_energies_range")
    return out[:n_slots]


def sv_param_shift_combine(problem: Problem, energies, energy_out=None, loss_out=None,
                           grad_out=None, stream=None):
    """(loss[1], energies[I], grad[P]) from a whole parameter-shift batch of energies."""
    e, l, g = _outputs(problem, energies.device, energy_out, loss_out, grad_out)
    _check(_lib.sv_param_shift_combine(ctypes.byref(problem.struct), _ptr(energies), _ptr(e),
                                       _ptr(l), _ptr(g), _stream(stream)), "sv_param_shift_combine")
    return l, e, g


def sv_grad_ddcl(problem: Problem, theta, target, js_out=None, grad_out=None, stream=None):
    """(JS[1], grad[P]) of data-driven circuit learning: the Jensen-Shannon
    divergence of the circuit's Z-basis output distribution from ``target``
    (float64 CUDA tensor [2^n]) and its adjoint gradient."""
    import torch
    f = dict(dtype=torch.float64, device=theta.device)
    js_out = torch.empty(1, **f) if js_out is None else js_out
    grad_out = torch.empty(max(1, problem.n_params), **f) if grad_out is None else grad_out
    _check(_lib.sv_grad_ddcl(ctypes.byref(problem.struct), _ptr(theta), _ptr(target),
                             _ptr(js_out), _ptr(grad_out), _stream(stream)), "sv_grad_ddcl")
    return js_out, grad_out


def sv_grad_ddcl_param_shift(problem: Problem, theta, target, js_out=None, grad_out=None,
                             stream=None):
    """(JS[1], grad[P]) as sv_grad_ddcl, by the parameter-shift rule over the
    2P + 1 circuits (the paper's form of the gradient)."""
    import torch
    f = dict(dtype=torch.float64, device=theta.device)
    js_out = torch.empty(1, **f) if js_out is None else js_out
    grad_out = torch.empty(max(1, problem.n_params), **f) if grad_out is None else grad_out
    _check(_lib.sv_grad_ddcl_param_shift(ctypes.byref(problem.struct), _ptr(theta), _ptr(target),
                                         _ptr(js_out), _ptr(grad_out), _stream(stream)),
           "sv_grad_ddcl_param_shift")
    return js_out, grad_out


def sv_grad_param_shift_plain(problem: Problem, theta, energy_out=None, loss_out=None,
                              grad_out=None, stream=None):
    """The plain one-circuit-at-a-time complex128 form (comparison only)."""
    e, l, g = _outputs(problem, theta.device, energy_out, loss_out, grad_out)
    _check(_lib.sv_grad_param_shift_plain(ctypes.byref(problem.struct), _ptr(theta), _ptr(e),
                                          _ptr(l), _ptr(g), _stream(stream)),
           "sv_grad_param_shift_plain")
    return l, e, g


def sv_grad_param_shift_noalloc(problem: Problem, theta, energy_out=None, loss_out=None,
                                grad_out=None, stream=None):
    """sv_grad_param_shift without any device allocation by the library: for
    callers whose device memory belongs to another allocator.  Its scratch is
    one fixed device array shared by all calls (serialise overlapping calls).
    Pass preallocated outputs to avoid torch allocations as well."""
    e, l, g = _outputs(problem, theta.device, energy_out, loss_out, grad_out)
    _check(_lib.sv_grad_param_shift_noalloc(ctypes.byref(problem.struct), _ptr(theta), _ptr(e),
                                            _ptr(l), _ptr(g), _stream(stream)),
           "sv_grad_param_shift_noalloc")
    return l, e, g


def sv_autotune(problem: Problem, theta, kinds: int = 3, stream=None) -> None:
    """Time launch shapes for the parameter-shift energies (kinds & 1) and the
    adjoint (kinds & 2) of this problem; later calls use the fastest."""
    _check(_lib.sv_autotune(ctypes.byref(problem.struct), _ptr(theta), int(kinds),
                            _stream(stream)), "sv_autotune")


def sv_tuned_shape(problem: Problem, kind: int):
    """(reg_bits, threads_per_block, microseconds) chosen by sv_autotune."""
    r, t, us = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_float()
    _check(_lib.sv_tuned_shape(ctypes.byref(problem.struct), int(kind), ctypes.byref(r),
                               ctypes.byref(t), ctypes.byref(us)), "sv_tuned_shape")
    return r.value, t.value, us.value


def sv_tuned_tile(problem: Problem, kind: int):
    """(tile_bits, reg_bits, tensor_blocks, microseconds) chosen by sv_autotune
    for a problem whose states live in device memory."""
    t, r, tc, us = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_float()
    _check(_lib.sv_tuned_tile(ctypes.byref(problem.struct), int(kind), ctypes.byref(t),
                              ctypes.byref(r), ctypes.byref(tc), ctypes.byref(us)),
           "sv_tuned_tile")
    return t.value, r.value, bool(tc.value), us.value


def sv_debug_wait_expiry(limit: int, stream=None) -> None:
    """Test hook: one block whose bounded wait on an mbarrier nothing arrives
    on gives up after `limit` tries and records it in the device error word
    (the next sv_sync_status raises SV_ERR_TIMEOUT)."""
    _check(_lib.sv_debug_wait_expiry(int(limit), _stream(stream)), "sv_debug_wait_expiry")


def sv_plan_info(circuit: Circuit, dtype="c64", opts: Optional[sv_plan_opts] = None) -> dict:
    """How the circuit runs: on chip, or as tile passes (count, tile size)."""
    vals = [ctypes.c_int32() for _ in range(5)]
    _check(_lib.sv_plan_info(ctypes.byref(circuit.struct), _dtype_code(dtype),
                             None if opts is None else ctypes.byref(opts),
                             *[ctypes.byref(v) for v in vals]), "sv_plan_info")
    keys = ("on_chip", "n_passes", "tile_bits", "n_stages", "n_groups")
    return {k: v.value for k, v in zip(keys, vals)}


def sv_h_plan_info(observable: PauliSum, dtype="c64") -> dict:
    """How lambda = H psi runs for states on the tile path: passes, tile size."""
    vals = [ctypes.c_int32() for _ in range(2)]
    _check(_lib.sv_h_plan_info(ctypes.byref(observable.struct), _dtype_code(dtype),
                               *[ctypes.byref(v) for v in vals]), "sv_h_plan_info")
    return {"n_passes": vals[0].value, "tile_bits": vals[1].value}


def sv_phase_timing(on: bool = True) -> None:
    """Turn CUDA-event phase timing of device-memory adjoint gradients on/off."""
    _check(_lib.sv_phase_timing(int(bool(on))), "sv_phase_timing")


def sv_last_phase_ms() -> dict:
    """Milliseconds of the last timed adjoint's forward, H and reverse phases."""
    vals = [ctypes.c_float() for _ in range(3)]
    _check(_lib.sv_last_phase_ms(*[ctypes.byref(v) for v in vals]), "sv_last_phase_ms")
    return {"forward_ms": vals[0].value, "h_ms": vals[1].value, "reverse_ms": vals[2].value}


def sv_last_adjoint_info() -> dict:
    """The checkpoint interval and the algorithmic bytes of the reverse tile
    passes of the last device-memory adjoint on the current device (both 0
    after an on-chip adjoint)."""
    every, nbytes = ctypes.c_int32(), ctypes.c_int64()
    _check(_lib.sv_last_adjoint_info(ctypes.byref(every), ctypes.byref(nbytes)),
           "sv_last_adjoint_info")
    return {"checkpoint_every": every.value, "reverse_bytes": nbytes.value}


def sv_status_string(status: int) -> str:
    return _lib.sv_status_string(int(status)).decode()


def sv_last_error() -> str:
    return _lib.sv_last_error().decode()


def sv_sync_status(stream=None) -> None:
    _check(_lib.sv_sync_status(_stream(stream)), "sv_sync_status")


def sv_shutdown() -> None:
    _check(_lib.sv_shutdown(), "sv_shutdown")


def sv_version() -> int:
    return int(_lib.sv_version())


def library():
    """The loaded ctypes library (for symbol checks)."""
    return _lib
