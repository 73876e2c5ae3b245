"""The virtual-QPU split (Sec. 3, Sec. 4.1): contiguous segments per rank
and one allgather, on CPU with gloo ranks; each rank evaluates only its
segment of the parameter-shift batch with the oracle, and the assembled
batch must give the oracle's gradient."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _vqpu():
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "vqpu", os.path.join(ROOT, "paper_2406_03466_gb300", "vqpu.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_segments_partition_the_batch():
    v = _vqpu()
    for n in (0, 1, 7, 33, 585):
        for world in (1, 2, 3, 8):
            segs = [v.segment(n, world, r) for r in range(world)]
            assert segs[0][0] == 0 and segs[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(segs, segs[1:]))
            sizes = [hi - lo for lo, hi in segs]
            assert max(sizes) - min(sizes) <= 1


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    import workloads as wl
    v = _vqpu()
    w = wl.mcvqe(6, 2, "all", n_refs=3)
    inst, sp, sh = oracle.param_shift_slots(w)
    seen = []

    def evaluate(lo, hi):
        seen.append((lo, hi))
        return torch.as_tensor(oracle.energies(w, None, inst[lo:hi], sp[lo:hi], sh[lo:hi]))

    E = v.distributed_energies(len(inst), evaluate, dist).numpy()
    q.put((rank, E, seen))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_assemble_the_oracle_batch(world):
    import oracle
    import workloads as wl
    w = wl.mcvqe(6, 2, "all", n_refs=3)
    inst, sp, sh = oracle.param_shift_slots(w)
    full = oracle.energies(w, None, inst, sp, sh)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = [q.get(timeout=180) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    v = _vqpu()
    for rank, E, seen in got:
        assert seen == [v.segment(len(inst), world, rank)]  # only its own segment
        np.testing.assert_allclose(E, full, rtol=0, atol=1e-14)
    # the assembled batch gives the oracle's gradient
    I = w.n_instances
    Es = full[I:].reshape(-1, 2, I)
    g = (0.5 * (Es[:, 0, :] - Es[:, 1, :])) @ oracle.cost_weights(w, full[:I])
    np.testing.assert_allclose(g, oracle.grad_param_shift(w)[2], atol=1e-13)
