"""Virtual QPUs over ranks (Sec. 3; Sec. 4.1 last paragraphs): the vector of
circuits of a gradient is split into one contiguous segment per rank, every
rank evaluates its segment, and one allgather assembles the batch.

Host-side logic only (partition and gather); the circuits run in the
library (`sv_param_shift_energies_range`) and the combination in
`sv_param_shift_combine`.
"""
from typing import Callable, Tuple


def segment(n_items: int, world: int, rank: int) -> Tuple[int, int]:
    """[lo, hi) of rank's contiguous segment; sizes differ by at most one, the
    first n_items % world ranks take one more."""
    if world < 1 or not 0 <= rank < world or n_items < 0:
        raise ValueError("bad segment request")
    base, extra = divmod(n_items, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def gather_segments(local, n_items: int, dist, device=None):
    """All segments, in rank order, on every rank.  `local` is this rank's
    segment (a float64 tensor); with dist None it is the whole vector."""
    import torch
    if dist is None:
        return local
    world, rank = dist.get_world_size(), dist.get_rank()
    width = -(-n_items // world)
    buf = torch.zeros(width, dtype=torch.float64, device=device or local.device)
    buf[: local.numel()] = local
    parts = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(parts, buf)
    out = [parts[r][: segment(n_items, world, r)[1] - segment(n_items, world, r)[0]]
           for r in range(world)]
    return torch.cat(out)


def distributed_energies(n_items: int, evaluate: Callable, dist, device=None):
    """Every item's value on every rank: rank r evaluates `evaluate(lo, hi)`
    for its own segment only."""
    if dist is None:
        return evaluate(0, n_items)
    lo, hi = segment(n_items, dist.get_world_size(), dist.get_rank())
    return gather_segments(evaluate(lo, hi), n_items, dist, device)


def param_shift_gradient(problem, theta, dist=None, stream=None):
    """(loss, energies, gradient) of one parameter-shift gradient with the
    batch split over the ranks of `dist` (one GPU per rank)."""
    import paper_2406_03466_gb300 as sv
    B = (2 * problem.n_params + 1) * problem.n_instances

    def evaluate(lo, hi):
        return sv.sv_param_shift_energies_range(problem, theta, lo, hi - lo, stream=stream)

    E = distributed_energies(B, evaluate, dist, theta.device)
    return sv.sv_param_shift_combine(problem, E.contiguous(), stream=stream)
