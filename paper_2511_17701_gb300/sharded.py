"""The adjoint of the pusher over frozen fields, sharded by particle across ranks.

Test particles in frozen fields (steps 2-11 of Sec. 3.1 of arXiv:2511.17701, no deposit, no
field update) do not interact, so the work splits by particle with no halo and no
migration: every rank pushes its own contiguous share of the particles through its own
copy of the field on its own GPU (the library's adjoint: forward with checkpoints, then the
reverse sweep). The gradients with respect to each particle's initial state stay on the
rank that owns the particle. The one exchange is the gradient with respect to the field
amplitude B0, a sum over every particle's term: each rank bins its terms exactly on its GPU
(grpic_sum_bins_add: integer sums per binary exponent), one all-reduce adds the int64 bins
across ranks (NCCL on GPUs, gloo without), and the library rounds the total once
(grpic_sum_bins_value). The result is the correctly rounded sum of all the terms: the same
bits for any number of ranks and any split of the particles.
"""
from __future__ import annotations

from .binding import SUM_BINS, sum_bins_add, sum_bins_value


def shard_bounds(n: int, rank: int, world: int) -> tuple[int, int]:
    """[lo, hi) of a rank's contiguous share of n particles: the first n % world ranks hold
    one particle more than the others."""
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError("bad shard request")
    q, r = divmod(n, world)
    lo = rank * q + min(rank, r)
    return lo, lo + q + (1 if rank < r else 0)


def library_adjoint(sim, qm: float, b0: float, n_steps: int, ckpt_every: int, n_iter: int):
    """One rank's local adjoint on its FP64 Sim: f(state0, cot) -> (final state, d/d state0,
    the int64 bins of the per-particle d/d B0 terms), all on the rank's GPU."""
    import torch

    def run(state0, cot):
        out, ckpt = sim.adjoint_forward(state0, qm, b0, n_steps, ckpt_every, n_iter)
        ok = ~torch.isnan(out[0])
        gout = (cot * ok).contiguous()
        gin, gpp, _ = sim.adjoint_backward(ckpt, gout, qm, b0, n_steps, ckpt_every, n_iter)
        bins = torch.zeros(2 * SUM_BINS, dtype=torch.int64, device=gpp.device)
        sum_bins_add(gpp.contiguous(), bins, sim.stream)
        return out, gin, bins
    return run


def sharded_adjoint(local_adjoint, state0, cot, group=None):
    """One rank's share of the sharded adjoint. state0, cot: this rank's (6, n_local) initial
    states and cotangents of the final states (its slice from shard_bounds);
    local_adjoint(state0, cot) -> (final state, d/d state0, int64 bins of the rank's d/d B0
    terms) runs the rank's particles (library_adjoint on a GPU). Returns (final state,
    d/d state0 of the rank's particles, dL/dB0 over every rank's particles), with L the sum
    over all particles of cot . final state."""
    import torch.distributed as dist
    out, gin, bins = local_adjoint(state0, cot)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(bins, op=dist.ReduceOp.SUM, group=group)
    return out, gin, sum_bins_value(bins.cpu())
