"""Event-sharded likelihood over several GPUs, one process per GPU.

The NLL and its gradient are sums over events (Sec. 3 of the paper: the PDF is
evaluated one thread per event and the log-likelihoods are summed).  Rank r of
W holds one contiguous range of the events whose start is a multiple of
IPA_SHARD_EVENTS (one 32-tile group of the kernel's reduction tree).  A pass
is: ipa_nll_grad_shard on the rank's events (its group partials), one
all-gather of the group partials in rank order, and ipa_nll_grad_combine on
all of them, which runs the kernel's last, fixed-order reduction level and the
gradient contraction.  Every rank ends with the bits that ipa_nll_grad gives
for all events on one GPU, for any W, so every rank's minimiser (ipa_fit_begin /
ipa_fit_advance) takes the same steps and no further exchange is needed.

This module only partitions, exchanges and sequences library calls: every
step of the computation runs in the library's kernels.
"""
from __future__ import annotations

import torch

from . import _capi as C
from . import api


def shard_bounds(n: int, rank: int, world: int) -> tuple[int, int]:
    """Events [lo, hi) of `rank` among `world` ranks: the ceil(n / IPA_SHARD_EVENTS)
    groups split into `world` contiguous runs of nearly equal length."""
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError("need 0 <= rank < world and n >= 0")
    g = api.shard_groups(n)
    g0, g1 = rank * g // world, (rank + 1) * g // world
    return min(g0 * C.IPA_SHARD_EVENTS, n), min(g1 * C.IPA_SHARD_EVENTS, n)


def shard_rows(n: int, world: int) -> list[int]:
    """Group partials each rank contributes, in rank order."""
    return [api.shard_groups(hi - lo) for lo, hi in (shard_bounds(n, r, world) for r in range(world))]


def gather_groups(local: torch.Tensor, rows: list[int], rank: int, group=None) -> torch.Tensor:
    """All-gather of the ranks' group partials (rank r contributes rows[r] rows of
    `local.shape[1]` doubles), concatenated in rank order on every rank.  The
    blocks are padded to the longest one for the collective and trimmed after."""
    import torch.distributed as dist
    world = len(rows)
    width = local.shape[1] if local.dim() == 2 else 1
    if local.shape[0] != rows[rank]:
        raise ValueError(f"rank {rank} holds {local.shape[0]} rows, expected {rows[rank]}")
    if world == 1:
        return local
    longest = max(rows)
    pad = torch.zeros(longest, width, dtype=local.dtype, device=local.device)
    pad[:rows[rank]] = local.view(-1, width)
    out = torch.empty(world * longest, width, dtype=local.dtype, device=local.device)
    dist.all_gather_into_tensor(out, pad, group=group)
    return torch.cat([out[r * longest:r * longest + rows[r]] for r in range(world)])


class ShardedNLL:
    """NLL and gradient of n_total events of which this rank holds `ev_local`
    (events shard_bounds(n_total, rank, world)), identical on every rank."""

    def __init__(self, model, ev_local: dict, n_total: int, rank: int = 0, world: int = 1, group=None,
                 cached: bool = False):
        lo, hi = shard_bounds(n_total, rank, world)
        if int(ev_local["t"].numel()) != hi - lo:
            raise ValueError(f"rank {rank} holds {ev_local['t'].numel()} events, its shard is [{lo}, {hi})")
        self.model, self.ev, self.rank, self.world, self.group = model, ev_local, rank, world, group
        self.cached = cached or ev_local.get("fk") is not None
        self.rows = shard_rows(n_total, world)
        dev = ev_local["t"].device
        self.width = api.ipa_shard_width(model)
        self.local_out = torch.empty(1 + model.n_par, dtype=torch.float64, device=dev)
        self.local_groups = torch.empty(self.rows[rank], self.width, dtype=torch.float64, device=dev)
        self.out = torch.empty(1 + model.n_par, dtype=torch.float64, device=dev)

    def nll_grad(self, theta: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        out = self.out if out is None else out
        api.ipa_nll_grad_shard(self.model, self.ev, theta, self.local_out, self.local_groups)
        groups = gather_groups(self.local_groups, self.rows, self.rank, self.group)
        return api.ipa_nll_grad_combine(self.model, theta, groups, self.cached, out)

    def fit(self, params: list, theta0: torch.Tensor, max_iter: int = 200, tol: float = 1e-9,
            check_every: int = 8, max_passes: int | None = None) -> dict:
        """One fit of all n_total events: the library's minimiser (the state
        machine of ipa_fit_batch) advanced one pass at a time, each pass the
        sharded NLL and gradient.  Every rank runs the same steps on the same
        bits and returns the same result."""
        P = self.model.n_par
        dev = theta0.device
        state = api.fit_state_new(1, P, dev)
        api.ipa_fit_begin(self.model, params, theta0.reshape(1, P), state, max_iter=max_iter, tol=tol)
        points = api.fit_state_points(state, 1, P)
        res = torch.empty(1, 1 + P, dtype=torch.float64, device=dev)
        n_active = torch.ones(1, dtype=torch.int32, device=dev)
        limit = max_passes if max_passes is not None else 6 * max_iter + 4 * P + 48
        passes = 0
        while passes < limit:
            for _ in range(check_every):
                self.nll_grad(points[0], res[0])
                api.ipa_fit_advance(self.model, 1, res, state, n_active)
                passes += 1
            if int(n_active.item()) == 0:
                break
        return api.ipa_fit_end(self.model, 1, state)
