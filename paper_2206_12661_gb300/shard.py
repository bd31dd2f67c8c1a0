"""One hologram split by pupil rows over several shards (devices or ranks).

Eq. 2 separates over the pupil rows: Theta_k is a sum over the rows n of
Fy[k,n] sum_m E[n,m] Fx[k,m].  A hologram can therefore be split into row shards,
each holding its rows of the pupil field and of Fy (and all of Fx).  One iteration of
the loop is then

  1. every shard computes its partial Theta over its rows (Eq. 2 restricted to them);
  2. the partials are summed over the shards: one all-reduce of K complex values;
  3. every shard runs the generalized weighting update on the sum -- the same sum and
     the same arithmetic, so every shard keeps identical weights -- and the inverse
     product for its own rows, which needs nothing from the other shards.

This module holds the orchestration only (which rows a shard owns, the order of the
three steps, the reduction); the arithmetic runs in the shard objects, which for GPU
shards call the library (ofa_shard_forward / ofa_shard_update).  A shard object has
``forward() -> partial`` and ``update(total)``; partials are [K, 2] arrays or tensors
(real, imaginary).
"""
from __future__ import annotations


def row_ranges(ny: int, shards: int) -> list[tuple[int, int]]:
    """Contiguous (first row, row count) slices of ny rows over `shards` shards, the
    first ny % shards of them one row longer."""
    if shards < 1 or shards > ny:
        raise ValueError("need 1 <= shards <= ny")
    base, extra = divmod(ny, shards)
    out, r0 = [], 0
    for g in range(shards):
        rows = base + (1 if g < extra else 0)
        out.append((r0, rows))
        r0 += rows
    return out


def fixed_order_sum(partials):
    """Sum of the partials in shard order (the same bits on every run)."""
    total = partials[0].clone() if hasattr(partials[0], "clone") else partials[0].copy()
    for p in partials[1:]:
        total += p
    return total


class DistributedSum:
    """All-reduce (sum) of this rank's partial over a torch.distributed group; each rank
    holds one shard.  Ranks that stop answering make the collective raise once the
    group's timeout expires, instead of hanging."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group

    def __call__(self, partials):
        total = fixed_order_sum(partials)
        self.dist.all_reduce(total, op=self.dist.ReduceOp.SUM, group=self.group)
        return total


class ShardedLoop:
    """Runs the loop over local shards with a reduction of their partials."""

    def __init__(self, shards, reduce=fixed_order_sum):
        self.shards = list(shards)
        self.reduce = reduce

    def step(self):
        partials = [s.forward() for s in self.shards]
        total = self.reduce(partials)
        for s in self.shards:
            s.update(total)
        return total

    def run(self, n_iter: int):
        for _ in range(int(n_iter)):
            self.step()


class PlanShard:
    """A GPU shard: an ofa plan over rows [row0, row0 + rows) of a workload's pupil."""

    def __init__(self, w, row0: int, rows: int, precision="f16x3", stream=None, **kw):
        """stream: the torch stream handle (non-zero) that the reduction of the partials
        also runs on; the library orders nothing across streams."""
        import numpy as np
        import torch

        from . import ofa
        if not stream:
            raise ValueError("a GPU shard needs the (non-default) stream its reduction runs on")
        self.ofa, self.torch = ofa, torch
        sl = slice(row0, row0 + rows)
        amp = np.ascontiguousarray(w.amplitude[sl])
        phi0 = np.ascontiguousarray(w.phi0[sl])
        self.plan = ofa.Plan(w.nx, rows, w.pitch_x, w.pitch_y, w.wavelength, w.focal_length,
                             w.focus_xy, w.target, precision=precision, amplitude=amp,
                             phi0=phi0, stream=stream, shard=(row0, w.ny), **kw)
        self.row0, self.rows, self.K = row0, rows, w.n_foci
        self.partial = torch.zeros(self.K, 2, dtype=torch.float32, device="cuda")

    def forward(self):
        self.ofa.ofa_shard_forward(self.plan.handle, self.partial)
        return self.partial

    def update(self, total):
        self.ofa.ofa_shard_update(self.plan.handle, total)

    def close(self):
        self.plan.close()
