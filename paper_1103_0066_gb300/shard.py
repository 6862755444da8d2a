"""One mesh split across torch.distributed ranks by elements.

Elements are independent units of the element integration (Sec. 4: every
A_e = G_e : K needs only its own element), so rank r of a world of N takes the
contiguous element range element_range(E, N, r) and runs the forward and the
adjoint kernels on that slice alone:

  * the forward writes A_e of its own elements: no exchange;
  * the adjoint's coefficient gradient dcoef_e is per element: no exchange;
  * the adjoint's vertex gradient dcoords[v] sums the contributions of every
    element at v, and the elements around a vertex on a range boundary lie on
    two ranks.  Each rank reduces its own elements into a partial [V][d] sum
    (the deterministic record reduction of its slice), and one all-reduce
    (NCCL on GPUs) adds the partials.  That sum is the path's one exchange
    step.  For a fixed world size and collective configuration it is
    reproducible run to run; its order across ranks is the collective's.

Every rank holds the whole vertex array (coords, dcoords); only the element
arrays are split.
"""
from __future__ import annotations

import torch
import torch.distributed as dist

from . import REDUCE_DETERMINISTIC, Workspace, integrate_bwd, integrate_fwd


def element_range(n_elem: int, world: int, rank: int) -> tuple[int, int]:
    """[e0, e1) of rank `rank`: contiguous ranges, sizes differing by at most
    one, covering [0, n_elem) in rank order."""
    if world < 1 or not 0 <= rank < world or n_elem < 0:
        raise ValueError("need world >= 1, 0 <= rank < world and n_elem >= 0")
    q, r = divmod(n_elem, world)
    e0 = rank * q + min(rank, r)
    return e0, e0 + q + (1 if rank < r else 0)


def _world(group):
    if not dist.is_available() or not dist.is_initialized():
        return 1, 0
    return dist.get_world_size(group), dist.get_rank(group)


def exchange_dcoords(partial: torch.Tensor, group=None) -> torch.Tensor:
    """Sums the ranks' partial vertex gradients in place (all-reduce); a
    no-op on one rank or without a process group."""
    world, _ = _world(group)
    if world > 1:
        dist.all_reduce(partial, op=dist.ReduceOp.SUM, group=group)
    return partial


class ShardedMesh:
    """This rank's slice of a mesh: coords [V][d] (whole) and conn [E][d+1]
    (whole; only rows e0..e1-1 are used).  The adjoint workspace of the slice
    is built on the first integrate_bwd and kept."""

    def __init__(self, coords: torch.Tensor, conn: torch.Tensor, form: int, group=None):
        self.group = group
        self.world, self.rank = _world(group)
        self.n_elem = conn.shape[0]
        self.e0, self.e1 = element_range(self.n_elem, self.world, self.rank)
        self.coords = coords
        self.conn = conn[self.e0:self.e1].contiguous()
        self.form = form
        self.ws = None

    def local(self, a: torch.Tensor | None) -> torch.Tensor | None:
        """Rows e0..e1-1 of a per-element array of the whole mesh."""
        return None if a is None else a[self.e0:self.e1]

    def integrate_fwd(self, coef=None, **kw) -> torch.Tensor:
        """A_e of this rank's elements ([e1 - e0][n][n]); coef: this rank's
        rows of a per-element coefficient, or the whole [V] vertex values of a
        P1 coefficient (the _W1 forms)."""
        return integrate_fwd(self.coords, self.conn, self.form, coef, **kw)

    def integrate_bwd(self, dA: torch.Tensor, coef=None, need_dcoef=True, **kw):
        """(dcoords [V][d] of the whole mesh, summed over the ranks; dcoef of
        this rank's elements) for this rank's upstream dA ([e1 - e0][n][n])."""
        if self.ws is None:
            self.ws = Workspace(self.coords, self.conn, self.form)
        dx, dw = integrate_bwd(self.coords, self.conn, self.form, dA, coef, ws=self.ws,
                               reduce=REDUCE_DETERMINISTIC, need_dcoef=need_dcoef, **kw)
        return exchange_dcoords(dx, self.group), dw
