"""Key-range decomposition of the short-range walk over ranks (one GPU each).

The paper distributes its walks over MPI ranks by domain and exports to
other ranks the particles their targets need (Sec. 2).  On a GB300 the
state of a whole set is small beside HBM (80 B per particle in the tree's
layout: 1.3 GB for 16.8M particles) and keys, sort and tree take a fraction
of a percent of a step, while the walk takes the rest.  So every rank keeps
all positions and builds the same keys, sort and tree, and the walk is what
is split: rank r walks a contiguous range of walk groups, i.e. a range of
Peano-Hilbert keys of its targets.  Per step:

  1. positions: each rank owns the rows of its previous targets; one
     all-reduce of disjoint rows (the others zero) gives every rank all of
     them (an all-gather by index);
  2. keys, sort, tree: identical on every rank (integer keys, a stable sort
     and a deterministic tree), no exchange;
  3. walk: rank r walks its range; its targets' accelerations are exactly
     those of the single-GPU walk (each group's walk is independent);
  4. forces, where every rank needs all of them: one all-reduce of disjoint
     rows;
  5. adjoint: rank r computes the gradient of its partial loss (the sum over
     its targets of w . a) for every particle; the loss is a sum over
     targets, so one all-reduce of the ranks' gradients gives the gradient;
  6. balance: the next ranges split this step's per-group interaction counts
     into equal parts (contiguous, so a rank's targets stay a key range).

The collectives go through torch.distributed (NCCL between GPUs).  The
compute is passed in: CudaCompute runs the og_* calls of libog.so; the tests
also run the same driver on CPU ranks with the oracle as the compute.
"""
from __future__ import annotations

import numpy as np
import torch

GROUP = 32  # targets per walk group


def partition(work, nranks: int) -> list[tuple[int, int]]:
    """Split groups 0..len(work)-1 into nranks contiguous ranges [g0, g1) whose
    sums of work are as equal as contiguous cuts allow: cut k sits at the
    first group where the running sum reaches k / nranks of the total.
    Every group is in exactly one range; a range may be empty when there are
    fewer groups than ranks."""
    w = np.asarray(work, dtype=np.float64)
    ng = w.shape[0]
    if nranks < 1:
        raise ValueError("nranks must be >= 1")
    if ng == 0:
        return [(0, 0)] * nranks
    w = np.maximum(w, 0.0)
    total = float(w.sum())
    if total <= 0.0:
        w = np.ones(ng)
        total = float(ng)
    csum = np.cumsum(w)
    cuts = [0]
    for k in range(1, nranks):
        c = int(np.searchsorted(csum, total * k / nranks, side="left")) + 1
        cuts.append(min(max(c, cuts[-1]), ng))
    cuts.append(ng)
    return [(cuts[r], cuts[r + 1]) for r in range(nranks)]


def group_work(counts_sorted, n_groups: int) -> np.ndarray:
    """Per-group sums of per-target work (interaction counts) given in sorted
    (Hilbert) order; a ragged last group sums what it has."""
    c = np.asarray(counts_sorted, dtype=np.float64)
    pad = n_groups * GROUP - c.shape[0]
    if pad > 0:
        c = np.concatenate([c, np.zeros(pad)])
    return c[: n_groups * GROUP].reshape(n_groups, GROUP).sum(axis=1)


class CudaCompute:
    """The per-rank compute on this rank's GPU: keys, sort, tree and the
    group-range walks of libog.so (buffers allocated once)."""

    def __init__(self, n: int, mass: torch.Tensor, eps, box: float, r_s: float, theta: float, p=None):
        from . import _workspace, lib, params
        import ctypes as C
        L = lib()
        dev = mass.device
        self.n, self.mass, self.eps, self.box, self.r_s, self.theta = n, mass, eps, float(box), float(r_s), float(theta)
        self.p = p or params()
        self.ws_keys = _workspace(L.og_keys_sort_ws_bytes(n), dev)
        self.keys = torch.empty(n, dtype=torch.int64, device=dev)
        self.order = torch.empty(n, dtype=torch.int32, device=dev)
        self.tree_mem = _workspace(L.og_tree_bytes(n, C.byref(self.p)), dev)
        self.tree = None
        self.ws_acc = None
        self.ws_adj = None

    def build(self, pos: torch.Tensor) -> torch.Tensor:
        """Keys, sort and tree of all positions; returns order (sorted -> original)."""
        from . import keys_sort, tree_build, lib
        import ctypes as C
        keys_sort(pos, self.box, ws=self.ws_keys, keys=self.keys, order=self.order)
        self.tree = tree_build(self.keys, self.order, pos, self.mass, self.eps, self.box, p=self.p, mem=self.tree_mem)
        if self.ws_acc is None:
            L = lib()
            from . import _workspace
            self.ws_acc = _workspace(L.og_accel_ws_bytes(C.byref(self.tree.header), 0), pos.device)
            self.ws_adj = _workspace(L.og_adjoint_ws_bytes(C.byref(self.tree.header), 1), pos.device)
        return self.order

    def n_groups(self) -> int:
        return int(self.tree.header.n_groups)

    def accel(self, g0: int, g1: int):
        """(acc [n,3] float32 with the range's target rows filled and the others
        zero, per-particle interaction counts likewise)."""
        from . import shortrange_accel
        dev = self.mass.device
        acc = torch.zeros((self.n, 3), dtype=torch.float32, device=dev)
        acc, _, cnt = shortrange_accel(self.tree, self.r_s, self.theta, counts=True, ws=self.ws_acc, out=acc,
                                       groups=(g0, g1))
        cnt = torch.where(cnt < 0, torch.zeros_like(cnt), cnt)
        mask = torch.zeros(self.n, dtype=torch.bool, device=dev)
        mask[self.order[GROUP * g0: min(GROUP * g1, self.n)].long()] = True
        return acc, torch.where(mask, cnt, torch.zeros_like(cnt))

    def adjoint(self, g0: int, g1: int, w: torch.Tensor):
        """Gradient (dpos [n,3], dmass [n], float64) of the partial loss over the
        range's targets."""
        from . import shortrange_adjoint
        return shortrange_adjoint(self.tree, self.r_s, self.theta, w.to(torch.float32).contiguous(),
                                  ws=self.ws_adj, groups=(g0, g1))


class KeyRangeDecomposition:
    """Rank `rank` of `world` ranks sharing the walk of one particle set.

    compute: an object with build(pos) -> order, n_groups(), accel(g0, g1) ->
    (acc, counts) and adjoint(g0, g1, w) -> (dpos, dmass) (CudaCompute on a
    GPU).  pg: the torch.distributed process group (None: the default)."""

    def __init__(self, rank: int, world: int, compute, pg=None):
        self.rank, self.world, self.compute, self.pg = rank, world, compute, pg
        self.ranges = None
        self.order = None

    def _sum(self, t: torch.Tensor) -> torch.Tensor:
        if self.world > 1:
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.SUM, group=self.pg)
        return t

    def owned_rows(self) -> torch.Tensor:
        """Original indices of this rank's targets (its rows), from the last build."""
        g0, g1 = self.ranges[self.rank]
        return self.order[GROUP * g0: min(GROUP * g1, self.order.shape[0])].long()

    def gather_rows(self, x: torch.Tensor, rows: torch.Tensor) -> torch.Tensor:
        """Every rank passes its full-size array with its own rows valid; the
        result holds every rank's rows on every rank (ranks' rows disjoint,
        the others zeroed before one all-reduce)."""
        y = torch.zeros_like(x)
        y[rows] = x[rows]
        return self._sum(y)

    def build(self, pos: torch.Tensor):
        """Keys, sort and tree of the full positions; the first call splits the
        groups evenly, later ranges come from rebalance()."""
        self.order = self.compute.build(pos)
        ng = self.compute.n_groups()
        if self.ranges is None or self.ranges[-1][1] != ng:
            self.ranges = partition(np.ones(ng), self.world)
        return self

    def accel(self, assemble: bool = True):
        """Accelerations of this rank's targets (assemble: of all particles, on
        every rank) and the interaction counts (assembled likewise)."""
        g0, g1 = self.ranges[self.rank]
        acc, cnt = self.compute.accel(g0, g1)
        if assemble:
            acc = self._sum(acc)
            cnt = self._sum(cnt)
        return acc, cnt

    def adjoint(self, w: torch.Tensor):
        """dL/dx, dL/dm of L = sum_i w_i . a_i over all targets, on every rank."""
        g0, g1 = self.ranges[self.rank]
        dpos, dmass = self.compute.adjoint(g0, g1, w)
        return self._sum(dpos.clone()), self._sum(dmass.clone())

    def rebalance(self, counts: torch.Tensor):
        """Ranges for the next step from per-particle interaction counts
        (original order, as assembled by accel())."""
        c = counts.detach().to("cpu").double().numpy()
        order = self.order.detach().to("cpu").long().numpy()
        self.ranges = partition(group_work(c[order], self.compute.n_groups()), self.world)
        return self.ranges
