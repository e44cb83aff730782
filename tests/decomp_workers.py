"""Workers for the key-range decomposition test on CPU ranks (a module of
its own so that spawned processes can import it).  The compute is the FP64
oracle: the decomposition's host logic and collectives are what is tested."""
import os

import numpy as np


class OracleCompute:
    """The per-rank compute of KeyRangeDecomposition, done by the oracle."""

    def __init__(self, w, theta):
        self.w, self.theta = w, theta
        self.T = None

    def build(self, pos_t):
        import oracle
        import torch
        pos = pos_t.numpy()
        k = oracle.keys(pos, self.w.box)[0]
        _, order = oracle.sort(k)
        self.order = np.asarray(order, dtype=np.int64)
        if self.T is not None:
            self.T.close()
        self.T = oracle.Tree(pos, self.w.mass, 2.8 * self.w.eps, box=self.w.box)
        return torch.tensor(self.order)

    def n_groups(self):
        return (self.w.n + 31) // 32

    def _targets(self, g0, g1):
        return self.order[32 * g0: min(32 * g1, self.w.n)]

    def accel(self, g0, g1):
        import torch
        tg = self._targets(g0, g1)
        acc = np.zeros((self.w.n, 3))
        cnt = np.zeros(self.w.n, np.int64)
        if len(tg):
            a, c = self.T.walk(self.w.r_s, self.w.rcut, self.theta, tg)
            acc[tg], cnt[tg] = a, c
        return torch.tensor(acc), torch.tensor(cnt)

    def adjoint(self, g0, g1, wt):
        import torch
        tg = self._targets(g0, g1)
        wm = np.zeros_like(wt.numpy())
        wm[tg] = wt.numpy()[tg]
        dp, dm = self.T.adjoint(self.w.r_s, self.w.rcut, self.theta, wm)
        return torch.tensor(dp), torch.tensor(dm)


def decomp_rank(rank, ws, port, q, name, scale):
    try:
        _decomp_rank(rank, ws, port, q, name, scale)
    except Exception:  # report instead of leaving the parent waiting
        import traceback
        q.put((rank, "error", traceback.format_exc()))
        raise


def _decomp_rank(rank, ws, port, q, name, scale):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import ics
    from paper_2606_17145_gb300.decomp import KeyRangeDecomposition
    w = ics.make(name, scale)
    wt = torch.tensor(ics.loss_weights(w.n, 41))
    D = KeyRangeDecomposition(rank, ws, OracleCompute(w, 0.5))
    pos = torch.tensor(w.pos)
    D.build(pos)
    rows = D.owned_rows()
    # a drift that only the owner applies, then the all-gather by rows
    moved = pos.clone()
    moved[rows] += 1e-4 * torch.tensor(np.random.default_rng(7).standard_normal((w.n, 3)))[rows]
    gathered = D.gather_rows(moved, rows)
    acc, cnt = D.accel()
    dpos, dmass = D.adjoint(wt)
    ranges1 = list(D.ranges)
    ranges2 = D.rebalance(cnt)
    D.build(pos)
    acc2, cnt2 = D.accel()
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, gathered.numpy(), rows.numpy(), acc.numpy(), cnt.numpy(), dpos.numpy(), dmass.numpy(), ranges1,
           ranges2, acc2.numpy()))
