"""Process-pool workers for oracle work in the tests (numpy + oracle only;
no torch, no GPU), started with the spawn method."""
import numpy as np


def fd_chunk(args):
    """Central finite differences of the oracle's frozen-list loss for the
    given particles of a named workload (weights rounded to float32 like the
    GPU input)."""
    name, samples, theta = args
    import ics
    import oracle
    w = ics.make(name)
    T = oracle.Tree(w.pos, w.mass, 2.8 * w.eps)
    wt = w.w.astype(np.float32).astype(np.float64)
    smp = np.asarray(samples, dtype=np.int64)
    fp, fm, fl = T.fd(w.r_s, w.rcut, theta, wt, smp, hx=1e-6, hm_rel=1e-6, with_flags=True)
    ap, am, sp, sm = T.adjoint(w.r_s, w.rcut, theta, wt, smp, with_scale=True)
    return fp, fm, fl, ap, am, sp, sm
