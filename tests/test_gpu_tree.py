"""K3/K4 parity: the GPU octree has exactly the oracle's nodes (same cells,
counts, leaf flags) and their FP64 moments agree to rounding."""
import numpy as np
import pytest

import ics
from gpu_util import build_tree, device, torch

pytestmark = pytest.mark.gpu


def _gpu_nodes(w, dev, leaf_size=8):
    tree, keys, order = build_tree(w, dev, leaf_size=leaf_size)
    nd = {k: v.cpu().numpy() for k, v in tree.nodes().items()}
    ks = keys.cpu().numpy().view(np.uint64)
    lev = nd["level"].astype(np.int64)
    shift = (63 - 3 * lev).astype(np.uint64)
    pref = np.where(lev > 0, ks[nd["first"]] >> shift, 0).astype(np.uint64)
    return nd, pref


def _oracle_nodes(orc, w, leaf_size=8):
    T = orc.Tree(w.pos, w.mass, 2.8 * w.eps, leaf_size=leaf_size)
    nd = T.nodes()
    pref = np.array([int(orc.hilbert_grid([c], l)[0]) if l > 0 else 0 for c, l in zip(nd["cell"], nd["level"])],
                    dtype=np.uint64)
    return nd, pref


@pytest.mark.parametrize("name,scale,B", [("uniform4096", None, 8), ("nfw256", 24, 8), ("zoom8m", 6000, 8),
                                          ("nfw256", 20, 1), ("uniform4096", 1000, 32), ("uniform4096", 5, 8)])
def test_nodes_match_oracle(orc, name, scale, B):
    dev = device()
    w = ics.make(name, scale)
    g, gp = _gpu_nodes(w, dev, B)
    o, op = _oracle_nodes(orc, w, B)
    assert len(gp) == len(op)
    gk = {(int(l), int(p)): i for i, (l, p) in enumerate(zip(g["level"], gp))}
    ok = {(int(l), int(p)): i for i, (l, p) in enumerate(zip(o["level"], op))}
    assert set(gk) == set(ok)
    gi = np.array([gk[k] for k in ok])
    oi = np.array([ok[k] for k in ok])
    assert np.array_equal(g["count"][gi], o["count"][oi])
    assert np.array_equal(g["nchild"][gi], o["nchild"][oi])
    # FP64 sums of positive terms in two different orders: each within
    # (count - 1) ulp of the exact sum
    cnt = np.maximum(o["count"][oi], 8).astype(np.float64)
    assert np.all(np.abs(g["mass"][gi] - o["mass"][oi]) <= 4.5e-16 * cnt * o["mass"][oi])
    tol = 2.3e-16 * cnt[:, None] * 2
    assert np.all(np.abs(g["com"][gi] - o["com"][oi]) <= tol * np.abs(o["com"][oi]) + 1e-300)
    assert np.array_equal(g["hmax"][gi], o["hmax"][oi])
    # parent links point at the node one level up whose cell contains the child
    par = g["parent"][gi]
    assert np.all((par >= 0) == (g["level"][gi] > 0))


def test_capacity_overflow_is_reported():
    dev = device()
    from gpu_util import og
    m = og()
    w = ics.make("uniform4096", None)
    pos = torch.tensor(w.pos, device=dev)
    mass = torch.tensor(w.mass, device=dev)
    keys, order = m.keys_sort(pos, 1.0)
    with pytest.raises(m.OGError) as e:
        m.tree_build(keys, order, pos, mass, 1.0 / 480, 1.0, p=m.params(node_capacity=50))
    assert e.value.code == 2
