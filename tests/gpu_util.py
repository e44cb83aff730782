"""Helpers shared by the GPU parity tests: move a seeded workload to the GPU,
run the CUDA path through the C ABI binding, and compare with the oracle."""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return torch.device("cuda:0")


def og():
    import paper_2606_17145_gb300 as m
    return m


def to_dev(w, dev):
    pos = torch.tensor(w.pos, dtype=torch.float64, device=dev)
    mass = torch.tensor(w.mass, dtype=torch.float64, device=dev)
    eps = torch.tensor(w.eps, dtype=torch.float64, device=dev)
    return pos, mass, eps


def build_tree(w, dev, **pkw):
    m = og()
    pos, mass, eps = to_dev(w, dev)
    keys, order = m.keys_sort(pos, w.box)
    p = m.params(**pkw) if pkw else None
    tree = m.tree_build(keys, order, pos, mass, eps, w.box, p=p)
    return tree, keys, order


def forward(w, dev, theta, prec="fp32", **pkw):
    m = og()
    tree, keys, order = build_tree(w, dev, **pkw)
    acc, total, cnt = m.shortrange_accel(tree, w.r_s, theta, prec=prec, counts=True)
    torch.cuda.synchronize()
    return acc.double().cpu().numpy(), int(total.item()), cnt.cpu().numpy(), tree


def rel_err(a, ref):
    num = np.linalg.norm(a - ref, axis=1)
    den = np.linalg.norm(ref, axis=1)
    return num / np.maximum(den, 1e-300)


def err_stats(a, ref):
    r = rel_err(a, ref)
    scale = np.sqrt(np.mean(np.sum(ref * ref, axis=1)))
    return dict(rms=float(np.sqrt(np.mean(r ** 2))), p99=float(np.percentile(r, 99)), max=float(r.max()),
                med=float(np.median(r)), norm_max=float(np.linalg.norm(a - ref, axis=1).max() / scale))



# FP32 terms: displacement rounding, rsqrt / ex2 approximations, the
# short-range polynomial and a handful of products give each term a relative
# error below about 2e-6; per-warp FP32 partial sums of up to 32 terms before
# the FP64 accumulation add about as much.  A gradient component is therefore
# within ~4e-6 of its terms' absolute sum; the tests allow 1e-5 of it.
GRAD_TOL = 1e-5


def grad_scaled_err(g, ref, scale):
    """max over particles and components of |g - ref| / scale, where scale is
    the oracle's sum of the absolute values of the terms of that component."""
    g = np.asarray(g, dtype=np.float64).reshape(len(g), -1)
    ref = np.asarray(ref, dtype=np.float64).reshape(len(ref), -1)
    sc = np.asarray(scale, dtype=np.float64).reshape(len(scale), -1)
    return float((np.abs(g - ref) / np.maximum(sc, 1e-300)).max())
