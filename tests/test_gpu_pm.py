"""PM long-range parity: the GPU mesh (FP32, cuFFT) against the FP64 numpy
oracle, plus the walk + mesh total against an Ewald sum.

Tolerance.  The GPU mesh is FP32 throughout: deposit, transforms, Green's
function, differences and interpolation.  A numpy FP32 emulation of the same
steps stays within 3e-7 rms and 2e-6 max of the FP64 oracle on the 32^3
sets, both relative to rms |a|.  The bounds below are 5e-6 and 5e-5. They
leave room for cuFFT's own rounding order and for the unordered FP32 atomics
of the deposit.
"""
import numpy as np
import pytest

import ics
from gpu_util import device, og, torch
from oracle import og_pm as P
from pm_ref import ewald

pytestmark = pytest.mark.gpu

RMS_TOL = 5e-6
MAX_TOL = 5e-5


def _run(pos, mass, box, N, r_s, dev, plan=None):
    m = og()
    own = plan is None
    plan = plan or m.PMPlan(N)
    a = m.pm_accel(plan, torch.tensor(pos, dtype=torch.float64, device=dev),
                   torch.tensor(mass, dtype=torch.float64, device=dev), box, r_s)
    torch.cuda.synchronize()
    if own:
        plan.close()
    return a.double().cpu().numpy()


def _err(a, ref):
    d = np.linalg.norm(a - ref, axis=1)
    s = np.sqrt(np.mean(np.sum(ref ** 2, axis=1)))
    return float(np.sqrt(np.mean(d ** 2)) / s), float(d.max() / s)


@pytest.mark.parametrize("name,side", [("zeldovich128", 32), ("nfw256", 32), ("nfw128_adjoint", 24)])
def test_sets_vs_oracle(name, side):
    """Mesh of 2 x side per axis (48^3 for the last set: not a power of two)."""
    dev = device()
    w = ics.make(name, side)
    N = 2 * side
    ref = P.pm_accel(w.pos, w.mass, w.box, N, w.r_s)
    a = _run(w.pos, w.mass, w.box, N, w.r_s, dev)
    rms, mx = _err(a, ref)
    assert rms < RMS_TOL and mx < MAX_TOL, (rms, mx)


def test_non_unit_box_and_positions_outside_it():
    dev = device()
    rng = np.random.default_rng(8)
    L = 3.0
    n = 5000
    pos = rng.random((n, 3)) * L + rng.integers(-2, 3, size=(n, 3)) * L
    mass = 0.5 + rng.random(n)
    N, r_s = 40, 1.25 * L / 40
    ref = P.pm_accel(pos, mass, L, N, r_s)
    a = _run(pos, mass, L, N, r_s, dev)
    rms, mx = _err(a, ref)
    assert rms < RMS_TOL and mx < MAX_TOL, (rms, mx)


def test_full_size_bench_configuration():
    """The bench's configuration: 128^3 Zel'dovich set on a 256^3 mesh, every particle."""
    dev = device()
    w = ics.make("zeldovich128")
    N = 256
    ref = P.pm_accel(w.pos, w.mass, w.box, N, w.r_s)
    a = _run(w.pos, w.mass, w.box, N, w.r_s, dev)
    rms, mx = _err(a, ref)
    assert rms < RMS_TOL and mx < MAX_TOL, (rms, mx)


def test_lone_particle_and_plan_reuse():
    dev = device()
    m = og()
    N = 32
    D = 1.0 / N
    plan = m.PMPlan(N)
    rng = np.random.default_rng(9)
    for _ in range(3):
        a = _run(rng.random((1, 3)), np.array([1.0]), 1.0, N, 1.25 * D, dev, plan)
        assert np.abs(a).max() < 1e-5 / D ** 2
    # the same plan and a second call give the same field: the mesh is cleared
    # per call (a stale mesh would double it).  The deposit's FP32 atomics add
    # in any order, so the calls agree to rounding (1.5e-6 seen), not bitwise.
    w = ics.make("uniform4096")
    a1 = _run(w.pos, w.mass, w.box, N, 1.25 * D, dev, plan)
    a2 = _run(w.pos, w.mass, w.box, N, 1.25 * D, dev, plan)
    assert _err(a2, a1)[1] < MAX_TOL
    plan.close()


def test_walk_plus_mesh_is_the_periodic_newtonian_force():
    """GPU short-range walk (theta = 0, cut at 10 r_s) + GPU mesh against an
    Ewald sum with an unrelated splitting parameter.  The bound is the mesh's
    discretisation error (the oracle shows at most 2.3 % at 2-4 cells)."""
    dev = device()
    m = og()
    N = 32
    D = 1.0 / N
    r_s = 1.25 * D
    plan = m.PMPlan(N)
    rng = np.random.default_rng(10)
    for r in (0.5, 2.0, 4.0, 12.0):
        for _ in range(4):
            x0 = rng.random(3)
            u = rng.normal(size=3)
            u /= np.linalg.norm(u)
            d = r * D * u
            pos = np.array([x0, x0 + d])
            mass = np.array([1.0, 1e-12])
            pt = torch.tensor(pos, dtype=torch.float64, device=dev)
            mt = torch.tensor(mass, dtype=torch.float64, device=dev)
            keys, order = m.keys_sort(pt, 1.0)
            tree = m.tree_build(keys, order, pt, mt, 1e-7, 1.0, p=m.params(rcut_factor=10.0))
            s, _, _ = m.shortrange_accel(tree, r_s, 0.0)
            a = m.pm_accel(plan, pt, mt, 1.0, r_s)
            tot = (s.double() + a.double()).cpu().numpy()[1]
            ew = ewald(d, 6.0)
            assert np.linalg.norm(tot - ew) / np.linalg.norm(ew) < 0.03, (r, tot, ew)
    plan.close()


def test_nonfinite_position_is_flagged():
    dev = device()
    m = og()
    w = ics.make("uniform4096")
    pos = w.pos.copy()
    pos[17, 1] = np.nan
    plan = m.PMPlan(32)
    with pytest.raises(m.OGError):
        m.pm_accel(plan, torch.tensor(pos, device=dev), torch.tensor(w.mass, device=dev), 1.0, 1.25 / 32)
    plan.close()
