"""CPU-side checks of the C ABI: the library loads, exports every function
include/og.h declares, and its host-side sizing / argument checks work
without a GPU (no kernel is launched here)."""
import ctypes as C

import pytest


@pytest.fixture(scope="module")
def L():
    import __graft_entry__
    from paper_2606_17145_gb300 import build as b
    b.build()
    from paper_2606_17145_gb300 import _native as N
    return N.load()


def test_every_header_symbol_is_exported(L):
    from paper_2606_17145_gb300 import _native as N
    names = N.header_symbols()
    assert len(names) >= 13
    for name in names:
        assert hasattr(L, name), name
        assert name in N.SIGNATURES, f"{name} has no ctypes signature"


def test_params_and_sizes(L):
    from paper_2606_17145_gb300 import _native as N
    p = N.og_params()
    L.og_params_default(C.byref(p))
    assert (p.leaf_size, p.rcut_factor, p.node_capacity, p.max_walk_iters) == (16, 4.5, 0, 0)
    assert L.og_keys_sort_ws_bytes(0) == 0
    assert L.og_keys_sort_ws_bytes(1000) >= 1000 * 12
    assert L.og_tree_bytes(1000, None) > L.og_tree_bytes(100, None) > 0
    big = N.og_params()
    L.og_params_default(C.byref(big))
    big.node_capacity = 10 ** 6
    assert L.og_tree_bytes(1000, C.byref(big)) > L.og_tree_bytes(1000, None)


def test_host_argument_checks(L):
    from paper_2606_17145_gb300 import _native as N
    ws = C.c_void_p(256)   # never dereferenced: every call below fails its host checks first
    assert L.og_keys_sort(None, 10, 1.0, ws, ws, ws, 1 << 20, None) == N.OG_EINVAL
    assert L.og_keys_sort(ws, 0, 1.0, ws, ws, ws, 1 << 20, None) == N.OG_EINVAL
    assert L.og_keys_sort(ws, 10, -1.0, ws, ws, ws, 1 << 20, None) == N.OG_EINVAL
    assert L.og_keys_sort(ws, 10, float("nan"), ws, ws, ws, 1 << 20, None) == N.OG_EINVAL
    assert L.og_keys_sort(ws, 10, 1.0, ws, ws, C.c_void_p(257), 1 << 20, None) == N.OG_EINVAL
    assert L.og_keys_sort(ws, 10, 1.0, ws, ws, ws, 16, None) == N.OG_ENOSPACE
    hdr = N.og_tree()
    p = N.og_params()
    L.og_params_default(C.byref(p))
    assert L.og_tree_build(ws, ws, ws, ws, None, 0.0, 10, 1.0, C.byref(p), ws, 1 << 30, C.byref(hdr),
                           None) == N.OG_EINVAL  # no eps array and eps_scalar = 0
    p.leaf_size = 0
    assert L.og_tree_build(ws, ws, ws, ws, None, 0.1, 10, 1.0, C.byref(p), ws, 1 << 30, C.byref(hdr),
                           None) == N.OG_EINVAL
    L.og_params_default(C.byref(p))
    for bad in (-1, 65):
        p.deep_stack = bad
        assert L.og_tree_build(ws, ws, ws, ws, None, 0.1, 10, 1.0, C.byref(p), ws, 1 << 30, C.byref(hdr),
                               None) == N.OG_EINVAL
    L.og_params_default(C.byref(p))
    assert L.og_tree_build(ws, ws, ws, ws, None, 0.1, 10, 1.0, C.byref(p), ws, 64, C.byref(hdr),
                           None) == N.OG_ENOSPACE
    # walks on a header that was never built
    assert L.og_shortrange_accel(C.byref(hdr), 0.01, 0.5, 0, ws, None, None, ws, 1 << 20, None) == N.OG_ETREE
    hdr.built = 1
    hdr.mem = 256
    hdr.box = 1.0
    hdr.rcut_factor = 4.5
    hdr.n = 10
    hdr.node_capacity = 100
    # rcut = 4.5 r_s must stay below box / 2
    assert L.og_shortrange_accel(C.byref(hdr), 0.2, 0.5, 0, ws, None, None, ws, 1 << 20, None) == N.OG_EINVAL
    assert L.og_shortrange_accel(C.byref(hdr), 0.01, -0.5, 0, ws, None, None, ws, 1 << 20, None) == N.OG_EINVAL
    assert L.og_shortrange_accel(C.byref(hdr), 0.01, 0.5, 7, ws, None, None, ws, 1 << 20, None) == N.OG_EINVAL
    assert L.og_shortrange_adjoint(C.byref(hdr), 0.01, 0.5, 0, ws, ws, ws, 0, ws, 1 << 30, None) == N.OG_ENOTIMPL
    assert L.og_shortrange_adjoint(C.byref(hdr), 0.01, 0.5, 1, ws, ws, ws, 1, ws, 1 << 30, None) == N.OG_ENOTIMPL
    for code in range(7):
        assert L.og_status_str(code)


def test_pm_host_argument_checks(L):
    """The PM entry points refuse bad arguments on the host, before cuFFT or
    any kernel is reached."""
    from paper_2606_17145_gb300 import _native as N
    h = C.c_void_p(1234)
    for bad in (0, 4, 7, 1025, -8):
        assert L.og_pm_plan_create(bad, C.byref(h)) == N.OG_EINVAL
        assert h.value is None  # *plan is cleared on error
    assert L.og_pm_plan_create(64, None) == N.OG_EINVAL
    assert L.og_pm_ws_bytes(None) == 0
    L.og_pm_plan_destroy(None)  # ignored
    buf = C.create_string_buffer(1024)
    p = C.cast(buf, C.c_void_p)
    assert L.og_pm_accel(None, p, p, 10, 1.0, 0.01, p, 1024, p, None) == N.OG_EINVAL


def test_sph_and_integrator_host_argument_checks(L):
    from paper_2606_17145_gb300 import _native as N
    assert L.og_sph_ws_bytes() >= 256
    buf = C.create_string_buffer(1024)
    p = C.cast(buf, C.c_void_p)
    assert L.og_sph_density(None, 32.0, p, 1024, p, p, p, None) == N.OG_ETREE
    assert L.og_kick(None, p, None, 10, 0.1, None) == N.OG_EINVAL
    assert L.og_kick(p, p, None, 0, 0.1, None) == N.OG_EINVAL
    assert L.og_drift(p, p, 10, float("nan"), None) == N.OG_EINVAL
