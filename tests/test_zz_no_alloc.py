"""og_keys_sort_noalloc: the keys and sort for callers that cannot allocate
device memory (their scratch lives in a static device array of the library).

Called through the C ABI (ctypes), its output must equal og_keys_sort's bit
for bit, on two calls in a row with different inputs (the shared array keeps
the previous call's contents, so the second call must not depend on them).
This file is collected last on purpose."""
import ctypes as C

import numpy as np
import pytest

import ics
from gpu_util import device, og, torch

pytestmark = pytest.mark.gpu


def _reference(L, pos, box):
    from paper_2606_17145_gb300 import _native as N  # noqa: F401
    n = pos.shape[0]
    ws = og()._workspace(L.og_keys_sort_ws_bytes(n), pos.device)
    keys = torch.empty(n, dtype=torch.int64, device=pos.device)
    order = torch.empty(n, dtype=torch.int32, device=pos.device)
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert L.og_keys_sort(C.c_void_p(pos.data_ptr()), n, box, C.c_void_p(keys.data_ptr()),
                          C.c_void_p(order.data_ptr()), C.c_void_p(ws.data_ptr()), ws.numel(), s) == 0
    torch.cuda.synchronize()
    assert og().poll_status(ws) == 0
    return keys.cpu().numpy(), order.cpu().numpy()


def _noalloc(L, pos, box):
    n = pos.shape[0]
    keys = torch.full((n,), -7, dtype=torch.int64, device=pos.device)
    order = torch.full((n,), -7, dtype=torch.int32, device=pos.device)
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    code = L.og_keys_sort_noalloc(C.c_void_p(pos.data_ptr()), n, box, C.c_void_p(keys.data_ptr()),
                                  C.c_void_p(order.data_ptr()), s)
    torch.cuda.synchronize()
    assert code == 0
    return keys.cpu().numpy(), order.cpu().numpy()


def test_noalloc_matches_workspace_version_twice():
    dev = device()
    L = og().lib()
    sets = [(ics.uniform(300_000, 61), 1.0),                      # first call on the device: set-up
            (ics.make("nfw256", 64).pos * 8.0, 8.0)]              # second call: other size, box, values
    for pos_np, box in sets:
        pos = torch.tensor(pos_np, dtype=torch.float64, device=dev)
        k_ref, o_ref = _reference(L, pos, box)
        k_na, o_na = _noalloc(L, pos, box)
        assert np.array_equal(k_na, k_ref)
        assert np.array_equal(o_na, o_ref)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    dev = device()
    L = og().lib()
    n = (1 << 20) + 1
    p = C.c_void_p(256)  # never dereferenced: the size check comes first
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert L.og_keys_sort_noalloc(p, n, 1.0, p, p, s) == 2   # OG_ENOSPACE
    assert L.og_keys_sort_noalloc(p, 0, 1.0, p, p, s) == 1   # OG_EINVAL
