"""GB300-native short-range TreePM gravity: Python binding of libog.so.

The functions mirror the C ABI in include/og.h (same names, same steps):

    keys_sort(pos, box)                               -> keys, order
    tree_build(keys, order, pos, mass, eps, box)      -> Tree
    shortrange_accel(tree, r_s, theta, prec)          -> acc (+ interaction count)
    shortrange_adjoint(tree, r_s, theta, w)           -> dpos, dmass
    ShortRangeAccel.apply(pos, mass, eps, box, r_s, theta) (torch.autograd.Function)

This layer only marshals arguments: every step runs in the CUDA kernels of
libog.so.  PyTorch provides device memory and the current CUDA stream.
Tensors must live on one CUDA device; positions/masses/softenings are float64.
"""
from __future__ import annotations

import ctypes as C

import torch

from . import _native as N

_lib = None

# Kernels libog.so launches per call (fixed sequences, see csrc/): keys (1) +
# 8 radix passes x (histogram, scan, scatter); permute + groups + root + 21
# expand levels + 22 moment levels; one walk; adjoint walk + 22 push-down
# levels + the particle gather.
LAUNCHES_PER_CALL = {"keys_sort": 1 + 8 * 3, "tree_build": 3 + 21 + 22, "accel": 1, "adjoint": 1 + 22 + 1,
                     "pm": 3, "kick": 1, "drift": 1, "sph": 1}  # pm: deposit, Green, interpolation (plus cuFFT's kernels)


def lib():
    """The loaded libog.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        _lib = N.load()
    return _lib


class OGError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = lib().og_status_str(code).decode() if code >= 0 else "unknown"
        super().__init__(f"{where}: {msg} (status {code})")
        self.code = code


def _check(code: int, where: str):
    if code != N.OG_OK:
        raise OGError(code, where)


def _stream(stream=None) -> C.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t) -> C.c_void_p:
    return C.c_void_p(0 if t is None else t.data_ptr())


def _cuda(t: torch.Tensor, dtype, shape_tail=None, name="tensor"):
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape_tail is not None and tuple(t.shape[1:]) != tuple(shape_tail):
        raise ValueError(f"{name} must have shape [n, {', '.join(map(str, shape_tail))}]")
    return t


def _workspace(nbytes: int, device) -> torch.Tensor:
    ws = torch.empty(max(int(nbytes), 256) + 256, dtype=torch.uint8, device=device)
    off = (-ws.data_ptr()) % 256
    return ws[off:off + max(int(nbytes), 256)]


def params(leaf_size: int = 16, rcut_factor: float = 4.5, node_capacity: int = 0,
           max_walk_iters: int = 0, deep_stack: int = 0) -> N.og_params:
    p = N.og_params()
    lib().og_params_default(C.byref(p))
    p.leaf_size = leaf_size
    p.rcut_factor = rcut_factor
    p.node_capacity = node_capacity
    p.max_walk_iters = max_walk_iters
    p.deep_stack = deep_stack
    return p


def poll_status(buf: torch.Tensor, stream=None) -> int:
    """Synchronise and return the device status of a workspace / tree buffer."""
    return lib().og_poll_status(_ptr(buf), _stream(stream))


def keys_sort(pos: torch.Tensor, box: float, stream=None, check: bool = True, ws: torch.Tensor | None = None,
              keys: torch.Tensor | None = None, order: torch.Tensor | None = None):
    """Hilbert keys (as non-negative int64; they are 63-bit) and order (int32)."""
    _cuda(pos, torch.float64, (3,), "pos")
    n = pos.shape[0]
    L = lib()
    need = L.og_keys_sort_ws_bytes(n)
    if ws is None:
        ws = _workspace(need, pos.device)
    if keys is None:
        keys = torch.empty(n, dtype=torch.int64, device=pos.device)
    if order is None:
        order = torch.empty(n, dtype=torch.int32, device=pos.device)
    _check(L.og_keys_sort(_ptr(pos), n, float(box), _ptr(keys), _ptr(order), _ptr(ws), ws.numel(),
                          _stream(stream)), "og_keys_sort")
    if check:
        _check(poll_status(ws, stream), "og_keys_sort (device)")
    return keys, order


class Tree:
    """A tree built by og_tree_build; owns its device buffer."""

    def __init__(self, mem: torch.Tensor, header: N.og_tree, inputs):
        self.mem = mem
        self.header = header
        self._inputs = inputs  # keep the input tensors alive while the tree is in use

    @property
    def n(self) -> int:
        return int(self.header.n)

    def node_count(self, stream=None) -> int:
        return int(lib().og_tree_node_count(C.byref(self.header), _stream(stream)))

    def nodes(self, stream=None) -> dict:
        m = self.node_count(stream)
        dev = self.mem.device
        out = dict(level=torch.empty(m, dtype=torch.int32, device=dev),
                   first=torch.empty(m, dtype=torch.int32, device=dev),
                   count=torch.empty(m, dtype=torch.int32, device=dev),
                   parent=torch.empty(m, dtype=torch.int32, device=dev),
                   mass=torch.empty(m, dtype=torch.float64, device=dev),
                   com=torch.empty((m, 3), dtype=torch.float64, device=dev),
                   hmax=torch.empty(m, dtype=torch.float64, device=dev),
                   child_first=torch.empty(m, dtype=torch.int32, device=dev),
                   nchild=torch.empty(m, dtype=torch.int32, device=dev))
        _check(lib().og_tree_copy_nodes(C.byref(self.header), *[_ptr(out[k]) for k in
                                                                 ("level", "first", "count", "parent", "mass", "com",
                                                                  "hmax", "child_first", "nchild")],
                                        _stream(stream)), "og_tree_copy_nodes")
        return out


def tree_build(keys: torch.Tensor, order: torch.Tensor, pos: torch.Tensor, mass: torch.Tensor, eps, box: float,
               p: N.og_params | None = None, stream=None, check: bool = True, mem: torch.Tensor | None = None) -> Tree:
    """Octree over the sorted particles.  eps: float64 tensor [n] or a float."""
    _cuda(pos, torch.float64, (3,), "pos")
    _cuda(mass, torch.float64, None, "mass")
    _cuda(keys, torch.int64, None, "keys")
    _cuda(order, torch.int32, None, "order")
    n = pos.shape[0]
    L = lib()
    p = p or params()
    need = L.og_tree_bytes(n, C.byref(p))
    if need == 0:
        raise ValueError("invalid particle count or node capacity")
    if mem is None:
        mem = _workspace(need, pos.device)
    if isinstance(eps, torch.Tensor):
        _cuda(eps, torch.float64, None, "eps")
        eps_t, eps_s = eps, 0.0
    else:
        eps_t, eps_s = None, float(eps)
    hdr = N.og_tree()
    _check(L.og_tree_build(_ptr(keys), _ptr(order), _ptr(pos), _ptr(mass), _ptr(eps_t), eps_s, n, float(box),
                           C.byref(p), _ptr(mem), mem.numel(), C.byref(hdr), _stream(stream)), "og_tree_build")
    if check:
        _check(poll_status(mem, stream), "og_tree_build (device)")
    return Tree(mem, hdr, (keys, order, pos, mass, eps_t))


def shortrange_accel(tree: Tree, r_s: float, theta: float, prec: str = "fp32", counts: bool = False,
                     stream=None, check: bool = True, ws: torch.Tensor | None = None, out: torch.Tensor | None = None,
                     total: torch.Tensor | None = None, groups: tuple[int, int] | None = None):
    """Short-range accelerations (original order).  Returns (acc, total, counts).
    groups=(g0, g1): walk only the groups [g0, g1) (og_shortrange_accel_range);
    only those targets' rows of acc / counts are written."""
    L = lib()
    code = N.OG_FP64 if prec == "fp64" else N.OG_FP32_KAHAN
    dev = tree.mem.device
    n = tree.n
    if out is None:
        out = torch.empty((n, 3), dtype=torch.float64 if code == N.OG_FP64 else torch.float32, device=dev)
    if total is None:
        total = torch.zeros(1, dtype=torch.int64, device=dev)
    cnt = torch.empty(n, dtype=torch.int32, device=dev) if counts else None
    if ws is None:
        ws = _workspace(L.og_accel_ws_bytes(C.byref(tree.header), code), dev)
    if groups is None:
        _check(L.og_shortrange_accel(C.byref(tree.header), float(r_s), float(theta), code, _ptr(out), _ptr(total),
                                     _ptr(cnt), _ptr(ws), ws.numel(), _stream(stream)), "og_shortrange_accel")
    else:
        _check(L.og_shortrange_accel_range(C.byref(tree.header), float(r_s), float(theta), code, int(groups[0]),
                                           int(groups[1]), _ptr(out), _ptr(total), _ptr(cnt), _ptr(ws), ws.numel(),
                                           _stream(stream)), "og_shortrange_accel_range")
    if check:
        _check(poll_status(ws, stream), "og_shortrange_accel (device)")
    return out, total, cnt


def shortrange_adjoint(tree: Tree, r_s: float, theta: float, w: torch.Tensor, stream=None, check: bool = True,
                       ws: torch.Tensor | None = None, dpos: torch.Tensor | None = None,
                       dmass: torch.Tensor | None = None, groups: tuple[int, int] | None = None):
    """dL/dx [n,3] and dL/dm [n] (float64, original order) for L = sum w . a.
    groups=(g0, g1): the gradient of the partial loss over the targets of the
    groups [g0, g1) only (og_shortrange_adjoint_range)."""
    _cuda(w, torch.float32, (3,), "w")
    L = lib()
    dev = tree.mem.device
    n = tree.n
    if ws is None:
        ws = _workspace(L.og_adjoint_ws_bytes(C.byref(tree.header), 1), dev)
    if dpos is None:
        dpos = torch.empty((n, 3), dtype=torch.float64, device=dev)
    if dmass is None:
        dmass = torch.empty(n, dtype=torch.float64, device=dev)
    if groups is None:
        _check(L.og_shortrange_adjoint(C.byref(tree.header), float(r_s), float(theta), N.OG_FP32_KAHAN, _ptr(w),
                                       _ptr(dpos), _ptr(dmass), 1, _ptr(ws), ws.numel(), _stream(stream)),
               "og_shortrange_adjoint")
    else:
        _check(L.og_shortrange_adjoint_range(C.byref(tree.header), float(r_s), float(theta), N.OG_FP32_KAHAN,
                                             _ptr(w), int(groups[0]), int(groups[1]), _ptr(dpos), _ptr(dmass), 1,
                                             _ptr(ws), ws.numel(), _stream(stream)), "og_shortrange_adjoint_range")
    if check:
        _check(poll_status(ws, stream), "og_shortrange_adjoint (device)")
    return dpos, dmass


def shortrange_accel_adjoint(tree: Tree, r_s: float, theta: float, w: torch.Tensor, counts: bool = False,
                             stream=None, check: bool = True, ws: torch.Tensor | None = None,
                             out: torch.Tensor | None = None, total: torch.Tensor | None = None,
                             dpos: torch.Tensor | None = None, dmass: torch.Tensor | None = None):
    """Forward and adjoint in one walk (og_shortrange_accel_adjoint), for
    L = sum w . a with w known in advance.  Returns (acc, total, counts, dpos,
    dmass), each as from shortrange_accel / shortrange_adjoint."""
    _cuda(w, torch.float32, (3,), "w")
    L = lib()
    dev = tree.mem.device
    n = tree.n
    if out is None:
        out = torch.empty((n, 3), dtype=torch.float32, device=dev)
    if total is None:
        total = torch.zeros(1, dtype=torch.int64, device=dev)
    cnt = torch.empty(n, dtype=torch.int32, device=dev) if counts else None
    if ws is None:
        ws = _workspace(L.og_adjoint_ws_bytes(C.byref(tree.header), 1), dev)
    if dpos is None:
        dpos = torch.empty((n, 3), dtype=torch.float64, device=dev)
    if dmass is None:
        dmass = torch.empty(n, dtype=torch.float64, device=dev)
    _check(L.og_shortrange_accel_adjoint(C.byref(tree.header), float(r_s), float(theta), N.OG_FP32_KAHAN, _ptr(w),
                                         _ptr(out), _ptr(total), _ptr(cnt), _ptr(dpos), _ptr(dmass), _ptr(ws),
                                         ws.numel(), _stream(stream)), "og_shortrange_accel_adjoint")
    if check:
        _check(poll_status(ws, stream), "og_shortrange_accel_adjoint (device)")
    return out, total, cnt, dpos, dmass


class PMPlan:
    """cuFFT plans for an N^3 long-range mesh (og_pm_plan_create); frees them when collected."""

    def __init__(self, ngrid: int):
        h = C.c_void_p()
        _check(lib().og_pm_plan_create(int(ngrid), C.byref(h)), "og_pm_plan_create")
        self.handle = h
        self.ngrid = int(ngrid)
        self._lib = lib()

    @property
    def ws_bytes(self) -> int:
        return int(self._lib.og_pm_ws_bytes(self.handle))

    def close(self):
        if self.handle is not None and self.handle.value:
            self._lib.og_pm_plan_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pm_accel(plan: PMPlan, pos: torch.Tensor, mass: torch.Tensor, box: float, r_s: float, stream=None,
             check: bool = True, ws: torch.Tensor | None = None, out: torch.Tensor | None = None) -> torch.Tensor:
    """Long-range (PM) accelerations, float32 [n, 3] in the order of pos."""
    _cuda(pos, torch.float64, (3,), "pos")
    _cuda(mass, torch.float64, None, "mass")
    n = pos.shape[0]
    if ws is None:
        ws = _workspace(plan.ws_bytes, pos.device)
    if out is None:
        out = torch.empty((n, 3), dtype=torch.float32, device=pos.device)
    _check(lib().og_pm_accel(plan.handle, _ptr(pos), _ptr(mass), n, float(box), float(r_s), _ptr(ws), ws.numel(),
                             _ptr(out), _stream(stream)), "og_pm_accel")
    if check:
        _check(poll_status(ws, stream), "og_pm_accel (device)")
    return out


def kick(vel: torch.Tensor, acc_a: torch.Tensor, acc_b: torch.Tensor | None, dt: float, stream=None):
    """vel += dt (acc_a + acc_b) in place (og_kick); acc_b may be None."""
    _cuda(vel, torch.float64, (3,), "vel")
    _cuda(acc_a, torch.float32, (3,), "acc_a")
    if acc_b is not None:
        _cuda(acc_b, torch.float32, (3,), "acc_b")
    _check(lib().og_kick(_ptr(vel), _ptr(acc_a), _ptr(acc_b), vel.shape[0], float(dt), _stream(stream)), "og_kick")


def drift(pos: torch.Tensor, vel: torch.Tensor, dt: float, stream=None):
    """pos += dt vel in place (og_drift)."""
    _cuda(pos, torch.float64, (3,), "pos")
    _cuda(vel, torch.float64, (3,), "vel")
    _check(lib().og_drift(_ptr(pos), _ptr(vel), pos.shape[0], float(dt), _stream(stream)), "og_drift")


def sph_density(tree: Tree, n_ngb: float, stream=None, check: bool = True, ws: torch.Tensor | None = None):
    """SPH smoothing lengths, densities and neighbour counts (og_sph_density),
    in the original particle order: (h float64 [n], rho float64 [n], ngb int32 [n])."""
    L = lib()
    dev = tree.mem.device
    n = tree.n
    if ws is None:
        ws = _workspace(L.og_sph_ws_bytes(), dev)
    h = torch.empty(n, dtype=torch.float64, device=dev)
    rho = torch.empty(n, dtype=torch.float64, device=dev)
    ngb = torch.empty(n, dtype=torch.int32, device=dev)
    _check(L.og_sph_density(C.byref(tree.header), float(n_ngb), _ptr(ws), ws.numel(), _ptr(h), _ptr(rho), _ptr(ngb),
                            _stream(stream)), "og_sph_density")
    if check:
        _check(poll_status(ws, stream), "og_sph_density (device)")
    return h, rho, ngb


class TreePMStepper:
    """Device-resident TreePM kick-drift-kick steps: positions, velocities,
    accelerations and every workspace stay on the GPU; each step rebuilds the
    keys and the tree and runs the FP32 walk and the PM mesh.  All buffers are
    allocated here, none in step()."""

    def __init__(self, pos: torch.Tensor, vel: torch.Tensor, mass: torch.Tensor, eps, box: float, r_s: float,
                 theta: float, ngrid: int, p=None):
        _cuda(pos, torch.float64, (3,), "pos")
        _cuda(vel, torch.float64, (3,), "vel")
        _cuda(mass, torch.float64, None, "mass")
        L = lib()
        dev = pos.device
        n = pos.shape[0]
        self.pos, self.vel, self.mass, self.eps = pos, vel, mass, eps
        self.box, self.r_s, self.theta = float(box), float(r_s), float(theta)
        self.p = p or params()
        self.ws_keys = _workspace(L.og_keys_sort_ws_bytes(n), dev)
        self.keys = torch.empty(n, dtype=torch.int64, device=dev)
        self.order = torch.empty(n, dtype=torch.int32, device=dev)
        self.tree_mem = _workspace(L.og_tree_bytes(n, C.byref(self.p)), dev)
        self.acc_s = torch.empty((n, 3), dtype=torch.float32, device=dev)
        self.acc_l = torch.empty((n, 3), dtype=torch.float32, device=dev)
        self.total = torch.zeros(1, dtype=torch.int64, device=dev)
        self.plan = PMPlan(ngrid)
        self.ws_pm = _workspace(self.plan.ws_bytes, dev)
        self.ws_acc = None
        self.forces(check=True)

    def forces(self, check: bool = False, stream=None):
        """Short-range (walk) and long-range (mesh) accelerations at the current positions."""
        keys_sort(self.pos, self.box, stream=stream, check=check, ws=self.ws_keys, keys=self.keys, order=self.order)
        tree = tree_build(self.keys, self.order, self.pos, self.mass, self.eps, self.box, p=self.p, stream=stream,
                          check=check, mem=self.tree_mem)
        if self.ws_acc is None:
            self.ws_acc = _workspace(lib().og_accel_ws_bytes(C.byref(tree.header), 0), self.pos.device)
        shortrange_accel(tree, self.r_s, self.theta, stream=stream, check=check, ws=self.ws_acc, out=self.acc_s,
                         total=self.total)
        pm_accel(self.plan, self.pos, self.mass, self.box, self.r_s, stream=stream, check=check, ws=self.ws_pm,
                 out=self.acc_l)

    def poll(self, stream=None):
        """Synchronise and raise OGError if keys, tree, walk or mesh recorded
        an error on the device since their last call."""
        for buf, where in ((self.ws_keys, "og_keys_sort"), (self.tree_mem, "og_tree_build"),
                           (self.ws_acc, "og_shortrange_accel"), (self.ws_pm, "og_pm_accel")):
            if buf is not None:
                _check(poll_status(buf, stream), f"{where} (device, stepper)")

    def step(self, dt: float, check: bool = True, stream=None):
        """One kick-drift-kick step of length dt.  With check (the default) the
        device status words are read once, after the second kick (one
        synchronisation per step); a failed tree makes the walk return NaN
        forces, so an unchecked step cannot silently reuse old ones."""
        kick(self.vel, self.acc_s, self.acc_l, 0.5 * dt, stream)
        drift(self.pos, self.vel, dt, stream)
        self.forces(check=False, stream=stream)
        kick(self.vel, self.acc_s, self.acc_l, 0.5 * dt, stream)
        if check:
            self.poll(stream)

    def close(self):
        self.plan.close()


class ShortRangeAccel(torch.autograd.Function):
    """acc = ShortRangeAccel.apply(pos, mass, eps, box, r_s, theta).

    Forward: keys, sort, tree and the FP32-Kahan walk.  Backward: the adjoint
    walk with the forward's opening / cut decisions frozen (recomputed on the
    same tree), giving gradients for pos and mass.  eps may be a float or a
    float64 tensor (it gets no gradient).
    """

    @staticmethod
    def forward(ctx, pos, mass, eps, box, r_s, theta):
        keys, order = keys_sort(pos, box, check=False)
        tree = tree_build(keys, order, pos, mass, eps, box, check=False)
        _check(poll_status(tree.mem), "tree_build (device)")
        # check=True: the walk's own status word is read after the call
        acc, total, _ = shortrange_accel(tree, r_s, theta, check=True)
        ctx.tree = tree
        ctx.r_s = r_s
        ctx.theta = theta
        ctx.total = total
        return acc

    @staticmethod
    def backward(ctx, grad_acc):
        w = grad_acc.contiguous().to(torch.float32)
        dpos, dmass = shortrange_adjoint(ctx.tree, ctx.r_s, ctx.theta, w)
        gm = dmass if ctx.needs_input_grad[1] else None
        gp = dpos if ctx.needs_input_grad[0] else None
        return gp, gm, None, None, None, None


class ShortRangeLinearLoss(torch.autograd.Function):
    """L = ShortRangeLinearLoss.apply(pos, mass, eps, w, box, r_s, theta):
    the scalar L = sum_i w_i . a_i of the short-range accelerations, for
    weights w (float32 [n, 3]) known before the forces.

    Forward: keys, sort, tree and one fused walk (og_shortrange_accel_adjoint)
    that writes the accelerations and dL/dx, dL/dm together.  Backward scales
    those by the incoming gradient; dL/dw = a.  The same gradients as
    ShortRangeAccel followed by (a * w).sum(), from one walk instead of two.
    """

    @staticmethod
    def forward(ctx, pos, mass, eps, w, box, r_s, theta):
        keys, order = keys_sort(pos, box, check=False)
        tree = tree_build(keys, order, pos, mass, eps, box, check=False)
        _check(poll_status(tree.mem), "tree_build (device)")
        # check=True: the walk's own status word (iteration cap, corrupt
        # queue entries) is read after the call
        acc, _, _, dpos, dmass = shortrange_accel_adjoint(tree, r_s, theta, w.detach().contiguous(), check=True)
        ctx.save_for_backward(acc, dpos, dmass)
        return (acc.double() * w.double()).sum()

    @staticmethod
    def backward(ctx, g):
        acc, dpos, dmass = ctx.saved_tensors
        gp = g * dpos if ctx.needs_input_grad[0] else None
        gm = g * dmass if ctx.needs_input_grad[1] else None
        gw = (g * acc).to(torch.float32) if ctx.needs_input_grad[3] else None
        return gp, gm, None, gw, None, None, None


def shortrange_accel_autograd(pos, mass, eps, box, r_s, theta):
    return ShortRangeAccel.apply(pos, mass, eps, box, r_s, theta)
