"""Thin Python binding of liblbfmm (include/lbfmm.h).

Argument marshalling only: every step of the method runs in the library's CUDA
kernels.  Device arrays are torch CUDA tensors (float64, contiguous); PyTorch
supplies device memory and the current stream.  The functions keep the C
names.  If the compiled library is missing, loading fails loudly: there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

from .build import LIB

LBF_OK = 0
LBF_NOCONV = 1
LBF_EINVAL = -1
LBF_EPOLE = -2
LBF_EDEPTH = -3
LBF_EWORKSPACE = -4
LBF_ECUDA = -5
LBF_ETIMEOUT = -6
LBF_ENOTBUILT = -7
LBF_ESINGULAR = -8

LBF_MATVEC_FMM = 0
LBF_MATVEC_DIRECT = 1
LBF_OP_FULL = 0
LBF_OP_K_ONLY = 1
LBF_OP_PRECONDITIONED = 2
LBF_OP_FP32 = 16
LBF_OP_TRANSPOSE = 32
LBF_PRECISION_FP64 = 0
LBF_PRECISION_FP32_REFINE = 1
LBF_SCHUR_AUTO = 0
LBF_SCHUR_GJ = 1
LBF_SCHUR_LU = 2


class lbf_options(C.Structure):
    _fields_ = [("tol", C.c_double), ("restart", C.c_int), ("maxit", C.c_int), ("p", C.c_int),
                ("leaf_size", C.c_int), ("max_depth", C.c_int), ("matvec", C.c_int),
                ("border", C.c_int), ("box_capacity", C.c_int64), ("precision", C.c_int),
                ("p32", C.c_int), ("inner_tol", C.c_double), ("max_refine", C.c_int),
                ("graphs", C.c_int), ("fmm64", C.c_int), ("schur", C.c_int),
                ("p2p_warps", C.c_int), ("precond", C.c_int)]


class lbf_batch_item(C.Structure):
    """Mirror of the C struct lbf_batch_item (one independent instance of a batch)."""
    _fields_ = [("M", C.c_int), ("island_ptr", C.c_void_p), ("x", C.c_void_p),
                ("dx", C.c_void_p), ("d2x", C.c_void_p), ("centres", C.c_void_p),
                ("workspace", C.c_void_p), ("bytes", C.c_size_t), ("nrhs", C.c_int),
                ("g", C.c_void_p), ("sigma", C.c_void_p), ("a", C.c_void_p), ("T", C.c_int64),
                ("targets", C.c_void_p), ("u", C.c_void_p), ("box_capacity", C.c_int64),
                ("status", C.c_int),
                ("iters", C.c_int), ("fp64_applies", C.c_int64), ("fp32_applies", C.c_int64),
                ("max_rel_res", C.c_double), ("box_capacity_needed", C.c_int64)]


class LbfError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {lbf_status_string(status)} ({status})")


_lib = None
_P = C.c_void_p


def load():
    """Load the in-tree liblbfmm.so (built by __graft_entry__.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise RuntimeError(f"liblbfmm is not built ({LIB}); run __graft_entry__.build()")
        lib = C.CDLL(LIB)
        i64 = C.c_int64
        sig = {
            "lbf_default_options": (C.c_int, [C.POINTER(lbf_options)]),
            "lbf_status_string": (C.c_char_p, [C.c_int]),
            "lbf_workspace_size": (C.c_int, [C.c_int, _P, C.POINTER(lbf_options), C.POINTER(C.c_size_t)]),
            "lbf_plan_create": (C.c_int, [C.POINTER(_P), C.c_int, _P, _P, _P, _P, _P, _P,
                                          C.POINTER(lbf_options), _P, C.c_size_t,
                                          C.POINTER(i64), _P]),
            "lbf_plan_create_planar": (C.c_int, [C.POINTER(_P), C.c_int, _P, _P, _P, _P, _P,
                                                 C.POINTER(lbf_options), _P, C.c_size_t,
                                                 C.POINTER(i64), _P]),
            "lbf_plan_destroy": (C.c_int, [_P]),
            "lbf_plan_info": (C.c_int, [_P, _P, _P, _P, _P, _P, _P]),
            "lbf_geometry_out": (C.c_int, [_P, _P, _P, _P, _P, _P]),
            "lbf_apply": (C.c_int, [_P, C.c_int, _P, _P, _P]),
            "lbf_gmres_solve": (C.c_int, [_P, _P, _P, _P, _P, _P, _P, _P]),
            "lbf_evaluate": (C.c_int, [_P, _P, _P, i64, _P, _P, _P]),
            "lbf_green_sum": (C.c_int, [i64, _P, i64, _P, _P, _P, _P]),
            "lbf_tree_export": (C.c_int, [_P, _P, _P, _P]),
            "lbf_list_export": (C.c_int, [_P, C.c_int, _P, _P, C.POINTER(i64), _P]),
            "lbf_plan_counts": (C.c_int, [_P, _P, _P]),
            "lbf_border_counts": (C.c_int, [_P, _P, _P]),
            "lbf_profile_enable": (C.c_int, [C.c_int]),
            "lbf_profile_reset": (C.c_int, []),
            "lbf_profile_read": (C.c_int, [C.c_int, C.POINTER(i64), C.POINTER(C.c_double)]),
            "lbf_evaluate_noalloc": (C.c_int, [i64, _P, _P, _P, C.c_int, _P, _P, i64, _P, _P, _P]),
            "lbf_solve_stats": (C.c_int, [_P, _P]),
            "lbf_gmres_solve_transpose": (C.c_int, [_P, _P, _P, _P, _P, _P, _P]),
            "lbf_batch_run": (C.c_int, [C.c_int, C.POINTER(lbf_batch_item), C.POINTER(lbf_options),
                                        C.c_int]),
            "lbf_evaluate_transpose": (C.c_int, [_P, i64, _P, _P, _P, _P, _P]),
            "lbf_gradient_nodes": (C.c_int, [_P, _P, _P, _P, i64, _P, _P, _P, _P]),
            "lbf_gradient_data": (C.c_int, [_P, _P, _P, _P]),
            "lbf_sync_status": (C.c_int, [_P, _P]),
            "lbf_selftest_rcp": (C.c_int, [C.c_int, i64, _P, _P, _P]),
            "lbf_debug_inject": (C.c_int, [_P, C.c_int, C.c_uint, _P]),
            "lbf_debug_clear": (C.c_int, [_P, _P]),
            "lbf_point_vortices": (C.c_int, [_P, i64, _P, _P, i64, _P, _P, _P, _P, _P, _P, _P]),
            "lbf_dipole_sum": (C.c_int, [i64, _P, i64, _P, _P, _P]),
            "lbf_autotune": (C.c_int, [C.c_int, _P, _P, _P, _P, _P, _P, C.POINTER(lbf_options),
                                       C.c_double, _P, C.c_size_t, C.POINTER(C.c_size_t),
                                       C.POINTER(lbf_options), C.c_char_p, C.c_size_t, _P]),
            "lbf_launch_count": (i64, []),
            "lbf_gmres_workspace_many": (C.c_int, [_P, C.c_int, C.POINTER(C.c_size_t)]),
            "lbf_gmres_solve_many": (C.c_int, [_P, C.c_int, _P, _P, _P, _P, _P, _P, C.c_size_t, _P]),
            "lbf_batch_workspace_size": (C.c_int, [C.c_int, _P, C.POINTER(lbf_options), C.c_int,
                                                   C.POINTER(C.c_size_t)]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def exported_symbols():
    return ["lbf_default_options", "lbf_status_string", "lbf_workspace_size", "lbf_plan_create",
            "lbf_plan_create_planar",
            "lbf_plan_destroy", "lbf_plan_info", "lbf_geometry_out", "lbf_apply",
            "lbf_gmres_solve", "lbf_evaluate", "lbf_green_sum", "lbf_tree_export",
            "lbf_list_export", "lbf_plan_counts", "lbf_border_counts", "lbf_profile_enable",
            "lbf_profile_reset", "lbf_profile_read", "lbf_gmres_solve_transpose",
            "lbf_evaluate_transpose", "lbf_gradient_nodes", "lbf_gradient_data", "lbf_batch_run", "lbf_evaluate_noalloc", "lbf_solve_stats", "lbf_sync_status", "lbf_selftest_rcp", "lbf_autotune", "lbf_debug_inject", "lbf_debug_clear", "lbf_point_vortices", "lbf_dipole_sum",
            "lbf_launch_count", "lbf_gmres_workspace_many", "lbf_gmres_solve_many",
            "lbf_batch_workspace_size"]


def lbf_status_string(status: int) -> str:
    try:
        return load().lbf_status_string(int(status)).decode()
    except Exception:  # noqa: BLE001 - message only
        return str(status)


def _check(rc: int, what: str):
    if rc < 0:
        raise LbfError(rc, what)
    return rc


def _dptr(t: torch.Tensor | None, n: int | None = None, name: str = "array"):
    if t is None:
        return None
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise ValueError(f"{name}: need a contiguous float64 CUDA tensor")
    if n is not None and t.numel() != n:
        raise ValueError(f"{name}: expected {n} entries, got {t.numel()}")
    return C.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def lbf_default_options(**kw) -> lbf_options:
    o = lbf_options()
    _check(load().lbf_default_options(C.byref(o)), "lbf_default_options")
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def lbf_workspace_size(island_ptr: np.ndarray, opt: lbf_options) -> int:
    ptr = np.ascontiguousarray(island_ptr, dtype=np.int64)
    out = C.c_size_t(0)
    _check(load().lbf_workspace_size(len(ptr) - 1, ptr.ctypes.data_as(_P), C.byref(opt),
                                     C.byref(out)), "lbf_workspace_size")
    return int(out.value)


def lbf_batch_workspace_size(island_ptr: np.ndarray, opt: lbf_options, nrhs: int) -> int:
    ptr = np.ascontiguousarray(island_ptr, dtype=np.int64)
    n = C.c_size_t(0)
    _check(load().lbf_batch_workspace_size(len(ptr) - 1, ptr.ctypes.data, C.byref(opt), int(nrhs),
                                           C.byref(n)), "lbf_batch_workspace_size")
    return n.value


class Plan:
    """A plan and the torch-owned workspace it lives in."""

    def __init__(self, handle, workspace, N, M, opt):
        self.handle = handle
        self.workspace = workspace
        self.N, self.M, self.opt = N, M, opt

    def info(self):
        return lbf_plan_info(self)

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.lbf_plan_destroy(self.handle)
            self.handle = None


def _create(planar, island_ptr, a, da, d2a, centres, pole_rotation, opt, stream, device):
    lib = load()
    opt = opt or lbf_default_options()
    ptr = np.ascontiguousarray(island_ptr, dtype=np.int64)
    M = len(ptr) - 1
    N = int(ptr[-1])
    k = 2 if planar else 3
    rot = None if pole_rotation is None else np.ascontiguousarray(pole_rotation, dtype=np.float64)
    dev = a.device if device is None else device
    name = "lbf_plan_create_planar" if planar else "lbf_plan_create"
    for _ in range(6):
        nbytes = lbf_workspace_size(ptr, opt)
        ws = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        h = C.c_void_p()
        need = C.c_int64(0)
        geo = (_dptr(a, k * N, "nodes"), _dptr(da, k * N, "first derivatives"),
               _dptr(d2a, k * N, "second derivatives"), _dptr(centres, 3 * M, "centres"))
        tail = (C.byref(opt), C.c_void_p(ws.data_ptr()), C.c_size_t(nbytes), C.byref(need),
                _stream(stream))
        if planar:
            rc = lib.lbf_plan_create_planar(C.byref(h), M, ptr.ctypes.data_as(_P), *geo, *tail)
        else:
            rc = lib.lbf_plan_create(C.byref(h), M, ptr.ctypes.data_as(_P), *geo,
                                     None if rot is None else rot.ctypes.data_as(_P), *tail)
        if rc == LBF_EWORKSPACE and need.value > opt.box_capacity:
            opt = lbf_options.from_buffer_copy(opt)
            opt.box_capacity = int(need.value)
            del ws
            continue
        _check(rc, name)
        return Plan(h, ws, N, M, opt)
    raise LbfError(LBF_EWORKSPACE, name)


def lbf_plan_create(island_ptr, x, dx, d2x, centres, pole_rotation=None, opt=None, stream=None,
                    device=None) -> Plan:
    """Build a plan from nodes on the sphere (synchronous).  Retries with a larger
    box capacity when the quadtree outgrows the first workspace estimate."""
    return _create(False, island_ptr, x, dx, d2x, centres, pole_rotation, opt, stream, device)


def lbf_plan_create_planar(island_ptr, xi, dxi, d2xi, centres, opt=None, stream=None,
                           device=None) -> Plan:
    """Build a plan from planar nodes xi, xi', xi'' (N x 2 each, synchronous)."""
    return _create(True, island_ptr, xi, dxi, d2xi, centres, None, opt, stream, device)


def lbf_plan_destroy(plan: Plan):
    if plan.handle:
        _check(load().lbf_plan_destroy(plan.handle), "lbf_plan_destroy")
        plan.handle = None


def lbf_plan_info(plan: Plan) -> dict:
    N, M, nb, nl, dep, p = (C.c_int64(), C.c_int(), C.c_int64(), C.c_int64(), C.c_int(), C.c_int())
    _check(load().lbf_plan_info(plan.handle, C.byref(N), C.byref(M), C.byref(nb), C.byref(nl),
                                C.byref(dep), C.byref(p)), "lbf_plan_info")
    return dict(N=N.value, M=M.value, nbox=nb.value, nleaf=nl.value, depth=dep.value, p=p.value)


def lbf_geometry_out(plan: Plan, xi=None, normal=None, weight=None, arc_weight=None, stream=None):
    N = plan.N
    _check(load().lbf_geometry_out(plan.handle, _dptr(xi, 2 * N, "xi"), _dptr(normal, 2 * N, "normal"),
                                   _dptr(weight, 2 * N, "weight"), _dptr(arc_weight, N, "arc_weight"),
                                   _stream(stream)), "lbf_geometry_out")


def lbf_solve_stats(plan: Plan) -> dict:
    st = (C.c_int64 * 4)()
    _check(load().lbf_solve_stats(plan.handle, C.cast(st, _P)), "lbf_solve_stats")
    return dict(arnoldi=int(st[0]), fp64_applies=int(st[1]), fp32_applies=int(st[2]),
                refine_steps=int(st[3]))


def lbf_apply(plan: Plan, op: int, inp: torch.Tensor, out: torch.Tensor, stream=None):
    n = plan.N if (op & ~(LBF_OP_FP32 | LBF_OP_TRANSPOSE)) == LBF_OP_K_ONLY else plan.N + plan.M
    _check(load().lbf_apply(plan.handle, int(op), _dptr(inp, n, "in"), _dptr(out, n, "out"),
                            _stream(stream)), "lbf_apply")


def lbf_gmres_solve(plan: Plan, g: torch.Tensor, sigma: torch.Tensor, a: torch.Tensor | None = None,
                    x0: torch.Tensor | None = None, stream=None):
    """Returns (status, iterations, relative residual); status LBF_NOCONV (> 0) if maxit hit."""
    it, rr = C.c_int(0), C.c_double(0.0)
    rc = load().lbf_gmres_solve(plan.handle, _dptr(g, plan.N, "g"), _dptr(sigma, plan.N, "sigma"),
                                _dptr(a, plan.M, "a"), _dptr(x0, plan.N + plan.M, "x0"),
                                C.byref(it), C.byref(rr), _stream(stream))
    _check(rc, "lbf_gmres_solve")
    return rc, it.value, rr.value


def lbf_gmres_workspace_many(plan: Plan, nrhs: int) -> int:
    n = C.c_size_t(0)
    _check(load().lbf_gmres_workspace_many(plan.handle, int(nrhs), C.byref(n)), "lbf_gmres_workspace_many")
    return n.value


def lbf_gmres_solve_many(plan: Plan, g: torch.Tensor, sigma: torch.Tensor,
                         a: torch.Tensor | None = None, work: torch.Tensor | None = None,
                         stream=None):
    """g: nrhs x N (device).  Returns (status, iterations per rhs, relative residual per rhs)."""
    nrhs = g.numel() // plan.N
    if nrhs < 1 or g.numel() != nrhs * plan.N:
        raise ValueError("g must hold nrhs x N values")
    need = lbf_gmres_workspace_many(plan, nrhs)
    if work is None and need > 0:
        work = torch.empty(need, dtype=torch.uint8, device=g.device)
    its = (C.c_int * nrhs)()
    rr = (C.c_double * nrhs)()
    rc = load().lbf_gmres_solve_many(plan.handle, nrhs, _dptr(g, nrhs * plan.N, "g"),
                                     _dptr(sigma, nrhs * plan.N, "sigma"),
                                     _dptr(a, nrhs * plan.M, "a"), its, rr,
                                     None if work is None else work.data_ptr(),
                                     0 if work is None else work.numel() * work.element_size(),
                                     _stream(stream))
    _check(rc, "lbf_gmres_solve_many")
    return rc, list(its), list(rr)


def lbf_evaluate(plan: Plan, sigma: torch.Tensor, a: torch.Tensor | None, targets: torch.Tensor,
                 u: torch.Tensor, stream=None):
    T = targets.numel() // 3
    _check(load().lbf_evaluate(plan.handle, _dptr(sigma, plan.N, "sigma"), _dptr(a, plan.M, "a"),
                               T, _dptr(targets, 3 * T, "targets"), _dptr(u, T, "u"),
                               _stream(stream)), "lbf_evaluate")


def lbf_gmres_solve_transpose(plan: Plan, r: torch.Tensor, lam: torch.Tensor,
                              x0: torch.Tensor | None = None, stream=None):
    """Adjoint solve A^T lam = r (N + M vectors); returns (status, iterations, residual)."""
    n = plan.N + plan.M
    it, rr = C.c_int(0), C.c_double(0.0)
    rc = load().lbf_gmres_solve_transpose(plan.handle, _dptr(r, n, "r"), _dptr(lam, n, "lam"),
                                          _dptr(x0, n, "x0"), C.byref(it), C.byref(rr),
                                          _stream(stream))
    _check(rc, "lbf_gmres_solve_transpose")
    return rc, it.value, rr.value


def lbf_evaluate_transpose(plan: Plan, targets: torch.Tensor, ubar: torch.Tensor,
                           sbar: torch.Tensor, abar: torch.Tensor | None = None, stream=None):
    T = targets.numel() // 3
    _check(load().lbf_evaluate_transpose(plan.handle, T, _dptr(targets, 3 * T, "targets"),
                                         _dptr(ubar, T, "ubar"), _dptr(sbar, plan.N, "sbar"),
                                         _dptr(abar, plan.M, "abar"), _stream(stream)),
           "lbf_evaluate_transpose")


def lbf_gradient_nodes(plan: Plan, sigma: torch.Tensor, a: torch.Tensor, lam: torch.Tensor,
                       targets: torch.Tensor, ubar: torch.Tensor, grad: torch.Tensor, stream=None):
    T = targets.numel() // 3
    _check(load().lbf_gradient_nodes(plan.handle, _dptr(sigma, plan.N, "sigma"),
                                     _dptr(a, plan.M, "a"), _dptr(lam, plan.N + plan.M, "lam"), T,
                                     _dptr(targets, 3 * T, "targets"), _dptr(ubar, T, "ubar"),
                                     _dptr(grad, 2 * plan.N, "grad"), _stream(stream)),
           "lbf_gradient_nodes")


def lbf_gradient_data(plan: Plan, lam: torch.Tensor, grad_g: torch.Tensor, stream=None):
    _check(load().lbf_gradient_data(plan.handle, _dptr(lam, plan.N + plan.M, "lam"),
                                    _dptr(grad_g, plan.N, "grad_g"), _stream(stream)),
           "lbf_gradient_data")


def lbf_batch_run(instances, opt=None, nworkers=8, lockstep=True):
    """Solve many independent instances (native scheduler, one CUDA stream per worker).

    instances: list of dicts with keys island_ptr (host int64, M + 1), x, dx, d2x,
    centres (CUDA float64), g (nrhs x N), and optionally targets (T x 3).  Returns a
    list of dicts with sigma (nrhs x N), a (nrhs x M), u (nrhs x T or None) and the
    item's status, iters, fp64_applies, fp32_applies, max_rel_res.  Instances whose
    quadtree outgrew the workspace estimate are rerun with the size they reported.
    lockstep: size each workspace for lbf_gmres_solve_many (lbf_batch_workspace_size), so
    that an instance's right-hand sides advance together; else one after another."""
    lib = load()
    opt = opt or lbf_default_options()
    n = len(instances)
    results = [None] * n
    todo = list(range(n))
    caps = [opt.box_capacity] * n
    for _ in range(4):
        if not todo:
            break
        items = (lbf_batch_item * len(todo))()
        keep = []
        for slot, q in enumerate(todo):
            ins = instances[q]
            ptr = np.ascontiguousarray(ins["island_ptr"], dtype=np.int64)
            M, N = len(ptr) - 1, int(ptr[-1])
            o = lbf_options.from_buffer_copy(opt)
            o.box_capacity = caps[q]
            g = ins["g"].reshape(-1)
            nrhs = g.numel() // N
            nbytes = lbf_batch_workspace_size(ptr, o, nrhs) if lockstep else lbf_workspace_size(ptr, o)
            dev = ins["x"].device
            ws = torch.empty(nbytes, dtype=torch.uint8, device=dev)
            sigma = torch.empty(nrhs * N, dtype=torch.float64, device=dev)
            a = torch.empty(nrhs * M, dtype=torch.float64, device=dev)
            t = ins.get("targets")
            T = 0 if t is None else t.numel() // 3
            u = torch.empty(nrhs * T, dtype=torch.float64, device=dev) if T else None
            it = items[slot]
            it.M, it.island_ptr = M, ptr.ctypes.data
            it.x = _dptr(ins["x"], 3 * N, "x").value
            it.dx = _dptr(ins["dx"], 3 * N, "dx").value
            it.d2x = _dptr(ins["d2x"], 3 * N, "d2x").value
            it.centres = _dptr(ins["centres"], 3 * M, "centres").value
            it.workspace, it.bytes = ws.data_ptr(), nbytes
            it.nrhs, it.g = nrhs, _dptr(g, nrhs * N, "g").value
            it.sigma, it.a = sigma.data_ptr(), a.data_ptr()
            it.T = T
            it.targets = None if T == 0 else _dptr(t, 3 * T, "targets").value
            it.u = None if u is None else u.data_ptr()
            it.box_capacity = caps[q]
            keep.append((q, ptr, ws, sigma, a, u, nrhs, N, M, T))
        _check(lib.lbf_batch_run(len(todo), items, C.byref(opt), int(nworkers)), "lbf_batch_run")
        nxt = []
        for slot, (q, ptr, ws, sigma, a, u, nrhs, N, M, T) in enumerate(keep):
            it = items[slot]
            if it.status == LBF_EWORKSPACE and it.box_capacity_needed > caps[q]:
                caps[q] = int(it.box_capacity_needed)
                nxt.append(q)
                continue
            results[q] = dict(sigma=sigma.view(nrhs, N), a=a.view(nrhs, M),
                              u=None if u is None else u.view(nrhs, T), status=it.status,
                              iters=it.iters, fp64_applies=it.fp64_applies,
                              fp32_applies=it.fp32_applies, max_rel_res=it.max_rel_res)
        todo = nxt
    for q in todo:
        raise LbfError(LBF_EWORKSPACE, f"lbf_batch_run item {q}")
    return results


def lbf_point_vortices(plan: Plan, vortices: torch.Tensor, gamma: torch.Tensor,
                       targets: torch.Tensor, u: torch.Tensor, sigma: torch.Tensor,
                       a: torch.Tensor, stream=None):
    """psi at the targets for point vortices in the ocean with psi = 0 on the curves
    (Sec. 6, Example 2).  Returns (status, iterations, relative residual)."""
    S, T = vortices.numel() // 3, targets.numel() // 3
    it, rr = C.c_int(0), C.c_double(0.0)
    rc = load().lbf_point_vortices(plan.handle, S, _dptr(vortices, 3 * S, "vortices"),
                                   _dptr(gamma, S, "gamma"), T, _dptr(targets, 3 * T, "targets"),
                                   _dptr(u, T, "u"), _dptr(sigma, plan.N, "sigma"),
                                   _dptr(a, plan.M, "a"), C.byref(it), C.byref(rr), _stream(stream))
    _check(rc, "lbf_point_vortices")
    return rc, it.value, rr.value


def lbf_dipole_sum(t: torch.Tensor, p: torch.Tensor, out: torch.Tensor, stream=None):
    T, S = t.numel() // 3, p.numel() // 3
    _check(load().lbf_dipole_sum(T, _dptr(t, 3 * T, "t"), S, _dptr(p, 3 * S, "p"),
                                 _dptr(out, T, "out"), _stream(stream)), "lbf_dipole_sum")


def lbf_green_sum(t: torch.Tensor, p: torch.Tensor, gamma: torch.Tensor, out: torch.Tensor,
                  stream=None):
    T, S = t.numel() // 3, p.numel() // 3
    _check(load().lbf_green_sum(T, _dptr(t, 3 * T, "t"), S, _dptr(p, 3 * S, "p"),
                                _dptr(gamma, S, "gamma"), _dptr(out, T, "out"), _stream(stream)),
           "lbf_green_sum")


def lbf_tree_export(plan: Plan, stream=None):
    """(perm, boxes) as int32 CUDA tensors; boxes rows are
    (level, ix, iy, parent, first_child, nchild, begin, end)."""
    nbox = lbf_plan_info(plan)["nbox"]
    dev = plan.workspace.device
    perm = torch.empty(plan.N, dtype=torch.int32, device=dev)
    boxes = torch.empty((nbox, 8), dtype=torch.int32, device=dev)
    _check(load().lbf_tree_export(plan.handle, C.c_void_p(perm.data_ptr()),
                                  C.c_void_p(boxes.data_ptr()), _stream(stream)), "lbf_tree_export")
    return perm, boxes


def lbf_list_export(plan: Plan, kind: int, stream=None):
    """(ptr, idx) of list kind 0..3 = U, V, W, X as int32 CUDA tensors."""
    nbox = lbf_plan_info(plan)["nbox"]
    dev = plan.workspace.device
    ptr = torch.empty(nbox + 1, dtype=torch.int32, device=dev)
    n = C.c_int64(0)
    lib = load()
    _check(lib.lbf_list_export(plan.handle, int(kind), C.c_void_p(ptr.data_ptr()), None,
                               C.byref(n), _stream(stream)), "lbf_list_export")
    idx = torch.empty(max(1, n.value), dtype=torch.int32, device=dev)
    _check(lib.lbf_list_export(plan.handle, int(kind), C.c_void_p(ptr.data_ptr()),
                               C.c_void_p(idx.data_ptr()), C.byref(n), _stream(stream)),
           "lbf_list_export")
    return ptr, idx[: n.value]


LBF_KERNEL_UP, LBF_KERNEL_DOWN, LBF_KERNEL_LEAF = 0, 1, 2
LBF_KERNEL_DIRECT, LBF_KERNEL_ARNOLDI, LBF_KERNEL_ESUM = 3, 4, 5
KERNEL_NAMES = ["up", "down", "leaf", "direct", "arnoldi", "esum", "up32", "down32", "leaf32",
                "esum32", "plan_geometry", "plan_border", "plan_inverse", "lu_panel", "lu_update",
                "lu_gemm", "lu_solve"]


def lbf_plan_counts(plan: Plan, stream=None) -> dict:
    c = (C.c_int64 * 8)()
    _check(load().lbf_plan_counts(plan.handle, C.cast(c, _P), _stream(stream)), "lbf_plan_counts")
    keys = ["N", "p2p_pairs", "m2m", "m2l", "l2l", "w_pairs", "x_pairs", "leaves"]
    return dict(zip(keys, [int(v) for v in c]))


def lbf_border_counts(plan: Plan, stream=None) -> dict:
    c = (C.c_int64 * 6)()
    _check(load().lbf_border_counts(plan.handle, C.cast(c, _P), _stream(stream)), "lbf_border_counts")
    keys = ["p2l_pairs", "direct_pairs", "global_centres", "walk_expansions", "terms", "terms32"]
    return dict(zip(keys, [int(v) for v in c]))


def lbf_profile_enable(on: bool = True):
    _check(load().lbf_profile_enable(1 if on else 0), "lbf_profile_enable")


def lbf_profile_reset():
    _check(load().lbf_profile_reset(), "lbf_profile_reset")


def lbf_profile_read(kernel: int):
    """(launches, total device ms) of one traced kernel."""
    n, t = C.c_int64(0), C.c_double(0.0)
    _check(load().lbf_profile_read(int(kernel), C.byref(n), C.byref(t)), "lbf_profile_read")
    return int(n.value), float(t.value)


LBF_NOALLOC_MAX_NODES = 262144


def lbf_evaluate_noalloc(xi: torch.Tensor, weight: torch.Tensor, sigma: torch.Tensor,
                         a: torch.Tensor | None, centres: torch.Tensor | None,
                         targets: torch.Tensor, u: torch.Tensor, stream=None, N: int | None = None):
    """Off-curve evaluation without any device allocation (static scratch in the
    library; N <= LBF_NOALLOC_MAX_NODES; overlapping calls race).  Every array is
    checked against N, M and T before the call.  N defaults to sigma's length; a
    larger N is accepted only beyond LBF_NOALLOC_MAX_NODES, where the library
    rejects the call before it reads any array."""
    N = sigma.numel() if N is None else int(N)
    if N > sigma.numel() and N <= LBF_NOALLOC_MAX_NODES:
        raise ValueError(f"N = {N} exceeds the {sigma.numel()} densities passed")
    checked = N <= LBF_NOALLOC_MAX_NODES
    M = 0 if a is None else a.numel()
    if (a is None) != (centres is None):
        raise ValueError("a and centres go together")
    T = targets.numel() // 3
    if targets.numel() != 3 * T:
        raise ValueError("targets: need T x 3 entries")
    _check(load().lbf_evaluate_noalloc(
        N, _dptr(xi, 2 * N if checked else None, "xi"),
        _dptr(weight, 2 * N if checked else None, "weight"),
        _dptr(sigma, N if checked else None, "sigma"), M, _dptr(a, M, "a"),
        _dptr(centres, 3 * M, "centres"), T, _dptr(targets, 3 * T, "targets"),
        _dptr(u, T, "u"), _stream(stream)), "lbf_evaluate_noalloc")


def lbf_autotune(island_ptr, x, dx, d2x, centres, target: float, opt=None, pole_rotation=None,
                 stream=None):
    """(options with p, leaf_size and p2p_warps chosen for this geometry, trial table)
    from the library's timed trials (synchronous; the workspace is a torch tensor)."""
    import json

    lib = load()
    opt = opt or lbf_default_options()
    ptr = np.ascontiguousarray(island_ptr, dtype=np.int64)
    M, N = len(ptr) - 1, int(ptr[-1])
    rot = None if pole_rotation is None else np.ascontiguousarray(pole_rotation, dtype=np.float64)
    need = C.c_size_t(0)
    best = lbf_options()
    _check(lib.lbf_autotune(M, ptr.ctypes.data_as(_P), None, None, None, None, None, C.byref(opt),
                            float(target), None, 0, C.byref(need), C.byref(best), None, 0,
                            _stream(stream)), "lbf_autotune")
    ws = torch.empty(int(need.value), dtype=torch.uint8, device=x.device)
    buf = C.create_string_buffer(1 << 16)
    rc = lib.lbf_autotune(M, ptr.ctypes.data_as(_P), _dptr(x, 3 * N, "x"), _dptr(dx, 3 * N, "dx"),
                          _dptr(d2x, 3 * N, "d2x"), _dptr(centres, 3 * M, "centres"),
                          None if rot is None else rot.ctypes.data_as(_P), C.byref(opt),
                          float(target), C.c_void_p(ws.data_ptr()), int(need.value), C.byref(need),
                          C.byref(best), buf, len(buf), _stream(stream))
    _check(rc, "lbf_autotune")
    del ws
    return best, json.loads(buf.value.decode())


def lbf_selftest_rcp(variant: int, a: torch.Tensor, out: torch.Tensor, stream=None):
    n = a.numel()
    _check(load().lbf_selftest_rcp(int(variant), n, _dptr(a, n, "a"), _dptr(out, n, "out"),
                                   _stream(stream)), "lbf_selftest_rcp")


LBF_INJECT_CHAIN = 1
LBF_INJECT_BARRIER = 2


def lbf_debug_inject(plan, what: int, polls: int, stream=None):
    _check(load().lbf_debug_inject(None if plan is None else plan.handle, int(what), int(polls),
                                   _stream(stream)), "lbf_debug_inject")


def lbf_debug_clear(plan: Plan, stream=None):
    _check(load().lbf_debug_clear(plan.handle, _stream(stream)), "lbf_debug_clear")


def lbf_sync_status(plan: Plan, stream=None) -> int:
    return load().lbf_sync_status(plan.handle, _stream(stream))


def lbf_launch_count() -> int:
    return int(load().lbf_launch_count())
