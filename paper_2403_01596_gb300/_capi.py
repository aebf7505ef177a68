"""ctypes binding of libp2p.so: the C ABI of include/p2p.h with the same names.

Argument marshalling only: every step of the operator runs in the library's
CUDA kernels.  Tensors are passed as raw device pointers, streams as the
cudaStream_t handle of a torch.cuda.Stream.  A missing library raises at first
use; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

P2P_OK = 0
P2P_ERR_INVALID = 1
P2P_ERR_WORKSPACE = 2
P2P_ERR_CUDA = 3
P2P_ERR_TIMEOUT = 4
P2P_ERR_UNSUPPORTED = 5
P2P_ERR_ALLOC = 6
P2P_ERR_STALE = 7

P2P_HELMHOLTZ = 0
P2P_LAPLACE = 1
P2P_LAYOUT_INDEXED = 0
P2P_LAYOUT_REDUNDANT = 1
P2P_LAYOUT_SYMMETRIC = 2
P2P_LAYOUT_REPETITION = 3
P2P_PATH_AUTO = 0
P2P_PATH_FP32_PER_RHS = 1
P2P_PATH_FP32_SHARED = 2
P2P_PATH_TC_BF16X3 = 3
P2P_PATH_TC_BF16X6 = 4

_lock = threading.Lock()
_lib = None


class P2PError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        lib = _lib
        msg = lib.p2p_status_string(status).decode() if lib else str(status)
        detail = lib.p2p_last_error_string().decode() if (lib and status == P2P_ERR_CUDA) else ""
        super().__init__(f"{where}: {msg}" + (f" ({detail})" if detail else ""))


class p2p_tuning(ctypes.Structure):
    _fields_ = [("chunk", ctypes.c_int32), ("warps_per_cta", ctypes.c_int32),
                ("target_group", ctypes.c_int32), ("warp_boxes", ctypes.c_int32)]


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Loads libp2p.so (building it in-tree first if it is missing)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = os.environ.get("P2P_LIBRARY") or _build.LIB
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError(f"libp2p.so not found at {path}")
            _build.build()
        lib = ctypes.CDLL(path)
        P, i32, i64, sz, dbl, flt = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t,
                                      ctypes.c_double, ctypes.c_float)
        PI64, PI32, PSZ = ctypes.POINTER(i64), ctypes.POINTER(i32), ctypes.POINTER(sz)
        sigs = {
            "p2p_status_string": ([ctypes.c_int], ctypes.c_char_p),
            "p2p_last_error_string": ([], ctypes.c_char_p),
            "p2p_version": ([], i32),
            "p2p_bin_workspace_size": ([i64, PSZ], ctypes.c_int),
            "p2p_bin_points": ([P, i64, P, dbl, i32, P, P, P, P, PI32, P, sz, P], ctypes.c_int),
            "p2p_bin_points_static": ([P, i64, P, dbl, i32, P, P, P, P, PI32, P], ctypes.c_int),
            "p2p_neighbors_workspace_size": ([i32, PSZ], ctypes.c_int),
            "p2p_build_neighbors": ([P, P, i32, i32, P, P, PI64, PI64, P, sz, P], ctypes.c_int),
            "p2p_apply_guarded_workspace_size": ([P, i32, PSZ], ctypes.c_int),
            "p2p_apply_guarded": ([P, P, P, i32, i64, i32, ctypes.c_int, dbl, P, sz, PI64, P], ctypes.c_int),
            "p2p_repetition_records": ([P, i32, P, P, PI64, P], ctypes.c_int),
            "p2p_plan_workspace_size_rep": ([i64, i32, i64, i64, i64, P, PSZ], ctypes.c_int),
            "p2p_plan_update_points": ([P, P, P, dbl, i32, PI64, P], ctypes.c_int),
            "p2p_build_neighbors_st": ([P, i32, P, P, i32, i32, P, P, P, PI64, PI64, P, sz, P], ctypes.c_int),
            "p2p_plan_workspace_size": ([i64, i32, i64, i64, ctypes.c_int, i32, P, PSZ], ctypes.c_int),
            "p2p_plan_workspace_size_st": ([i64, i32, i64, i32, i64, i64, ctypes.c_int, i32, P, PSZ], ctypes.c_int),
            "p2p_plan_create_st": ([ctypes.POINTER(P), P, i64, P, P, i32, P, i64, P, P, i32, P, P, P, i64, i64,
                                    ctypes.c_int, flt, ctypes.c_int, i32, P, P, sz, P], ctypes.c_int),
            "p2p_plan_create": ([ctypes.POINTER(P), P, i64, P, P, i32, P, P, i64, i64, ctypes.c_int, flt,
                                 ctypes.c_int, i32, P, P, sz, P], ctypes.c_int),
            "p2p_plan_destroy": ([P], ctypes.c_int),
            "p2p_plan_info": ([P, PI64, PI32, PI64, PI64, ctypes.POINTER(ctypes.c_int), P], ctypes.c_int),
            "p2p_plan_pair_count": ([P, PI64, P], ctypes.c_int),
            "p2p_apply": ([P, P, P, i32, i64, P], ctypes.c_int),
            "p2p_apply_adjoint": ([P, P, P, i32, i64, P], ctypes.c_int),
            "p2p_apply_path": ([P, P, P, i32, i64, i32, ctypes.c_int, P], ctypes.c_int),
            "p2p_apply_stage": ([P, P, i32, i64, ctypes.c_int, P], ctypes.c_int),
            "p2p_apply_staged": ([P, P, i32, i64, i32, ctypes.c_int, P], ctypes.c_int),
            "p2p_grad_points": ([P, P, P, P, i32, i64, P], ctypes.c_int),
            "p2p_last_async_status": ([P, P], ctypes.c_int),
            "p2p_diag_tc_gemm": ([P, P, P, i32, i32, P, P], ctypes.c_int),
            "p2p_diag_wait_timeout": ([P, i32, P], ctypes.c_int),
            "p2p_diag_tc_wait_limit": ([P, i32], ctypes.c_int),
            "p2p_batch_workspace_size": ([P, i32, i32, PSZ], ctypes.c_int),
            "p2p_batch_create": ([ctypes.POINTER(P), P, i32, i32, i32, P, sz, P], ctypes.c_int),
            "p2p_batch_apply": ([P, P, P, i64, P], ctypes.c_int),
            "p2p_batch_graph_create": ([P, P, P, i64], ctypes.c_int),
            "p2p_batch_graph_launch": ([P, P], ctypes.c_int),
            "p2p_batch_info": ([P, PI64, PI32, PI32], ctypes.c_int),
            "p2p_batch_destroy": ([P], ctypes.c_int),
            "p2p_host_pipe_workspace_size": ([i64, i32, PSZ], ctypes.c_int),
            "p2p_host_pipe_create": ([ctypes.POINTER(P), i64, i32, P, sz], ctypes.c_int),
            "p2p_apply_host": ([P, P, i32, P, P, P], ctypes.c_int),
            "p2p_host_pipe_destroy": ([P], ctypes.c_int),
        }
        for name, (args, res) in sigs.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        _lib = lib
        return lib


def check(status: int, where: str):
    if status != P2P_OK:
        raise P2PError(status, where)


def _ptr(t) -> ctypes.c_void_p:
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _stream(stream) -> ctypes.c_void_p:
    return ctypes.c_void_p(0 if stream is None else int(stream.cuda_stream))


def _lo(lo):
    return (ctypes.c_double * 3)(*[float(v) for v in lo])


# --------------------------------------------------------------- C ABI calls --

def p2p_bin_workspace_size(n: int) -> int:
    out = ctypes.c_size_t(0)
    check(load().p2p_bin_workspace_size(n, ctypes.byref(out)), "p2p_bin_workspace_size")
    return out.value


def p2p_bin_points(pts, lo, h, ng, perm, point_box, box_keys, box_ptr, work, stream=None) -> int:
    nb = ctypes.c_int32(0)
    st = load().p2p_bin_points(_ptr(pts), pts.shape[0], _lo(lo), float(h), int(ng), _ptr(perm), _ptr(point_box),
                               _ptr(box_keys), _ptr(box_ptr), ctypes.byref(nb), _ptr(work), work.numel(),
                               _stream(stream))
    check(st, "p2p_bin_points")
    return nb.value


P2P_BIN_STATIC_MAX_POINTS = 65536


def p2p_bin_points_static(pts, lo, h, ng, perm, point_box, box_keys, box_ptr, stream=None) -> int:
    """p2p_bin_points without a workspace (scratch in a fixed device array, n <= 65536)."""
    nb = ctypes.c_int32(0)
    st = load().p2p_bin_points_static(_ptr(pts), pts.shape[0], _lo(lo), float(h), int(ng), _ptr(perm),
                                      _ptr(point_box), _ptr(box_keys), _ptr(box_ptr), ctypes.byref(nb),
                                      _stream(stream))
    check(st, "p2p_bin_points_static")
    return nb.value


def p2p_neighbors_workspace_size(num_boxes: int) -> int:
    out = ctypes.c_size_t(0)
    check(load().p2p_neighbors_workspace_size(num_boxes, ctypes.byref(out)), "p2p_neighbors_workspace_size")
    return out.value


def p2p_build_neighbors(box_keys, box_ptr, num_boxes, ng, nbr_ptr, nbr_idx, work, stream=None):
    nnz, src = ctypes.c_int64(0), ctypes.c_int64(0)
    st = load().p2p_build_neighbors(_ptr(box_keys), _ptr(box_ptr), int(num_boxes), int(ng), _ptr(nbr_ptr),
                                    _ptr(nbr_idx), ctypes.byref(nnz), ctypes.byref(src), _ptr(work), work.numel(),
                                    _stream(stream))
    check(st, "p2p_build_neighbors")
    return nnz.value, src.value


def p2p_build_neighbors_st(tgt_keys, num_tgt_boxes, src_keys, src_box_ptr, num_src_boxes, ng, nbr_ptr, nbr_idx,
                           nbr_self, work, stream=None):
    nnz, src = ctypes.c_int64(0), ctypes.c_int64(0)
    st = load().p2p_build_neighbors_st(_ptr(tgt_keys), int(num_tgt_boxes), _ptr(src_keys), _ptr(src_box_ptr),
                                       int(num_src_boxes), int(ng), _ptr(nbr_ptr), _ptr(nbr_idx), _ptr(nbr_self),
                                       ctypes.byref(nnz), ctypes.byref(src), _ptr(work), work.numel(),
                                       _stream(stream))
    check(st, "p2p_build_neighbors_st")
    return nnz.value, src.value


def _tuning(t):
    if t is None:
        return None
    return ctypes.byref(p2p_tuning(int(t.get("chunk", 0)), int(t.get("warps_per_cta", 0)),
                                   int(t.get("target_group", 0)), int(t.get("warp_boxes", 0))))


def p2p_plan_workspace_size(n, num_boxes, nnz, sources, layout, max_nrhs, tuning=None) -> int:
    out = ctypes.c_size_t(0)
    check(load().p2p_plan_workspace_size(n, num_boxes, nnz, sources, layout, max_nrhs, _tuning(tuning),
                                         ctypes.byref(out)), "p2p_plan_workspace_size")
    return out.value


def p2p_plan_create(pts, perm, box_ptr, num_boxes, nbr_ptr, nbr_idx, nnz, sources, kernel, k, layout, max_nrhs,
                    tuning, workspace, stream=None) -> ctypes.c_void_p:
    plan = ctypes.c_void_p(0)
    st = load().p2p_plan_create(ctypes.byref(plan), _ptr(pts), pts.shape[0], _ptr(perm), _ptr(box_ptr),
                                int(num_boxes), _ptr(nbr_ptr), _ptr(nbr_idx), int(nnz), int(sources), int(kernel),
                                float(k), int(layout), int(max_nrhs), _tuning(tuning), _ptr(workspace),
                                workspace.numel(), _stream(stream))
    check(st, "p2p_plan_create")
    return plan


def p2p_plan_workspace_size_st(n_tgt, num_tgt_boxes, n_src, num_src_boxes, nnz, sources, layout, max_nrhs,
                               tuning=None) -> int:
    out = ctypes.c_size_t(0)
    check(load().p2p_plan_workspace_size_st(n_tgt, num_tgt_boxes, n_src, num_src_boxes, nnz, sources, layout,
                                            max_nrhs, _tuning(tuning), ctypes.byref(out)),
          "p2p_plan_workspace_size_st")
    return out.value


def p2p_plan_create_st(tgt_pts, tgt_perm, tgt_box_ptr, num_tgt_boxes, src_pts, src_perm, src_box_ptr, num_src_boxes,
                       nbr_ptr, nbr_idx, nbr_self, nnz, sources, kernel, k, layout, max_nrhs, tuning, workspace,
                       stream=None) -> ctypes.c_void_p:
    plan = ctypes.c_void_p(0)
    st = load().p2p_plan_create_st(ctypes.byref(plan), _ptr(tgt_pts), tgt_pts.shape[0], _ptr(tgt_perm),
                                   _ptr(tgt_box_ptr), int(num_tgt_boxes), _ptr(src_pts), src_pts.shape[0],
                                   _ptr(src_perm), _ptr(src_box_ptr), int(num_src_boxes), _ptr(nbr_ptr),
                                   _ptr(nbr_idx), _ptr(nbr_self), int(nnz), int(sources), int(kernel), float(k),
                                   int(layout), int(max_nrhs), _tuning(tuning), _ptr(workspace), workspace.numel(),
                                   _stream(stream))
    check(st, "p2p_plan_create_st")
    return plan


def p2p_plan_destroy(plan):
    if plan:
        load().p2p_plan_destroy(plan)


def p2p_plan_info(plan) -> dict:
    n, nb, src, items = ctypes.c_int64(0), ctypes.c_int32(0), ctypes.c_int64(0), ctypes.c_int64(0)
    layout = ctypes.c_int(0)
    t = p2p_tuning()
    check(load().p2p_plan_info(plan, ctypes.byref(n), ctypes.byref(nb), ctypes.byref(src), ctypes.byref(items),
                               ctypes.byref(layout), ctypes.byref(t)), "p2p_plan_info")
    return {"n": n.value, "num_boxes": nb.value, "sources": src.value, "work_items": items.value,
            "layout": layout.value, "tuning": {"chunk": t.chunk, "warps_per_cta": t.warps_per_cta,
                                               "target_group": t.target_group, "warp_boxes": t.warp_boxes}}


def p2p_repetition_records(box_ptr, num_boxes, nbr_ptr, nbr_idx, stream=None) -> int:
    out = ctypes.c_int64(0)
    check(load().p2p_repetition_records(_ptr(box_ptr), int(num_boxes), _ptr(nbr_ptr), _ptr(nbr_idx),
                                        ctypes.byref(out), _stream(stream)), "p2p_repetition_records")
    return out.value


def p2p_plan_workspace_size_rep(n, num_boxes, nnz, sources, records, tuning=None) -> int:
    out = ctypes.c_size_t(0)
    check(load().p2p_plan_workspace_size_rep(n, num_boxes, nnz, sources, records, _tuning(tuning),
                                             ctypes.byref(out)), "p2p_plan_workspace_size_rep")
    return out.value


def p2p_plan_update_points(plan, pts, lo, h, ng, stream=None):
    """New coordinates for a plan; returns (status, moved): P2P_OK, or P2P_ERR_STALE when `moved` points would
    change leaf box (the plan is then unchanged).  Other failures raise."""
    lo_arr = (ctypes.c_double * 3)(*[float(v) for v in lo])
    moved = ctypes.c_int64(0)
    st = load().p2p_plan_update_points(plan, _ptr(pts), lo_arr, float(h), int(ng), ctypes.byref(moved),
                                       _stream(stream))
    if st not in (P2P_OK, P2P_ERR_STALE):
        check(st, "p2p_plan_update_points")
    return st, moved.value


def p2p_plan_pair_count(plan, stream=None) -> int:
    out = ctypes.c_int64(0)
    check(load().p2p_plan_pair_count(plan, ctypes.byref(out), _stream(stream)), "p2p_plan_pair_count")
    return out.value


def p2p_apply(plan, lam, out, nrhs, ld, stream=None):
    check(load().p2p_apply(plan, _ptr(lam), _ptr(out), int(nrhs), int(ld), _stream(stream)), "p2p_apply")


def p2p_apply_adjoint(plan, g, out, nrhs, ld, stream=None):
    check(load().p2p_apply_adjoint(plan, _ptr(g), _ptr(out), int(nrhs), int(ld), _stream(stream)),
          "p2p_apply_adjoint")


def p2p_apply_path(plan, lam, out, nrhs, ld, adjoint, path, stream=None):
    check(load().p2p_apply_path(plan, _ptr(lam), _ptr(out), int(nrhs), int(ld), int(adjoint), int(path),
                                _stream(stream)), "p2p_apply_path")


def p2p_apply_stage(plan, lam, nrhs, ld, path, stream=None):
    check(load().p2p_apply_stage(plan, _ptr(lam), int(nrhs), int(ld), int(path), _stream(stream)),
          "p2p_apply_stage")


def p2p_apply_staged(plan, out, nrhs, ld, adjoint, path, stream=None):
    check(load().p2p_apply_staged(plan, _ptr(out), int(nrhs), int(ld), int(adjoint), int(path), _stream(stream)),
          "p2p_apply_staged")


def p2p_grad_points(plan, lam, g, grad, nrhs, ld, stream=None):
    check(load().p2p_grad_points(plan, _ptr(lam), _ptr(g), _ptr(grad), int(nrhs), int(ld), _stream(stream)),
          "p2p_grad_points")


def p2p_last_async_status(plan, stream=None) -> int:
    return load().p2p_last_async_status(plan, _stream(stream))


def p2p_diag_tc_gemm(A, B, D, status, stream=None):
    check(load().p2p_diag_tc_gemm(_ptr(A), _ptr(B), _ptr(D), int(A.shape[1]), int(B.shape[0]), _ptr(status), _stream(stream)),
          "p2p_diag_tc_gemm")


def _ptr_array(items):
    arr = (ctypes.c_void_p * len(items))()
    for i, t in enumerate(items):
        arr[i] = t if isinstance(t, int) else (t.value if isinstance(t, ctypes.c_void_p) else t.data_ptr())
    return arr


def p2p_batch_workspace_size(plans, nrhs) -> int:
    out = ctypes.c_size_t(0)
    check(load().p2p_batch_workspace_size(_ptr_array(plans), len(plans), int(nrhs), ctypes.byref(out)),
          "p2p_batch_workspace_size")
    return out.value


def p2p_batch_create(plans, nrhs, warps_per_cta, workspace, stream=None):
    batch = ctypes.c_void_p(0)
    check(load().p2p_batch_create(ctypes.byref(batch), _ptr_array(plans), len(plans), int(nrhs), int(warps_per_cta),
                                  _ptr(workspace), workspace.numel(), _stream(stream)), "p2p_batch_create")
    return batch


def p2p_batch_apply(batch, lams, outs, ld, stream=None):
    check(load().p2p_batch_apply(batch, _ptr_array(lams), _ptr_array(outs), int(ld), _stream(stream)),
          "p2p_batch_apply")


def p2p_batch_graph_create(batch, lams, outs, ld):
    check(load().p2p_batch_graph_create(batch, _ptr_array(lams), _ptr_array(outs), int(ld)), "p2p_batch_graph_create")


def p2p_batch_graph_launch(batch, stream=None):
    check(load().p2p_batch_graph_launch(batch, _stream(stream)), "p2p_batch_graph_launch")


def p2p_batch_info(batch) -> dict:
    items, grid, warps = ctypes.c_int64(0), ctypes.c_int32(0), ctypes.c_int32(0)
    check(load().p2p_batch_info(batch, ctypes.byref(items), ctypes.byref(grid), ctypes.byref(warps)), "p2p_batch_info")
    return {"work_items": items.value, "grid": grid.value, "warps_per_cta": warps.value}


def p2p_batch_destroy(batch):
    if batch:
        load().p2p_batch_destroy(batch)


def p2p_diag_wait_timeout(status, limit, stream=None):
    check(load().p2p_diag_wait_timeout(_ptr(status), int(limit), _stream(stream)), "p2p_diag_wait_timeout")


def p2p_host_pipe_workspace_size(max_n, nrhs) -> int:
    out = ctypes.c_size_t(0)
    check(load().p2p_host_pipe_workspace_size(int(max_n), int(nrhs), ctypes.byref(out)), "p2p_host_pipe_workspace_size")
    return out.value


def p2p_host_pipe_create(max_n, nrhs, workspace):
    pipe = ctypes.c_void_p(0)
    check(load().p2p_host_pipe_create(ctypes.byref(pipe), int(max_n), int(nrhs), _ptr(workspace), workspace.numel()),
          "p2p_host_pipe_create")
    return pipe


def p2p_apply_host(pipe, plans, lams_host, outs_host, stream=None):
    check(load().p2p_apply_host(pipe, _ptr_array(plans), len(plans), _ptr_array(lams_host), _ptr_array(outs_host),
                                _stream(stream)), "p2p_apply_host")


def p2p_host_pipe_destroy(pipe):
    if pipe:
        load().p2p_host_pipe_destroy(pipe)


def p2p_diag_tc_wait_limit(plan, polls: int):
    check(load().p2p_diag_tc_wait_limit(plan, int(polls)), "p2p_diag_tc_wait_limit")


def p2p_apply_guarded_workspace_size(plan, nrhs) -> int:
    out = ctypes.c_size_t(0)
    check(load().p2p_apply_guarded_workspace_size(plan, int(nrhs), ctypes.byref(out)),
          "p2p_apply_guarded_workspace_size")
    return out.value


def p2p_apply_guarded(plan, lam, out, nrhs, ld, adjoint, path, tol, work, stream=None) -> int:
    refined = ctypes.c_int64(0)
    check(load().p2p_apply_guarded(plan, _ptr(lam), _ptr(out), int(nrhs), int(ld), int(adjoint), int(path),
                                   float(tol), _ptr(work), work.numel(), ctypes.byref(refined), _stream(stream)),
          "p2p_apply_guarded")
    return refined.value
