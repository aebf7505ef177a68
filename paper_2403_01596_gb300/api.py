"""Python API of the GB300 P2P library on top of the C ABI.

    plan = Plan(points, lo, h, ng, k, kernel="helmholtz", layout="indexed")
    out = plan.apply(lam)                 # out = A lam   (complex64, original point order)
    gl = plan.apply(g, adjoint=True)      # A^H g
    gx = plan.grad_points(lam, g)         # dL/dx for dL/dout = g
    out = p2p(lam, points, plan)          # autograd-aware: d/dlam and d/dpoints

All device memory is owned by the Plan as torch tensors; the library only
receives raw pointers.  Everything runs on the current CUDA stream.  There is
no CPU fallback: points must be a CUDA tensor and libp2p.so must be loadable.
"""
from __future__ import annotations

import math

import torch

from . import _capi as C

KERNELS = {"helmholtz": C.P2P_HELMHOLTZ, "laplace": C.P2P_LAPLACE}
LAYOUTS = {"indexed": C.P2P_LAYOUT_INDEXED, "redundant": C.P2P_LAYOUT_REDUNDANT,
           "symmetric": C.P2P_LAYOUT_SYMMETRIC, "repetition": C.P2P_LAYOUT_REPETITION}
PATHS = {"auto": C.P2P_PATH_AUTO, "fp32_per_rhs": C.P2P_PATH_FP32_PER_RHS, "fp32_shared": C.P2P_PATH_FP32_SHARED,
         "tc_bf16x3": C.P2P_PATH_TC_BF16X3, "tc_bf16x6": C.P2P_PATH_TC_BF16X6}


def _stream():
    return torch.cuda.current_stream()


def _bytes(n: int, device) -> torch.Tensor:
    # torch's caching allocator returns blocks aligned to at least 512 bytes
    return torch.empty(max(int(n), 1), dtype=torch.uint8, device=device)


class Binning:
    """Leaf binning of one point set (device tensors): perm, point_box, box_keys, box_ptr."""

    def __init__(self, points: torch.Tensor, lo, h: float, ng: int):
        if not points.is_cuda:
            raise RuntimeError("P2P requires CUDA tensors (no CPU path)")
        if points.dtype != torch.float32 or points.dim() != 2 or points.shape[1] != 3:
            raise ValueError("points must be a float32 tensor of shape (n, 3)")
        self.points = points.contiguous()
        self.lo, self.h, self.ng = tuple(float(v) for v in lo), float(h), int(ng)
        n = self.points.shape[0]
        dev = self.points.device
        s = _stream()
        self.perm = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
        self.point_box = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
        keys = torch.empty(max(n, 1), dtype=torch.int64, device=dev)
        ptr = torch.empty(n + 1, dtype=torch.int32, device=dev)
        work = _bytes(C.p2p_bin_workspace_size(n), dev)
        self.num_boxes = C.p2p_bin_points(self.points, self.lo, self.h, self.ng, self.perm, self.point_box, keys, ptr,
                                          work, s)
        del work
        B = self.num_boxes
        self.box_keys = keys[:B].clone() if B else keys[:0]
        self.box_ptr = ptr[:B + 1].clone()
        self.n = n


class BoxStructure(Binning):
    """Leaf binning + neighbour lists of one point set (device tensors)."""

    def __init__(self, points: torch.Tensor, lo, h: float, ng: int):
        super().__init__(points, lo, h, ng)
        dev = self.points.device
        s = _stream()
        B = self.num_boxes
        self.nbr_ptr = torch.empty(B + 1, dtype=torch.int32, device=dev)
        self.nbr_idx = torch.empty(max(27 * B, 1), dtype=torch.int32, device=dev)
        work = _bytes(C.p2p_neighbors_workspace_size(B), dev)
        self.nnz, self.sources = C.p2p_build_neighbors(self.box_keys, self.box_ptr, B, self.ng, self.nbr_ptr,
                                                       self.nbr_idx, work, s)
        del work


class Plan:
    """A P2P operator bound to a point set, kernel, wavenumber and source layout."""

    def __init__(self, points: torch.Tensor, lo, h: float, ng: int, k: float = 0.0, kernel: str = "helmholtz",
                 layout: str = "indexed", max_nrhs: int = 1, tuning: dict | None = None,
                 structure: BoxStructure | None = None):
        self.kernel, self.layout, self.k = kernel, layout, float(k)
        self.max_nrhs = int(max_nrhs)
        self.tuning = tuning
        self._build(structure if structure is not None else BoxStructure(points, lo, h, ng))
        self.rebuilds = 0

    def _build(self, structure: "BoxStructure"):
        self.structure = structure
        st = self.structure
        kernel, layout, tuning = self.kernel, self.layout, self.tuning
        dev = st.points.device
        if layout == "repetition":
            # the paper's per-target records: sum over boxes of n_b (1 + S_b) entries
            self.records = C.p2p_repetition_records(st.box_ptr, st.num_boxes, st.nbr_ptr, st.nbr_idx, _stream())
            ws = C.p2p_plan_workspace_size_rep(st.n, st.num_boxes, st.nnz, st.sources, self.records, tuning)
        else:
            ws = C.p2p_plan_workspace_size(st.n, st.num_boxes, st.nnz, st.sources, LAYOUTS[layout], self.max_nrhs,
                                           tuning)
        self.workspace = _bytes(ws, dev)
        self._plan = C.p2p_plan_create(st.points, st.perm, st.box_ptr, st.num_boxes, st.nbr_ptr, st.nbr_idx, st.nnz,
                                       st.sources, KERNELS[kernel], self.k, LAYOUTS[layout], self.max_nrhs, tuning,
                                       self.workspace, _stream())
        self.info = C.p2p_plan_info(self._plan)
        self._pairs = None
        self._seen = (st.points.data_ptr(), st.points._version)

    # ------------------------------------------------------ moving points --
    def update_points(self, points: torch.Tensor) -> bool:
        """Takes new coordinates for the plan's points (original order).  Returns True when every point stays in
        its leaf box (only the coordinates are gathered again), else rebuilds the box structure and the plan from
        the new coordinates on the same grid and returns False."""
        pts = points.detach().contiguous()
        if pts.shape != self.structure.points.shape or pts.dtype != torch.float32 or not pts.is_cuda:
            raise ValueError("new coordinates must be a float32 CUDA tensor of the plan's shape")
        st = self.structure
        status, _ = C.p2p_plan_update_points(self._plan, pts, st.lo, st.h, st.ng, _stream())
        if status == C.P2P_OK:
            st.points = pts      # the plan reads this array from now on
            self._seen = (pts.data_ptr(), pts._version)
            return True
        self.close()
        self._build(BoxStructure(pts, st.lo, st.h, st.ng))
        self.rebuilds += 1
        return False

    def follow(self, points: torch.Tensor):
        """update_points(points) if `points` is not the array (and version) the plan last took."""
        if (points.data_ptr(), points._version) != self._seen:
            self.update_points(points)

    # ----------------------------------------------------------------- info --
    @property
    def n(self) -> int:
        return self.structure.n

    @property
    def n_src(self) -> int:
        """Rows of the strengths (the sources; the points themselves for a one-set plan)."""
        return self.structure.n

    @property
    def num_boxes(self) -> int:
        return self.structure.num_boxes

    @property
    def device(self):
        return self.workspace.device

    def pair_count(self) -> int:
        if self._pairs is None:
            self._pairs = C.p2p_plan_pair_count(self._plan, _stream())
        return self._pairs

    def async_status(self) -> int:
        return C.p2p_last_async_status(self._plan, _stream())

    # ---------------------------------------------------------------- apply --
    def _check_lam(self, lam: torch.Tensor, rows: int | None = None):
        rows = self.n_src if rows is None else rows
        if not lam.is_cuda or lam.dtype != torch.complex64:
            raise ValueError("strengths must be a complex64 CUDA tensor")
        if lam.shape[0] != rows:
            raise ValueError(f"expected {rows} rows, got {lam.shape[0]}")
        lam2 = lam.reshape(rows, 1) if lam.dim() == 1 else lam
        if lam2.dim() != 2:
            raise ValueError("strengths must have shape (n,) or (n, nrhs)")
        if lam2.stride(1) != 1:
            lam2 = lam2.contiguous()
        return lam2

    def apply(self, lam: torch.Tensor, out: torch.Tensor | None = None, adjoint: bool = False,
              path: str = "auto") -> torch.Tensor:
        lam2 = self._check_lam(lam)
        nrhs = lam2.shape[1]
        if lam2.stride(0) != nrhs:
            lam2 = lam2.contiguous()
        if out is None:
            out = torch.empty_like(lam2)
        C.p2p_apply_path(self._plan, lam2, out, nrhs, nrhs, int(adjoint), PATHS[path], _stream())
        return out.reshape(lam.shape)

    def apply_guarded(self, lam: torch.Tensor, tol: float = 1e-6, adjoint: bool = False, path: str = "auto",
                      out: torch.Tensor | None = None):
        """apply() with every result within relative `tol` of the exact sum: targets whose FP32 error bound
        (2^-20 sum_j |G lambda_j|) exceeds tol |out| are re-evaluated in FP64 on the GPU.  Returns (out, number
        of targets re-evaluated)."""
        lam2 = self._check_lam(lam).contiguous()
        nrhs = lam2.shape[1]
        if out is None:
            out = torch.empty((self.n, nrhs), dtype=torch.complex64, device=lam.device)
        work = _bytes(C.p2p_apply_guarded_workspace_size(self._plan, nrhs), lam.device)
        refined = C.p2p_apply_guarded(self._plan, lam2, out, nrhs, nrhs, int(adjoint), PATHS[path], tol, work,
                                      _stream())
        return (out.reshape(self.n) if lam.dim() == 1 else out), refined

    def grad_points(self, lam: torch.Tensor, g: torch.Tensor) -> torch.Tensor:
        lam2 = self._check_lam(lam).contiguous()
        g2 = self._check_lam(g).contiguous()
        grad = torch.empty((self.n, 3), dtype=torch.float32, device=lam.device)
        C.p2p_grad_points(self._plan, lam2, g2, grad, lam2.shape[1], lam2.shape[1], _stream())
        return grad

    def close(self):
        if getattr(self, "_plan", None):
            C.p2p_plan_destroy(self._plan)
            self._plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class TwoSetStructure:
    """Binnings of a target set and a source set on one grid, and the target-box -> source-box neighbour lists
    (with the position of each target box's own-cell source box, nbr_self)."""

    def __init__(self, targets: torch.Tensor, sources: torch.Tensor, lo, h: float, ng: int,
                 tgt: Binning | None = None, src: Binning | None = None):
        self.tgt = tgt if tgt is not None else Binning(targets, lo, h, ng)
        self.src = src if src is not None else Binning(sources, lo, h, ng)
        t, sb = self.tgt, self.src
        dev = t.points.device
        B = t.num_boxes
        self.nbr_ptr = torch.empty(B + 1, dtype=torch.int32, device=dev)
        self.nbr_idx = torch.empty(max(27 * B, 1), dtype=torch.int32, device=dev)
        self.nbr_self = torch.empty(max(B, 1), dtype=torch.int32, device=dev)
        work = _bytes(C.p2p_neighbors_workspace_size(B), dev)
        self.nnz, self.sources = C.p2p_build_neighbors_st(t.box_keys, B, sb.box_keys, sb.box_ptr, sb.num_boxes,
                                                          t.ng, self.nbr_ptr, self.nbr_idx, self.nbr_self, work,
                                                          _stream())
        del work

    def exchanged(self) -> "TwoSetStructure":
        """The same two binnings with the roles of targets and sources exchanged."""
        return TwoSetStructure(self.src.points, self.tgt.points, self.tgt.lo, self.tgt.h, self.tgt.ng,
                               tgt=self.src, src=self.tgt)


class TwoSetPlan(Plan):
    """out (n_tgt rows) = A lam (n_src rows): the near field from a source point set to a separate target point
    set binned on the same grid.  plan.apply(lam), plan.adjoint_plan().apply(g, adjoint=True) = A^H g."""

    def __init__(self, targets: torch.Tensor, sources: torch.Tensor, lo, h: float, ng: int, k: float = 0.0,
                 kernel: str = "helmholtz", layout: str = "indexed", max_nrhs: int = 1, tuning: dict | None = None,
                 structure: TwoSetStructure | None = None):
        self.structure = structure if structure is not None else TwoSetStructure(targets, sources, lo, h, ng)
        st = self.structure
        t, sb = st.tgt, st.src
        self.kernel, self.layout, self.k = kernel, layout, float(k)
        self.max_nrhs = int(max_nrhs)
        self.tuning = tuning
        ws = C.p2p_plan_workspace_size_st(t.n, t.num_boxes, sb.n, sb.num_boxes, st.nnz, st.sources,
                                          LAYOUTS[layout], self.max_nrhs, tuning)
        self.workspace = _bytes(ws, t.points.device)
        self._plan = C.p2p_plan_create_st(t.points, t.perm, t.box_ptr, t.num_boxes, sb.points, sb.perm, sb.box_ptr,
                                          sb.num_boxes, st.nbr_ptr, st.nbr_idx, st.nbr_self, st.nnz, st.sources,
                                          KERNELS[kernel], self.k, LAYOUTS[layout], self.max_nrhs, tuning,
                                          self.workspace, _stream())
        self.info = C.p2p_plan_info(self._plan)
        self._pairs = None

    @property
    def n(self) -> int:
        return self.structure.tgt.n

    @property
    def n_src(self) -> int:
        return self.structure.src.n

    @property
    def num_boxes(self) -> int:
        return self.structure.tgt.num_boxes

    def apply(self, lam: torch.Tensor, out: torch.Tensor | None = None, adjoint: bool = False,
              path: str = "auto") -> torch.Tensor:
        """A lam (adjoint=True: conj(A) lam, which is the adjoint of the plan with the sets exchanged)."""
        lam2 = self._check_lam(lam).contiguous()
        nrhs = lam2.shape[1]
        if out is None:
            out = torch.empty((self.n, nrhs), dtype=torch.complex64, device=lam.device)
        C.p2p_apply_path(self._plan, lam2, out, nrhs, nrhs, int(adjoint), PATHS[path], _stream())
        return out.reshape(self.n) if lam.dim() == 1 else out

    def adjoint_plan(self) -> "TwoSetPlan":
        """The plan with targets and sources exchanged; its apply(g, adjoint=True) is A^H g."""
        st = self.structure.exchanged()
        return TwoSetPlan(st.tgt.points, st.src.points, st.tgt.lo, st.tgt.h, st.tgt.ng, self.k, self.kernel,
                          self.layout, self.max_nrhs, self.tuning, structure=st)

    def grad_points(self, lam, g):
        raise NotImplementedError("coordinate gradients are provided for one-set plans")


class Batch:
    """Several plans applied in one persistent launch (optionally replayed from a CUDA graph)."""

    def __init__(self, plans, nrhs: int = 1, warps_per_cta: int = 0):
        self.plans = list(plans)
        self.nrhs = int(nrhs)
        handles = [p._plan for p in self.plans]
        dev = self.plans[0].device
        self.workspace = _bytes(C.p2p_batch_workspace_size(handles, self.nrhs), dev)
        self._b = C.p2p_batch_create(handles, self.nrhs, warps_per_cta, self.workspace, _stream())
        self.info = C.p2p_batch_info(self._b)
        self._graph_buffers = None

    def _views(self, lams, outs):
        if len(lams) != len(self.plans):
            raise ValueError("one strength tensor per plan is required")
        lam2 = [p._check_lam(l).contiguous() for p, l in zip(self.plans, lams)]
        for l in lam2:
            if l.shape[1] != self.nrhs:
                raise ValueError(f"expected {self.nrhs} right-hand sides")
        if outs is None:
            outs = [torch.empty((p.n, self.nrhs), dtype=torch.complex64, device=l.device)
                    for p, l in zip(self.plans, lam2)]
        outs2 = [o.reshape(p.n, self.nrhs) for o, p in zip(outs, self.plans)]
        return lam2, outs2

    def apply(self, lams, outs=None):
        lam2, outs2 = self._views(lams, outs)
        C.p2p_batch_apply(self._b, lam2, outs2, self.nrhs, _stream())
        return outs2

    def capture(self, lams, outs=None):
        """Captures one batched apply on these buffers into a CUDA graph; returns the outputs."""
        lam2, outs2 = self._views(lams, outs)
        C.p2p_batch_graph_create(self._b, lam2, outs2, self.nrhs)
        self._graph_buffers = (lam2, outs2)
        return outs2

    def replay(self):
        if self._graph_buffers is None:
            raise RuntimeError("capture() first")
        C.p2p_batch_graph_launch(self._b, _stream())
        return self._graph_buffers[1]

    def close(self):
        if getattr(self, "_b", None):
            C.p2p_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class HostPipe:
    """Applies a sequence of plans to strengths held in (page-locked) host memory and writes the results back
    to host memory; uploads and downloads of neighbouring plans overlap each plan's kernels."""

    def __init__(self, max_n: int, nrhs: int = 1, device=None):
        self.max_n = int(max_n)
        self.nrhs = int(nrhs)
        dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.workspace = _bytes(C.p2p_host_pipe_workspace_size(self.max_n, self.nrhs), dev)
        self._p = C.p2p_host_pipe_create(self.max_n, self.nrhs, self.workspace)

    def apply(self, plans, lams_host, outs_host=None):
        """lams_host[g]: plan g's (n_g,) or (n_g, nrhs) complex64 CPU tensor; returns the CPU results, complete
        once the current stream has reached this call's end."""
        if len(lams_host) != len(plans):
            raise ValueError("one strength tensor per plan is required")
        lam2 = []
        for p, l in zip(plans, lams_host):
            if l.device.type != "cpu" or l.dtype != torch.complex64 or not l.is_contiguous():
                raise ValueError("host strengths must be contiguous complex64 CPU tensors")
            if l.numel() != p.n_src * self.nrhs:
                raise ValueError(f"expected {p.n_src} x {self.nrhs} strengths")
            lam2.append(l)
        if outs_host is None:
            outs_host = [torch.empty(p.n * self.nrhs, dtype=torch.complex64, pin_memory=True) for p in plans]
        for o, p in zip(outs_host, plans):
            if (o.device.type != "cpu" or o.dtype != torch.complex64 or not o.is_contiguous()
                    or o.numel() != p.n * self.nrhs):
                raise ValueError("host results must be contiguous complex64 CPU tensors of n x nrhs elements")
        C.p2p_apply_host(self._p, [p._plan for p in plans], lam2, outs_host, _stream())
        return outs_host

    def close(self):
        if getattr(self, "_p", None):
            C.p2p_host_pipe_destroy(self._p)
            self._p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def choose_grid_ct(points: torch.Tensor, lo, extent: float, ct: int, ng_start: int = 1,
                   ng_max: int = 1 << 21) -> BoxStructure:
    """Leaf grid by clustering threshold (Sec. 3.1): raise the tree level, doubling
    the boxes per axis, until no leaf box holds more than `ct` points."""
    ng = max(1, int(ng_start))
    while True:
        st = BoxStructure(points, lo, float(extent) / ng, ng)
        occ = int((st.box_ptr[1:] - st.box_ptr[:-1]).max().item()) if st.num_boxes else 0
        if occ <= ct or ng * 2 > ng_max:
            st.max_occupancy = occ
            return st
        ng *= 2


class P2PFunction(torch.autograd.Function):
    """out = A(x) lam with gradients for lam (A^H g) and for x (radial-derivative kernel).

    The plan follows the coordinates it is given: when `points` is not the
    array (or version of it) the plan last took, the plan takes the new
    coordinates (p2p_plan_update_points) or, when a point has left its leaf
    box, is rebuilt from them on the same grid.  A coordinate gradient is the
    derivative with box membership held fixed (a perturbation that moves no
    point across a box face).
    """

    @staticmethod
    def forward(ctx, lam, points, plan: Plan):
        plan.follow(points)
        ctx.plan = plan
        ctx.save_for_backward(lam)
        return plan.apply(lam)

    @staticmethod
    def backward(ctx, g):
        (lam,) = ctx.saved_tensors
        plan: Plan = ctx.plan
        g = g.contiguous()
        glam = plan.apply(g, adjoint=True) if ctx.needs_input_grad[0] else None
        gx = plan.grad_points(lam, g) if ctx.needs_input_grad[1] else None
        return glam, gx, None


def p2p(lam: torch.Tensor, points: torch.Tensor, plan: Plan) -> torch.Tensor:
    """Autograd entry: the plan must have been built from `points`."""
    return P2PFunction.apply(lam, points, plan)


def inv4pi() -> float:
    return 1.0 / (4.0 * math.pi)
