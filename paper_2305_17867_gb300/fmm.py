"""User API of the GB300 compressed-Taylor FMM.

``FMM`` wraps one C-ABI plan (``include/ctfmm.h``) and a device workspace
taken from the PyTorch caching allocator; ``fmm_potential`` is the autograd
entry point (a ``torch.autograd.Function`` whose backward calls
``fmm_eval_backward``).  Every arithmetic step runs in the CUDA library;
this module only moves tensors and pointers.
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib
from ._lib import KERNELS, M2L_PATHS, PRECISIONS, PlanDesc, Pde, check


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


class FMM:
    """A compressed-Taylor FMM plan on a uniform tree.

    kernel     "laplace" (d = 2, 3), "yukawa" (d = 3), "biharmonic" (d = 3),
               "helmholtz" (d = 3, uniform trees; lam = kappa; complex potentials)
    p          expansion order;  levels: leaf depth L of the uniform tree, or
               -D for an adaptive tree (3D, fp64 or fp32) refined to at most level D,
               splitting boxes that hold more than ``max_leaf`` points
    root_lo, root_size  root box; root_size <= 0 picks the bounding cube per call
    precision  "fp64" | "fp32" | "tf32" | "tf32x3" | "bf16x3" | "f16x3"
    m2l        "dense" (eq. (m2l_toeplitz) as dense products) | "fft" (its
               convolution form, eq. (convolution_m2l); fp64 and fp32 only) |
               "auto" (fft for fp64/fp32, dense tensor cores otherwise)
    pde        optional (multi_idx [n,d] ints, coeff [n] floats) overriding the
               kernel's own PDE (eq. (define_pde_op))
    """

    def __init__(self, kernel: str = "laplace", d: int = 3, p: int = 10, levels: int = 5,
                 lam: float = 0.0, root_lo=None, root_size: float = 1.0,
                 precision: str = "fp64", pde=None, device=None, m2l: str = "dense",
                 max_leaf: int = 64):
        self.L = _lib.load()
        self.kernel, self.d, self.p, self.levels, self.lam = kernel, d, p, levels, lam
        self.precision = precision
        self.m2l = m2l
        self.device = torch.device("cuda" if device is None else device)
        desc = PlanDesc()
        desc.kernel = KERNELS[kernel]
        desc.lam = float(lam)
        desc.d, desc.p, desc.levels = d, p, levels
        lo = [0.0, 0.0, 0.0] if root_lo is None else list(root_lo) + [0.0] * (3 - len(root_lo))
        desc.root_lo = (ctypes.c_double * 3)(*lo)
        desc.root_size = float(root_size)
        desc.precision = PRECISIONS[precision]
        desc.m2l = M2L_PATHS[m2l]
        desc.max_leaf = int(max_leaf)
        self._pde_keep = None
        if pde is not None:
            mi, co = pde
            mi_a = (ctypes.c_int * (len(co) * d))(*[int(v) for row in mi for v in row])
            co_a = (ctypes.c_double * len(co))(*[float(v) for v in co])
            pd = Pde(len(co), ctypes.cast(mi_a, ctypes.POINTER(ctypes.c_int)),
                     ctypes.cast(co_a, ctypes.POINTER(ctypes.c_double)))
            self._pde_keep = (mi_a, co_a, pd)
            desc.pde = ctypes.pointer(pd)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            check(self.L.fmm_plan_create(ctypes.byref(h), ctypes.byref(desc)), "fmm_plan_create")
        self._h = h
        nf, nj, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        check(self.L.fmm_plan_info(h, ctypes.byref(nf), ctypes.byref(nj), ctypes.byref(c)),
              "fmm_plan_info")
        self.nfull, self.nj, self.c = nf.value, nj.value, c.value
        self._ws = None

    def close(self):
        if getattr(self, "_h", None):
            self.L.fmm_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- workspace -------------------------------------------------------
    def workspace_bytes(self, n_src: int, n_tgt: int) -> int:
        b = ctypes.c_size_t()
        check(self.L.fmm_workspace_size(self._h, n_src, n_tgt, ctypes.byref(b)),
              "fmm_workspace_size")
        return b.value

    def _workspace(self, n_src: int, n_tgt: int):
        need = self.workspace_bytes(n_src, n_tgt)
        if self._ws is None or self._ws.numel() < need:
            self._ws = torch.empty(need + 256, dtype=torch.uint8, device=self.device)
        base = self._ws.data_ptr()
        aligned = (base + 255) // 256 * 256
        return ctypes.c_void_p(aligned), self._ws.numel() - (aligned - base)

    def set_timing(self, on: bool = True):
        check(self.L.fmm_set_timing(self._h, int(on)), "fmm_set_timing")

    def phase_times(self) -> dict:
        out = (ctypes.c_float * _lib.NUM_PHASES)()
        check(self.L.fmm_phase_times(self._h, out), "fmm_phase_times")
        return dict(zip(_lib.PHASES, list(out)))

    def m2l_kernel_time(self) -> float:
        """Milliseconds of the M2L contraction launch(es) of the last timed evaluation."""
        out = ctypes.c_float()
        check(self.L.fmm_m2l_kernel_time(self._h, ctypes.byref(out)), "fmm_m2l_kernel_time")
        return float(out.value)

    def last_stats(self) -> dict:
        """fmm_last_stats: phase times, tree, M2L count, near-field pairs, status."""
        st = _lib.Stats()
        check(self.L.fmm_last_stats(self._h, ctypes.byref(st)), "fmm_last_stats")
        return {"phase_ms": dict(zip(_lib.PHASES, list(st.phase_ms))),
                "m2l_kernel_ms": st.m2l_kernel_ms, "boxes": st.boxes, "depth": st.depth,
                "m2l_translations": st.m2l_translations, "p2p_pairs": st.p2p_pairs,
                "status": st.status, "launches": st.launches}

    def last_status(self) -> int:
        return self.L.fmm_last_status(self._h)

    def last_tree(self):
        """(boxes, deepest level) of the last evaluation's tree."""
        nb, dp = ctypes.c_int64(), ctypes.c_int()
        check(self.L.fmm_last_tree(self._h, ctypes.byref(nb), ctypes.byref(dp), None),
              "fmm_last_tree")
        return nb.value, dp.value

    def last_m2l_count(self) -> int:
        """M2L translations of the last evaluation (uniform: exact count of the lists)."""
        n = ctypes.c_int64()
        check(self.L.fmm_last_tree(self._h, None, None, ctypes.byref(n)), "fmm_last_tree")
        return n.value

    def last_launch_count(self) -> int:
        return self.L.fmm_last_launch_count(self._h)

    # ---- evaluation --------------------------------------------------------
    def _dev(self, t, shape_last=None):
        t = t.to(device=self.device, dtype=torch.float64, non_blocking=True)
        return t.contiguous()

    def eval(self, src, w, tgt=None, grad: bool = False, check_status: bool = False):
        """phi(tgt) (and grad phi) for sources ``src`` [n, d] with weights ``w`` [n].

        Accepts device or host tensors; host inputs are copied in and the
        results copied back to the host (the end-to-end path)."""
        host = not src.is_cuda
        s = self._dev(src)
        wd = self._dev(w)
        t = s if tgt is None else (s if tgt is src else self._dev(tgt))
        ns, nt = s.shape[0], t.shape[0]
        cplx = self.kernel == "helmholtz"  # complex phi: (re, im) pairs
        phi = torch.empty((nt, 2) if cplx else (nt,), dtype=torch.float64, device=self.device)
        g = (torch.empty((nt, self.d, 2) if cplx else (nt, self.d), dtype=torch.float64,
                         device=self.device) if grad else None)
        ws, wb = self._workspace(ns, nt)
        stream = torch.cuda.current_stream(self.device).cuda_stream
        check(self.L.fmm_eval(self._h, ns, _ptr(s), _ptr(wd), nt, _ptr(t), _ptr(phi), _ptr(g),
                              ws, wb, ctypes.c_void_p(stream)), "fmm_eval")
        if check_status:
            check(self.last_status(), "fmm_eval (device status)")
        if cplx:
            phi = torch.view_as_complex(phi)
            g = torch.view_as_complex(g) if g is not None else None
        if host:
            phi = phi.cpu()
            g = g.cpu() if g is not None else None
        return (phi, g) if grad else phi

    def eval_f32(self, src, w, tgt=None, grad: bool = False, check_status: bool = False):
        """fmm_eval_f32: float32 device tensors in and out (widened to float64 on
        the device for the evaluation, results rounded to float32)."""
        s = src.to(device=self.device, dtype=torch.float32).contiguous()
        wd = w.to(device=self.device, dtype=torch.float32).contiguous()
        t = s if tgt is None else tgt.to(device=self.device, dtype=torch.float32).contiguous()
        ns, nt = s.shape[0], t.shape[0]
        cplx = self.kernel == "helmholtz"
        phi = torch.empty((nt, 2) if cplx else (nt,), dtype=torch.float32, device=self.device)
        g = (torch.empty((nt, self.d, 2) if cplx else (nt, self.d), dtype=torch.float32,
                         device=self.device) if grad else None)
        b = ctypes.c_size_t()
        check(self.L.fmm_workspace_size_f32(self._h, ns, nt, ctypes.byref(b)),
              "fmm_workspace_size_f32")
        if self._ws is None or self._ws.numel() < b.value + 256:
            self._ws = torch.empty(b.value + 256, dtype=torch.uint8, device=self.device)
        base = self._ws.data_ptr()
        aligned = (base + 255) // 256 * 256
        stream = torch.cuda.current_stream(self.device).cuda_stream
        check(self.L.fmm_eval_f32(self._h, ns, _ptr(s), _ptr(wd), nt, _ptr(t), _ptr(phi),
                                  _ptr(g), ctypes.c_void_p(aligned),
                                  self._ws.numel() - (aligned - base), ctypes.c_void_p(stream)),
              "fmm_eval_f32")
        if check_status:
            check(self.last_status(), "fmm_eval_f32 (device status)")
        if cplx:
            phi = torch.view_as_complex(phi)
            g = torch.view_as_complex(g) if g is not None else None
        return (phi, g) if grad else phi

    def backward(self, src, w, tgt, u, need_w=True, need_src=True, need_tgt=True,
                 grad_phi=None):
        """Gradients of sum(u * phi); grad_phi (grad phi at tgt from a forward
        eval with grad=True) saves the second FMM for the target gradient."""
        s, wd, t, ud = self._dev(src), self._dev(w), self._dev(tgt), self._dev(u)
        gp = None if grad_phi is None else self._dev(grad_phi)
        ns, nt = s.shape[0], t.shape[0]
        gw = torch.empty(ns, dtype=torch.float64, device=self.device) if need_w else None
        gs = torch.empty(ns, self.d, dtype=torch.float64, device=self.device) if need_src else None
        gt = torch.empty(nt, self.d, dtype=torch.float64, device=self.device) if need_tgt else None
        n = max(ns, nt)
        ws, wb = self._workspace(n, n)
        stream = torch.cuda.current_stream(self.device).cuda_stream
        check(self.L.fmm_eval_backward(self._h, ns, _ptr(s), _ptr(wd), nt, _ptr(t), _ptr(ud),
                                       _ptr(gp), _ptr(gw), _ptr(gs), _ptr(gt), ws, wb,
                                       ctypes.c_void_p(stream)), "fmm_eval_backward")
        return gw, gs, gt


class _FMMFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, plan, src, w, tgt):
        # when the targets need a gradient, grad phi comes with phi in the
        # same evaluation and the backward needs only the transposed FMM
        if ctx.needs_input_grad[3]:
            phi, gphi = plan.eval(src, w, tgt, grad=True)
        else:
            phi, gphi = plan.eval(src, w, tgt), None
        ctx.plan = plan
        ctx.gphi = gphi
        ctx.save_for_backward(src, w, tgt)
        return phi.to(src.dtype)

    @staticmethod
    def backward(ctx, gphi):
        src, w, tgt = ctx.saved_tensors
        plan = ctx.plan
        _, ns, nw, nt = ctx.needs_input_grad
        gw, gs, gt = plan.backward(src, w, tgt, gphi, need_w=bool(nw), need_src=bool(ns),
                                   need_tgt=bool(nt), grad_phi=ctx.gphi)
        ctx.gphi = None
        cast = lambda g, ref: None if g is None else g.to(ref.dtype)
        return None, cast(gs, src), cast(gw, w), cast(gt, tgt)


def fmm_potential(plan: FMM, src, w, tgt):
    """phi = FMM(src, w) at tgt, differentiable w.r.t. src, w and tgt."""
    return _FMMFunction.apply(plan, src, w, tgt)
