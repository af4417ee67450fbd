"""Python API over the C ABI: a grid object, the forward and backward traces, the
neutral-fraction update and a ``torch.autograd.Function``.

PyTorch supplies device memory and streams; every step of the trace runs in the CUDA
library. Tensors handed to the library must be contiguous float32 CUDA tensors on the
grid's device; the library borrows them for the duration noted in ``include/art.h``.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib as C


@dataclass
class Params:
    """Trace parameters (Sec. 2.1 / 2.3 of Kim et al. 2017); see ``art_params`` in art.h."""

    level0: int = 4
    level_max: int = -1
    m_ray: float = 4.0
    tau_max: float = 7.0
    sigma_H: float = 1.0
    sigma_d: float = 0.0
    rot: np.ndarray | None = None
    schedule: str = "persistent"          # or "plain"
    block_threads: int = 0
    chunk: int = 0
    queue_capacity: int = 0
    wait_limit_s: float = 0.0
    blocks_per_sm: int = 0
    d_max: float = 0.0                    # > 0: rays end this far from their source (Sec. 3.1)

    def to_c(self) -> C.ArtParams:
        p = C.ArtParams()
        C.lib().art_params_default(ctypes.byref(p))
        p.level0 = int(self.level0)
        p.level_max = int(self.level_max)
        p.m_ray = float(self.m_ray)
        p.tau_max = float(self.tau_max)
        p.sigma_H = float(self.sigma_H)
        p.sigma_d = float(self.sigma_d)
        if self.rot is not None:
            r = np.asarray(self.rot, dtype=np.float64).reshape(9)
            for i in range(9):
                p.rot[i] = float(r[i])
            p.flags |= C.ART_F_ROTATE
        p.schedule = {"persistent": C.ART_SCHED_PERSISTENT, "plain": C.ART_SCHED_PLAIN}[self.schedule]
        p.block_threads = int(self.block_threads)
        p.chunk = int(self.chunk)
        p.queue_capacity = int(self.queue_capacity)
        p.wait_limit_s = float(self.wait_limit_s)
        p.blocks_per_sm = int(self.blocks_per_sm)
        p.d_max = float(self.d_max)
        return p


def _dev_ptr(t: torch.Tensor | None, what: str):
    if t is None:
        return None
    if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise ValueError(f"{what} must be a contiguous float32 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


class Grid:
    """A uniform grid with its density fields and point sources (library-owned state).

    ``nH0`` (and ``nH``) are CUDA float32 tensors of shape (nz, ny, nx); they are borrowed,
    and read again by every trace.
    """

    def __init__(self, nH0: torch.Tensor, dx: float, lo=(0.0, 0.0, 0.0),
                 nH: torch.Tensor | None = None, stream: torch.cuda.Stream | None = None):
        if nH0.dim() != 3:
            raise ValueError("nH0 must have shape (nz, ny, nx)")
        self.shape = tuple(nH0.shape)
        self.device = nH0.device
        self.dx = float(dx)
        self.lo = tuple(float(v) for v in lo)
        self.stream = stream if stream is not None else torch.cuda.current_stream(nH0.device)
        self._nH0, self._nH = nH0, nH
        self._h = ctypes.c_void_p()
        lo_arr = (ctypes.c_double * 3)(*self.lo)
        nz, ny, nx = self.shape
        with torch.cuda.device(self.device):
            C.check(C.lib().art_create_grid(ctypes.byref(self._h), nx, ny, nz, lo_arr, self.dx,
                                            _dev_ptr(nH0, "nH0"), _dev_ptr(nH, "nH"),
                                            ctypes.c_void_p(self.stream.cuda_stream)),
                    "art_create_grid")
        self.nsrc = 0

    @property
    def ncell(self) -> int:
        return self.shape[0] * self.shape[1] * self.shape[2]

    def close(self):
        if self._h:
            C.lib().art_destroy_grid(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def update_fields(self, nH0: torch.Tensor, nH: torch.Tensor | None = None):
        C.check(C.lib().art_update_fields(self._h, _dev_ptr(nH0, "nH0"), _dev_ptr(nH, "nH")),
                "art_update_fields")
        self._nH0, self._nH = nH0, nH

    def add_sources(self, pos, L):
        pos = np.ascontiguousarray(np.asarray(pos, dtype=np.float64).reshape(-1, 3))
        L = np.ascontiguousarray(np.asarray(L, dtype=np.float64).reshape(-1))
        if len(pos) != len(L):
            raise ValueError("pos and L differ in length")
        P = ctypes.POINTER(ctypes.c_double)
        C.check(C.lib().art_add_sources(self._h, len(L), pos.ctypes.data_as(P),
                                        L.ctypes.data_as(P)), "art_add_sources")
        self.nsrc += len(L)

    def set_nonionizing(self, Ln):
        """Second, non-ionizing frequency bin per source (dust-attenuated); None removes it."""
        if Ln is None:
            C.check(C.lib().art_set_nonionizing(self._h, None), "art_set_nonionizing")
            return
        Ln = np.ascontiguousarray(np.asarray(Ln, dtype=np.float64).reshape(-1))
        if len(Ln) != self.nsrc:
            raise ValueError("one non-ionizing luminosity per source")
        C.check(C.lib().art_set_nonionizing(self._h, Ln.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
                "art_set_nonionizing")

    def clear_sources(self):
        C.check(C.lib().art_clear_sources(self._h), "art_clear_sources")
        self.nsrc = 0

    def trace(self, params: Params, force: bool = True, energy: bool = False,
              stats: bool = True, out: dict | None = None) -> dict:
        """One full trace. Returns gamma (nz,ny,nx), force (3,nz,ny,nx) or None, energy or
        None, and the counters (a dict) when ``stats`` (which synchronizes)."""
        nz, ny, nx = self.shape
        o = out or {}
        g = o.get("gamma")
        if g is None:
            g = torch.empty(self.shape, device=self.device, dtype=torch.float32)
        f = o.get("force")
        if force and f is None:
            f = torch.empty((3, nz, ny, nx), device=self.device, dtype=torch.float32)
        e = o.get("energy")
        if energy and e is None:
            e = torch.empty(self.shape, device=self.device, dtype=torch.float32)
        st = C.ArtStats()
        cp = params.to_c()
        rc = C.lib().art_trace(self._h, ctypes.byref(cp), _dev_ptr(g, "gamma"),
                               _dev_ptr(f if force else None, "force"),
                               _dev_ptr(e if energy else None, "energy"),
                               ctypes.byref(st) if stats else None)
        C.check(rc, "art_trace")
        return {"gamma": g, "force": f if force else None, "energy": e if energy else None,
                "stats": st.as_dict() if stats else None}

    def estimate_work(self, params: Params) -> np.ndarray:
        """Per-source estimate of a trace's crossings (float64, one per source), for
        balancing a trace split over several GPUs; synchronizes."""
        work = np.zeros(self.nsrc, dtype=np.float64)
        cp = params.to_c()
        C.check(C.lib().art_estimate_work(self._h, ctypes.byref(cp),
                                          work.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
                "art_estimate_work")
        return work

    def stats(self) -> dict:
        st = C.ArtStats()
        C.check(C.lib().art_get_stats(self._h, ctypes.byref(st)), "art_get_stats")
        return st.as_dict()

    def trace_backward(self, params: Params, w: torch.Tensor | None, stats: bool = True,
                       v: torch.Tensor | None = None):
        """Gradient of sum(w * gamma) + sum(v * force) w.r.t. log n_H0 (per cell) and L (per
        source). w: (nz, ny, nx) or None; v: (3, nz, ny, nx) or None; not both None."""
        grad = torch.empty(self.shape, device=self.device, dtype=torch.float32)
        dL = torch.empty(self.nsrc, device=self.device, dtype=torch.float64)
        st = C.ArtStats()
        cp = params.to_c()
        wc = None if w is None else w.float().contiguous()
        vc = None if v is None else v.float().contiguous()
        rc = C.lib().art_trace_backward(self._h, ctypes.byref(cp), _dev_ptr(wc, "w"),
                                        _dev_ptr(vc, "v"), _dev_ptr(grad, "grad"),
                                        ctypes.c_void_p(dL.data_ptr()),
                                        ctypes.byref(st) if stats else None)
        C.check(rc, "art_trace_backward")
        return grad, dL, (st.as_dict() if stats else None)


def xn_update(gamma: torch.Tensor, nH: torch.Tensor, xn: torch.Tensor, alpha_B: float,
              dt: float, nH0_out: torch.Tensor | None = None, method: str = "b",
              stream: torch.cuda.Stream | None = None):
    """In-place neutral-fraction update of ``xn`` (Eq. e:xn3 for "b", Eq. e:xn2 for "a")."""
    s = stream if stream is not None else torch.cuda.current_stream(xn.device)
    rc = C.lib().art_xn_update(ctypes.c_void_p(s.cuda_stream), xn.numel(),
                               _dev_ptr(gamma, "gamma"), _dev_ptr(nH, "nH"), _dev_ptr(xn, "xn"),
                               _dev_ptr(nH0_out, "nH0"), float(alpha_B), float(dt),
                               {"b": 0, "a": 1}[method])
    C.check(rc, "art_xn_update")


def dt_substep(gamma: torch.Tensor, nH: torch.Tensor, xn: torch.Tensor, alpha_B: float,
               C_coef: float = 0.1, stream: torch.cuda.Stream | None = None) -> torch.Tensor:
    """Eq. e:dtss as a 1-element float64 CUDA tensor (no host synchronization)."""
    s = stream if stream is not None else torch.cuda.current_stream(xn.device)
    nbytes = C.lib().art_dt_scratch_bytes(xn.numel())
    scratch = torch.empty(int(nbytes), device=xn.device, dtype=torch.uint8)
    out = torch.empty(1, device=xn.device, dtype=torch.float64)
    rc = C.lib().art_dt_substep(ctypes.c_void_p(s.cuda_stream), xn.numel(), _dev_ptr(gamma, "gamma"),
                                _dev_ptr(nH, "nH"), _dev_ptr(xn, "xn"), float(alpha_B),
                                float(C_coef), ctypes.c_void_p(scratch.data_ptr()),
                                ctypes.c_void_p(out.data_ptr()))
    C.check(rc, "art_dt_substep")
    return out


class ARTFunction(torch.autograd.Function):
    """gamma = ART(log n_H0, L), or (gamma, force) with ``with_force``: forward trace,
    hand-written adjoint in ``backward``.

    Inputs: log_nH0 (nz,ny,nx) float32 CUDA, L (n_src,) float64 (any device); ``grid`` is a
    Grid (its total-density field, if any, is kept for the dust term); ``positions`` the
    (n_src, 3) source positions; ``params`` the trace parameters. gamma and force carry
    gradients. The grid is shared state: ``forward`` points it at this call's neutral
    density and sources, and ``backward`` points it back at them before the reverse sweep,
    so other traces of the same grid between the two calls do not change the gradient.
    """

    @staticmethod
    def forward(ctx, log_nH0: torch.Tensor, L: torch.Tensor, grid: Grid, params: Params,
                positions, with_force: bool = False):
        nH0 = torch.exp(log_nH0.detach()).contiguous()
        nH = grid._nH
        pos = np.array(positions, dtype=np.float64).reshape(-1, 3)
        Lh = L.detach().double().cpu().numpy().copy()
        grid.update_fields(nH0, nH)
        grid.clear_sources()
        grid.add_sources(pos, Lh)
        out = grid.trace(params, force=with_force, stats=False)
        ctx.grid, ctx.params, ctx.nH0, ctx.nH = grid, params, nH0, nH
        ctx.pos, ctx.L = pos, Lh
        ctx.L_device = L.device
        ctx.with_force = with_force
        if with_force:
            return out["gamma"], out["force"]
        return out["gamma"]

    @staticmethod
    def backward(ctx, dgamma: torch.Tensor, dforce: torch.Tensor | None = None):
        if dgamma is None and dforce is None:
            return None, None, None, None, None, None
        grid = ctx.grid
        grid.update_fields(ctx.nH0, ctx.nH)
        grid.clear_sources()
        grid.add_sources(ctx.pos, ctx.L)
        grad, dL, _ = grid.trace_backward(ctx.params, dgamma, stats=False, v=dforce)
        return grad, dL.to(ctx.L_device), None, None, None, None
