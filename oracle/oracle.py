"""ctypes wrapper of the FP64 CPU oracle (``art_oracle.c``) plus the photochemistry closed forms.

TEST INFRASTRUCTURE ONLY: the test suite, the package smoke check and the bench's
CPU-baseline leg use this module; the library never imports it. It shares no code with the
CUDA path.

The ray-tracing part follows Sec. 2.1 of Kim, Kim, Ostriker & Skinner (2017); the
neutral-fraction updates follow Sec. 2.3 (Eqs. e:xn, e:xn2, e:xn3, e:dtss and the
Gamma = 0 solution) and the one-cell scheme of the Appendix (Eq. e:bdf1).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "art_oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
NLEVELS = 20

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, no fused multiply-add contraction, OpenMP)."""
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        os.makedirs(os.path.dirname(_OUT), exist_ok=True)
        tmp = _OUT + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _OUT)
    return _OUT


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        dp, fp, lp = P(ctypes.c_double), P(ctypes.c_float), P(ctypes.c_longlong)
        i, d = ctypes.c_int, ctypes.c_double
        lib.or_pix2vec.argtypes = [i, ctypes.c_uint64, dp]
        lib.or_pix2vec.restype = None
        lib.or_vec2pix.argtypes = [i, dp]
        lib.or_vec2pix.restype = ctypes.c_uint64
        lib.or_trace.argtypes = [i, i, i, dp, d, fp, fp, i, dp, dp, dp, i, i, d, d, d, d, dp,
                                 d, dp, dp, lp, i, i, lp]
        lib.or_trace.restype = i
        lib.or_ray_segments.argtypes = [i, i, i, dp, d, fp, fp, dp, i, i, d, d, d, d, dp, d,
                                        i, ctypes.c_ulonglong, d, d, lp, dp, i, P(ctypes.c_int)]
        lib.or_ray_segments.restype = i
        lib.or_trace_adjoint.argtypes = [i, i, i, dp, d, fp, fp, i, dp, dp, i, i, d, d, d, d,
                                         dp, d, dp, dp, dp, dp, dp, i]
        lib.or_trace_adjoint.restype = i
        _lib = lib
    return _lib


def _ptr(a, ctype):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctype))


@dataclass
class Problem:
    """A grid, its fields, its sources and the trace parameters (code units c = h nu = 1)."""

    nH0: np.ndarray                       # (nz, ny, nx) neutral density
    pos: np.ndarray                       # (nsrc, 3) source positions
    L: np.ndarray                         # (nsrc,) luminosities
    dx: float
    lo: tuple = (0.0, 0.0, 0.0)
    nH: np.ndarray | None = None          # total density for the dust term
    sigma_H: float = 1.0
    sigma_d: float = 0.0
    level0: int = 4
    level_cap: int = -1
    m_ray: float = 4.0
    tau_max: float = 30.0
    rot: np.ndarray | None = None
    Ln: np.ndarray | None = None          # non-ionizing luminosities: a second, dust-only bin
    d_max: float = 0.0                    # rays end this far from their source (> 0), else none

    def _args(self):
        nz, ny, nx = self.nH0.shape
        self._nH0 = np.ascontiguousarray(self.nH0, dtype=np.float32)
        self._nH = None if self.nH is None else np.ascontiguousarray(self.nH, dtype=np.float32)
        self._pos = np.ascontiguousarray(np.asarray(self.pos, dtype=np.float64).reshape(-1, 3))
        self._L = np.ascontiguousarray(np.asarray(self.L, dtype=np.float64).reshape(-1))
        self._Ln = None if self.Ln is None else np.ascontiguousarray(
            np.asarray(self.Ln, dtype=np.float64).reshape(-1))
        self._lo = np.ascontiguousarray(np.asarray(self.lo, dtype=np.float64))
        self._rot = None if self.rot is None else np.ascontiguousarray(
            np.asarray(self.rot, dtype=np.float64).reshape(9))
        return nx, ny, nz


@dataclass
class TraceResult:
    G: np.ndarray          # (nz, ny, nx) sum L_in ds phi(dtau)
    F: np.ndarray          # (3, nz, ny, nx) sum dL n
    L_in: float
    absorbed: float
    escaped: float
    dropped: float
    crossings: int
    rays: int
    near_tie_rays: int
    destroy: int
    Ln_in: float
    absorbed_n: float
    escaped_n: float
    dropped_n: float
    destroy_expected: int
    level_reached: int
    level_max: int
    rays_per_level: np.ndarray = field(default_factory=lambda: np.zeros(NLEVELS, np.int64))
    dV: float = 1.0
    sigma_H: float = 1.0
    hits: np.ndarray | None = None     # (nz, ny, nx) deposits per cell, when asked for

    @property
    def gamma(self):
        """Photoionization rate per neutral atom (Eq. e:photrate2 / n_HI)."""
        return self.sigma_H * self.G / self.dV

    @property
    def energy(self):
        """Radiation energy density (Eq. e:Erad, c = 1)."""
        return self.G / self.dV

    @property
    def force(self):
        """Radiation force density chi F / c (Eq. e:Frad, c = 1)."""
        return self.F / self.dV


def trace(prob: Problem, nthreads: int = 1, pix_stride: int = 1,
          count_hits: bool = False) -> TraceResult:
    """The full trace; ``pix_stride`` > 1 traces only the base rays whose pixel index is a
    multiple of it (a bounded sample, for timing); ``count_hits`` also returns the number
    of deposits per cell."""
    lib = _load()
    nx, ny, nz = prob._args()
    ncell = nx * ny * nz
    acc = np.zeros(4 * ncell, dtype=np.float64)
    hits = np.zeros(ncell, dtype=np.int64) if count_hits else None
    dstat = np.zeros(8, dtype=np.float64)
    istat = np.zeros(8 + NLEVELS, dtype=np.int64)
    rc = lib.or_trace(nx, ny, nz, _ptr(prob._lo, ctypes.c_double), prob.dx,
                      _ptr(prob._nH0, ctypes.c_float), _ptr(prob._nH, ctypes.c_float),
                      len(prob._L), _ptr(prob._pos, ctypes.c_double),
                      _ptr(prob._L, ctypes.c_double), _ptr(prob._Ln, ctypes.c_double),
                      prob.level0, prob.level_cap,
                      prob.m_ray, prob.tau_max, prob.sigma_H, prob.sigma_d,
                      _ptr(prob._rot, ctypes.c_double), prob.d_max, _ptr(acc, ctypes.c_double),
                      _ptr(dstat, ctypes.c_double), _ptr(istat, ctypes.c_longlong), nthreads,
                      int(pix_stride), _ptr(hits, ctypes.c_longlong))
    if rc != 0:
        raise ValueError("oracle rejected the problem")
    acc = acc.reshape(4, nz, ny, nx)
    return TraceResult(G=acc[0], F=acc[1:4], L_in=dstat[0], absorbed=dstat[1],
                       escaped=dstat[2], dropped=dstat[3], crossings=int(istat[0]),
                       rays=int(istat[1]), near_tie_rays=int(istat[2]), destroy=int(istat[3]),
                       Ln_in=dstat[4], absorbed_n=dstat[5], escaped_n=dstat[6],
                       dropped_n=dstat[7],
                       destroy_expected=int(istat[4]), level_reached=int(istat[5]),
                       level_max=int(istat[6]), rays_per_level=istat[8:].copy(),
                       dV=prob.dx**3, sigma_H=prob.sigma_H,
                       hits=None if hits is None else hits.reshape(nz, ny, nx))


def ray_segments(prob: Problem, level: int, pix: int, L: float = 1.0, tau: float = 0.0,
                 cap: int = 1 << 20):
    """Cells and physical lengths of the segments of one ray of source 0; and the end reason
    (0 exit or d_max cutoff, 1 tau_max, 2 split)."""
    lib = _load()
    nx, ny, nz = prob._args()
    cells = np.zeros(cap, dtype=np.int64)
    ds = np.zeros(cap, dtype=np.float64)
    end = ctypes.c_int(-1)
    n = lib.or_ray_segments(nx, ny, nz, _ptr(prob._lo, ctypes.c_double), prob.dx,
                            _ptr(prob._nH0, ctypes.c_float), _ptr(prob._nH, ctypes.c_float),
                            _ptr(prob._pos[:1].copy(), ctypes.c_double), prob.level0,
                            prob.level_cap, prob.m_ray, prob.tau_max, prob.sigma_H,
                            prob.sigma_d, _ptr(prob._rot, ctypes.c_double), prob.d_max, level,
                            pix, L, tau,
                            _ptr(cells, ctypes.c_longlong), _ptr(ds, ctypes.c_double), cap,
                            ctypes.byref(end))
    if n < 0:
        raise ValueError("oracle rejected the ray")
    n = min(n, cap)
    return cells[:n].copy(), ds[:n].copy(), end.value


def trace_adjoint(prob: Problem, w: np.ndarray, nthreads: int = 1, v: np.ndarray | None = None):
    """d loss / d log n_H0 per cell and d loss / d L per source for
    loss = sum_c (w_c Gamma_c + v_c . f_rad,c); v has shape (3, nz, ny, nx) or is None."""
    lib = _load()
    nx, ny, nz = prob._args()
    ncell = nx * ny * nz
    w64 = np.ascontiguousarray(np.asarray(w, dtype=np.float64).reshape(-1))
    if w64.size != ncell:
        raise ValueError("w must have one entry per cell")
    v64 = None
    if v is not None:
        v64 = np.ascontiguousarray(np.asarray(v, dtype=np.float64).reshape(-1))
        if v64.size != 3 * ncell:
            raise ValueError("v must have three entries per cell")
    grad = np.zeros(ncell, dtype=np.float64)
    dL = np.zeros(len(prob._L), dtype=np.float64)
    loss = ctypes.c_double(0.0)
    rc = lib.or_trace_adjoint(nx, ny, nz, _ptr(prob._lo, ctypes.c_double), prob.dx,
                              _ptr(prob._nH0, ctypes.c_float), _ptr(prob._nH, ctypes.c_float),
                              len(prob._L), _ptr(prob._pos, ctypes.c_double),
                              _ptr(prob._L, ctypes.c_double), prob.level0, prob.level_cap,
                              prob.m_ray, prob.tau_max, prob.sigma_H, prob.sigma_d,
                              _ptr(prob._rot, ctypes.c_double), prob.d_max,
                              _ptr(w64, ctypes.c_double),
                              _ptr(v64, ctypes.c_double), _ptr(grad, ctypes.c_double),
                              _ptr(dL, ctypes.c_double), ctypes.byref(loss), nthreads)
    if rc != 0:
        raise ValueError("oracle rejected the problem")
    return grad.reshape(nz, ny, nx), dL, loss.value


def pix2vec(level: int, pix: int) -> np.ndarray:
    v = np.zeros(3, dtype=np.float64)
    _load().or_pix2vec(level, pix, _ptr(v, ctypes.c_double))
    return v


def vec2pix(level: int, v) -> int:
    a = np.ascontiguousarray(np.asarray(v, dtype=np.float64))
    return int(_load().or_vec2pix(level, _ptr(a, ctypes.c_double)))


# ---------------------------------------------------------------------------------------
# Neutral-fraction updates (Sec. 2.3), FP64 numpy, elementwise
# ---------------------------------------------------------------------------------------

def xn_method_b(xn0, gamma, nH, alpha, dt):
    """Eq. e:xn3: electron density held at n_H (1 - x_0) over the step."""
    xn0 = np.asarray(xn0, dtype=np.float64)
    ne = nH * (1.0 - xn0)
    rate = gamma + alpha * ne
    out = np.empty_like(xn0)
    pos = rate > 0
    xeq = np.where(pos, alpha * ne / np.where(pos, rate, 1.0), xn0)
    out = xeq + (xn0 - xeq) * np.exp(-dt * rate)
    return np.clip(out, 0.0, 1.0)


def xn_equilibrium(gamma, nH, alpha):
    """Equilibrium neutral fraction of Eq. e:xn (root of the quadratic in [0, 1])."""
    a = alpha * nH
    return 2.0 * a / (gamma + 2.0 * a + np.sqrt(gamma**2 + 4.0 * a * gamma))


def xn_method_a(xn0, gamma, nH, alpha, dt):
    """Eq. e:xn2 (exact quadratic solution), with the Gamma = 0 solution for shielded cells."""
    xn0 = np.asarray(xn0, dtype=np.float64)
    gamma = np.asarray(gamma, dtype=np.float64) * np.ones_like(xn0)
    a = alpha * nH * np.ones_like(xn0)
    out = np.empty_like(xn0)
    z = gamma <= 0
    out[z] = xn_gamma_zero(xn0[z], a[z], dt)
    nzm = ~z
    xeq = xn_equilibrium(gamma[nzm], a[nzm], 1.0)
    xp = 1.0 / xeq
    K = np.exp(-(xp - xeq) * dt * a[nzm])
    x0 = xn0[nzm]
    out[nzm] = xeq + (xp - xeq) * (x0 - xeq) * K / ((xp - x0) + (x0 - xeq) * K)
    return np.clip(out, 0.0, 1.0)


def xn_gamma_zero(xn0, a, t):
    """Solution of Eq. e:xn with Gamma = 0, a = alpha_B n_H."""
    return (xn0 + (1.0 - xn0) * a * t) / (1.0 + (1.0 - xn0) * a * t)


def xn_method_c(xn0, gamma, nH, alpha, dt):
    """Eq. e:bdf1 (semi-implicit backward difference, Appendix)."""
    return (xn0 + (1.0 - xn0) ** 2 * alpha * nH * dt) / (1.0 + gamma * dt)


def dt_substep(xn, gamma, nH, alpha, C=0.1):
    """Eq. e:dtss: C min(n_H / |I - R|) over cells, I = x_n n_H Gamma, R = alpha n_e n_H+."""
    xn = np.asarray(xn, dtype=np.float64)
    ne = nH * (1.0 - xn)
    I = xn * nH * gamma
    R = alpha * ne * ne
    d = np.abs(I - R)
    with np.errstate(divide="ignore"):
        q = np.where(d > 0, nH / np.where(d > 0, d, 1.0), np.inf)
    return C * float(np.min(q))
