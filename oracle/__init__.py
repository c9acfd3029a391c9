"""FP64 CPU oracle of the halfway-domain scene-flow solve (arXiv 1610.07159).

TEST INFRASTRUCTURE ONLY. This package is the parity reference for the CUDA
library. Only the tests, the package's smoke check and the benchmark's CPU
baseline leg import it; the product path never does. It shares no code with
the CUDA path: the arithmetic lives in ``sfo.c`` (plain single-threaded C in
double precision) and this module only marshals numpy arrays through ctypes.

Parity status of each function (what pins it, see the ``-m "not gpu"`` tests):
  pyramid / gradients     pinned: numpy block means, closed forms on ramps
  sample, grid weights    pinned: scipy map_coordinates, partition of unity
  pixel terms (Eqs. 1-6)  pinned: closed forms on linear ramp images, FD Jacobian
  energy, assemble        pinned: b = -grad(E)/2 by finite differences, A by FD
                          directional derivatives (IRLS and the paper-literal
                          square-root residuals), closed-form priors
  pcg                     pinned: dense Cholesky solve on tiny grids, monotone model
  upsample, temporal      pinned: constant and linear fields, closed forms
  solve_frame             pinned: static plane -> analytic disparity, rigid
                          translation -> m = v/2, stereo-only symmetry, identical
                          images -> zero, energy monotone per step
  halfway image           pinned: closed form on ramps at non-zero fields, exact
                          shifted means at integer fields
  feature weight          eigenvalue step pinned by numpy eigvalsh on the exact
                          halfway image; its constants (gain 9, tau 1e-3) are a
                          reading, since the paper gives none
Every pin is itself checked: tests/test_oracle_mutations.py plants 22
plausible mistakes in copies of sfo.c and each one fails a pin.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sfo.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libsfo.so")

MAX_LEVELS = 8
MAX_GN = 16
STEP_STATS = 10
STATS_LEN = 16 + MAX_LEVELS * MAX_GN * STEP_STATS

IRLS, SQRT_PAPER = 0, 1
GRAD_BROX, GRAD_LITERAL = 0, 1
WFEAT_EIG, WFEAT_OFF = 0, 1
TEMPORAL_PROPAGATE, TEMPORAL_COPY, TEMPORAL_ZERO = 0, 1, 2
SOLVER_PCG, SOLVER_SCHWARZ = 0, 1


def build(force: bool = False) -> str:
    """Compiles sfo.c into _build/libsfo.so (gcc, C99, no FP contraction)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Params(ctypes.Structure):
    _fields_ = [
        ("w_reg", ctypes.c_double), ("w_photo", ctypes.c_double), ("w_grad", ctypes.c_double),
        ("w_epi", ctypes.c_double), ("w_smooth", ctypes.c_double), ("w_mag", ctypes.c_double),
        ("w_s", ctypes.c_double), ("w_m", ctypes.c_double), ("w_d", ctypes.c_double),
        ("m_s", ctypes.c_double), ("m_m", ctypes.c_double), ("m_d", ctypes.c_double),
        ("eps", ctypes.c_double), ("eps_p", ctypes.c_double), ("F", ctypes.c_double * 9),
        ("gn_iters", ctypes.c_int * MAX_LEVELS), ("pcg_iters", ctypes.c_int * MAX_LEVELS),
        ("robust_mode", ctypes.c_int), ("grad_mode", ctypes.c_int), ("wfeat_mode", ctypes.c_int),
        ("wfeat_gain", ctypes.c_double), ("wfeat_tau", ctypes.c_double),
        ("temporal_mode", ctypes.c_int), ("max_backtracks", ctypes.c_int),
        ("solver", ctypes.c_int), ("patch_iters", ctypes.c_int * MAX_LEVELS),
        ("schwarz_tile", ctypes.c_int), ("schwarz_overlap", ctypes.c_int),
        ("occlusion", ctypes.c_int), ("occ_tau", ctypes.c_double),
        ("illumination", ctypes.c_int), ("illum_sigma", ctypes.c_double),
    ]


# Table 1 (Appendix A): columns "Figure 2", "Figures 5, 6, 8", "Figures 7, 9";
# w_smooth = w_mag = 1 in all experiments.
TABLE1 = {
    "fig2": dict(w_reg=1.0, w_photo=1.0, w_grad=2.0, w_epi=0.0, w_s=5.0, w_m=5.0, w_d=0.5,
                 m_s=5.0, m_m=100.0, m_d=1000.0),
    "fig568": dict(w_reg=0.5, w_photo=0.5, w_grad=5.0, w_epi=0.5, w_s=0.75, w_m=0.5, w_d=0.01,
                   m_s=0.5, m_m=10.0, m_d=100.0),
    "fig79": dict(w_reg=5.0, w_photo=1.0, w_grad=5.0, w_epi=0.5, w_s=0.5, w_m=1.0, w_d=1.0,
                  m_s=0.1, m_m=10000.0, m_d=10000.0),
}

RECTIFIED_F = (0.0, 0.0, 0.0, 0.0, 0.0, -1.0, 0.0, 1.0, 0.0)


@dataclass
class Params:
    """Solver parameters; defaults are the Figure-2 column of Table 1."""
    w_reg: float = 1.0
    w_photo: float = 1.0
    w_grad: float = 2.0
    w_epi: float = 0.0
    w_smooth: float = 1.0
    w_mag: float = 1.0
    w_s: float = 5.0
    w_m: float = 5.0
    w_d: float = 0.5
    m_s: float = 5.0
    m_m: float = 100.0
    m_d: float = 1000.0
    eps: float = 1e-3
    eps_p: float = 0.2
    F: tuple = RECTIFIED_F
    gn_iters: tuple = (5,) * MAX_LEVELS
    pcg_iters: tuple = (10,) * MAX_LEVELS
    robust_mode: int = IRLS
    grad_mode: int = GRAD_BROX
    wfeat_mode: int = WFEAT_EIG
    wfeat_gain: float = 9.0
    wfeat_tau: float = 1e-3
    temporal_mode: int = TEMPORAL_PROPAGATE
    max_backtracks: int = 4
    solver: int = SOLVER_PCG
    patch_iters: tuple = (5,) * MAX_LEVELS
    schwarz_tile: int = 8
    schwarz_overlap: int = 1
    occlusion: int = 0
    occ_tau: float = 0.5
    illumination: int = 0
    illum_sigma: float = 3.2

    @classmethod
    def preset(cls, name: str, **kw) -> "Params":
        d = dict(TABLE1[name])
        d.update(kw)
        return cls(**d)

    def to_c(self) -> _Params:
        p = _Params()
        for k in ("w_reg", "w_photo", "w_grad", "w_epi", "w_smooth", "w_mag", "w_s", "w_m", "w_d",
                  "m_s", "m_m", "m_d", "eps", "eps_p", "wfeat_gain", "wfeat_tau", "occ_tau", "illum_sigma"):
            setattr(p, k, float(getattr(self, k)))
        for k in ("robust_mode", "grad_mode", "wfeat_mode", "temporal_mode", "max_backtracks", "solver",
                  "schwarz_tile", "schwarz_overlap", "occlusion", "illumination"):
            setattr(p, k, int(getattr(self, k)))
        qi = list(self.patch_iters) + [0] * MAX_LEVELS
        p.patch_iters = (ctypes.c_int * MAX_LEVELS)(*[int(v) for v in qi[:MAX_LEVELS]])
        p.F = (ctypes.c_double * 9)(*[float(v) for v in self.F])
        gi = list(self.gn_iters) + [0] * MAX_LEVELS
        pi = list(self.pcg_iters) + [0] * MAX_LEVELS
        p.gn_iters = (ctypes.c_int * MAX_LEVELS)(*[int(v) for v in gi[:MAX_LEVELS]])
        p.pcg_iters = (ctypes.c_int * MAX_LEVELS)(*[int(v) for v in pi[:MAX_LEVELS]])
        return p


_lib = None


def lib():
    global _lib
    if _lib is None:
        # SFO_LIB: a different build of sfo.c (the mutation tests load planted
        # mistakes this way); by default the library built from sfo.c here
        path = os.environ.get("SFO_LIB") or build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        up = ctypes.POINTER(ctypes.c_ubyte)
        pp = ctypes.POINTER(_Params)
        i, d = ctypes.c_int, ctypes.c_double
        L.sfo_downsample.argtypes = [i, i, dp, dp]
        L.sfo_gradients.argtypes = [i, i, dp, dp, dp]
        L.sfo_level_planes.argtypes = [i, i, dp, dp]
        L.sfo_sample.argtypes = [i, i, dp, d, d, dp, dp]
        L.sfo_sample.restype = d
        L.sfo_grid_weights.argtypes = [i, i, i, i, i, ip, dp]
        L.sfo_pixel_terms.argtypes = [i, i, dp, d, d, dp, dp, dp, dp, dp]
        L.sfo_level_F.argtypes = [dp, i, dp]
        L.sfo_feature_weights.argtypes = [i, i, i, i, i, dp, dp, pp, dp]
        L.sfo_halfway_image.argtypes = [i, i, i, i, i, dp, dp, dp]
        L.sfo_energy.argtypes = [i, i, i, i, i, i, dp, dp, dp, dp, up, pp, dp, up]
        L.sfo_energy.restype = d
        L.sfo_assemble.argtypes = [i, i, i, i, i, i, dp, dp, dp, dp, up, pp, dp, dp, up]
        L.sfo_assemble.restype = d
        L.sfo_apply.argtypes = [i, i, dp, dp, dp]
        L.sfo_pcg.argtypes = [i, i, dp, dp, i, dp, dp]
        L.sfo_pcg.restype = i
        L.sfo_schwarz.argtypes = [i, i, dp, dp, i, i, i, i, dp]
        L.sfo_schwarz.restype = i
        L.sfo_upsample.argtypes = [i, i, dp, i, i, dp]
        L.sfo_temporal.argtypes = [i, i, i, dp, dp, i, dp]
        L.sfo_packed_size.argtypes = [i, i, i, i]
        L.sfo_packed_size.restype = ctypes.c_long
        u32p = ctypes.POINTER(ctypes.c_uint)
        lp = ctypes.POINTER(ctypes.c_long)
        L.sfo_solve_frame.argtypes = [i, i, i, i, pp, dp, dp, dp, dp, up, u32p, lp, up, dp, dp, dp]
        L.sfo_occlusion_map.argtypes = [i, i, i, i, i, dp, d, up]
        L.sfo_vis_upsample.argtypes = [i, i, up, i, i, up]
        L.sfo_illum_residual.argtypes = [i, i, i, i, i, dp, dp, dp]
        L.sfo_gauss_blur.argtypes = [i, i, dp, d, dp]
        L.sfo_illum_upsample.argtypes = [i, i, dp, i, i, dp]
        L.sfo_energy_maps.argtypes = [i, i, i, i, i, i, dp, dp, dp, dp, up, pp, up, dp, dp, up]
        L.sfo_energy_maps.restype = d
        L.sfo_assemble_maps.argtypes = [i, i, i, i, i, i, dp, dp, dp, dp, up, pp, up, dp, dp, dp, up]
        L.sfo_assemble_maps.restype = d
        L.sfo_solve_frame.restype = i
        _lib = L
    return _lib


def _d(a: np.ndarray | None):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _u8(a: np.ndarray | None):
    if a is None:
        return None
    assert a.dtype == np.uint8 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# --------------------------------------------------------------------------- #
# geometry helpers (pure integer bookkeeping)
# --------------------------------------------------------------------------- #

def level_dims(w0: int, h0: int, level: int) -> tuple[int, int]:
    w, h = w0, h0
    for _ in range(level):
        w, h = (w + 1) // 2, (h + 1) // 2
    return w, h


def grid_dims(w: int, h: int, s: int) -> tuple[int, int]:
    return (w + s - 1) // s, (h + s - 1) // s


def packed_offsets(w0: int, h0: int, s: int, levels: int) -> list[tuple[int, int, int, int, int]]:
    """Per level (offset, nx, ny, w, h) of the packed per-level node arrays."""
    out, off = [], 0
    for l in range(levels):
        w, h = level_dims(w0, h0, l)
        nx, ny = grid_dims(w, h, s)
        out.append((off, nx, ny, w, h))
        off += 6 * nx * ny
    return out


# --------------------------------------------------------------------------- #
# step-level functions
# --------------------------------------------------------------------------- #

def downsample(img: np.ndarray) -> np.ndarray:
    img = _f64(img)
    h, w = img.shape
    out = np.zeros(((h + 1) // 2, (w + 1) // 2))
    lib().sfo_downsample(w, h, _d(img), _d(out))
    return out


def gradients(img: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    img = _f64(img)
    h, w = img.shape
    gx, gy = np.zeros_like(img), np.zeros_like(img)
    lib().sfo_gradients(w, h, _d(img), _d(gx), _d(gy))
    return gx, gy


def pyramid(imgs4: np.ndarray, levels: int) -> list[np.ndarray]:
    """Per level the four intensity images [4, h, w]."""
    cur = _f64(imgs4)
    out = [cur]
    for _ in range(1, levels):
        cur = np.stack([downsample(cur[c]) for c in range(4)])
        out.append(cur)
    return out


def level_planes(imgs4: np.ndarray) -> np.ndarray:
    """[4, 3, h, w]: (I, dI/dx, dI/dy) of the four images."""
    imgs4 = _f64(imgs4)
    _, h, w = imgs4.shape
    planes = np.zeros((4, 3, h, w))
    lib().sfo_level_planes(w, h, _d(imgs4), _d(planes))
    return planes


def sample(plane: np.ndarray, px: float, py: float) -> tuple[float, float, float]:
    plane = _f64(plane)
    h, w = plane.shape
    dx, dy = ctypes.c_double(), ctypes.c_double()
    v = lib().sfo_sample(w, h, _d(plane), float(px), float(py), ctypes.byref(dx), ctypes.byref(dy))
    return v, dx.value, dy.value


def grid_weights(x: int, y: int, s: int, nx: int, ny: int) -> tuple[np.ndarray, np.ndarray]:
    nodes = (ctypes.c_int * 4)()
    wts = np.zeros(4)
    lib().sfo_grid_weights(int(x), int(y), int(s), int(nx), int(ny), nodes, _d(wts))
    return np.array(list(nodes)), wts


def pixel_terms(planes: np.ndarray, x: float, y: float, f6) -> dict:
    planes = _f64(planes)
    _, _, h, w = planes.shape
    f = _f64(f6)
    e, g, Je, Jg = np.zeros(6), np.zeros(12), np.zeros(36), np.zeros(72)
    lib().sfo_pixel_terms(w, h, _d(planes), float(x), float(y), _d(f), _d(e), _d(g), _d(Je), _d(Jg))
    return {"e": e, "g": g.reshape(6, 2), "Je": Je.reshape(6, 6), "Jg": Jg.reshape(12, 6)}


def level_F(F, level: int) -> np.ndarray:
    F = _f64(F)
    out = np.zeros(9)
    lib().sfo_level_F(_d(F), int(level), _d(out))
    return out.reshape(3, 3)


@dataclass
class Level:
    """One hierarchy level: its planes and grid geometry."""
    planes: np.ndarray  # [4, 3, h, w]
    s: int
    level: int = 0
    w: int = field(init=False)
    h: int = field(init=False)
    nx: int = field(init=False)
    ny: int = field(init=False)

    def __post_init__(self):
        self.planes = _f64(self.planes)
        self.h, self.w = self.planes.shape[2], self.planes.shape[3]
        self.nx, self.ny = grid_dims(self.w, self.h, self.s)

    @property
    def G(self) -> int:
        return self.nx * self.ny


def halfway_image(lv: Level, T: np.ndarray) -> np.ndarray:
    """[h, w]: the mean of the four images warped by the totals T (6 x G)."""
    T = _f64(T)
    H = np.zeros((lv.h, lv.w))
    lib().sfo_halfway_image(lv.w, lv.h, lv.s, lv.nx, lv.ny, _d(lv.planes), _d(T), _d(H))
    return H


def feature_weights(lv: Level, T: np.ndarray, p: Params) -> np.ndarray:
    T = _f64(T)
    wf = np.zeros(lv.G)
    pc = p.to_c()
    lib().sfo_feature_weights(lv.w, lv.h, lv.s, lv.nx, lv.ny, _d(lv.planes), _d(T), ctypes.byref(pc), _d(wf))
    return wf


def energy(lv: Level, base, delta, wf, p: Params, W: np.ndarray | None = None) -> tuple[float, np.ndarray, np.ndarray]:
    """(E, unweighted terms [photo, grad, smooth, epi, mag], W used)."""
    base, delta, wf = _f64(base), _f64(delta), _f64(wf)
    terms = np.zeros(5)
    Wout = np.zeros(lv.w * lv.h, dtype=np.uint8)
    Win = None if W is None else np.ascontiguousarray(W, dtype=np.uint8).reshape(-1)
    pc = p.to_c()
    E = lib().sfo_energy(lv.w, lv.h, lv.s, lv.nx, lv.ny, lv.level, _d(lv.planes), _d(base), _d(delta), _d(wf),
                         _u8(Win), ctypes.byref(pc), _d(terms), _u8(Wout))
    return E, terms, (Win if Win is not None else Wout).reshape(lv.h, lv.w)


def assemble(lv: Level, base, delta, wf, p: Params, W: np.ndarray | None = None):
    """(A [G, 9, 6, 6], b [G, 6], E, W [h, w]) at the state base + delta."""
    base, delta, wf = _f64(base), _f64(delta), _f64(wf)
    A = np.zeros((lv.G, 9, 6, 6))
    b = np.zeros((lv.G, 6))
    Wout = np.zeros(lv.w * lv.h, dtype=np.uint8)
    Win = None if W is None else np.ascontiguousarray(W, dtype=np.uint8).reshape(-1)
    pc = p.to_c()
    E = lib().sfo_assemble(lv.w, lv.h, lv.s, lv.nx, lv.ny, lv.level, _d(lv.planes), _d(base), _d(delta), _d(wf),
                           _u8(Win), ctypes.byref(pc), _d(A), _d(b), _u8(Wout))
    return A, b, E, (Win if Win is not None else Wout).reshape(lv.h, lv.w)


def _maps(lv: Level, V, Lmap):
    Vc = None if V is None else np.ascontiguousarray(V, dtype=np.uint8).reshape(-1)
    Lc = None if Lmap is None else _f64(Lmap).reshape(-1)
    if Vc is not None:
        assert Vc.size == lv.w * lv.h
    if Lc is not None:
        assert Lc.size == 2 * lv.w * lv.h
    return Vc, Lc


def energy_maps(lv: Level, base, delta, wf, p: Params, V=None, Lmap=None, W=None):
    """energy() with a level's occlusion map V [h, w] and illumination
    differences Lmap [2, h, w] (either may be None)."""
    base, delta, wf = _f64(base), _f64(delta), _f64(wf)
    Vc, Lc = _maps(lv, V, Lmap)
    terms = np.zeros(5)
    Wout = np.zeros(lv.w * lv.h, dtype=np.uint8)
    Win = None if W is None else np.ascontiguousarray(W, dtype=np.uint8).reshape(-1)
    pc = p.to_c()
    E = lib().sfo_energy_maps(lv.w, lv.h, lv.s, lv.nx, lv.ny, lv.level, _d(lv.planes), _d(base), _d(delta),
                              _d(wf), _u8(Win), ctypes.byref(pc), _u8(Vc), _d(Lc), _d(terms), _u8(Wout))
    return E, terms, (Win if Win is not None else Wout).reshape(lv.h, lv.w)


def assemble_maps(lv: Level, base, delta, wf, p: Params, V=None, Lmap=None, W=None):
    """assemble() with a level's occlusion map and illumination differences."""
    base, delta, wf = _f64(base), _f64(delta), _f64(wf)
    Vc, Lc = _maps(lv, V, Lmap)
    A = np.zeros((lv.G, 9, 6, 6))
    b = np.zeros((lv.G, 6))
    Wout = np.zeros(lv.w * lv.h, dtype=np.uint8)
    Win = None if W is None else np.ascontiguousarray(W, dtype=np.uint8).reshape(-1)
    pc = p.to_c()
    E = lib().sfo_assemble_maps(lv.w, lv.h, lv.s, lv.nx, lv.ny, lv.level, _d(lv.planes), _d(base), _d(delta),
                                _d(wf), _u8(Win), ctypes.byref(pc), _u8(Vc), _d(Lc), _d(A), _d(b), _u8(Wout))
    return A, b, E, (Win if Win is not None else Wout).reshape(lv.h, lv.w)


def occlusion_map(w: int, h: int, s: int, T: np.ndarray, tau: float = 0.5) -> np.ndarray:
    """[h, w] uint8 visibility of a level at totals T (6 x G)."""
    nx, ny = grid_dims(w, h, s)
    T = _f64(T)
    assert T.size == 6 * nx * ny
    O = np.zeros(w * h, dtype=np.uint8)
    lib().sfo_occlusion_map(w, h, s, nx, ny, _d(T), float(tau), _u8(O))
    return O.reshape(h, w)


def vis_upsample(Oc: np.ndarray, w: int, h: int) -> np.ndarray:
    Oc = np.ascontiguousarray(Oc, dtype=np.uint8)
    hc, wc = Oc.shape
    V = np.zeros(w * h, dtype=np.uint8)
    lib().sfo_vis_upsample(wc, hc, _u8(Oc.reshape(-1)), w, h, _u8(V))
    return V.reshape(h, w)


def illum_residual(lv: Level, T: np.ndarray) -> np.ndarray:
    """[2, h, w] stereo intensity residuals (right - left at times 0 and 1)."""
    r = np.zeros(2 * lv.w * lv.h)
    lib().sfo_illum_residual(lv.w, lv.h, lv.s, lv.nx, lv.ny, _d(lv.planes), _d(_f64(T)), _d(r))
    return r.reshape(2, lv.h, lv.w)


def gauss_blur(img: np.ndarray, sigma: float = 3.2) -> np.ndarray:
    img = _f64(img)
    h, w = img.shape
    out = np.zeros_like(img)
    lib().sfo_gauss_blur(w, h, _d(img), float(sigma), _d(out))
    return out


def illum_upsample(Rc: np.ndarray, w: int, h: int) -> np.ndarray:
    Rc = _f64(Rc)
    _, hc, wc = Rc.shape
    out = np.zeros(2 * w * h)
    lib().sfo_illum_upsample(wc, hc, _d(Rc), w, h, _d(out))
    return out.reshape(2, h, w)


def apply(nx: int, ny: int, A: np.ndarray, x: np.ndarray) -> np.ndarray:
    A, x = _f64(A), _f64(x)
    y = np.zeros_like(x)
    lib().sfo_apply(nx, ny, _d(A), _d(x), _d(y))
    return y


def pcg(nx: int, ny: int, A: np.ndarray, b: np.ndarray, iters: int):
    """(x [G, 6], model trace, iterations run)."""
    A, b = _f64(A), _f64(b)
    x = np.zeros_like(b)
    model = np.zeros(max(iters, 1))
    its = lib().sfo_pcg(nx, ny, _d(A), _d(b), int(iters), _d(x), _d(model))
    return x, model[:its], its


def schwarz(nx: int, ny: int, A: np.ndarray, b: np.ndarray, sweeps: int, patch_iters: int, tile: int = 8,
            overlap: int = 1) -> np.ndarray:
    """x [G, 6] after `sweeps` alternating Schwarz iterations (Section 5.2)."""
    A, b = _f64(A), _f64(b)
    x = np.zeros_like(b)
    if lib().sfo_schwarz(nx, ny, _d(A), _d(b), int(sweeps), int(patch_iters), int(tile), int(overlap), _d(x)) != 0:
        raise ValueError("invalid Schwarz tiling")
    return x


def upsample(Tc: np.ndarray, nxc: int, nyc: int, nx: int, ny: int) -> np.ndarray:
    Tc = _f64(Tc)
    base = np.zeros(6 * nx * ny)
    lib().sfo_upsample(nxc, nyc, _d(Tc), nx, ny, _d(base))
    return base


def temporal(s: int, nx: int, ny: int, delta_prev, T_prev, mode: int = TEMPORAL_PROPAGATE) -> np.ndarray:
    delta_prev, T_prev = _f64(delta_prev), _f64(T_prev)
    out = np.zeros(6 * nx * ny)
    lib().sfo_temporal(s, nx, ny, _d(delta_prev), _d(T_prev), int(mode), _d(out))
    return out


@dataclass
class FrameResult:
    delta: np.ndarray   # packed per-level deltas
    total: np.ndarray   # packed per-level totals
    stats: np.ndarray   # SFO stats vector
    offsets: list

    @property
    def energy(self) -> float:
        return float(self.stats[0])

    def fields(self, level: int = 0) -> np.ndarray:
        off, nx, ny, _, _ = self.offsets[level]
        return self.total[off:off + 6 * nx * ny].reshape(6, ny, nx)

    def deltas(self, level: int = 0) -> np.ndarray:
        off, nx, ny, _, _ = self.offsets[level]
        return self.delta[off:off + 6 * nx * ny].reshape(6, ny, nx)

    def step(self, level: int, g: int) -> np.ndarray:
        """E at the linearisation point, E accepted, t, pixels with W = 0, PCG
        iterations, replayed W decisions that differ from the oracle's own and
        their largest margin, replayed cell decisions that differ and their
        largest distance from an integer position."""
        i = 16 + (level * MAX_GN + g) * STEP_STATS
        return self.stats[i:i + STEP_STATS]


def solve_frame(imgs4: np.ndarray, s: int, levels: int, p: Params, prev: FrameResult | None = None,
                init_coarsest: np.ndarray | None = None, W_given: list | None = None,
                cells_given: list | None = None, V_given: list | None = None) -> FrameResult:
    """Algorithm 1 for one quadruple (without occlusion and illumination maps).

    W_given: optional outlier masks to use instead of taking W in FP64, as
    W_given[level][step] arrays of the level's image shape.
    cells_given: optional bilinear cell decisions to use in the assembly of
    each step instead of taking them in FP64, as cells_given[level][step]
    uint32 arrays [n, 2] of (pixel y*w + x, cell << 4 | clamped << 3 |
    image << 1 | axis), any order.
    V_given: optional occlusion maps to use instead of the oracle's own
    prolongated ones, as V_given[level] arrays of the level's image shape."""
    imgs4 = _f64(imgs4)
    _, h, w = imgs4.shape
    n = int(lib().sfo_packed_size(w, h, s, levels))
    delta, total, stats = np.zeros(n), np.zeros(n), np.zeros(STATS_LEN)
    pc = p.to_c()
    ic = None if init_coarsest is None else _f64(init_coarsest).reshape(-1)
    wg = None
    if W_given is not None:
        parts = []
        for l in range(levels):
            lw, lh = level_dims(w, h, l)
            for g in range(p.gn_iters[l]):
                m = np.ascontiguousarray(W_given[l][g], dtype=np.uint8).reshape(-1)
                assert m.size == lw * lh
                parts.append(m)
        wg = np.ascontiguousarray(np.concatenate(parts) if parts else np.zeros(1, np.uint8))
    recs_p = offs_p = None
    if cells_given is not None:
        offs = np.zeros(MAX_LEVELS * MAX_GN + 1, dtype=np.int64)
        parts, k = [], 0
        for l in range(MAX_LEVELS):
            for g in range(MAX_GN):
                offs[l * MAX_GN + g] = k
                if l < levels and l < len(cells_given) and g < len(cells_given[l]):
                    r = np.asarray(cells_given[l][g], dtype=np.uint32).reshape(-1, 2)
                    r = r[np.lexsort((r[:, 1], r[:, 0]))]
                    parts.append(r)
                    k += len(r)
        offs[-1] = k
        recs = np.ascontiguousarray(np.concatenate(parts) if parts else np.zeros((1, 2), np.uint32))
        offs = np.ascontiguousarray(offs.astype(np.int_))
        recs_p = recs.ctypes.data_as(ctypes.POINTER(ctypes.c_uint))
        offs_p = offs.ctypes.data_as(ctypes.POINTER(ctypes.c_long))
    vg = None
    if V_given is not None:
        parts = []
        for l in range(levels):
            lw, lh = level_dims(w, h, l)
            m = np.ascontiguousarray(V_given[l], dtype=np.uint8).reshape(-1)
            assert m.size == lw * lh
            parts.append(m)
        vg = np.ascontiguousarray(np.concatenate(parts))
    rc = lib().sfo_solve_frame(w, h, s, levels, ctypes.byref(pc), _d(imgs4),
                               _d(prev.delta) if prev is not None else None,
                               _d(prev.total) if prev is not None else None,
                               _d(ic), _u8(wg), recs_p, offs_p, _u8(vg), _d(delta), _d(total), _d(stats))
    if rc != 0:
        raise ValueError("invalid sizes for the oracle solve")
    return FrameResult(delta, total, stats, packed_offsets(w, h, s, levels))
