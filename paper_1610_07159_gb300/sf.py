"""Thin ctypes binding of the C ABI in include/sf.h (libsf_gb300.so).

Argument marshalling only: every step of the solve runs in the library's CUDA
kernels. Tensors passed in must be contiguous CUDA tensors of the stated
dtype; the binding hands their data pointers and the current CUDA stream to
the library. There is no CPU path: if the library is missing or fails to
load, loading raises.
"""

from __future__ import annotations

import ctypes
import os

import torch

from . import build as _build

MAX_LEVELS = 8
MAX_GN = 16

OK, ERR_ARG, ERR_CUDA, ERR_OOM, ERR_NUMERIC, ERR_TIMEOUT, ERR_STATE = range(7)
IRLS, SQRT_PAPER = 0, 1
GRAD_BROX, GRAD_LITERAL = 0, 1
WFEAT_EIG, WFEAT_OFF = 0, 1
TEMPORAL_PROPAGATE, TEMPORAL_COPY, TEMPORAL_ZERO = 0, 1, 2
FP32, MIXED_BF16, MIXED_FP16 = 0, 1, 2
K_PYRAMID, K_LEVEL, K_ASSEMBLE, K_GATHER, K_PCG, K_ENERGY = range(6)
PCG_AUTO, PCG_CLUSTER, PCG_GRID, PCG_DSM, PCG_ONE_REDUCTION, PCG_PIPELINED = 0, 1, 2, 3, 4, 5
SOLVER_PCG, SOLVER_SCHWARZ = 0, 1
PRESET_FIG2, PRESET_FIG568, PRESET_FIG79 = 0, 1, 2

EXPORTED = (
    "sf_params_preset", "sf_create", "sf_solve", "sf_solve_host", "sf_solve_video", "sf_solve_video_host",
    "sf_grid_dims", "sf_set_init", "sf_reset",
    "sf_get_stats", "sf_get_state", "sf_kernel_times", "sf_destroy", "sf_status_string", "sf_last_error", "sf_probe_pyramid",
    "sf_probe_feature_weights", "sf_probe_assemble", "sf_probe_pcg", "sf_probe_wmask", "sf_probe_energy",
    "sf_probe_cells", "sf_probe_fma_rate", "sf_probe_schwarz", "sf_probe_vmask", "sf_probe_occlusion",
    "sf_probe_illum", "sf_probe_barrier_timeout", "sf_probe_mbarrier_timeout", "sf_probe_tagged_timeout",
    "sf_pcg_static", "sf_batch_create", "sf_batch_layout", "sf_batch_solve", "sf_batch_set_schedule",
    "sf_batch_get_schedule", "sf_batch_tune", "sf_batch_sequence", "sf_batch_reset", "sf_batch_destroy",
    "sf_probe_gemm_bf16", "sf_net_param_count", "sf_net_create", "sf_net_set_params", "sf_net_get_params",
    "sf_net_forward", "sf_net_gradients", "sf_net_train_step", "sf_net_status", "sf_net_destroy",
    "sf_coarsest_images", "sf_warm_start", "sf_tune_pcg", "sf_pcg_schedule", "sf_set_pcg_schedule",
)
STATIC_PCG_MAX_NODES = 4096


class SFError(RuntimeError):
    pass


class Params(ctypes.Structure):
    _fields_ = [
        ("w_reg", ctypes.c_float), ("w_photo", ctypes.c_float), ("w_grad", ctypes.c_float),
        ("w_epi", ctypes.c_float), ("w_smooth", ctypes.c_float), ("w_mag", ctypes.c_float),
        ("w_s", ctypes.c_float), ("w_m", ctypes.c_float), ("w_d", ctypes.c_float),
        ("m_s", ctypes.c_float), ("m_m", ctypes.c_float), ("m_d", ctypes.c_float),
        ("eps", ctypes.c_float), ("eps_p", ctypes.c_float), ("F", ctypes.c_float * 9),
        ("gn_iters", ctypes.c_int * MAX_LEVELS), ("pcg_iters", ctypes.c_int * MAX_LEVELS),
        ("robust_mode", ctypes.c_int), ("grad_mode", ctypes.c_int), ("wfeat_mode", ctypes.c_int),
        ("wfeat_gain", ctypes.c_float), ("wfeat_tau", ctypes.c_float),
        ("temporal_mode", ctypes.c_int), ("precision", ctypes.c_int), ("max_backtracks", ctypes.c_int),
        ("use_graph", ctypes.c_int), ("profile_mask", ctypes.c_int), ("pcg_mode", ctypes.c_int),
        ("video", ctypes.c_int), ("record_cells", ctypes.c_int),
        ("solver", ctypes.c_int), ("patch_iters", ctypes.c_int * MAX_LEVELS),
        ("schwarz_tile", ctypes.c_int), ("schwarz_overlap", ctypes.c_int),
        ("occlusion", ctypes.c_int), ("occ_tau", ctypes.c_float),
        ("illumination", ctypes.c_int), ("illum_sigma", ctypes.c_float),
    ]


class Stats(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int), ("frames", ctypes.c_int), ("levels", ctypes.c_int), ("n_excluded", ctypes.c_int),
        ("launches", ctypes.c_int), ("pad", ctypes.c_int),
        ("energy", ctypes.c_double), ("terms", ctypes.c_double * 5),
        ("step_energy", (ctypes.c_double * MAX_GN) * MAX_LEVELS),
        ("step_accepted", (ctypes.c_double * MAX_GN) * MAX_LEVELS),
        ("step_t", (ctypes.c_float * MAX_GN) * MAX_LEVELS),
        ("step_excluded", (ctypes.c_int * MAX_GN) * MAX_LEVELS),
    ]


_lib = None


def lib_path() -> str:
    return _build.LIB_PATH


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Loads libsf_gb300.so (building it first if needed); raises if it cannot."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing and not _build.up_to_date():
        _build.build()
    path = _build.LIB_PATH
    if not os.path.exists(path):
        raise SFError(f"CUDA library missing: {path}")
    L = ctypes.CDLL(path)
    vp, i, fp = ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p
    ip = ctypes.POINTER(ctypes.c_int)
    L.sf_params_preset.argtypes = [ctypes.POINTER(Params), i]
    L.sf_create.argtypes = [i, i, i, i, ctypes.POINTER(Params)]
    L.sf_create.restype = vp
    L.sf_solve.argtypes = [vp, fp, fp, fp, fp, fp, vp]
    L.sf_solve_host.argtypes = [vp, fp, fp, fp, fp, fp, vp]
    L.sf_solve_video.argtypes = [vp, fp, i, fp, vp]
    L.sf_solve_video_host.argtypes = [vp, fp, i, fp, vp]
    L.sf_grid_dims.argtypes = [vp, i, ip, ip, ip, ip]
    L.sf_set_init.argtypes = [vp, fp, vp]
    L.sf_reset.argtypes = [vp]
    L.sf_get_stats.argtypes = [vp, ctypes.POINTER(Stats)]
    L.sf_get_state.argtypes = [vp, i, fp, fp, vp]
    L.sf_kernel_times.argtypes = [vp, i, ctypes.POINTER(ctypes.c_double), ip]
    L.sf_destroy.argtypes = [vp]
    L.sf_destroy.restype = None
    L.sf_status_string.argtypes = [i]
    L.sf_status_string.restype = ctypes.c_char_p
    L.sf_last_error.argtypes = []
    L.sf_probe_pyramid.argtypes = [vp, fp, fp, fp, fp, i, fp, vp]
    L.sf_probe_feature_weights.argtypes = [vp, i, fp, fp, vp]
    L.sf_probe_assemble.argtypes = [vp, i, fp, fp, fp, fp, fp, fp, fp, vp]
    L.sf_probe_pcg.argtypes = [vp, i, i, fp, vp]
    L.sf_probe_schwarz.argtypes = [vp, i, i, i, fp, vp]
    L.sf_probe_vmask.argtypes = [vp, i, fp, vp]
    L.sf_probe_barrier_timeout.argtypes = [i, ctypes.c_longlong, ip, ip]
    L.sf_probe_mbarrier_timeout.argtypes = [i, ctypes.c_longlong, ip]
    L.sf_probe_tagged_timeout.argtypes = [i, i, ctypes.c_longlong, ip, ip]
    L.sf_probe_occlusion.argtypes = [vp, i, fp, fp, vp]
    L.sf_probe_illum.argtypes = [vp, i, fp, fp, vp]
    L.sf_probe_wmask.argtypes = [vp, i, i, fp, vp]
    L.sf_probe_energy.argtypes = [vp, i, fp, fp, fp, fp, fp, vp]
    L.sf_probe_cells.argtypes = [vp, i, i, ctypes.POINTER(ctypes.c_uint), i, ip]
    L.sf_probe_fma_rate.argtypes = [i, ctypes.POINTER(ctypes.c_double), vp]
    L.sf_pcg_static.argtypes = [i, i, fp, fp, i, fp, vp]
    sz = ctypes.POINTER(ctypes.c_size_t)
    L.sf_batch_create.argtypes = [i, ip, ip, ip, i, ctypes.POINTER(Params), ctypes.POINTER(vp)]
    L.sf_batch_layout.argtypes = [vp, sz, sz, sz, sz]
    L.sf_batch_solve.argtypes = [vp, fp, fp, vp]
    L.sf_batch_set_schedule.argtypes = [vp, i, i]
    L.sf_batch_get_schedule.argtypes = [vp, ip, ip]
    L.sf_batch_tune.argtypes = [vp, fp, fp, i, vp, ctypes.POINTER(ctypes.c_float)]
    L.sf_batch_sequence.argtypes = [vp, i]
    L.sf_batch_sequence.restype = vp
    L.sf_batch_reset.argtypes = [vp]
    L.sf_batch_destroy.argtypes = [vp]
    L.sf_batch_destroy.restype = None
    L.sf_probe_gemm_bf16.argtypes = [vp, vp, i, i, i, i, i, fp, vp]
    L.sf_net_param_count.argtypes = []
    L.sf_net_create.argtypes = [i, ctypes.POINTER(vp)]
    L.sf_net_set_params.argtypes = [vp, fp, vp]
    L.sf_net_get_params.argtypes = [vp, fp, vp]
    L.sf_net_forward.argtypes = [vp, fp, i, fp, vp]
    L.sf_net_gradients.argtypes = [vp, fp, fp, i, fp, fp, vp]
    L.sf_net_train_step.argtypes = [vp, fp, fp, i, ctypes.c_float, fp, vp]
    L.sf_net_status.argtypes = [vp]
    L.sf_net_destroy.argtypes = [vp]
    L.sf_net_destroy.restype = None
    L.sf_coarsest_images.argtypes = [vp, fp, fp, fp, fp, fp, vp]
    L.sf_warm_start.argtypes = [vp, vp, fp, fp, fp, fp, vp]
    L.sf_tune_pcg.argtypes = [vp, fp, fp, fp, fp, i, vp]
    L.sf_pcg_schedule.argtypes = [vp, i, ip, ip, ip]
    L.sf_set_pcg_schedule.argtypes = [vp, i, i, i, i]
    _lib = L
    return L


def status_string(code: int) -> str:
    return load().sf_status_string(int(code)).decode()


def _check(rc: int, what: str) -> None:
    if rc != OK:
        raise SFError(f"{what}: {status_string(rc)} ({rc})")


def preset(which: int = PRESET_FIG2, **kw) -> Params:
    p = Params()
    _check(load().sf_params_preset(ctypes.byref(p), int(which)), "sf_params_preset")
    for k, v in kw.items():
        if k in ("gn_iters", "pcg_iters", "patch_iters"):
            vals = list(v) + [list(v)[-1]] * MAX_LEVELS
            setattr(p, k, (ctypes.c_int * MAX_LEVELS)(*[int(x) for x in vals[:MAX_LEVELS]]))
        elif k == "F":
            p.F = (ctypes.c_float * 9)(*[float(x) for x in v])
        else:
            setattr(p, k, v)
    return p


def _ptr(t: torch.Tensor | None, dtype: torch.dtype | None = None) -> int | None:
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise SFError("tensors passed to the library must be contiguous CUDA tensors")
    if dtype is not None and t.dtype != dtype:
        raise SFError(f"expected {dtype}, got {t.dtype}")
    return t.data_ptr()


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


def barrier_timeout_probe(skip_block: int, limit_cycles: int) -> tuple[int, int]:
    """(latched status, blocks back from the barrier) of one grid barrier that
    block skip_block never reaches (-1: all arrive)."""
    st, ret = ctypes.c_int(), ctypes.c_int()
    _check(load().sf_probe_barrier_timeout(int(skip_block), int(limit_cycles), ctypes.byref(st), ctypes.byref(ret)),
           "sf_probe_barrier_timeout")
    return st.value, ret.value


def tagged_timeout_probe(mode: int, skip_block: int, limit_cycles: int) -> tuple[int, int]:
    """(latched status, blocks back) of the self-tagged exchange's waits: mode 0
    the partial-sum poll, mode 1 a halo word; block skip_block never publishes
    (-1: all do)."""
    st, ret = ctypes.c_int(), ctypes.c_int()
    _check(load().sf_probe_tagged_timeout(int(mode), int(skip_block), int(limit_cycles), ctypes.byref(st),
                                          ctypes.byref(ret)), "sf_probe_tagged_timeout")
    return st.value, ret.value


def mbarrier_timeout_probe(arrive: bool, limit_cycles: int) -> int:
    """1 if an mbarrier wait saw its phase complete, 0 if it ran out."""
    out = ctypes.c_int()
    _check(load().sf_probe_mbarrier_timeout(int(bool(arrive)), int(limit_cycles), ctypes.byref(out)),
           "sf_probe_mbarrier_timeout")
    return out.value


def fma_rate(reps: int = 5) -> float:
    """The FP32 FMA rate of the current GPU in flops/s (measurement aid)."""
    out = ctypes.c_double()
    _check(load().sf_probe_fma_rate(int(reps), ctypes.byref(out), _stream()), "sf_probe_fma_rate")
    return out.value


def gemm_bf16(A: torch.Tensor, B: torch.Tensor, BN: int = 256, splits: int = 1) -> torch.Tensor:
    """[splits, M, N] FP32 partial products of A[M, K] @ B[N, K]^T (BF16 CUDA
    tensors, K % 64 == 0, N % 16 == 0) on the tensor cores."""
    L = load()
    assert A.dtype == torch.bfloat16 and B.dtype == torch.bfloat16 and A.is_contiguous() and B.is_contiguous()
    M, K = A.shape
    N = B.shape[0]
    C = torch.empty((splits, M, N), device="cuda", dtype=torch.float32)
    _check(L.sf_probe_gemm_bf16(A.data_ptr(), B.data_ptr(), M, N, K, int(BN), int(splits), _ptr(C), _stream()),
           "sf_probe_gemm_bf16")
    return C


def pcg_static(nx: int, ny: int, blocks: torch.Tensor, rhs: torch.Tensor, iters: int,
               x: torch.Tensor | None = None) -> torch.Tensor:
    """sf_pcg_static: PCG on a [G,5,6,6] block system with no device allocation
    inside the call (the caller allocates x, or this wrapper does before it)."""
    G = int(nx) * int(ny)
    if x is None:
        x = torch.empty((G, 6), device=blocks.device, dtype=torch.float32)
    _check(load().sf_pcg_static(int(nx), int(ny), _ptr(blocks, torch.float32), _ptr(rhs, torch.float32), int(iters),
                                _ptr(x, torch.float32), _stream()), "sf_pcg_static")
    return x


class Solver:
    """One solver context (sf_create ... sf_destroy)."""

    def __init__(self, width: int, height: int, grid_stride: int, levels: int, params: Params | None = None,
                 _view_of: int | None = None):
        self.L = load()
        self.params = params if params is not None else preset()
        torch.cuda.init()
        self.owned = _view_of is None
        if self.owned:
            self.ctx = self.L.sf_create(int(width), int(height), int(grid_stride), int(levels),
                                        ctypes.byref(self.params))
        else:
            self.ctx = _view_of
        if not self.ctx:
            raise SFError(f"sf_create: {status_string(self.L.sf_last_error())}")
        self.width, self.height, self.stride, self.levels = int(width), int(height), int(grid_stride), int(levels)

    def close(self) -> None:
        if getattr(self, "ctx", None):
            if self.owned:
                self.L.sf_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def dims(self, level: int = 0) -> tuple[int, int, int, int]:
        w, h, nx, ny = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(self.L.sf_grid_dims(self.ctx, int(level), ctypes.byref(w), ctypes.byref(h), ctypes.byref(nx),
                                   ctypes.byref(ny)), "sf_grid_dims")
        return w.value, h.value, nx.value, ny.value

    def solve(self, imgs: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        """imgs: float32 CUDA [4, H, W] (L_t, R_t, L_t1, R_t1); returns fields [6, ny, nx]."""
        _, _, nx, ny = self.dims(0)
        if out is None:
            out = torch.empty((6, ny, nx), device=imgs.device, dtype=torch.float32)
        if imgs.shape != (4, self.height, self.width):
            raise SFError(f"expected images of shape (4, {self.height}, {self.width})")
        base = _ptr(imgs, torch.float32)
        n = self.width * self.height * 4
        _check(self.L.sf_solve(self.ctx, base, base + n, base + 2 * n, base + 3 * n, _ptr(out, torch.float32),
                               _stream()), "sf_solve")
        return out

    def solve_ptrs(self, p0: int, p1: int, p2: int, p3: int, out_ptr: int, stream: int) -> None:
        _check(self.L.sf_solve(self.ctx, p0, p1, p2, p3, out_ptr, stream), "sf_solve")

    def solve_host(self, imgs, out) -> None:
        """imgs: float32 CPU tensor [4, H, W] (pinned for full speed); out: float32 CPU [6, ny, nx]."""
        if imgs.is_cuda or out.is_cuda or not imgs.is_contiguous() or not out.is_contiguous():
            raise SFError("solve_host takes contiguous host tensors")
        base = imgs.data_ptr()
        n = self.width * self.height * 4
        _check(self.L.sf_solve_host(self.ctx, base, base + n, base + 2 * n, base + 3 * n, out.data_ptr(), _stream()),
               "sf_solve_host")

    def solve_video(self, frames: torch.Tensor, outs: torch.Tensor | None = None) -> torch.Tensor:
        """frames: float32 CUDA [n, 4, H, W]; returns fields [n, 6, ny, nx] (level pipeline)."""
        n = frames.shape[0]
        _, _, nx, ny = self.dims(0)
        if outs is None:
            outs = torch.empty((n, 6, ny, nx), device=frames.device, dtype=torch.float32)
        if tuple(frames.shape[1:]) != (4, self.height, self.width) or tuple(outs.shape) != (n, 6, ny, nx):
            raise SFError("solve_video: shape mismatch")
        _check(self.L.sf_solve_video(self.ctx, _ptr(frames, torch.float32), int(n), _ptr(outs, torch.float32),
                                     _stream()), "sf_solve_video")
        return outs

    def solve_video_host(self, frames, outs) -> None:
        """frames: float32 CPU [n, 4, H, W] (pinned for speed); outs: float32 CPU [n, 6, ny, nx]."""
        if frames.is_cuda or outs.is_cuda or not frames.is_contiguous() or not outs.is_contiguous():
            raise SFError("solve_video_host takes contiguous host tensors")
        _check(self.L.sf_solve_video_host(self.ctx, frames.data_ptr(), int(frames.shape[0]), outs.data_ptr(),
                                          _stream()), "sf_solve_video_host")

    def tune_pcg(self, imgs: torch.Tensor, reps: int = 5) -> list:
        """Autotunes the PCG schedule of every level on one frame of imgs [4, h, w]; returns the schedules."""
        base = _ptr(imgs, torch.float32)
        n = self.width * self.height * 4
        _check(self.L.sf_tune_pcg(self.ctx, base, base + n, base + 2 * n, base + 3 * n, int(reps), _stream()),
               "sf_tune_pcg")
        return [self.pcg_schedule(l) for l in range(self.levels)]

    def pcg_schedule(self, level: int) -> tuple[int, int, int]:
        k, b, t = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(self.L.sf_pcg_schedule(self.ctx, int(level), ctypes.byref(k), ctypes.byref(b), ctypes.byref(t)),
               "sf_pcg_schedule")
        return k.value, b.value, t.value

    def set_pcg_schedule(self, level: int, kind: int, blocks: int, npt: int) -> None:
        """Sets a level's PCG schedule (as pcg_schedule reports it); SFError if the level cannot run it."""
        _check(self.L.sf_set_pcg_schedule(self.ctx, int(level), int(kind), int(blocks), int(npt)),
               "sf_set_pcg_schedule")

    def set_init(self, coarsest_delta: torch.Tensor) -> None:
        _check(self.L.sf_set_init(self.ctx, _ptr(coarsest_delta, torch.float32), _stream()), "sf_set_init")

    def reset(self) -> None:
        _check(self.L.sf_reset(self.ctx), "sf_reset")

    def stats(self) -> Stats:
        st = Stats()
        rc = self.L.sf_get_stats(self.ctx, ctypes.byref(st))
        if rc not in (OK, ERR_NUMERIC, ERR_TIMEOUT):
            _check(rc, "sf_get_stats")
        return st

    def kernel_times(self, klass: int) -> tuple[float, int]:
        """(total ms, launches) of kernel class `klass` in the last frame."""
        ms, n = ctypes.c_double(), ctypes.c_int()
        _check(self.L.sf_kernel_times(self.ctx, int(klass), ctypes.byref(ms), ctypes.byref(n)), "sf_kernel_times")
        return ms.value, n.value

    def state(self, level: int) -> tuple[torch.Tensor, torch.Tensor]:
        _, _, nx, ny = self.dims(level)
        d = torch.empty((6, ny, nx), device="cuda", dtype=torch.float32)
        t = torch.empty_like(d)
        _check(self.L.sf_get_state(self.ctx, int(level), _ptr(d), _ptr(t), _stream()), "sf_get_state")
        return d, t

    # ---- step-level probes ------------------------------------------------
    def probe_pyramid(self, imgs: torch.Tensor, level: int) -> torch.Tensor:
        w, h, _, _ = self.dims(level)
        planes = torch.empty((4, 3, h, w), device="cuda", dtype=torch.float32)
        base = _ptr(imgs, torch.float32)
        n = self.width * self.height * 4
        _check(self.L.sf_probe_pyramid(self.ctx, base, base + n, base + 2 * n, base + 3 * n, int(level), _ptr(planes),
                                       _stream()), "sf_probe_pyramid")
        return planes

    def probe_feature_weights(self, level: int, T: torch.Tensor) -> torch.Tensor:
        _, _, nx, ny = self.dims(level)
        wf = torch.empty(nx * ny, device="cuda", dtype=torch.float32)
        _check(self.L.sf_probe_feature_weights(self.ctx, int(level), _ptr(T, torch.float32), _ptr(wf), _stream()),
               "sf_probe_feature_weights")
        return wf

    def probe_assemble(self, level: int, base: torch.Tensor, delta: torch.Tensor, wfeat: torch.Tensor):
        w, h, nx, ny = self.dims(level)
        G = nx * ny
        blocks = torch.empty((G, 5, 6, 6), device="cuda", dtype=torch.float32)
        rhs = torch.empty((G, 6), device="cuda", dtype=torch.float32)
        energy = torch.empty(1, device="cuda", dtype=torch.float64)
        W = torch.empty((h, w), device="cuda", dtype=torch.uint8)
        _check(self.L.sf_probe_assemble(self.ctx, int(level), _ptr(base, torch.float32), _ptr(delta, torch.float32),
                                        _ptr(wfeat, torch.float32), _ptr(blocks), _ptr(rhs), _ptr(energy), _ptr(W),
                                        _stream()), "sf_probe_assemble")
        return blocks, rhs, energy, W

    def probe_pcg(self, level: int, iters: int) -> torch.Tensor:
        _, _, nx, ny = self.dims(level)
        x = torch.empty((nx * ny, 6), device="cuda", dtype=torch.float32)
        _check(self.L.sf_probe_pcg(self.ctx, int(level), int(iters), _ptr(x), _stream()), "sf_probe_pcg")
        return x

    def probe_schwarz(self, level: int, sweeps: int, patch: int) -> torch.Tensor:
        _, _, nx, ny = self.dims(level)
        x = torch.empty((nx * ny, 6), device="cuda", dtype=torch.float32)
        _check(self.L.sf_probe_schwarz(self.ctx, int(level), int(sweeps), int(patch), _ptr(x), _stream()),
               "sf_probe_schwarz")
        return x

    def probe_vmask(self, level: int) -> torch.Tensor:
        w, h, _, _ = self.dims(level)
        V = torch.empty((h, w), device="cuda", dtype=torch.uint8)
        _check(self.L.sf_probe_vmask(self.ctx, int(level), _ptr(V), _stream()), "sf_probe_vmask")
        return V

    def vmasks(self) -> list:
        """The occlusion maps every level used in the last frame (needs occlusion=1)."""
        return [self.probe_vmask(l).cpu().numpy() for l in range(self.levels)]

    def probe_occlusion(self, level: int, T: torch.Tensor) -> torch.Tensor:
        w, h, _, _ = self.dims(level)
        O = torch.empty((h, w), device="cuda", dtype=torch.uint8)
        _check(self.L.sf_probe_occlusion(self.ctx, int(level), _ptr(T, torch.float32), _ptr(O), _stream()),
               "sf_probe_occlusion")
        return O

    def probe_illum(self, level: int, T: torch.Tensor) -> torch.Tensor:
        w, h, _, _ = self.dims(level)
        R = torch.empty((2, h, w), device="cuda", dtype=torch.float32)
        _check(self.L.sf_probe_illum(self.ctx, int(level), _ptr(T, torch.float32), _ptr(R), _stream()),
               "sf_probe_illum")
        return R

    def probe_wmask(self, level: int, step: int) -> torch.Tensor:
        w, h, _, _ = self.dims(level)
        W = torch.empty((h, w), device="cuda", dtype=torch.uint8)
        _check(self.L.sf_probe_wmask(self.ctx, int(level), int(step), _ptr(W), _stream()), "sf_probe_wmask")
        return W

    def wmasks(self) -> list:
        """The outlier masks of every Gauss-Newton step of the last frame, [level][step]."""
        return [[self.probe_wmask(l, g).cpu().numpy() for g in range(self.params.gn_iters[l])]
                for l in range(self.levels)]

    def cell_records(self) -> list:
        """The bilinear cell decisions at cell edges of every Gauss-Newton step
        of the last frame, [level][step] uint32 arrays [n, 2] (needs
        record_cells=1 at creation)."""
        import numpy as np
        out = []
        for l in range(self.levels):
            per = []
            for g in range(self.params.gn_iters[l]):
                n = ctypes.c_int()
                _check(self.L.sf_probe_cells(self.ctx, l, g, None, 0, ctypes.byref(n)), "sf_probe_cells")
                buf = np.zeros((max(n.value, 1), 2), dtype=np.uint32)
                _check(self.L.sf_probe_cells(self.ctx, l, g, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_uint)),
                                             n.value, ctypes.byref(n)), "sf_probe_cells")
                per.append(buf[:n.value])
            out.append(per)
        return out

    def probe_energy(self, level: int, base: torch.Tensor, delta: torch.Tensor, wfeat: torch.Tensor,
                     W: torch.Tensor | None = None) -> torch.Tensor:
        out = torch.empty(6, device="cuda", dtype=torch.float64)
        _check(self.L.sf_probe_energy(self.ctx, int(level), _ptr(base, torch.float32), _ptr(delta, torch.float32),
                                      _ptr(wfeat, torch.float32), _ptr(W, torch.uint8) if W is not None else None,
                                      _ptr(out), _stream()), "sf_probe_energy")
        return out


class Batch:
    """n independent sequences solved together (sf_batch_create ... sf_batch_destroy):
    one launch per frame step, one thread-block cluster per sequence."""

    def __init__(self, sizes, levels, grid_stride: int, params: Params | None = None):
        self.L = load()
        self.params = params if params is not None else preset()
        torch.cuda.init()
        self.sizes = [(int(w), int(h)) for w, h in sizes]
        self.levels = [int(l) for l in levels]
        self.n = len(self.sizes)
        self.stride = int(grid_stride)
        W = (ctypes.c_int * self.n)(*[w for w, _ in self.sizes])
        H = (ctypes.c_int * self.n)(*[h for _, h in self.sizes])
        Lv = (ctypes.c_int * self.n)(*self.levels)
        out = ctypes.c_void_p()
        _check(self.L.sf_batch_create(self.n, W, H, Lv, self.stride, ctypes.byref(self.params), ctypes.byref(out)),
               "sf_batch_create")
        self.b = out.value
        ino = (ctypes.c_size_t * self.n)()
        outo = (ctypes.c_size_t * self.n)()
        it, ot = ctypes.c_size_t(), ctypes.c_size_t()
        _check(self.L.sf_batch_layout(self.b, ino, outo, ctypes.byref(it), ctypes.byref(ot)), "sf_batch_layout")
        self.in_offsets, self.out_offsets = list(ino), list(outo)
        self.in_total, self.out_total = it.value, ot.value
        self._views = {}

    def close(self) -> None:
        if getattr(self, "b", None):
            self._views.clear()
            self.L.sf_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def pack(self, quads) -> torch.Tensor:
        """Packed device input from n arrays/tensors of shape [4, h_i, w_i]."""
        buf = torch.empty(self.in_total, device="cuda", dtype=torch.float32)
        for i, q in enumerate(quads):
            t = torch.as_tensor(q, dtype=torch.float32).reshape(-1)
            buf[self.in_offsets[i]:self.in_offsets[i] + t.numel()].copy_(t, non_blocking=True)
        return buf

    def unpack(self, out: torch.Tensor) -> list:
        """Per-sequence views [6, ny_i, nx_i] of a packed output."""
        res = []
        for i, (w, h) in enumerate(self.sizes):
            nx, ny = -(-w // self.stride), -(-h // self.stride)
            o = self.out_offsets[i]
            res.append(out[o:o + 6 * nx * ny].view(6, ny, nx))
        return res

    def solve(self, packed_in: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        if out is None:
            out = torch.empty(self.out_total, device="cuda", dtype=torch.float32)
        _check(self.L.sf_batch_solve(self.b, _ptr(packed_in, torch.float32), _ptr(out, torch.float32), _stream()),
               "sf_batch_solve")
        return out

    def set_schedule(self, cluster: int, cpb_div: int = 1) -> None:
        _check(self.L.sf_batch_set_schedule(self.b, int(cluster), int(cpb_div)), "sf_batch_set_schedule")

    def schedule(self) -> tuple[int, int]:
        c, d = ctypes.c_int(), ctypes.c_int()
        _check(self.L.sf_batch_get_schedule(self.b, ctypes.byref(c), ctypes.byref(d)), "sf_batch_get_schedule")
        return c.value, d.value

    def tune(self, packed_in: torch.Tensor, out: torch.Tensor, steps: int = 2) -> float:
        ms = ctypes.c_float()
        _check(self.L.sf_batch_tune(self.b, _ptr(packed_in, torch.float32), _ptr(out, torch.float32), int(steps),
                                    _stream(), ctypes.byref(ms)), "sf_batch_tune")
        return ms.value

    def reset(self) -> None:
        _check(self.L.sf_batch_reset(self.b), "sf_batch_reset")

    def sequence(self, i: int) -> Solver:
        """A non-owning Solver view of sequence i (stats, state, wmasks)."""
        if i not in self._views:
            ctx = self.L.sf_batch_sequence(self.b, int(i))
            if not ctx:
                raise SFError("sf_batch_sequence: bad index")
            w, h = self.sizes[i]
            self._views[i] = Solver(w, h, self.stride, self.levels[i], self.params, _view_of=ctx)
        return self._views[i]


NET_IN = (4, 60, 80)
NET_OUT = (6, 8, 10)


class Net:
    """The warm-start network (sf_net_create ... sf_net_destroy)."""

    def __init__(self, max_batch: int = 256):
        self.L = load()
        torch.cuda.init()
        out = ctypes.c_void_p()
        _check(self.L.sf_net_create(int(max_batch), ctypes.byref(out)), "sf_net_create")
        self.n = out.value
        self.max_batch = int(max_batch)
        self.n_params = int(self.L.sf_net_param_count())

    def close(self) -> None:
        if getattr(self, "n", None):
            self.L.sf_net_destroy(self.n)
            self.n = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, flat: torch.Tensor) -> None:
        assert flat.numel() == self.n_params
        _check(self.L.sf_net_set_params(self.n, _ptr(flat, torch.float32), _stream()), "sf_net_set_params")

    def get_params(self) -> torch.Tensor:
        p = torch.empty(self.n_params, device="cuda", dtype=torch.float32)
        _check(self.L.sf_net_get_params(self.n, _ptr(p), _stream()), "sf_net_get_params")
        return p

    def forward(self, imgs: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        B = imgs.shape[0]
        if out is None:
            out = torch.empty((B,) + NET_OUT, device="cuda", dtype=torch.float32)
        _check(self.L.sf_net_forward(self.n, _ptr(imgs, torch.float32), B, _ptr(out, torch.float32), _stream()),
               "sf_net_forward")
        return out

    def gradients(self, imgs: torch.Tensor, target: torch.Tensor):
        g = torch.empty(self.n_params, device="cuda", dtype=torch.float32)
        loss = torch.empty(1, device="cuda", dtype=torch.float32)
        _check(self.L.sf_net_gradients(self.n, _ptr(imgs, torch.float32), _ptr(target, torch.float32),
                                       imgs.shape[0], _ptr(g), _ptr(loss), _stream()), "sf_net_gradients")
        return g, loss

    def train_step(self, imgs: torch.Tensor, target: torch.Tensor, lr: float, loss: torch.Tensor | None = None):
        if loss is None:
            loss = torch.empty(1, device="cuda", dtype=torch.float32)
        _check(self.L.sf_net_train_step(self.n, _ptr(imgs, torch.float32), _ptr(target, torch.float32),
                                        imgs.shape[0], ctypes.c_float(lr), _ptr(loss), _stream()),
               "sf_net_train_step")
        return loss

    def status(self) -> None:
        _check(self.L.sf_net_status(self.n), "sf_net_status")

    def warm_start(self, solver: "Solver", imgs: torch.Tensor) -> None:
        """Sets solver's coarsest initial delta for its next solve from the quadruple imgs [4, h, w]."""
        base = _ptr(imgs, torch.float32)
        n = solver.width * solver.height * 4
        _check(self.L.sf_warm_start(self.n, solver.ctx, base, base + n, base + 2 * n, base + 3 * n, _stream()),
               "sf_warm_start")


def coarsest_images(solver: "Solver", imgs: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
    """The four coarsest-level intensities [4, h, w] of a quadruple imgs [4, H, W]."""
    w, h, _, _ = solver.dims(solver.levels - 1)
    if out is None:
        out = torch.empty((4, h, w), device="cuda", dtype=torch.float32)
    base = _ptr(imgs, torch.float32)
    n = solver.width * solver.height * 4
    _check(load().sf_coarsest_images(solver.ctx, base, base + n, base + 2 * n, base + 3 * n, _ptr(out, torch.float32),
                                     _stream()), "sf_coarsest_images")
    return out
