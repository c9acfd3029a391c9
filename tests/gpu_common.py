"""Shared helpers of the GPU parity tests: one parameter set mapped to both the
CUDA library's sf_params and the oracle's parameters, and block-format
conversions. No arithmetic of the method lives here."""

from __future__ import annotations

import numpy as np

import oracle as O

PRESET_IDS = {"fig2": 0, "fig568": 1, "fig79": 2}
# node blocks of the library: self, E, S, SE, SW; oracle neighbour slot = 3*(dy+1) + (dx+1)
LIB_SLOTS = (4, 5, 7, 8, 6)


def make_params(gn, pcg, preset: str = "fig2", **kw):
    """(sf.Params, oracle.Params) for the same configuration."""
    from paper_1610_07159_gb300 import sf
    d = dict(O.TABLE1[preset])
    lib_only = {k: kw.pop(k) for k in ("use_graph", "precision", "pcg_mode", "profile_mask", "video",
                                       "record_cells") if k in kw}
    if "patch_iters" in kw:  # per level, like gn and pcg
        kw["patch_iters"] = tuple(list(kw["patch_iters"]) + [kw["patch_iters"][-1]] * 8)[:8]
    d.update(kw)
    op = O.Params(gn_iters=tuple(list(gn) + [gn[-1]] * 8)[:8], pcg_iters=tuple(list(pcg) + [pcg[-1]] * 8)[:8], **d)
    sp = sf.preset(PRESET_IDS[preset], gn_iters=list(gn), pcg_iters=list(pcg), **{**kw, **lib_only})
    return sp, op


def lib_blocks_to_oracle(blocks: np.ndarray, nx: int, ny: int) -> np.ndarray:
    """[G, 5, 6, 6] (self, E, S, SE, SW) -> the oracle's [G, 9, 6, 6] neighbour slots."""
    G = nx * ny
    A = np.zeros((G, 9, 6, 6))
    for k, slot in enumerate(LIB_SLOTS):
        A[:, slot] = blocks[:, k]
    for n in range(G):
        i, j = n % nx, n // nx
        if i > 0:
            A[n, 3] = blocks[n - 1, 1]
        if j > 0:
            A[n, 1] = blocks[n - nx, 2]
            if i > 0:
                A[n, 0] = blocks[n - nx - 1, 3]
            if i + 1 < nx:
                A[n, 2] = blocks[n - nx + 1, 4]
    return A


def rel_max(a, b) -> float:
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-30))
