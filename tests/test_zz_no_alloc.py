"""sf_pcg_static, the PCG entry point that allocates nothing, against the
context's PCG (sf_probe_pcg) and the FP64 oracle's PCG on the same systems.

It serves callers that cannot allocate device memory where they solve:
real-time loops that must not meet the allocator's implicit device
synchronisation, and host applications whose memory pool or fixed device
budget forbids a library's raw allocations after start-up. Its scratch is a
fixed device array inside the library, shared by every call.

This file sorts last, so a run that stops at the first failure has already
run every other test. It also passes alone in a fresh process.
"""

import numpy as np
import pytest
import torch

import oracle as O
from paper_1610_07159_gb300 import scenes, sf
from tests.gpu_common import lib_blocks_to_oracle, make_params, rel_max

pytestmark = pytest.mark.gpu

ITERS = 20
TOL = 2e-4 * ITERS  # the tolerance of the PCG parity tests for this many iterations


def _system(solver, level, seed):
    _, _, nx, ny = solver.dims(level)
    G = nx * ny
    rng = np.random.default_rng(seed)
    base = (rng.uniform(-1, 1, (6, 1)) + 0.2 * rng.standard_normal((6, G))).astype(np.float32)
    delta = (0.2 * rng.standard_normal((6, G))).astype(np.float32)
    wf = (1.0 + rng.random(G)).astype(np.float32)
    blocks, rhs, _, _ = solver.probe_assemble(level, torch.from_numpy(base).cuda(), torch.from_numpy(delta).cuda(),
                                              torch.from_numpy(wf).cuda())
    return nx, ny, blocks, rhs


def test_static_pcg_matches_the_context_pcg_on_consecutive_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    w, h = 160, 120
    q = torch.from_numpy(scenes.random_quadruple(w, h, 5, sigma=0.01)).cuda()
    sp, _ = make_params([1], [1])
    solver = sf.Solver(w, h, 4, 3, sp)
    solver.probe_pyramid(q, 0)
    results = []
    # two calls in a row on one system, then one on a smaller system: the
    # shared scratch keeps the previous call's contents between calls
    for level, seed in ((0, 11), (0, 11), (1, 12)):
        nx, ny, blocks, rhs = _system(solver, level, seed)
        x_ctx = solver.probe_pcg(level, ITERS)
        x_static = sf.pcg_static(nx, ny, blocks, rhs, ITERS)
        torch.cuda.synchronize()
        assert rel_max(x_static.cpu().numpy(), x_ctx.cpu().numpy()) < TOL
        # and against the FP64 oracle's PCG on the same blocks and right-hand side
        A = lib_blocks_to_oracle(blocks.cpu().numpy().astype(np.float64), nx, ny)
        x_ref, _, its = O.pcg(nx, ny, A, rhs.cpu().numpy().astype(np.float64), ITERS)
        assert its == ITERS and rel_max(x_static.cpu().numpy(), x_ref) < TOL
        results.append(x_static.cpu().numpy())
    assert np.array_equal(results[0], results[1])  # deterministic across calls


def test_static_pcg_rejects_systems_beyond_its_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    L = sf.load()
    n = sf.STATIC_PCG_MAX_NODES + 1
    buf = torch.zeros(n * 5 * 36, device="cuda")
    assert L.sf_pcg_static(n, 1, buf.data_ptr(), buf.data_ptr(), 1, buf.data_ptr(), None) == sf.ERR_ARG
    assert L.sf_pcg_static(0, 4, buf.data_ptr(), buf.data_ptr(), 1, buf.data_ptr(), None) == sf.ERR_ARG
