"""Failure detection, exercised without a GPU fault.

The device-wide waits of the library are bounded: a wait that runs out latches
a status bit and returns, so a lost block never hangs the GPU. The tests run
the library's own grid barrier, the waits of the self-tagged PCG exchange and
the mbarrier wait with a limit of about a millisecond on a condition they
control (a block that never arrives or publishes, an mbarrier that nothing
completes), and feed non-finite images, which the
solve must report as SF_ERR_NUMERIC and then recover from after sf_reset.
Nothing here traps, faults or waits without a bound."""

import numpy as np
import pytest
import torch

from paper_1610_07159_gb300 import scenes, sf
from tests.gpu_common import make_params

pytestmark = pytest.mark.gpu

LIMIT = 2_000_000  # SM clock cycles: about a millisecond


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sf.load()
    yield
    torch.cuda.synchronize()


def test_grid_barrier_passes_when_every_block_arrives():
    status, returned = sf.barrier_timeout_probe(-1, LIMIT)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert status == sf.OK and returned == sms


def test_grid_barrier_times_out_when_a_block_never_arrives():
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    for skip in (0, sms - 1):
        status, returned = sf.barrier_timeout_probe(skip, LIMIT)
        assert status == sf.ERR_TIMEOUT, status
        assert returned == sms - 1  # every waiting block came back
    # the GPU stays usable: the next barrier passes
    assert sf.barrier_timeout_probe(-1, LIMIT) == (sf.OK, sms)


@pytest.mark.parametrize("mode", [0, 1])
def test_self_tagged_waits_time_out_when_a_block_never_publishes(mode):
    """The waits of the self-tagged PCG exchange (kinds 5 and 6): the poll of
    the partial-sum words (mode 0) and a halo reader's wait for a word (mode
    1) pass when every block publishes, and run out, latch SF_ERR_TIMEOUT and
    return in every block when one block never does."""
    nb = min(torch.cuda.get_device_properties(0).multi_processor_count, 160)
    assert sf.tagged_timeout_probe(mode, -1, LIMIT) == (sf.OK, nb)
    for skip in (0, nb - 1):
        status, returned = sf.tagged_timeout_probe(mode, skip, LIMIT)
        assert status == sf.ERR_TIMEOUT, status
        assert returned == nb  # every block came back
    assert sf.tagged_timeout_probe(mode, -1, LIMIT) == (sf.OK, nb)


def test_mbarrier_wait_completes_or_times_out():
    assert sf.mbarrier_timeout_probe(True, LIMIT) == 1
    assert sf.mbarrier_timeout_probe(False, LIMIT) == 0
    assert sf.mbarrier_timeout_probe(True, LIMIT) == 1


@pytest.mark.parametrize("bad", [float("nan"), float("inf"), -float("inf")])
@pytest.mark.parametrize("solver", [0, 1])
def test_non_finite_images_latch_numeric_and_reset_recovers(bad, solver):
    q = scenes.plane_quadruple()
    sp, _ = make_params([2], [10] if solver == 0 else [3], solver=solver, patch_iters=[4])
    s = sf.Solver(160, 120, 4, 3, sp)
    qb = q.copy()
    qb[2, 40:44, 60:70] = bad
    s.solve(torch.from_numpy(qb).cuda())
    st = s.stats()
    assert st.status == sf.ERR_NUMERIC, sf.status_string(st.status)
    s.reset()
    f = s.solve(torch.from_numpy(q).cuda()).cpu().numpy()
    st = s.stats()
    assert st.status == sf.OK and np.all(np.isfinite(f)) and np.isfinite(st.energy)
