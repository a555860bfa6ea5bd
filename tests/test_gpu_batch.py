"""Independent optimisations side by side (CUDA graphs on separate streams) equal the
same optimisations run one at a time with eager launches, bit for bit: every kernel
of the path is deterministic and the specifications share nothing."""

import pytest
import torch

from paper_1707_09898_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    import __graft_entry__

    __graft_entry__.build()


def test_batched_runs_equal_sequential_runs():
    from paper_1707_09898_gb300.batch import BatchedRuns, sequential

    wls = [W.config5(s) for s in list(W.CONFIG5_HELDOUT_SEEDS)[:4]]
    assert len({wl.mask_z for wl in wls}) > 1 or len({wl.mask_xy for wl in wls}) > 1  # different targets
    runs = BatchedRuns(wls, steps_per_graph=5)
    runs.run(20)
    torch.cuda.synchronize()
    for wl, r in zip(wls, runs.rho):
        ref = sequential(wl, 20)
        torch.cuda.synchronize()
        assert torch.equal(r, ref), wl.name
        assert not torch.equal(r, torch.from_numpy(wl.rho()).to(r.device))  # the run moved
    Js = runs.objectives()
    assert all(J > 0 for J in Js)
    with pytest.raises(ValueError):
        runs.run(7)
