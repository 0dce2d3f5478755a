"""Failure detection without a GPU fault: the bounded mbarrier wait of the
pipelined kernels gives up when nothing arrives, reports it through a device
flag, and the context stays usable afterwards."""
import numpy as np
import pytest
import torch

import gtt_inputs as gi
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    from paper_2507_02420_gb300 import build
    build.build()
    import paper_2507_02420_gb300 as g
    torch.cuda.set_device(0)
    return g


@pytest.mark.parametrize("polls", [1, 64, 4096])
def test_bounded_wait_expires_and_is_reported(g, polls):
    assert g.selftest_bounded_wait(polls) is True


def test_context_is_usable_after_an_expired_wait(g):
    assert g.selftest_bounded_wait(256)
    rng = np.random.default_rng(9900)
    W = gi.haar_unitary(4, rng).astype(np.complex64)
    x = gi.complex_normal_x((2, 4 ** 9), rng, np.complex64)
    plan = g.Plan(W, 9, "c64", 2)
    y = plan.forward(torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    plan.check()  # the plan's own flag is untouched by the self-test
    ref = oracle.modes(W.astype(np.complex128), x.astype(np.complex128))
    assert np.linalg.norm(y.cpu().numpy() - ref) / np.linalg.norm(ref) <= 2e-6


def test_selftest_rejects_bad_arguments(g):
    for polls in (0, -3, (1 << 20) + 1):
        with pytest.raises(g.GTTError) as ei:
            g.selftest_bounded_wait(polls)
        assert ei.value.status == 1
