"""The timeout path of the bounded device waits, made to run out on purpose
without a fault: a wait on an mbarrier that nothing completes gives up after
its bound and records TTO_E_TIMEOUT; the host reads it, the context stays
usable, a tcgen05 sweep launched while the timeout is recorded returns at once,
and evaluation is exact again once the status is cleared."""
import numpy as np
import pytest

from oracle import dcflow
from synth import config_grid, limits_from_flows, random_topologies

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")


def test_bounded_wait_runs_out_and_the_context_survives():
    from paper_2605_10128_b300 import Grid, TTOError, _lib
    sg = config_grid("tto30")
    sg = sg.with_limits(limits_from_flows(dcflow.base_flows(sg)[0], 5))
    g = Grid(sg)
    topo = torch.tensor(random_topologies(sg, 64, seed=3), dtype=torch.int32, device="cuda")
    g.set_sweep_shape(3, 4)  # the tcgen05 sweep
    ref = g.evaluate(topo, precision=3, fmax=True)
    g.sync_status()
    ref_fmax = ref["fmax"].cpu().numpy()

    g.debug_bounded_wait(cycles=2_000_000)  # about a millisecond
    with pytest.raises(TTOError) as e:
        g.sync_status()
    assert e.value.code == _lib.TTO_E_TIMEOUT
    g.sync_status()  # cleared by the read

    # while a timeout is recorded, the sweep's CTAs return at once
    g.debug_bounded_wait(cycles=2_000_000)
    out = g.evaluate(topo, precision=3, fmax=True)
    out["fmax"].zero_()
    out = g.evaluate(topo, precision=3, fmax=True, out=out)
    torch.cuda.synchronize()
    assert not np.any(out["fmax"].cpu().numpy())
    with pytest.raises(TTOError):
        g.sync_status()

    # cleared: exact again, and the context is fine
    again = g.evaluate(topo, precision=3, fmax=True)
    g.sync_status()
    np.testing.assert_array_equal(again["fmax"].cpu().numpy(), ref_fmax)
    with pytest.raises(TTOError):
        g.debug_bounded_wait(cycles=0)
