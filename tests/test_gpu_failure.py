"""Failure detection without a GPU fault: the kernels' waits on
asynchronous copies are bounded.  A wait on a transaction that nothing
completes must give up (the patch step then records GEOFLOOD_ERR_TIMEOUT
and returns) and the context must stay usable; a non-finite state is
reported as an error, not stepped on."""
import numpy as np
import pytest

from paper_2403_15435_gb300 import geoflood, inputs

pytestmark = pytest.mark.gpu


def test_bounded_wait_gives_up_and_the_gpu_stays_usable():
    assert geoflood.check_bounded_wait() == 0
    assert geoflood.check_bounded_wait() == 0
    prob = inputs.stoker(64, patch=32)
    g = geoflood.Forest(prob.cfg, prob.dem)
    g.set_state(prob.ic)
    t, n = g.step(2.0)
    assert t == 2.0 and n > 0


def test_non_finite_state_is_an_error():
    prob = inputs.stoker(64, patch=32)
    g = geoflood.Forest(prob.cfg, prob.dem)
    g.set_state(prob.ic)
    h, hu, hv, _ = g.read()
    hu[0, 5, 5] = np.nan
    g.write(h, hu, hv)
    with pytest.raises(geoflood.GeoFloodError) as e:
        g.step(2.0)
    assert e.value.code == -5  # GEOFLOOD_ERR_NAN
