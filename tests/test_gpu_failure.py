"""Failure detection on the GPU without a fault: a bounded device-side wait
that runs out reports LGS_ERR_TIMEOUT in the status words and returns, and the
CUDA context stays usable."""
import pytest
import torch

from paper_2606_16566_gb300 import lgs, scenes
from paper_2606_16566_gb300 import _lib as L

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("spin_limit", [0, 1000])
def test_bounded_wait_reports_timeout_and_context_survives(spin_limit):
    st = lgs.selftest_wait_timeout(spin_limit)
    assert st[L.ST_CODE] == L.LGS_ERR_TIMEOUT
    assert st[L.ST_DETAIL] == 1
    sc, cams = scenes.random_small(500, seed=1)
    res = lgs.render(lgs.to_device(sc), cams)        # raises on any device status
    torch.cuda.synchronize()
    assert res["K"] > 0


def test_capacity_one_short_reports_needed_count():
    sc, cams = scenes.random_small(800, seed=2)
    g = lgs.to_device(sc)
    K = lgs.render(g, cams)["K"]
    with pytest.raises(L.LgsError) as e:
        lgs.render(g, cams, capacity=K - 1)
    assert e.value.code == L.LGS_ERR_CAPACITY
