"""The ALU issue-rate probe behind the pair kernel's roofline denominator:
both kinds report a rate between a quarter of and just above the nominal
152 SMs x 128 lanes x 2.07 GHz, and bad arguments are refused."""
import pytest

import paper_1311_0402_gb300 as dpd
from gpu_util import need_gpu

pytestmark = pytest.mark.gpu

NOMINAL = 152 * 128 * 2.07e9


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


@pytest.mark.parametrize("kind", [0, 1])
def test_issue_rate_is_near_the_lane_count(kind):
    r = dpd.dpd_alu_peak(kind, 10)
    assert 0.25 * NOMINAL < r["lane_ops_per_s"] < 1.1 * NOMINAL, r
    assert r["ms_per_launch"] > 0.0


def test_bad_arguments_are_refused():
    for kind, reps in ((2, 10), (0, 0), (1, 1001)):
        with pytest.raises(dpd.DPDError):
            dpd.dpd_alu_peak(kind, reps)
