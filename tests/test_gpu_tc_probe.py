"""The wide-N tensor-core probe (plan_probe_tc_wide): it runs to the end on
every SM, reports positive cycle counts for every part, and the split mode
(three passes) costs more than one pass."""
import pytest

from paper_2212_02224_gb300 import binding

pytestmark = pytest.mark.gpu


def test_probe_reports_every_part():
    one = binding.plan_probe_tc_wide(1, 20)
    three = binding.plan_probe_tc_wide(3, 20)
    assert one["ctas"] >= 1 and three["ctas"] == one["ctas"]
    for res in (one, three):
        for key in ("forward_cycles", "transposed_n16_cycles", "transposed_n128_cycles",
                    "transposed_n16_4acc_cycles", "transposed_n128_4acc_cycles"):
            assert res[key] > 0.0, key
    assert three["transposed_n16_cycles"] > one["transposed_n16_cycles"]


@pytest.mark.parametrize("passes,iters", [(2, 10), (1, 0), (3, 10001)])
def test_probe_rejects_bad_arguments(passes, iters):
    with pytest.raises(binding.PlanError) as e:
        binding.plan_probe_tc_wide(passes, iters)
    assert e.value.status == binding.PLAN_EINVAL
