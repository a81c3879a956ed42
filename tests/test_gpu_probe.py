"""The integer issue-rate probe (et_probe.h) used beside the nominal peak in
the tube-count roofline: its rates are positive, below the device's nominal
lane rate with a margin for clock reporting, and ordered as the op mixes
imply (a step of xor + add + multiply-add costs at least as much as either
part)."""
import pytest

pytestmark = pytest.mark.gpu


def test_int_throughput_rates():
    from paper_1311_5334_gb300 import et
    with et.Context(0) as c:
        r = c.int_throughput()
        sms = c.info()["sm_count"]
    nominal = sms * 128 * 2.2e9 * 2   # ops/s: 128 lanes per SM, <= 2.2 GHz, two pipes at most
    for k in ("alu", "mad", "mix"):
        assert 0 < r[k] < nominal, (k, r[k])
    # a mix step (3 ops) takes at least as long as each of its parts
    assert r["mix"] / 3 <= min(r["alu"] / 2, r["mad"]) * 1.05
