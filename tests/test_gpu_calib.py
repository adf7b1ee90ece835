"""fbn_measure_unit_rates: the measured throughput of the counting units.

The rates are the denominators of the counting kernels' rooflines; they must
come out positive and, per SM and clock, within what a GPU of this kind can
do (a shared-memory reduction or a POPC takes at least one lane slot: at most
128 per SM and clock; the bit-plane count assumes tens of POPC per SM and
clock, the histograms a few reductions)."""
import pytest

pytestmark = pytest.mark.gpu


def test_unit_rates_are_plausible():
    from paper_2212_04259_gb300 import build
    build.build()
    import paper_2212_04259_gb300 as F
    r = F.fbn_measure_unit_rates()
    per = r["sms"] * r["sm_clock_hz"]
    assert r["sms"] > 0 and r["sm_clock_hz"] > 0
    assert 1.0 <= r["smem_red_per_s"] / per <= 128.0, r
    assert 4.0 <= r["popc_per_s"] / per <= 128.0, r
    with pytest.raises(F.FbnError) as e:
        F.fbn._check(F.fbn.lib().fbn_measure_unit_rates(-1, None, 4))
    assert e.value.code == -1
