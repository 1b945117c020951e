"""Host-side helpers of bench.py without a GPU: the clock-sample summary used for the
bench line's clocks record, and the algorithmic flop count's descriptor size."""
import bench
from paper_2603_01234_gb300 import inputs


def line(sm, smax=2070, power=900.0, hw="Not Active", hwt="Not Active", swt="Not Active", cap="Not Active"):
    return f"0, {sm}, {smax}, {power}, 0x0000000000000000, {hw}, {hwt}, {swt}, {cap}"


def test_clock_summary_uses_the_timed_region():
    samples = [(0.0, line(1000)), (1.0, line(2070)), (1.1, line(2055, cap="Active")), (1.2, line(2070, power=1200.0)),
               (5.0, line(600, hwt="Active"))]
    c = bench.summarize_clocks(samples, 0.95, 1.25)
    assert c["samples"] == 3 and c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"] and c["power_w_max"] == 1200.0 and c["window"] == "timed region"
    # a throttle reason inside the window is reported; outside it is not
    c = bench.summarize_clocks(samples, 4.0, 6.0)
    assert c["reasons"] == ["hw_thermal_slowdown"] and c["sm_mhz"] == 600.0


def test_clock_summary_without_samples_in_the_window():
    samples = [(0.0, line(1900)), (2.0, line(2000))]
    c = bench.summarize_clocks(samples[:2], 0.5, 1.5)
    assert c["samples"] == 2 and c["sm_mhz"] == 1950.0 and "none fell inside" in c["window"]
    assert bench.summarize_clocks([], 0.0, 1.0)["samples"] == 0
    assert bench.summarize_clocks([(0.1, "0, N/A, 2070, 1, 0x0, Not Active")], 0.0, 1.0)["samples"] == 0


def test_flop_count_follows_the_descriptor_size():
    base = inputs.random_model(seed=1)
    mb = inputs.random_model(seed=1, l_max_4b=2, l_max_5b=1)
    a = bench.algorithmic_flops(base, 7700, 1800, 100)
    b = bench.algorithmic_flops(mb, 7700, 1800, 100)
    # only the network's per-bead term grows: H (4 N_des + 6) with N_des 21 -> 29
    assert b["force_virial"] == a["force_virial"]
    assert b["descriptor_network"] - a["descriptor_network"] == 100 * base.hidden * 4 * (mb.n_des - base.n_des)
