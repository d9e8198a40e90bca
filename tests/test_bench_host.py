"""Host-side parts of the benchmark that need no GPU: the oracle baseline on
several host cores (one spawned process per core, each on its own sample, the
slowest process's time for the job), the reference arm's JSON line, the
parsing of the clock samples taken during the timed region, and the DRAM
traffic lookup, which answers only for the pair-kernel sources it was
captured on."""
import types

import pytest


def test_oracle_on_cores_counts_every_process():
    import bench
    value, sec, cores, n = bench.oracle_on_cores(1, cores=2)
    assert cores == 2 and n == 78125
    assert sec > 0 and value == pytest.approx(n * cores * 1 / sec)


def test_reference_arm_line():
    import bench
    args = types.SimpleNamespace(steps=1, warmup=0, gpus=1)
    line = bench.run_reference(args, 0)
    assert line["impl"] == "reference" and line["unit"] == bench.UNIT and line["metric"] == bench.METRIC
    assert line["cpu_baseline"]["cores"] == bench.host_cores()
    assert line["cpu_baseline"]["value"] == line["value"] == line["e2e"]["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert bench.run_reference(args, 1) is None          # other ranks do no work


def test_clock_summary_reads_reasons():
    import bench
    c = bench.ClockSampler(0)
    c.lines = ["0, 2070, 2070, 910.2, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
               "0, 2055, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
               "0, 1980, 2070, 1401.5, 0x0000000000000024, Not Active, Not Active, Active, Not Active",
               "garbage line", ""]
    out = c.summary()
    assert out["samples"] == 3 and out["sm_mhz"] == 2055.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap", "sw_thermal_slowdown"]
    assert bench.ClockSampler(0).summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_traffic_only_for_the_current_kernel_sources(tmp_path):
    import bench
    args = types.SimpleNamespace(beta=0.15, precision="mixed")
    f = tmp_path / "k_pair_lists_plate_impact_387k.md"
    f.write_text(f"kernel_sha1: {bench.kernel_rev()}\ntraffic_bytes_per_launch_1125k: 123456\n")
    assert bench.pair_traffic_bytes(args, str(tmp_path)) == 123456
    f.write_text("kernel_sha1: 000000000000\ntraffic_bytes_per_launch_1125k: 123456\n")
    assert bench.pair_traffic_bytes(args, str(tmp_path)) is None          # another source revision
    assert bench.pair_traffic_bytes(types.SimpleNamespace(beta=0.15, precision="fp64"), str(tmp_path)) is None
    assert bench.pair_traffic_bytes(types.SimpleNamespace(beta=0.0, precision="mixed"), str(tmp_path)) is None
