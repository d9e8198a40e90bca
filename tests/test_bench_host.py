"""Host-side parts of the benchmark that need no GPU: the oracle baseline on
several host cores (one spawned process per core, each on its own sample, the
slowest process's time for the job) and the reference arm's JSON line."""
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
