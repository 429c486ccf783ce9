"""The reference arm of bench.py (the FP64 oracle on one host core) prints
one JSON line on the same workload config, metric and unit as the GPU arm,
with its cpu_baseline and an end-to-end entry that moves no bytes."""
import io
import json
import contextlib

import bench


import pytest


@pytest.mark.parametrize("procs", [1, 2])
def test_reference_arm_line(procs):
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        out = bench.main(["--impl", "reference", "--steps", "1", "--warmup", "0", "--ref-outer", "1",
                          "--ref-inner", "5", "--ref-procs", str(procs)])
    line = json.loads(buf.getvalue().strip().splitlines()[-1])
    assert line == json.loads(json.dumps(out))
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["higher_is_better"] is True and line["value"] > 0
    # the GPU arm's config at the parser defaults (608 slices through 304 slots)
    ours = bench.workload_config(type("A", (), {"queue": 608, "batch": 304, "outer": bench.OUTER,
                                                "inner": bench.INNER, "inner_late": bench.INNER_LATE,
                                                "outer_late": bench.OUTER_LATE,
                                                "boundary_period": bench.BOUNDARY_PERIOD,
                                                "outer_tol": bench.OUTER_TOL, "stall_tol": bench.STALL_TOL,
                                                "steady": 0, "precond": "paper"})(), 1)
    assert line["config"] == ours
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == procs
    assert line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_auxiliary_measurement_failure_is_reported_not_fatal(capsys):
    """A measurement beside the main line that raises leaves an error entry
    in its key; the main line still prints."""
    def boom(x):
        raise KeyError(x)
    r = bench._aux(boom, "missing")
    assert r == {"error": "KeyError: 'missing'"} and not bench._ok(r)
    assert "KeyError" in capsys.readouterr().err
    assert bench._aux(lambda a, b: {"value": a + b}, 1, 2) == {"value": 3} and bench._ok({"value": 3})
    assert not bench._ok(None)
