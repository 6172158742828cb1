"""Host logic of bench.py that the reported numbers depend on: the cube
census behind the roofline's algorithmic bytes (checked against the oracle's
own footprint assembly, Algorithm 1), the DRAM-traffic record's validity rule
and the JSON contract of the command line."""
import json
import os

import numpy as np

import bench
import oracle
from paper_2009_02702_gb300 import synth


def test_cube_census_matches_the_oracle_footprint():
    dims = (512, 512, 384)
    boxes = synth.make_boxes(2)[:200]
    extra = np.array([[0, 0, 0, 512, 512, 384], [511, 511, 383, 1, 1, 1], [3, 7, 5, 600, 2, 900]], np.int32)
    boxes = np.concatenate([boxes, extra])
    census = bench.cube_levels(boxes, dims)
    want = np.zeros(40, np.int64)
    for b in boxes:
        cubes = oracle.fa_cubes(b, *dims)
        want += np.bincount(cubes[:, 0], minlength=40)[:40]
    assert np.array_equal(census, want)


def test_traffic_record_applies_only_to_its_source_and_workload():
    with open(os.path.join(bench.ROOT, "profiles", "traffic.json")) as f:
        recs = json.load(f)["records"]
    assert recs
    for rec in recs:
        k, c, Q = rec["kernel"], rec["config"], rec["queries"]
        t = bench.measured_traffic(k, c, Q)
        assert t is None or t == rec["dram_bytes_per_launch"]
        assert bench.measured_traffic(k, c, Q + 1) is None
        assert bench.measured_traffic(k, 99, Q) is None
        assert bench.measured_traffic("no_such_kernel", c, Q) is None


def test_error_sample_spans_the_size_range():
    boxes = synth.make_boxes(3)
    pick, vol = bench.error_sample(boxes, synth.CONFIGS[3]["dims"], 500, 21)
    assert len(pick) == 500 and len(np.unique(pick)) == 500
    # every decile of box volume contributes, so the largest boxes are in it
    assert vol[pick].max() >= np.percentile(vol, 90) and vol[pick].min() <= np.percentile(vol, 10)


def test_command_line_defaults_fit_the_contract():
    a = bench.parse([])
    assert a.gpus == 1 and a.steps >= 1 and a.warmup >= 3
    # the headline is the largest single-GPU workload: 2048x2048x300, 100,000 boxes
    assert a.config == 3 and synth.CONFIGS[a.config]["queries"] == 100000 and a.secondary == 2
    r = bench.parse(["--impl", "reference", "--steps", "2", "--warmup", "3"])
    assert r.impl == "reference" and r.steps == 2
    assert bench.whole_job_rate(1, 10000, 0.5) == 10000 / 0.5e-3
