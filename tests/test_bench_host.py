"""Host-side logic of bench.py that needs no GPU: the oracle samples behind
the CPU baselines and the reference arm.

A sample steps with the full-size patch's timestep, C min(h/c) with the
full-size h (R7), held fixed.  When the sample is the full-size patch
itself (the 20^3 workload), that step must be the oracle's own first
Courant step, which pins the formula to the oracle's EOS (R9) and Courant
rule rather than to a retyped copy of them.
"""
import argparse
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _args(config="c1", steps=2):
    return argparse.Namespace(config=config, kernel="wendland", grad_h=False, steps=steps)


def test_sample_timestep_is_the_oracles_first_courant_step():
    import bench
    import oracle
    from paper_1905_03344_gb300 import inputs
    pairs, el, k, n_edge, dt = bench.oracle_sample(_args(), 1, 100, warmup=0, nsteps=1)
    assert n_edge == 20 and k == 1 and pairs > 0 and el > 0.0
    sim = oracle.Sim(inputs.square_patch(20))
    sim.step(1)
    assert abs(dt - sim.dt) <= 1e-12 * sim.dt, (dt, sim.dt)


def test_sample_timestep_follows_h():
    """A smaller sample of a larger workload steps with the larger patch's
    step: the sample's own Courant step scaled by the ratio of the edges."""
    import bench
    _, _, _, n_small, dt_small = bench.oracle_sample(_args("c1"), 1, 10, warmup=0, nsteps=1)
    _, _, _, n_full, dt_full = bench.oracle_sample(_args("c1"), 1, 20, warmup=0, nsteps=1)
    assert (n_small, n_full) == (10, 20)
    # both samples take the 20^3 patch's step; the lattice u differs only by
    # where the points sit, so c_max agrees to the series' resolution
    assert np.isclose(dt_small, dt_full, rtol=2e-2), (dt_small, dt_full)


def test_baselines_stop_at_the_step_count():
    import bench
    a = _args("c1", steps=3)
    b = bench.cpu_baseline(a)
    assert b["sample"].startswith("3 full oracle steps") and b["kind"] == "oracle" and b["value"] > 0
    b1 = bench.cpu_baseline_1thread(a)
    assert b1["cores"] == 1 and b1["sample"].startswith("3 full oracle steps") and b1["value"] > 0


def test_reference_arm_line():
    import json
    import subprocess
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--config", "c1",
                        "--steps", "2"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["steps"] == 2 and line["warmup"] == 3 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["value"] == line["value"] and line["e2e"]["h2d_bytes_per_step"] == 0
