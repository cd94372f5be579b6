"""bench.py's kick/push roofline model (no GPU): the FP64-pipe instruction
counts per element were measured with ncu on the kernel sources the model
names, and those must be the sources in the tree (a kernel change without a
new capture would make the reported ALU fraction a guess); the model
reproduces the measured per-segment counts of the c2 ring's three segment
types and the ring's element mix."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2010_11540_gb300 import synth  # noqa: E402

# ncu sm__thread_inst_executed_pipe_fp64_pred_on / particle of the three c2
# segment types (A: QF, drift, SF, drift; B: drift, QD, drift, SD, drift;
# C: drift), split-TF32 form, mean of two captures (profiles/kick_push_c2.md)
MEASURED = {"A": 55.775, "B": 67.97, "C": 17.96}


def test_model_fitted_on_the_sources_in_the_tree():
    assert bench.kp_sources_sha() == bench.FP64_INST_SOURCES_SHA, (
        "kick/push sources changed since the FP64 counts were measured: re-capture them with ncu "
        "(profiles/kick_push_c2.md) and update bench.py")
    assert bench.KP_TRAFFIC_TF32["c2"][1] == bench.FP64_INST_SOURCES_SHA


def test_model_reproduces_the_segments():
    f, d, q, s = (bench.FP64_INST_BASE_F32, bench.FP64_INST["drift"], bench.FP64_INST["quad"],
                  bench.FP64_INST["sext"])
    model = {"A": f + q + 2 * d + s, "B": f + q + 3 * d + s, "C": f + d}
    for seg, v in MEASURED.items():
        assert model[seg] == pytest.approx(v, abs=0.1), (seg, model[seg], v)


def test_c2_ring_mix_and_count_per_kick():
    lat = synth.lattice("c2")
    mix = bench.element_mix(lat)
    assert mix == {"drift": 432, "quad": 144, "sext": 144, "bend": 0, "rf": 0, "kicks": 216}
    per_turn, kicks = bench.fp64_inst_per_turn(lat, "tf32x3")
    assert kicks == 216
    assert per_turn / kicks == pytest.approx(np.mean(list(MEASURED.values())), abs=0.1)
