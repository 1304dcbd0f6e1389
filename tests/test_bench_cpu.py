"""bench.py's own measurement logic, without a GPU: the DRAM traffic it
reports comes only from a capture of the kernel source as it stands, and the
ALU term counts rounds and accepts the way its docstring states."""
import hashlib
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402
import oracle as O  # noqa: E402


def test_traffic_needs_the_captured_source():
    for kind, e in bench.NCU_TRAFFIC.items():
        path = os.path.join(ROOT, "paper_2509_12086_gb300", "csrc", e["src"])
        sha = hashlib.sha1(open(path, "rb").read()).hexdigest()
        got = bench.traffic_per_launch(kind, e["workload"], e["precision"], 1000)
        if sha == e["sha1"]:
            assert got == e["bytes_per_row"] * 1000
        else:
            assert got is None
        # another workload or precision has no capture
        assert bench.traffic_per_launch(kind, "c1_d128", e["precision"], 1000) is None
        assert bench.traffic_per_launch(kind, e["workload"], "bf16", 1000) is None


def test_traffic_is_withheld_once_the_source_changes(monkeypatch):
    kind = "quantize_adjust_pack"
    e = dict(bench.NCU_TRAFFIC[kind])
    e["sha1"] = "0" * 40
    monkeypatch.setitem(bench.NCU_TRAFFIC, kind, e)
    assert bench.traffic_per_launch(kind, e["workload"], e["precision"], 1000) is None


def test_alu_count_follows_rounds_and_accepts():
    """Two kept segments; accepts per round given by hand: a vector-segment
    runs through its first round without an accept."""
    mo = O.Model(d=96, mean=np.zeros(96), W=np.eye(96), plan=[(0, 64, 3), (64, 32, 2)])

    class Enc:
        pass

    enc = Enc()
    # vector 0: segment 0 stops after round 2 (round 2 has no accept), segment 1 runs all 3
    # vector 1: segment 0 runs all 3 rounds, segment 1 stops after round 1
    enc.accepts = np.array([[[4, 0, 0], [2, 1, 1]],
                            [[3, 2, 1], [0, 0, 0]]])
    ops, steps = bench.alu_ops_per_vector(enc, mo, 3)
    ran0 = np.array([2, 3]).mean()   # segment 0
    ran1 = np.array([3, 1]).mean()   # segment 1
    want_steps = 64 * ran0 + 32 * ran1
    want_ops = (64 * (bench.ALU_INIT + bench.ALU_PACK * 3) + 64 * bench.ALU_TRIAL * ran0
                + bench.ALU_ACCEPT * np.array([4, 6]).mean()
                + 32 * (bench.ALU_INIT + bench.ALU_PACK * 2) + 32 * bench.ALU_TRIAL * ran1
                + bench.ALU_ACCEPT * np.array([4, 0]).mean())
    assert steps == want_steps
    assert abs(ops - want_ops) < 1e-9


def test_one_core_baseline_runs_the_oracle_on_one_thread():
    """The one-core figure beside the all-core CPU baseline: a child process
    pinned to one CPU encodes the given rows with the oracle on one OpenMP
    thread and reports their rate."""
    rng = np.random.default_rng(5)
    X = rng.standard_normal((2000, 64)).astype(np.float32)
    mo = O.fit(X, 4.0)
    one = bench.cpu_baseline_one_core(mo, X[:300], 2)
    assert one["cores"] == 1 and one["omp_threads"] == 1
    assert one["value"] > 0 and "300 rows" in one["sample"]


def test_a_failing_one_core_child_is_reported(monkeypatch):
    """The all-core baseline still comes back when the one-core child fails;
    the failure is named in its field."""
    import subprocess
    import torch

    def fail(*args, **kwargs):
        raise subprocess.CalledProcessError(1, "child")

    monkeypatch.setattr(bench, "cpu_baseline_one_core", fail)
    X = torch.from_numpy(np.random.default_rng(6).standard_normal((3000, 64)).astype(np.float32))
    cpu, mo, enc = bench.cpu_baseline({"n": 3000, "avg_bits": 4.0, "rounds": 2}, X, target_s=0.2)
    assert cpu["value"] > 0 and cpu["kind"] == "oracle"
    assert cpu["one_core"]["value"] is None and "CalledProcessError" in cpu["one_core"]["error"]
