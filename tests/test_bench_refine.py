"""The bench's operating-point search (host logic, no GPU): between the last
swept L below a recall target and the first one reaching it, bisection finds
the smallest integer L that reaches the target, measuring recall only at the
L it tries."""
import bench


def sweep(recall, Ls):
    return [{"L": L, "recall10": recall(L), "qps": 1e6 / L} for L in Ls]


def test_finds_smallest_L_reaching_target():
    recall = lambda L: min(1.0, 0.8 + L / 1000.0)  # reaches 0.95 at L = 150
    tried = []

    def at(L):
        tried.append(L)
        return recall(L)

    p = bench.refine_L(sweep(recall, [100, 125, 175, 200]), 0.95, at, lambda L: 1e6 / L)
    assert p["L"] == 150 and p["recall10"] >= 0.95 and p["refined"]
    assert all(125 < L < 175 for L in tried) and len(tried) <= 6


def test_grid_point_already_smallest():
    # no L below the grid point reaches the target: nothing new to add
    recall = lambda L: 0.95 if L >= 125 else 0.90
    assert bench.refine_L(sweep(recall, [100, 125, 150]), 0.95, recall, lambda L: 1.0) is None


def test_target_unreached_or_reached_at_first_point():
    recall = lambda L: 0.5
    assert bench.refine_L(sweep(recall, [10, 20]), 0.95, recall, lambda L: 1.0) is None
    recall = lambda L: 0.99
    assert bench.refine_L(sweep(recall, [10, 20]), 0.95, recall, lambda L: 1.0) is None


def test_result_is_measured_not_interpolated():
    # a plateau: recall jumps at L = 133; the point returned carries the
    # recall measured there
    recall = lambda L: 0.96 if L >= 133 else 0.94
    p = bench.refine_L(sweep(recall, [125, 150]), 0.95, recall, lambda L: 7.0)
    assert p == {"L": 133, "recall10": 0.96, "qps": 7.0, "refined": True}


def test_cpu_alg1_baseline_on_an_oracle_graph():
    # the CPU baseline times the oracle's Alg. 1 on a given index: one sample
    # on one thread, one on every host thread
    import numpy as np

    import oracle
    from paper_1707_00143_gb300 import datagen

    base, q = datagen.workload("tiny", n=2000, nq=64)
    ref = oracle.build(base, 16, 30, 12, 100, seed=0)
    out, counts = bench.cpu_alg1(ref["adj"], ref["deg"], base, ref["nav"], q, 10, 40, budget_s=0.2)
    # the counts of the all-thread sample are the oracle's own
    m = len(counts["n_expand"])
    _, _, ne, nd = oracle.search(ref["adj"], base, ref["nav"], q[:m], 10, 40, deg=ref["deg"])
    assert np.array_equal(counts["n_expand"], ne) and np.array_equal(counts["n_dist"], nd)
    assert out["kind"] == "oracle" and out["unit"] == bench.UNIT
    assert out["value"] > 0 and out["single_thread"]["value"] > 0
    assert out["cores"] >= 1 and "Alg. 1" in out["sample"]
    assert np.isfinite(out["value"])


def test_both_arms_share_the_config():
    import numpy as np

    W = bench.WORKLOADS["sift"]
    base = np.zeros((4, 128), np.float32)
    a, b = bench.bench_config(W, 1, base), bench.bench_config(W, 1, base)
    assert a == b and a["workload"] == W["desc"] and a["target_recall10"] == bench.TARGET


def test_config_runs_summarise_children(monkeypatch):
    # the default line's configuration runs: each child's last JSON line is
    # summarised; a failing child or one past its time limit is an error entry
    import json
    import subprocess
    import types

    line = {"metric": "m", "value": 2.0, "unit": "queries/s", "config": {"workload": "w"},
            "operating_point": {"L": 300}, "batched": {"value": 5.0},
            "at_recall10": {"0.95": {"best": {"u8": {"L": 300, "qps": 2.0, "recall10": 0.95}, "plain": None},
                                     "stop_vs_fixed_L": {}}}}
    calls = []

    def fake_run(cmd, capture_output, text, timeout):
        calls.append((cmd, timeout))
        wl = cmd[cmd.index("--workload") + 1]
        assert "--compact" in cmd and "--no-cpu" in cmd
        if wl == "gist":
            return types.SimpleNamespace(returncode=0, stdout="noise\n" + json.dumps(line) + "\n", stderr="")
        raise subprocess.TimeoutExpired(cmd, timeout)

    monkeypatch.setattr(bench.subprocess, "run", fake_run)
    args = types.SimpleNamespace(steps=7, warmup=3)
    out = bench.config_runs(args)
    assert [c[0][c[0].index("--workload") + 1] for c in calls] == [wl for wl, _ in bench.CONFIG_RUNS]
    g = out["gist"]
    assert g["value"] == 2.0 and g["batched"] == {"value": 5.0} and g["operating_point"] == {"L": 300}
    assert g["at_recall10"]["0.95"]["u8"] == {"L": 300, "qps": 2.0} and g["at_recall10"]["0.95"]["plain"] is None
    assert "--steps 7" in g["command"] and "error" not in g
    assert out["deep"] == {"error": "no result within %d s" % dict(bench.CONFIG_RUNS)["deep"]}


def test_build_index_follows_the_workloads_knn_stage():
    # the DEEP-shaped workload builds on an nn-descent kNN stage, the others on
    # the exact one; the line's config names which
    import types

    calls = []
    fake = types.SimpleNamespace(
        nsg_build=lambda bt, K, L, R, C, seed=0: calls.append(("exact", K, L, R, C, seed)) or "idx",
        nsg_build_ex=lambda bt, K, L, R, C, seed=0, knn_params=None: calls.append(
            ("nndescent", K, L, R, C, seed, knn_params)) or "idx",
        NnDescentParams=lambda *a: tuple(a))
    assert bench.build_index(fake, None, bench.WORKLOADS["sift"]) == "idx"
    assert bench.build_index(fake, None, bench.WORKLOADS["deep"], seed=3) == "idx"
    assert calls[0] == ("exact", 100, 40, 50, 500, 0)
    assert calls[1][:6] == ("nndescent", 64, 60, 32, 500, 3) and calls[1][6][:3] == bench.WORKLOADS["deep"]["knn"]
    import numpy as np
    base = np.zeros((4, 2), np.float32)
    assert "nn-descent" in bench.bench_config(bench.WORKLOADS["deep"], 1, base)["knn_stage"]
    assert bench.bench_config(bench.WORKLOADS["sift"], 1, base)["knn_stage"].startswith("exact")
