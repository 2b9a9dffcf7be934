"""Host-side logic that needs no GPU: the batch strategy search of the
autotuner (against a fake batch whose launch time depends on the knobs) and
the benchmark's reading of the committed ncu summaries."""
import types

import pytest


class FakeJob:
    def __init__(self, g, op):
        self.g, self.op = g, op
        self.big_degree, self.do_a, self.do_b, self.delta = 0, 0.0, 0.0, 0


def test_batch_strategy_search_keeps_the_fastest_knobs(monkeypatch):
    from paper_1701_01170_gb300 import GR_OP_BFS, GR_OP_SSSP, tune

    jobs = [FakeJob("g1", GR_OP_BFS), FakeJob("g1", GR_OP_SSSP), FakeJob("g2", GR_OP_BFS)]
    created = []

    def cost(opts):
        # cluster 4, BFS split 256, do (0.2, 0.05), SSSP split 1024, delta x0.5 are best
        c = {1: 9.0, 2: 8.0, 4: 5.0, 8: 6.0}[opts["cluster_size"]]
        for j in jobs:
            if j.op == GR_OP_BFS:
                c += {0: 3.0, 64: 2.0, 256: 1.0, 1024: 2.5}[j.big_degree]
                c += {(0.0, 0.0): 2.0, (0.01, 0.01): 1.5, (0.05, 0.05): 1.2,
                      (0.2, 0.05): 0.5}[(round(j.do_a, 2), round(j.do_b, 2))]
            else:
                c += {0: 3.0, 256: 2.0, 1024: 0.5, 4096: 1.0}[j.big_degree]
                c += {0: 3.0, 50: 0.25, 100: 1.0, 200: 2.0}[j.delta]
        return c

    def fake_create(js, opts):
        created.append(dict(cluster_size=opts.cluster_size))
        return types.SimpleNamespace()

    monkeypatch.setattr(tune, "gr_batch_create", fake_create)
    monkeypatch.setattr(tune, "gr_batch_run", lambda b: None)
    monkeypatch.setattr(tune, "gr_batch_status", lambda b: (0, []))
    monkeypatch.setattr(tune, "gr_batch_destroy", lambda b: None)
    monkeypatch.setattr(tune, "batch_opts", lambda **kw: types.SimpleNamespace(**kw))
    monkeypatch.setattr(tune, "default_delta", lambda G: 100)
    # a launch "takes" the cost of the knobs the jobs hold when it is timed
    monkeypatch.setattr(tune, "_time", lambda fn, reps, warm=1: cost(
        {"cluster_size": created[-1]["cluster_size"]}))
    opts, ms, chosen = tune.tune_batch_strategy(jobs, {"g1": object(), "g2": object()}, reps=1)
    assert opts["cluster_size"] == 4
    assert chosen["bfs_big_degree"] == 256 and chosen["bfs_do"] == (0.2, 0.05)
    assert chosen["sssp_big_degree"] == 1024 and chosen["sssp_delta_factor"] == 0.5
    assert [j.big_degree for j in jobs] == [256, 1024, 256]
    assert jobs[1].delta == 50 and (round(jobs[0].do_a, 2), round(jobs[0].do_b, 2)) == (0.2, 0.05)
    assert ms == pytest.approx(cost({"cluster_size": 4}))


def test_profiled_traffic_reads_matching_summaries(tmp_path, monkeypatch):
    import bench
    from paper_1701_01170_gb300 import _build

    (tmp_path / "profiles").mkdir()
    dig = {k: _build.source_digest(k) for k in ("bfs", "sssp")}
    (tmp_path / "profiles" / "bfs_persistent_rmat_s22.md").write_text(
        f"# x\n\n- kernel_source_digest: `{dig['bfs']}` (comment)\n"
        "- traffic_bytes_per_launch: 1234\n")
    (tmp_path / "profiles" / "sssp_persistent_rmat_s22.md").write_text(
        "- kernel_source_digest: `0000000000000000`\n- traffic_bytes_per_launch: 99\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    got = bench.profiled_traffic()
    # a stale summary gives no traffic, and so does a missing one
    assert got == {"bfs": 1234, "sssp": None, "push_bfs": None}


def test_roofline_bytes_follow_the_per_unit_formulas():
    import bench
    n, m_r, n_r = 1000, 50_000, 800
    # push BFS: 4 B per column of a reached row, 24 B per reached vertex, 8 B per vertex
    assert bench.algorithmic_bytes("push_bfs", n, m_r=m_r, n_r=n_r) == 4 * m_r + 24 * n_r + 8 * n
    # SSSP lower bound: every edge of a reached vertex relaxed once (column + weight),
    # 28 B per vertex; repeated relaxations are not counted
    assert bench.algorithmic_bytes("sssp", n, m_r=m_r, n_r=n_r) == 8 * m_r + 28 * n
    st = {"edges": 7000, "vertices": 300, "updates": 250}
    assert bench.algorithmic_bytes("bfs", n, st=st) == 4 * 7000 + 12 * 300 + 12 * 250 + 8 * n
    e = bench.roofline_entry("k", "l", 2e9, 1.0, 4000.0, "measured", None)
    assert abs(e["achieved"] - 2000.0) < 1e-9 and abs(e["frac"] - 0.5) < 1e-12


def test_timed_sources_start_at_the_hub_and_warmup_uses_others():
    import bench
    srcs = list(range(100, 165))          # 65 entries, entry 0 plays the hub
    assert bench.timed_sources(srcs, 0, 20) == srcs[:20]
    assert bench.timed_sources(srcs, 1, 3) == srcs[7:10]
    assert bench.timed_sources(srcs, 0, 70)[65:] == srcs[:5]      # wraps around the list
    w = bench.warmup_sources(srcs, 5)
    assert w == srcs[-5:][::-1] and srcs[0] not in w


def test_operator_bytes_and_peak_fallback(tmp_path, monkeypatch):
    import json

    import bench
    # advance: 4 B frontier + 8 B row bounds + 16 B offsets per row, 8 B per edge;
    # filters: 4 B per input item and 4 B per output item
    assert bench.ops_algorithmic_bytes("advance", 10, 100, 100) == 10 * 28 + 800
    assert bench.ops_algorithmic_bytes("filter", 10, 100, 7) == 400 + 28
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.hbm_peak() == (6800.0, "fallback")          # no measured peaks file
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6794.1}))
    assert bench.hbm_peak() == (6794.1, "measured")
    (tmp_path / "MEASURED_PEAKS.json").write_text("not json")
    assert bench.hbm_peak() == (6800.0, "fallback")


def test_reference_arm_prints_the_contract_line():
    # `--impl reference` times the CPU oracle (no GPU) and prints one JSON line with the
    # same metric and config keys as the GPU arm, plus its own cpu_baseline and e2e
    import json
    import os
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cmd = [sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--scale", "12",
           "--steps", "2", "--warmup", "3"]
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=300, cwd=root)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == "GTEPS" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 2 and d["warmup"] == 3
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": "GTEPS", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert d["config"]["graph"]["n"] == 4096
    # a non-zero rank of a multi-rank launch prints nothing and exits 0
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=300, cwd=root, env=env)
    assert out.returncode == 0 and not [l for l in out.stdout.splitlines() if l.startswith("{")]


def test_kernel_digest_ignores_comments_but_not_code(tmp_path, monkeypatch):
    # the ncu summaries are matched to a kernel by this digest: editing a comment must keep
    # them valid, any code change must not
    import shutil

    from paper_1701_01170_gb300 import _build
    src = tmp_path / "csrc"
    shutil.copytree(_build.CSRC, src)
    monkeypatch.setattr(_build, "CSRC", str(src))
    before = {k: _build.source_digest(k) for k in ("bfs", "sssp")}
    body = src / "gr_sssp_body.cuh"
    text = body.read_text()
    body.write_text("// a new comment line\n" + text.replace("{", "{  /* inline comment */", 1))
    assert {k: _build.source_digest(k) for k in ("bfs", "sssp")} == before
    body.write_text(text.replace("GR_BULK_MIN_ROWS 4096", "GR_BULK_MIN_ROWS 4097", 1))
    after = {k: _build.source_digest(k) for k in ("bfs", "sssp")}
    assert after["sssp"] != before["sssp"] and after["bfs"] == before["bfs"]
