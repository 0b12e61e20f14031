"""Host logic of the benchmark that needs no GPU: when the committed ncu DRAM traffic may be
reported, how the fused-step kernel is named from the plan a solve reports, and how the clock
samples taken during the timed region are summarised."""

import json
import os
import shutil

import bench


def _tree_with_traffic(tmp_path, record, source_hash=None):
    """A copy of the files `_traffic_per_launch` reads (kernel source and traffic summary)."""
    root = tmp_path / "repo"
    src = root / "paper_2110_11738_b300" / "csrc"
    src.mkdir(parents=True)
    shutil.copy(os.path.join(bench.ROOT, "paper_2110_11738_b300", "csrc", "drot_kernels.cuh"), src)
    (root / "profiles").mkdir()
    doc = {"kernel_source_sha256_16": source_hash or bench._kernel_source_hash(),
           "workloads": {"plain_8192x6144": record}}
    (root / "profiles" / "step_kernel_traffic.json").write_text(json.dumps(doc))
    return root


def test_traffic_reported_only_for_a_current_capture_of_the_kernel_that_ran(tmp_path, monkeypatch):
    rec = {"dram_bytes_per_launch": 123456789.0, "kernel": "drot_step_kernel<4,1,0>"}
    root = _tree_with_traffic(tmp_path, rec)
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench._traffic_per_launch("plain_8192x6144", "drot_step_kernel<4,1,0>") == 123456789.0
    assert bench._traffic_per_launch("plain_8192x6144", "drot_step_kernel<2,1,0>") is None  # another plan ran
    assert bench._traffic_per_launch("plain_20000", "drot_step_kernel<4,1,0>") is None  # never captured
    # the kernel source changed after the capture: the counters no longer describe it
    with open(root / "paper_2110_11738_b300" / "csrc" / "drot_kernels.cuh", "a") as fh:
        fh.write("\n// edited\n")
    assert bench._traffic_per_launch("plain_8192x6144", "drot_step_kernel<4,1,0>") is None


def test_traffic_absent_summary(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._traffic_per_launch("plain_8192x6144") is None


def test_committed_traffic_summary_matches_the_kernel_source():
    # the committed capture is the one the benchmark reports: it must describe the current source
    with open(os.path.join(bench.ROOT, "profiles", "step_kernel_traffic.json")) as fh:
        doc = json.load(fh)
    assert doc["kernel_source_sha256_16"] == bench._kernel_source_hash()
    for rec in doc["workloads"].values():
        assert rec["dram_bytes_per_launch"] == rec["dram_read_bytes"] + rec["dram_write_bytes"]


def test_step_kernel_name_follows_the_reported_plan():
    prof = {"step_variant": 1, "tile_k": 4, "stages": 0}
    assert bench._step_kernel_name(prof, c_skip=False) == "drot_step_kernel<4,1,0>"
    assert bench._step_kernel_name(prof, c_skip=True) == "drot_step_kernel<4,1,1|2>"
    assert bench._step_kernel_name({"step_variant": 2, "tile_k": 2, "stages": 6}, False) == "drot_step_tma_kernel<2,6>"
    assert bench._step_kernel_name({"step_variant": 3, "tile_k": 4, "stages": 3}, False) == \
        "drot_step_async_kernel<4,3>"
    assert bench._step_kernel_name({"step_variant": 4, "tile_k": 0, "stages": 16}, False) == \
        "drot_cluster_kernel<16>"


class _FakeProc:
    def __init__(self, text):
        self.text = text

    def terminate(self):
        pass

    def communicate(self, timeout=None):
        return self.text, ""


def test_clock_samples_and_throttle_reasons():
    rows = [
        "0, 2032, 2032, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2032, 1099.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2032, 2032, 950.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, [N/A], 2032, 950.0, 0x0, Not Active, Not Active, Not Active, Not Active",  # unreadable: skipped
        "garbage",
    ]
    s = bench.ClockSampler(0)
    s.proc = _FakeProc("\n".join(rows) + "\n")
    out = s.stop()
    assert out == {"sm_mhz": 2032.0, "sm_max_mhz": 2032.0, "reasons": ["sw_power_cap"], "samples": 3}
    s.proc = _FakeProc("0, 1200, 2032, 500, 0x0, Active, Not Active, Active, Not Active\n")
    assert s.stop()["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    s.proc = None
    assert s.stop() is None


def test_certificate_brackets_the_exact_optimum():
    """The benchmark's optimality certificate: the rounded plan's cost is an upper bound and the
    c-transform dual objective a lower bound of the exact LP optimum (HiGHS), for an optimal pair,
    for an infeasible plan and for perturbed duals; both meet the optimum at an exact solution."""
    import numpy as np
    import torch

    import oracle
    import workloads

    pr = workloads.make_problem("plain_8192x6144", seed=3, m=9, n=7)
    C64 = pr.C.astype(np.float64)
    X, mu, nu, opt = oracle.lp_primal_dual(C64, pr.p, pr.q)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a))  # noqa: E731
    C = t(pr.C)
    cert = bench._certificate(C, t(pr.p), t(pr.q), t(X.astype(np.float32)), t(mu), t(nu), block_rows=4)
    assert cert["lower_c_transform"] <= opt + 1e-9
    assert cert["upper_rounded_plan"] >= opt - 1e-7
    assert abs(cert["lower_c_transform"] - opt) <= 1e-9
    assert abs(cert["upper_rounded_plan"] - opt) <= 1e-6
    rng = np.random.default_rng(0)
    for trial in range(5):
        Xb = (X * rng.uniform(0.5, 1.5, size=X.shape) + rng.uniform(0, 1e-3, size=X.shape)).astype(np.float32)
        mub = mu + rng.normal(0, 0.05, size=mu.shape)
        c = bench._certificate(C, t(pr.p), t(pr.q), t(Xb), t(mub), t(nu), block_rows=3)
        assert c["lower_c_transform"] <= opt + 1e-12
        assert c["upper_rounded_plan"] >= opt - 1e-7
        assert c["certified_rel_gap"] >= 0.0
        # the rounded plan is feasible: recompute its cost independently
        xs = np.minimum(pr.p / Xb.astype(np.float64).sum(1), 1.0)
        X1 = Xb.astype(np.float64) * xs[:, None]
        ys = np.minimum(pr.q / X1.sum(0), 1.0)
        X2 = X1 * ys[None, :]
        er, ec = pr.p - X2.sum(1), pr.q - X2.sum(0)
        Xf = X2 + np.outer(er, ec) / er.sum()
        assert np.abs(Xf.sum(1) - pr.p).max() < 1e-12 and np.abs(Xf.sum(0) - pr.q).max() < 1e-12
        assert abs((C64 * Xf).sum() - c["upper_rounded_plan"]) < 1e-12
