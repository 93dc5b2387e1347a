"""Host logic of the benchmark's measurement, on the CPU: the clock record
taken during the timed region, the algorithmic work model, the lookup of
profiled DRAM bytes by source hash and the reference arm's line (no GPU)."""
import hashlib
import os
import shutil
import types

import numpy as np
import pytest

import bench


class _Proc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _line(sm, mx, hw="Not Active", hwt="Not Active", swt="Not Active", cap="Not Active"):
    return "0, %s, %s, 900.00, 0x0, %s, %s, %s, %s" % (sm, mx, hw, hwt, swt, cap)


def test_clocks_summary_within_the_timed_region():
    c = bench.Clocks(0)
    c.proc = _Proc()
    c.lines = [_line(2070, 2070), _line(2055, 2070, cap="Active"), _line(2070, 2070), "garbage",
               _line("[N/A]", 2070)]
    c.pause()                                    # samples after the timed region are dropped
    c.lines += [_line(1200, 2070, hwt="Active")]
    r = c.stop()
    assert r["samples"] == 3
    assert r["sm_mhz"] == 2070.0 and r["sm_max_mhz"] == 2070.0
    assert r["reasons"] == ["sw_power_cap"]


def test_clocks_summary_reports_thermal_slowdown():
    c = bench.Clocks(0)
    c.proc = _Proc()
    c.lines = [_line(1500, 2070, hwt="Active"), _line(1600, 2070, swt="Active", hw="Active")]
    r = c.stop()
    assert r["sm_mhz"] == 1550.0
    assert r["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]


def test_clocks_without_nvidia_smi():
    c = bench.Clocks(0)
    assert c.stop() is None                      # never started: no record, no error


def test_algorithmic_ops_counts():
    w = types.SimpleNamespace(n=64000, box=(126.0, 126.0, 126.0))
    rho = 64000 / 126.0 ** 3
    sphere = lambda r: 4.0 / 3.0 * np.pi * r ** 3 * rho
    ops, slots, tests = bench.algorithmic_ops(w, 500, 20)
    assert tests == pytest.approx(sphere(12.0))
    n_core = sphere(6.0)
    assert ops["near"] == pytest.approx(w.n * (bench.OPS_TEST * sphere(12.0) + bench.OPS_PAIR * (n_core + 20)))
    assert ops["rho"] == pytest.approx(bench.OPS_RHO * w.n * 500)
    assert ops["farforce"] == pytest.approx(bench.OPS_FAR * w.n * 500)
    assert slots["farforce"] < ops["farforce"] and slots["rho"] < ops["rho"]   # packed pairs share a slot
    # kept lists: the tests of the list radius, charged by the builds per step
    ops_k, _, tests_k = bench.algorithmic_ops(w, 500, 20, list_every=-1, skin=1.5, builds_per_step=0.05)
    assert tests_k == pytest.approx(0.05 * sphere(13.5))
    assert ops_k["near"] < ops["near"]
    # a fixed schedule: one build every list_every steps
    _, _, tests_f = bench.algorithmic_ops(w, 500, 20, list_every=10, skin=1.5)
    assert tests_f == pytest.approx(0.1 * sphere(13.5))


def test_profiled_traffic_follows_the_source_hash(tmp_path, monkeypatch):
    root = bench.ROOT
    summ = os.path.join(root, "profiles", "traffic_nacl64k.txt")
    rows = {}
    for line in open(summ):
        f = line.split()
        if len(f) >= 3 and not line.startswith("#"):
            rows[f[0]] = (f[1], float(f[2]))
    near_src = os.path.join(root, "paper_2512_24970_gb300", "csrc", "k_near.cu")
    h = hashlib.sha256(open(near_src, "rb").read()).hexdigest()[:16]
    got = bench.profiled_traffic("near", kept=True)
    if rows["k_sample_batch"][0] == h and rows["k_near_kept"][0] == h:
        assert got == rows["k_sample_batch"][1] + rows["k_near_kept"][1]
    else:
        assert got is None
    # a changed source: no traffic figure
    fake = tmp_path / "repo"
    (fake / "profiles").mkdir(parents=True)
    (fake / "paper_2512_24970_gb300" / "csrc").mkdir(parents=True)
    shutil.copy(summ, fake / "profiles" / "traffic_nacl64k.txt")
    for src in ("k_near.cu", "k_far.cu"):
        data = open(os.path.join(root, "paper_2512_24970_gb300", "csrc", src), "rb").read()
        (fake / "paper_2512_24970_gb300" / "csrc" / src).write_bytes(data + b"\n// changed\n")
    monkeypatch.setattr(bench, "ROOT", str(fake))
    assert bench.profiled_traffic("near", kept=True) is None
    assert bench.profiled_traffic("rho") is None
    assert bench.profiled_traffic("unknown") is None


def test_reference_arm_line(monkeypatch, capsys, orc):
    """The reference arm times the oracle on the host cores and prints one
    line with the same metric as the GPU arm, its own cpu_baseline and an
    end-to-end figure without copies (a short sample per step here)."""
    import argparse
    import json
    real = bench.oracle_sample
    monkeypatch.setattr(bench, "oracle_sample",
                        lambda w, cfg, P_F, P_R, budget_s=15.0: real(w, cfg, P_F, P_R, budget_s=0.2))
    monkeypatch.delenv("RANK", raising=False)
    args = argparse.Namespace(config="nacl_1k", P_F=None, P_R=None, steps=2, warmup=1, gpus=1)
    bench.run_reference(args)
    out = [l for l in capsys.readouterr().out.splitlines() if l.startswith("{")]
    assert len(out) == 1
    line = json.loads(out[0])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC
    assert line["unit"] == "atom-steps/s" and line["higher_is_better"] is True
    assert line["steps"] == 2 and line["warmup"] == 1 and line["value"] > 0
    assert line["ms_per_step"] == pytest.approx(1000.0 * 1000 / line["value"])
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1 and cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": "atom-steps/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    # other ranks of a multi-process launch print nothing
    monkeypatch.setenv("RANK", "1")
    bench.run_reference(args)
    assert capsys.readouterr().out == ""
