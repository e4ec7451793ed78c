"""Host logic of bench.py that needs no GPU: the recorded-traffic digest ignores comments and
layout but not code, the FP64 peak follows from the unit counts and clock, every workload the
benchmark offers builds and names its configuration, and the reference arm stays time-boxed."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_digest_ignores_comments_and_layout_but_not_code(tmp_path, monkeypatch):
    src = tmp_path / "paper_0910_1531_gb300" / "csrc"
    src.mkdir(parents=True)
    (src / "k.cuh").write_text("int f(int a) { return a + 1; }  // one\n/* block */\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    d0 = bench.csrc_digest()
    (src / "k.cuh").write_text("int f(int a)   {\n  return a + 1;   // two\n}\n")
    assert bench.csrc_digest() == d0
    (src / "k.cuh").write_text("int f(int a) { return a + 2; }\n")
    assert bench.csrc_digest() != d0


def test_digest_covers_the_build_flags(tmp_path, monkeypatch):
    pkg = tmp_path / "paper_0910_1531_gb300"
    (pkg / "csrc").mkdir(parents=True)
    (pkg / "csrc" / "k.cuh").write_text("int f(int a) { return a + 1; }\n")
    (pkg / "build.py").write_text('"""doc"""\nFLAGS = ["-O3"]  # flags\n')
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    d0 = bench.csrc_digest()
    (pkg / "build.py").write_text('"""other doc"""\nFLAGS = ["-O3"]   # other comment\n')
    assert bench.csrc_digest() == d0
    (pkg / "build.py").write_text('"""doc"""\nFLAGS = ["-O2"]\n')
    assert bench.csrc_digest() != d0


def test_recorded_traffic_is_well_formed_and_dropped_once_stale(monkeypatch):
    # every entry names kernel kinds the bench reports (a workload may record only its largest
    # passes) and always the Phi' pass
    for key, per in bench.NCU_TRAFFIC["captures"].items():
        assert set(per) <= set(bench.KERNELS) and "xphi" in per, key
        assert all(v >= 0 for v in per.values())
    key = next(iter(bench.NCU_TRAFFIC["captures"]))
    name, prec = key.rsplit("/", 1)
    monkeypatch.setitem(bench.NCU_TRAFFIC, "digest", bench.csrc_digest())
    assert bench.recorded_traffic(name, prec, "xphi") == bench.NCU_TRAFFIC["captures"][key]["xphi"]
    monkeypatch.setitem(bench.NCU_TRAFFIC, "digest", "0" * 16)
    assert bench.recorded_traffic(name, prec, "xphi") is None


def test_fp64_peak_from_unit_counts():
    # 152 SMs x 2 FP64 FMAs (4 flop) per clock x 2.07 GHz: the part's nominal 1.25 TFLOP/s
    assert bench.FP64_TFLOPS == pytest.approx(1.25, rel=0.01)


@pytest.mark.parametrize("name", ["obstacles128", "wall161", "hswall", "sphere32"])
def test_workloads_build_and_name_their_configuration(name):
    class A:
        workload = name
        n = 32 if name == "obstacles128" else None
        eta = 0.2
    w = bench.workload(A)
    assert w.V.shape == (w.nspecies,) + tuple(w.shape)
    cfg = bench.workload_config(w)
    assert isinstance(cfg, dict) and cfg


def test_reference_arm_is_time_boxed():
    assert 0 < bench.REFERENCE_BUDGET_S <= 180


def test_cpu_model_is_named():
    assert isinstance(bench.cpu_model(), str) and bench.cpu_model()
