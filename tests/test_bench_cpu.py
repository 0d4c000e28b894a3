"""Host logic of bench.py (no GPU): workload parameters from the frozen
windows, the traffic reader's source-hash check and the peak lookup."""
import os

import pytest

import bench


class _Args:
    def __init__(self, workload, Np=0):
        self.workload, self.Np = workload, Np


@pytest.mark.parametrize("name,N_p,ns", [("topi", 309, 256), ("graphene", 1779, 512),
                                         ("topi_large", 807, 256)])
def test_workload_parameters_follow_the_rule(name, N_p, ns):
    """N_p = N_0 S_w / delta' with delta' = (sqrt(N_S/N_T) - 1) delta (Sec. 2.4)."""
    w, a, b, delta, Np = bench.workload_params(_Args(name))
    assert w["ns"] == ns and Np == N_p
    assert a < -delta < 0 < delta < b
    assert bench.workload_params(_Args(name, Np=500))[4] == 500


def test_traffic_only_while_the_profiled_source_is_unchanged(tmp_path, monkeypatch):
    # a summary whose hash matches its source gives the traffic, else None
    import hashlib
    src = os.path.join(bench.ROOT, "paper_1510_04895_gb300", "csrc", "step_bell.cu")
    digest = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    prof = tmp_path / "profiles"
    (prof / "paper_1510_04895_gb300" / "csrc").mkdir(parents=True)
    (prof / "paper_1510_04895_gb300" / "csrc" / "step_bell.cu").write_bytes(open(src, "rb").read())
    (prof / "good.txt").write_text(
        "kernel_source paper_1510_04895_gb300/csrc/step_bell.cu\n"
        "kernel_source_sha256_16 %s\ntraffic_bytes_per_launch 123.0\n" % digest)
    (prof / "stale.txt").write_text(
        "kernel_source paper_1510_04895_gb300/csrc/step_bell.cu\n"
        "kernel_source_sha256_16 0000000000000000\ntraffic_bytes_per_launch 1.0\n")
    root = tmp_path / "root"
    root.mkdir()
    os.symlink(str(prof), str(root / "profiles"))
    os.symlink(str(prof / "paper_1510_04895_gb300"), str(root / "paper_1510_04895_gb300"))
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.read_traffic("good.txt") == 123.0
    assert bench.read_traffic("stale.txt") is None


def test_peaks_fall_back_without_the_measured_file(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    peaks, kind = bench.measured_peaks()
    assert kind == "fallback" and peaks["hbm_gbs"] == 6800.0
