"""Host logic of bench.py (no GPU): workload parameters from the frozen
windows, the traffic reader's source-hash check, the peak lookup and the
sequence of solve forms (against a stand-in for the library)."""
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


class _FakeLib:
    """Stands in for the library in bench_solve: records the solve calls and
    fails the one form a test names."""

    class ChebFDError(Exception):
        pass

    def __init__(self, fail=None):
        self.calls, self.fail = [], fail

    def chebfd_solve(self, H, lo, hi, ns, Np, eps, kernel, precision, a, b, max_iter, seed,
                     extraction="ritz", window_inset=0.0):
        import numpy as np
        key = (precision, extraction, window_inset)
        self.calls.append(dict(ns=ns, Np=Np, kernel=kernel, precision=precision,
                               extraction=extraction, window_inset=window_inset))
        if self.fail == key:
            raise self.ChebFDError("planted failure")
        lam = np.array([-0.1, -0.05, 0.05, 0.1])
        rec = dict(fp64_filter=0, in_window=4, ghosts=0, accepted=4, res_max=1e-10,
                   seconds_gram=0.1, seconds_block_gemm=0.1, seconds_eigensolve=0.1,
                   seconds_hy=0.05, seconds_residuals=0.05, seconds_other=0.0)
        return dict(a=a, b=b, lam=lam, res=np.full(4, 1e-10), nev=4, iterations=5,
                    fp64_iterations=1, converged=True, seconds_filter=1.0, seconds_dense=0.5,
                    n_mvm=5 * ns * Np, log=[rec] * 5)

    def set_matrix_free(self, on):
        self.calls.append(dict(matrix_free=on))

    class MLP:
        def __init__(self, n_in, n_h):
            pass

        def set_params(self, p):
            pass

    def chebfd_choose_params(self, H, lo, hi, mlp, a, b, m_feat):
        return 192, 610, "lanczos", 94.0


@pytest.mark.parametrize("fail", [None, ("mixed_df", "harmonic", 0.5),
                                  ("mixed_df", "harmonic", 0.0)])
def test_solve_forms_of_the_benchmark(monkeypatch, fail):
    """bench_solve runs every form with the parameters it reports (the inset
    form at half the MLP's degree), restores the matrix-free switch, and a
    failing harmonic form is reported without losing the others."""
    import torch
    monkeypatch.setattr(torch.cuda, "synchronize", lambda: None)
    monkeypatch.setattr(bench, "warm_up_solves", lambda pkg: None)
    fake = _FakeLib(fail)
    H = fake
    out = bench.bench_solve(fake, H, -4.2, 4.2, 0.14, 309, 256, "fake", precisions=("fp64",),
                            matrix_free=True)
    forms = ("fp64", "mixed_df_mlp", "mixed_df_mlp_matrix_free",
             "mixed_df_mlp_matrix_free_harmonic", "mixed_df_mlp_matrix_free_harmonic_inset")
    for f in forms:
        assert f in out
    solves = [c for c in fake.calls if "Np" in c]
    assert [c["extraction"] for c in solves] == ["ritz", "ritz", "ritz", "harmonic", "harmonic"]
    assert solves[-1]["window_inset"] == 0.5 and solves[-1]["Np"] == 305
    assert fake.calls[-1] == dict(matrix_free=False)
    assert out["fp64"]["dense_breakdown_seconds"]["gram"] == pytest.approx(0.5)
    assert len(out["fp64"]["iterations_log"]) == 5
    if fail is None:
        assert out["mixed_df_mlp_matrix_free_harmonic_inset"]["Np"] == 305
        assert out["speedup_mixed_df_mlp_matrix_free_harmonic_inset_over_fp64"] > 0
    else:
        name = ("mixed_df_mlp_matrix_free_harmonic_inset" if fail[2] else
                "mixed_df_mlp_matrix_free_harmonic")
        assert out[name] == {"error": "planted failure"}
        assert out["mixed_df_mlp_matrix_free"]["converged"]


def test_solves_are_warmed_up_outside_the_timed_region():
    """Every precision and extraction is run once, stored-matrix and
    matrix-free, on a small insulator before the timed solves."""
    fake = _FakeLib()
    made = []

    def create(kind, Lx, Ly, Lz, **kw):
        made.append((kind, Lx, Ly, Lz, kw.get("also_single")))
        return fake
    fake.chebfd_matrix_create_lattice = create
    bench.warm_up_solves(fake)
    assert made == [("topi", 8, 8, 8, True)]
    solves = [(c["precision"], c["extraction"]) for c in fake.calls if "Np" in c]
    assert sorted(solves) == sorted([(p, e) for p in ("fp64", "mixed", "mixed_df")
                                     for e in ("ritz", "harmonic")] * 2)
    assert [c for c in fake.calls if "matrix_free" in c] == [dict(matrix_free=False),
                                                             dict(matrix_free=True)]
