#!/usr/bin/env python
"""Throughput of the ChebFD polynomial filter (Fig. ChebFD) on GB300.

Default workload (--workload topi): the 64x64x32x4 topological insulator
(N = 524288, W = 1.0, seed 1), a search space of n_s = 256 vectors filtered in
four row-major blocks of n_b = 64, complex64 recurrence with FP32
accumulation, Lanczos kernel (mu = 2), central window [-delta, delta] holding
~100 eigenpairs (oracle KPM, frozen in tests/golden/topi_64x64x32_window.txt),
N_p from the Lanczos-kernel scaling N_p = N_0 S_w / delta' with N_0 = 6.23 and
delta' = (sqrt(N_S / N_T) - 1) delta (linear DOS, Sec. 2.4).

--workload graphene: the 1024x1024 disordered honeycomb lattice (N = 2097152,
real symmetric, W = 1.0, seed 2), n_s = 512 in four blocks of n_b = 128, FP32
recurrence, window of ~200 eigenpairs (tests/golden/graphene_1024x1024_window.txt),
N_p by the same rule with N_T = 200.

One step = one application p[H] X of the degree-N_p filter to the whole
search block.  metric = filter row-vector updates per second
(N * n_s * N_p / t).  Prints one JSON line (rank 0).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "filter row-vector updates/s (N * n_s * N_p / t)"
UNIT = "row-vector updates/s"
N0_LANCZOS = 6.23

# Per workload: lattice (from workloads), frozen window, KPM target count N_T,
# stored entries per row, value type, and the ncu summary of its fused step.
WORKLOADS = {
    "topi": dict(spec="TOPI_MEDIUM", window="topi_64x64x32_window.txt", NT=100, nnz_row=13,
                 cplx=True, label="topi 64x64x32x4 (N=524288) W=1.0 seed 1",
                 profile="cheb_step_c64_nb64_topi64x64x32.txt", profile_nb=64,
                 profile_blocked="bell_step_c64_nb64_topi64x64x32.txt"),
    "graphene": dict(spec="GRAPHENE", window="graphene_1024x1024_window.txt", NT=200, nnz_row=4,
                     cplx=False, label="graphene 1024x1024x2 (N=2097152) W=1.0 seed 2",
                     profile="cheb_step_r32_nb128_graphene1024x1024.txt", profile_nb=128),
    "topi_large": dict(spec="TOPI_LARGE", window="topi_200x200x100_window.txt", NT=100,
                       nnz_row=13, cplx=True,
                       label="topi 200x200x100x4 (N=16000000) W=0.5 seed 3",
                       profile=None, profile_nb=64),
}


def load_window(name="topi"):
    vals = {}
    with open(os.path.join(ROOT, "tests", "golden", WORKLOADS[name]["window"])) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    return vals["a"], vals["b"], vals["delta"]


def workload_params(args):
    """N_p by the rule of Sec. 3.1 step 3 / Sec. 2.4: the search-interval margin
    delta' follows from N_S and the KPM count N_T for the linear DOS of the
    insulator and of graphene (delta'/delta = sqrt(N_S/N_T) - 1), and
    N_p = N_0 S_w / delta' with N_0 = 6.23 (Tab. lanczoskernel, centre)."""
    from paper_1510_04895_gb300 import workloads
    name = getattr(args, "workload", "topi")
    spec = WORKLOADS[name]
    w = dict(getattr(workloads, spec["spec"]), **spec)
    a, b, delta = load_window(name)
    S_w = 0.5 * (b - a)
    margin = (np.sqrt(w["ns"] / float(spec["NT"])) - 1.0) * delta
    Np = args.Np or int(round(N0_LANCZOS * S_w / margin))
    return w, a, b, delta, Np


def read_traffic(profile):
    """DRAM bytes per launch of the fused step from the committed ncu summary,
    or None when the kernel source changed since that capture."""
    import hashlib
    vals = {}
    try:
        with open(os.path.join(ROOT, "profiles", profile)) as f:
            for line in f:
                if line.strip() and not line.startswith("#"):
                    parts = line.split()
                    vals[parts[0]] = parts[1] if len(parts) > 1 else ""
        src = os.path.join(ROOT, vals.get("kernel_source",
                                          "paper_1510_04895_gb300/csrc/filter_kernels.cuh"))
        with open(src, "rb") as f:
            digest = hashlib.sha256(f.read()).hexdigest()[:16]
    except OSError:
        return None
    if vals.get("kernel_source_sha256_16") != digest:
        return None
    return float(vals["traffic_bytes_per_launch"])


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            p = [x.strip() for x in l.split(",")]
            if len(p) < 8:
                continue
            try:
                sm.append(float(p[0]))
                mx.append(float(p[1]))
            except ValueError:
                continue
            for name, v in zip(names, p[4:8]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = os.environ.get("CHEBFD_BENCH_BACKEND", "nccl")
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier_max(world, value):
    """Barrier across ranks and the maximum of a host float."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def aggregate(world, units_per_rank, t_local):
    """Whole-job throughput: every rank did units_per_rank units; the job took
    the slowest rank's time.  Returns (units per second, max time)."""
    t_max = barrier_max(world, t_local)
    return world * units_per_rank / t_max, t_max


# ------------------------------------------------------------------ CPU legs


def oracle_sample(w, a, b, delta, steps_per_sample, nb=64, seed=0):
    """Time the oracle's FP64 filter recurrence on one nb-wide block of the
    same matrix: returns (row-vector updates/s, seconds, description)."""
    from oracle import coeffs, filter as ofilt, lattice
    from paper_1510_04895_gb300 import workloads
    if w["kind"] == "topi":
        csr = lattice.topi_csr(w["Lx"], w["Ly"], w["Lz"], t=w["t"], m=w["m"], W=w["W"],
                               seed=w["seed"])
    else:
        csr = lattice.graphene_csr(w["Lx"], w["Ly"], t=w["t"], W=w["W"], seed=w["seed"])
    Ho = lattice.to_scipy(*csr)
    alpha, beta = coeffs.scaling(a, b)
    gc = coeffs.filter_coeffs(a, b, -delta, delta, steps_per_sample, "lanczos")
    X = workloads.random_block(seed, Ho.shape[0], nb, w["cplx"])
    t0 = time.perf_counter()
    ofilt.filter_block(Ho, alpha, beta, gc, X)
    dt = time.perf_counter() - t0
    units = Ho.shape[0] * nb * steps_per_sample
    desc = ("oracle FP64 %s filter, %d Chebyshev steps on one %d-vector block of the "
            "N=%d matrix (scipy CSR product, single thread)" % (
                "complex128" if w["cplx"] else "float64", steps_per_sample, nb, Ho.shape[0]))
    return units / dt, dt, desc


def run_reference(args):
    world, rank, _ = dist_setup(args)
    if rank != 0:
        return 0
    w, a, b, delta, Np = workload_params(args)
    samples = []
    for i in range(args.warmup + args.steps):
        v, dt, desc = oracle_sample(w, a, b, delta, 2, seed=i)
        if i >= args.warmup:
            samples.append((v, dt))
    value = statistics.median(v for v, _ in samples)
    ms = 1e3 * statistics.median(dt for _, dt in samples)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c128" if w["cplx"] else "f64",
            "data": "synthetic",
            "config": {"workload": "%s, n_b=64, window [-%.6g, %.6g]" % (w["label"], delta, delta)},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ GPU arm


def bench_ensemble(pkg, workloads, dev, peak_gbs):
    """The 512-member disorder ensemble filtered together: autotuned layout,
    one CUDA-graph launch per filter (N_p = 300 fused steps over all members)."""
    import torch
    w = workloads.ENSEMBLE
    members = workloads.ensemble_members(w["count"], w["first_seed"])
    mats = [pkg.chebfd_matrix_create_lattice("topi", L, L, L, t=w["t"], m=w["m"], W=W, seed=s,
                                             also_single=True) for L, W, s in members]
    n = sum(4 * L ** 3 for L, _, _ in members)
    X = torch.empty((n, w["ns"]), dtype=torch.complex64, device=dev)
    E, ms_step_tune = pkg.chebfd_ensemble_autotune(mats, X)
    al, be, gcs = [], [], []
    for L, W, s in members:
        bound = 1.01 * (abs(w["m"]) + 3 * w["t"] + W / 2)   # Weyl: clean radius m+3t plus W/2
        a, b = -bound, bound
        al.append(2.0 / (b - a))
        be.append((a + b) / (a - b))
        gcs.append(pkg.chebfd_window_coeffs(a, b, w["window"][0], w["window"][1], w["Np"],
                                            w["kernel"], 2.0))
    E.set_coeffs(np.array(al), np.array(be), np.array(gcs))
    pkg.chebfd_random_block(X, ns_total=w["ns"], seed=1)
    del mats
    stream = torch.cuda.current_stream()
    E.filter(X)                    # capture + warm-up
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 2
    e0.record(stream)
    for _ in range(reps):
        E.filter(X)
    e1.record(stream)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3 / reps
    ns = w["ns"]
    bytes_step = n * (13 * (8 + 4) + 5 * ns * 8)
    gbs = bytes_step * w["Np"] / t / 1e9
    return {"workload": "%d insulators, L in U{10..20} (N = 4L^3), W in U[0.2, 2.0], seeds "
                        "%d-%d, window [%g, %g], n_s = %d, N_p = %d, complex64"
                        % (w["count"], w["first_seed"], w["first_seed"] + w["count"] - 1,
                           w["window"][0], w["window"][1], ns, w["Np"]),
            "n_total": n, "sell_C": E.sell_C, "panel": E.panel, "tile": E.tile,
            "ms_per_filter": 1e3 * t, "graph_launches_per_filter": 1,
            "value": n * ns * w["Np"] / t, "unit": UNIT,
            "achieved_gbs": gbs, "frac_of_measured_hbm": gbs / peak_gbs,
            "autotune_ms_per_step": ms_step_tune}


def fp64_class_kernels(pkg, H, N, alpha, beta, a, b, delta, peaks, stream):
    """The FP64-class Chebyshev steps of the plain and mixed solves on the
    insulator, each against its own bound: the native complex128 step on the
    FP64 pipe (118 executed flops per row-vector update; peak = a cuBLAS
    DGEMM measured here, and the nominal 1.25 TFLOP/s), and the double-float
    steps (SELL and matrix-free, 16 bytes
    per complex entry) against HBM on their own algorithmic bytes.  A
    double-float step's time is the difference of two filters of degree 12
    and 36, divided by the 24 extra steps (the conversions and the two start
    steps cancel)."""
    import torch
    out = {}
    nb = 32
    # measured FP64 peak: cuBLAS DGEMM 4096^3, best of 3
    A = torch.randn(4096, 4096, dtype=torch.float64, device="cuda")
    B = torch.randn_like(A)
    torch.matmul(A, B)
    best = None
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        torch.matmul(A, B)
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3
        best = t if best is None else min(best, t)
    fp64_peak = 2.0 * 4096 ** 3 / best / 1e12
    del A, B
    U = torch.empty((N, nb), dtype=torch.complex128, device="cuda")
    Wv = torch.empty_like(U)
    Y = torch.zeros_like(U)
    pkg.chebfd_random_block(U, ns_total=nb, seed=11)
    pkg.chebfd_random_block(Wv, ns_total=nb, seed=12)
    for _ in range(3):
        pkg.chebfd_chebyshev_step(H, alpha, beta, 1e-3, U, Wv, Y)
    reps = 20
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for i in range(reps):
        if i % 2 == 0:
            pkg.chebfd_chebyshev_step(H, alpha, beta, 1e-3, U, Wv, Y)
        else:
            pkg.chebfd_chebyshev_step(H, alpha, beta, 1e-3, Wv, U, Y)
    e1.record(stream)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3 / reps
    # executed FP64 flops per row-vector update: 13 complex multiply-adds
    # (4 FMAs = 8 flops each) for H u as sums P = sum Re h u, Q = sum Im h u,
    # their combination (2), w = 2 alpha H u + 2 beta u - w and y += c w with
    # real scalars (8 + 4); the paper's intensity model (Sec. 4) counts 146
    # (complex multiplies as 6 flops, complex scalars)
    flops = N * nb * 118.0
    out["c128_step"] = {"kernel": "cheb_step_kernel (MODE_STEP, c128, n_b=32)", "bound": "fp64",
                        "launch_us": t * 1e6, "flops_per_launch": flops,
                        "flops_per_update": 118, "paper_model_flops_per_update": 146,
                        "achieved_tflops": flops / t / 1e12, "peak_tflops": fp64_peak,
                        "peak_kind": "cuBLAS DGEMM 4096^3 measured in this run",
                        "frac": flops / t / 1e12 / fp64_peak,
                        "frac_of_nominal_1.25_tflops": flops / t / 1e12 / 1.25,
                        "hbm_gbs": N * (13 * 20 + 5 * nb * 16) / t / 1e9}
    del Y, Wv
    X = U
    gc12 = pkg.chebfd_window_coeffs(a, b, -delta, delta, 12, "lanczos", 2.0)
    gc36 = pkg.chebfd_window_coeffs(a, b, -delta, delta, 36, "lanczos", 2.0)

    def df_step_time():
        pkg.chebfd_filter_block_df(H, alpha, beta, gc12, X)   # warm-up
        times = []
        for gc in (gc12, gc36):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            pkg.chebfd_filter_block_df(H, alpha, beta, gc, X)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
        return (times[1] - times[0]) / 24.0

    peak = peaks["hbm_gbs"]
    t_df = df_step_time()
    b_df = N * (13 * (16 + 4) + 5 * nb * 16)
    out["df_sell_step"] = {"kernel": "cheb_df_kernel (MODE_STEP, double-float complex, n_b=32)",
                           "bound": "hbm", "launch_us": t_df * 1e6, "bytes_per_launch": b_df,
                           "achieved": b_df / t_df / 1e9, "frac": b_df / t_df / 1e9 / peak}
    H.set_matrix_free(True)
    try:
        t_dff = df_step_time()
    finally:
        H.set_matrix_free(False)
    b_dff = N * 5 * nb * 16
    out["df_matrix_free_step"] = {
        "kernel": "stencil_df_kernel (MODE_STEP, double-float complex, n_b=32)", "bound": "hbm",
        "launch_us": t_dff * 1e6, "bytes_per_launch": b_dff, "achieved": b_dff / t_dff / 1e9,
        "frac": b_dff / t_dff / 1e9 / peak}
    out["peak_hbm_gbs"] = peak
    return out


DENSE_PHASES = ("gram", "block_gemm", "eigensolve", "hy", "residuals", "other")


LEARNED_FORMS = ("mlp", "mlp_matrix_free", "mlp_matrix_free_harmonic",
                 "mlp_matrix_free_harmonic_inset")


def warm_up_solves(pkg):
    """One-time initialisation outside the timed solves (the library's cuBLAS
    and cuSOLVER handles, lazily loaded kernels, the workspace pool): every
    precision and extraction once, stored-matrix and matrix-free, on the
    8x8x8x4 insulator with the benchmark's panel widths (n_s = 64)."""
    Hw = pkg.chebfd_matrix_create_lattice("topi", 8, 8, 8, t=1.0, m=1.0, W=0.5, seed=0,
                                          also_single=True)
    for free in (False, True):
        Hw.set_matrix_free(free)
        for prec in ("fp64", "mixed", "mixed_df"):
            for extraction in ("ritz", "harmonic"):
                pkg.chebfd_solve(Hw, -0.1, 0.1, 64, 40, eps=1e-9, kernel="lanczos",
                                 precision=prec, a=-4.6, b=4.6, max_iter=2, seed=0,
                                 extraction=extraction)


def bench_solve(pkg, H, a, b, delta, Np, ns, label, eps=1e-9, learned=True, chiral=True,
                precisions=("fp64", "mixed", "mixed_df"), matrix_free=False,
                learned_forms=LEARNED_FORMS):
    """Wall time of the whole ChebFD solve (Sec. 3.1 steps 4-8) to residual
    <= eps ||H|| for every accepted pair in [-delta, delta]: plain FP64 against
    the mixed forms (single-precision filter until the residuals stall, then
    FP64 or double-float sweeps; FP64 Gram, Rayleigh-Ritz and residuals
    throughout), and the mixed double-float form with the MLP's parameters,
    with `matrix_free` once more with H's entries rebuilt in registers in
    both the single-precision and the double-float steps, that once more
    with harmonic Ritz pairs for the window centre (Sec. 6), and that with
    the filter window narrowed by half its half-width at half the degree.
    A precision "mixed_df_matrix_free" is the heuristic-parameter MIXED_DF
    form with the matrix-free steps; learned_forms picks the learned ones."""
    import torch
    out = {}
    lams = {}
    warm_up_solves(pkg)
    torch.cuda.synchronize()

    def run(name, ns_r, Np_r, kern, prec, extra=None, t_pre=0.0, extraction="ritz",
            window_inset=0.0):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = pkg.chebfd_solve(H, -delta, delta, ns_r, Np_r, eps=eps, kernel=kern, precision=prec,
                             a=a, b=b, max_iter=40, seed=0, extraction=extraction,
                             window_inset=window_inset)
        torch.cuda.synchronize()
        t = time.perf_counter() - t0 + t_pre
        normH = max(abs(r["a"]), abs(r["b"]))
        lam = np.sort(r["lam"])
        lams[name] = lam
        out[name] = dict(extra or {})
        out[name].update({"seconds": t, "precision": prec, "iterations": r["iterations"],
                          "fp64_filter_iterations": r["fp64_iterations"], "nev": r["nev"],
                          "converged": r["converged"], "max_residual_over_normH":
                              float(r["res"].max() / normH) if r["nev"] else None,
                          "seconds_filter": r["seconds_filter"],
                          "seconds_dense": r["seconds_dense"], "n_mvm": r["n_mvm"],
                          "dense_breakdown_seconds": {
                              ph: sum(rec["seconds_" + ph] for rec in r["log"])
                              for ph in DENSE_PHASES},
                          "iterations_log": [
                              {"fp64_filter": rec["fp64_filter"], "in_window": rec["in_window"],
                               "ghosts": rec["ghosts"], "accepted": rec["accepted"],
                               "res_max": rec["res_max"]} for rec in r["log"]]})
        if chiral and r["nev"]:
            # spec(H) = -spec(H) for the insulator: the window set is +- paired
            out[name]["chiral_pairing_error"] = float(np.abs(lam + lam[::-1]).max())
        # against the first precision timed (the baseline: FP64 by default)
        base = precisions[0] if precisions else None
        if base and name != base and base in lams and len(lam) == len(lams[base]) and len(lam):
            out[name]["max_eigenvalue_difference_vs_%s" % base] = float(
                np.abs(lam - lams[base]).max())
        if base and name != base and base in out:
            out["speedup_%s_over_%s" % (name, base)] = out[base]["seconds"] / t

    for prec in precisions:
        if prec == "mixed_df_matrix_free":
            H.set_matrix_free(True)
            try:
                run(prec, ns, Np, "lanczos", "mixed_df")
            finally:
                H.set_matrix_free(False)
        else:
            run(prec, ns, Np, "lanczos", prec)
    # learned parameters: (N_p, n_s, kernel) from the trained MLP on the KPM
    # features of this matrix and window (its time is part of the solve's)
    wpath = os.path.join(ROOT, "paper_1510_04895_gb300", "data", "mlp_weights.npy")
    if learned and os.path.exists(wpath):
        from paper_1510_04895_gb300 import mlp_train
        net = pkg.MLP(mlp_train.N_IN, 128)
        net.set_params(np.load(wpath).astype(np.float32))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ns_m, Np_m, kern_m, nt = pkg.chebfd_choose_params(H, -delta, delta, mlp=net, a=a, b=b,
                                                          m_feat=mlp_train.M_FEAT)
        t_choose = time.perf_counter() - t0
        extra = {"ns": ns_m, "Np": Np_m, "kernel": kern_m, "kpm_n_target": nt,
                 "seconds_parameter_choice": t_choose}
        if "mlp" in learned_forms:
            run("mixed_df_mlp", ns_m, Np_m, kern_m, "mixed_df", extra=extra, t_pre=t_choose)
        if matrix_free:
            H.set_matrix_free(True)
            try:
                if "mlp_matrix_free" in learned_forms:
                    run("mixed_df_mlp_matrix_free", ns_m, Np_m, kern_m, "mixed_df", extra=extra,
                        t_pre=t_choose)
                if "mlp_matrix_free_harmonic" in learned_forms:
                    try:
                        run("mixed_df_mlp_matrix_free_harmonic", ns_m, Np_m, kern_m, "mixed_df",
                            extra=extra, t_pre=t_choose, extraction="harmonic")
                    except pkg.ChebFDError as e:     # reported; the other forms stand
                        out["mixed_df_mlp_matrix_free_harmonic"] = {"error": str(e)}
                # the window narrowed by half its half-width, half the degree
                Np_i = max(8, int(round(0.5 * Np_m)))
                if "mlp_matrix_free_harmonic_inset" in learned_forms:
                    try:
                        run("mixed_df_mlp_matrix_free_harmonic_inset", ns_m, Np_i, kern_m,
                            "mixed_df", extra=dict(extra, Np=Np_i, window_inset=0.5),
                            t_pre=t_choose, extraction="harmonic", window_inset=0.5)
                    except pkg.ChebFDError as e:
                        out["mixed_df_mlp_matrix_free_harmonic_inset"] = {"error": str(e)}
            finally:
                H.set_matrix_free(False)
    out["eps"] = eps
    out["workload"] = "%s, window [-%.6g, %.6g], n_s = %d, N_p = %d, Lanczos mu=2" % (
        label, delta, delta, ns, Np)
    return out


def run_ours(args):
    import torch

    import paper_1510_04895_gb300 as pkg
    from paper_1510_04895_gb300 import workloads

    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w, a, b, delta, Np = workload_params(args)
    cplx = w["cplx"]
    ns = w["ns"]
    single = args.precision in ("single", "c64", "r32")
    dtype_name = ("c64" if single else "c128") if cplx else ("r32" if single else "r64")
    panel = min(ns, {"c64": 64, "c128": 32, "r32": 128, "r64": 128}[dtype_name])
    nb = args.nb or panel
    H = pkg.chebfd_matrix_create_lattice(w["kind"], w["Lx"], w["Ly"], w["Lz"], t=w["t"],
                                         m=w["m"], W=w["W"], seed=w["seed"], sell_C=args.sell_C,
                                         also_single=True)
    N = H.n
    alpha, beta = 2.0 / (b - a), (a + b) / (a - b)
    gc = pkg.chebfd_window_coeffs(a, b, -delta, delta, Np, "lanczos", 2.0)
    cdt = {"c64": torch.complex64, "c128": torch.complex128, "r32": torch.float32,
           "r64": torch.float64}[dtype_name]
    X = torch.empty((N, ns), dtype=cdt, device=dev)
    pkg.chebfd_random_block(X, col0=0, ns_total=ns, seed=rank)
    stream = torch.cuda.current_stream()

    def step():
        # the library filters the n_s columns in row-major panels of its
        # widest panel for the value type (complex64 64, complex128 32, real 128)
        pkg.chebfd_filter_block(H, alpha, beta, gc, X)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier(world)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
    t_dev = e0.elapsed_time(e1) / 1e3
    barrier(world)
    units_rank = N * ns * Np * args.steps
    value, t_max = aggregate(world, units_rank, t_dev)
    launches = args.steps * ((ns + panel - 1) // panel) * Np

    # ---- dominant kernel alone: the fused Chebyshev step on one n_b block ------
    U = torch.empty((N, nb), dtype=cdt, device=dev)
    Wv = torch.empty_like(U)
    Y = torch.empty_like(U)
    pkg.chebfd_random_block(U, ns_total=nb, seed=11)
    pkg.chebfd_random_block(Wv, ns_total=nb, seed=12)
    Y.zero_()

    def time_step(reps=50, width=None):
        # width < nb: the step on the first `width` columns of the same blocks
        u_, w_, y_ = (U, Wv, Y) if width is None else (U[:, :width], Wv[:, :width], Y[:, :width])
        for _ in range(5):
            pkg.chebfd_chebyshev_step(H, alpha, beta, 1e-3, u_, w_, y_)
        torch.cuda.synchronize()
        k0, k1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        k0.record(stream)
        for i in range(reps):
            if i % 2 == 0:
                pkg.chebfd_chebyshev_step(H, alpha, beta, 1e-3, u_, w_, y_)
            else:
                pkg.chebfd_chebyshev_step(H, alpha, beta, 1e-3, w_, u_, y_)
        k1.record(stream)
        torch.cuda.synchronize()
        return k0.elapsed_time(k1) / 1e3 / reps

    blocked = single and H.blocked_width > 0
    t_launch = time_step()
    S_v = U.element_size()                      # bytes of one vector entry
    S_d = S_v                                   # matrix values stored at the same precision
    bytes_launch = N * (w["nnz_row"] * (S_d + 4) + 5 * nb * S_v)
    peaks, peak_kind = measured_peaks()
    achieved = bytes_launch / t_launch / 1e9
    kname = "bell_step_kernel" if blocked else "cheb_step_kernel"
    profile = w.get("profile_blocked") if blocked else w["profile"]
    traffic = read_traffic(profile) if profile and single and nb == w["profile_nb"] else None
    roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
            "kernel": "%s (MODE_STEP, %s, n_b=%d)" % (kname, dtype_name, nb),
            "bytes_per_launch": bytes_launch, "launch_us": t_launch * 1e6,
            "peak_kind": peak_kind + " (burst copy)"}
    if blocked:
        # the same step on the SELL arrays alone (row-wise kernel)
        H.set_blocked(False)
        t_sell = time_step()
        H.set_blocked(True)
        roof["sell_kernel"] = {"kernel": "cheb_step_kernel (MODE_STEP, %s, n_b=%d)" % (
            dtype_name, nb), "launch_us": t_sell * 1e6,
            "achieved": bytes_launch / t_sell / 1e9,
            "frac": bytes_launch / t_sell / 1e9 / peaks["hbm_gbs"]}
    # the same step at narrower block widths (strided panels of the same blocks)
    by_width = {}
    for width in (16, 32):
        if width < nb and (width * S_v) % 16 == 0:
            t_w = time_step(width=width)
            b_w = N * (w["nnz_row"] * (S_d + 4) + 5 * width * S_v)
            by_width[str(width)] = {"launch_us": t_w * 1e6, "achieved": b_w / t_w / 1e9,
                                    "frac": b_w / t_w / 1e9 / peaks["hbm_gbs"]}
    by_width[str(nb)] = {"launch_us": t_launch * 1e6, "achieved": achieved,
                         "frac": achieved / peaks["hbm_gbs"]}
    roof["by_block_width"] = by_width
    if single and w["kind"] == "topi":
        # matrix-free step: the insulator's entries rebuilt in registers
        H.set_matrix_free(True)
        t_mf = time_step()
        H.set_matrix_free(False)
        # its own algorithmic bytes: the five vector streams, no matrix
        vb = N * 5 * nb * S_v
        roof["matrix_free_kernel"] = {
            "kernel": "stencil_step_kernel (MODE_STEP, %s, n_b=%d)" % (dtype_name, nb),
            "launch_us": t_mf * 1e6, "bytes_per_launch": vb, "achieved": vb / t_mf / 1e9,
            "frac": vb / t_mf / 1e9 / peaks["hbm_gbs"],
            "speedup_over_stored_matrix_step": t_launch / t_mf}
    del U, Wv, Y
    if single and w["kind"] == "topi" and not args.no_fp64_kernels:
        torch.cuda.empty_cache()
        roof["fp64_kernels"] = fp64_class_kernels(pkg, H, N, alpha, beta, a, b, delta, peaks,
                                                  stream)

    # ---- end to end through the C ABI with host buffers ------------------------
    # chebfd_filter_block_host: the page-locked host block is streamed through
    # the device panel by panel (each panel copied in, filtered, copied back;
    # the copies of neighbouring panels overlap the filter); the whole block
    # crosses the link both ways every step
    Xh = torch.empty((N, ns), dtype=cdt, pin_memory=True)
    Xh.copy_(X)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e_steps = max(1, min(args.steps, 3))
    for _ in range(e_steps):
        pkg.chebfd_filter_block_host(H, alpha, beta, gc, Xh)
        torch.cuda.synchronize()
    t_e2e = (time.perf_counter() - t0) / e_steps
    t_e2e = barrier_max(world, t_e2e)
    e2e = {"value": world * N * ns * Np / t_e2e, "unit": UNIT,
           "h2d_bytes_per_step": X.numel() * X.element_size(),
           "d2h_bytes_per_step": X.numel() * X.element_size(),
           "api": "chebfd_filter_block_host (page-locked host block, copies overlapped)"}
    del Xh

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": dtype_name, "data": "synthetic",
           "config": {"workload": w["label"], "n_s": ns, "n_b": panel,
                      "N_p": Np, "kernel": "lanczos mu=2",
                      "window": [-delta, delta], "spectral_interval": [a, b],
                      "sell_C": args.sell_C,
                      "l2": "inputs larger than L2 (search block %.2f GB)" % (
                          X.numel() * X.element_size() / 1e9),
                      "parallelism": "independent search blocks per GPU (no collective)"},
           "roofline": roof, "e2e": e2e, "gpu_launches": launches,
           "clocks": clk.summary(),
           "hbm_gbs_filter_region": bytes_launch * launches / t_max / 1e9}
    del X

    if not args.no_ensemble and w["kind"] == "topi":
        out["ensemble"] = bench_ensemble(pkg, workloads, dev, peaks["hbm_gbs"])
    torch.cuda.empty_cache()     # the solve allocates its own blocks
    if not args.no_solve:
        # the MLP was trained on insulators only: learned parameters for those
        try:
            out["time_to_solution"] = bench_solve(pkg, H, a, b, delta, Np, ns, w["label"],
                                                  learned=w["kind"] == "topi",
                                                  chiral=w["kind"] == "topi",
                                                  precisions=args.solve_precisions,
                                                  matrix_free=w["kind"] == "topi",
                                                  learned_forms=args.solve_forms)
        except pkg.ChebFDError as e:     # reported, the throughput line still prints
            out["time_to_solution"] = {"error": str(e)}

    if rank == 0 and not args.no_cpu_baseline:
        v, dt, desc = oracle_sample(w, a, b, delta, args.cpu_steps)
        out["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                               "sample": desc, "seconds": dt}
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_profile(args):
    """Short, self-contained launch sequences for an ncu capture (no timing):
    `step`  five fused Chebyshev steps on the workload's lattice (n_b = --nb,
            value type --precision, --form blocked | sell | free);
    `df`    one double-float filter of degree 8 on --nb complex columns
            (--form sell | free);
    `solve` one ChebFD iteration (filter of degree 20, SVQB, Rayleigh-Ritz) on
            the 32x32x32x4 insulator (N = 131072, W = 1, seed 1), n_s = 256,
            --solve-precisions[0] (fp64 | mixed_df);
    `pairs` a complex64 filter of degree 4 on 16 columns of the insulator,
            matrix-free: first with the fused two-step kernel (one launch for
            steps 3-4), then with single steps (two launches);
    `gram`  the tall Gram A^H A of a 131072 x 256 complex128 block (seeded
            uniform entries), once by each method of chebfd_gram: tensor,
            double_float, fp64 (cuBLAS)."""
    import torch

    import paper_1510_04895_gb300 as pkg
    from paper_1510_04895_gb300 import workloads
    if args.profile == "gram":
        A = torch.from_numpy(workloads.random_block(7, 131072, 256, True)).to("cuda")
        for method in ("tensor", "double_float", "fp64"):
            pkg.chebfd_gram(A, method=method)
        torch.cuda.synchronize()
        print("profile target done")
        return 0
    name = args.workload
    w = dict(getattr(workloads, WORKLOADS[name]["spec"]))
    if args.profile == "solve":
        w.update(Lx=32, Ly=32, Lz=32)
    H = pkg.chebfd_matrix_create_lattice(w["kind"], w["Lx"], w["Ly"], w.get("Lz", 1), t=w["t"],
                                         m=w.get("m", 0.0), W=w["W"], seed=w["seed"],
                                         also_single=True)
    if args.form == "sell" and H.blocked_width:
        H.set_blocked(False)
    if args.form == "free":
        H.set_matrix_free(True)
    if args.profile == "pairs":
        X = torch.empty((H.n, 16), dtype=torch.complex64, device="cuda")
        gc = pkg.chebfd_window_coeffs(-4.2, 4.2, -0.14, 0.14, 4, "lanczos", 2.0)
        for pairs in (True, False):
            pkg.chebfd_random_block(X, ns_total=16, seed=1)
            H.set_matrix_free(True, pairs=pairs)
            pkg.chebfd_filter_block(H, 2.0 / 8.4, 0.0, gc, X)
    elif args.profile == "df":
        nb = args.nb or 32
        X = torch.empty((H.n, nb), dtype=torch.complex128, device="cuda")
        pkg.chebfd_random_block(X, ns_total=nb, seed=1)
        gc = pkg.chebfd_window_coeffs(-4.3, 4.3, -0.1, 0.1, 8, "lanczos", 2.0)
        pkg.chebfd_filter_block_df(H, 2.0 / 8.6, 0.0, gc, X)
    elif args.profile == "solve":
        pkg.chebfd_solve(H, -0.14, 0.14, 256, 20, eps=1e-9, kernel="lanczos",
                         precision=args.solve_precisions[0], a=-4.2, b=4.2, max_iter=1, seed=0)
    else:
        single = args.precision in ("single", "c64", "r32")
        cplx = w["kind"] != "graphene"
        dt = ({True: torch.complex64, False: torch.complex128} if cplx else
              {True: torch.float32, False: torch.float64})[single]
        nb = args.nb or w["nb"]
        U = torch.empty((H.n, nb), dtype=dt, device="cuda")
        W = torch.empty_like(U)
        Y = torch.zeros_like(U)
        pkg.chebfd_random_block(U, ns_total=nb, seed=1)
        pkg.chebfd_random_block(W, ns_total=nb, seed=2)
        for _ in range(5):
            pkg.chebfd_chebyshev_step(H, 0.24, 0.0, 1e-3, U, W, Y)
    torch.cuda.synchronize()
    print("profile target done")
    return 0


def main():
    p = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="topi", choices=sorted(WORKLOADS))
    p.add_argument("--nb", type=int, default=0, help="block width (0: the workload's)")
    p.add_argument("--precision", default="single",
                   choices=["single", "double", "c64", "c128", "r32", "r64"])
    p.add_argument("--Np", type=int, default=0)
    p.add_argument("--sell-C", dest="sell_C", type=int, default=1)
    p.add_argument("--cpu-steps", dest="cpu_steps", type=int, default=8)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-ensemble", action="store_true")
    p.add_argument("--no-solve", action="store_true")
    p.add_argument("--no-fp64-kernels", dest="no_fp64_kernels", action="store_true")
    p.add_argument("--solve-precisions", dest="solve_precisions", nargs="*",
                   default=["fp64", "mixed", "mixed_df"],
                   help="precisions of the time-to-solution runs (the MLP run is extra)")
    p.add_argument("--solve-forms", dest="solve_forms", nargs="*", default=list(LEARNED_FORMS),
                   choices=list(LEARNED_FORMS),
                   help="the learned-parameter solve forms to time")
    p.add_argument("--profile", choices=["step", "df", "solve", "pairs", "gram"], default=None,
                   help="run a short launch sequence for an ncu capture and exit")
    p.add_argument("--form", choices=["blocked", "sell", "free"], default="blocked",
                   help="--profile: insulator step on the blocked copy, the SELL arrays, or "
                        "matrix-free")
    args = p.parse_args()
    if args.profile:
        return run_profile(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
