"""Benchmark: Newton solves/s of the 3D Bratu problem on the NURBS quarter annulus.

Workload (default, one GPU): -lap u - 2 e^u = 0 on the quarter annulus extruded in z
(radii 1 and 2, height 1; rational quadratic in theta raised to cubic C2), 64^3
elements, 4^3 Gauss points, homogeneous Dirichlet on all faces, FP64 throughout;
one step = one Newton-GMRES(Jacobi) solve from U = 0 to ||F||_2 <= 1e-10 through
the C ABI (residual assembly, Jacobian assembly, Krylov, line search).
The discretisation (knots, tables, CSR pattern, geometry factors) is set up once
per process, outside the timed region; its time is reported as setup_ms.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank solves its own replica (weak scaling); rank 0
prints one JSON line.  --impl reference times the oracle (plain C, one thread) on
a bounded sample of the same workload and prints the same metric.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "assembled Jacobian nnz/s & Newton solves/s to ||F||≤1e-10, FP64 vs mixed/NN"
UNIT = "solves/s"
NEL, P, LAM = 64, 3, 2.0
# FP64 peak of GB300: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.070 GHz (max SM clock)
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ----------------------------------------------------------------- clocks ---
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.dev = dev
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.dev)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=2)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------ CPU oracle ---
def oracle_sample(min_seconds=10.0, newton_its=3):
    """Time the oracle's residual and Jacobian assembly on an 8x8x8-element block of
    the same discretisation (degree, rule, rational geometry, lambda) until at
    least min_seconds of CPU work, extrapolate per element to the 64^3 mesh, and
    convert to solves/s with one Jacobian + one residual per Newton step (plus the
    final residual).  The oracle's linear solves are not counted, so the figure
    favours the CPU."""
    import numpy as np
    import oracle as O
    from paper_1305_4452_gb300 import workloads as W
    sub = 8
    kn, ctrl, w = W.quarter_annulus(sub, P)
    prob = O.Problem(kn, [P] * 3, ctrl=ctrl, weights=w, lam=LAM, dirichlet={(a, s): 0.0 for a in range(3) for s in range(2)})
    U = W.interior_field([sub + P] * 3, 2)
    prob.pattern()
    tr, tj, reps = 0.0, 0.0, 0
    t_start = time.time()
    while reps == 0 or time.time() - t_start < min_seconds:
        t = time.perf_counter(); prob.residual(U); tr += time.perf_counter() - t
        t = time.perf_counter(); prob.jacobian(U); tj += time.perf_counter() - t
        reps += 1
    scale = (NEL ** 3) / float(sub ** 3)
    tr_full, tj_full = tr / reps * scale, tj / reps * scale
    t_solve = newton_its * (tr_full + tj_full) + tr_full
    return {"value": 1.0 / t_solve, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "oracle residual+Jacobian assembly of an 8^3-element block of the annulus (p=3, 4^3 Gauss points, "
                      "lambda=2), %d repetitions (%.1f s), extrapolated x%d to 64^3 and to %d Newton steps; linear solves "
                      "not counted" % (reps, time.time() - t_start, int(scale), newton_its),
            "residual_s_full_mesh": tr_full, "jacobian_s_full_mesh": tj_full}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle as O
    O.build()
    per_step = []
    for _ in range(args.warmup):
        oracle_sample(min_seconds=0.0)
    cb = None
    for _ in range(args.steps):
        cb = oracle_sample(min_seconds=0.0)
        per_step.append(1.0 / cb["value"])
    value = len(per_step) / sum(per_step)
    cb = dict(cb)
    cb["value"] = value
    line = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(per_step) / len(per_step),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(None), "cpu_baseline": cb,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def config_dict(disc):
    d = {"workload": "bratu3d_quarter_annulus_%dcubed_p3_C2_lambda2_fp64_newton_gmres_jacobi" % NEL,
         "elements": NEL ** 3, "degree": P, "gauss_points_per_elem": (P + 1) ** 3, "lambda": LAM,
         "newton_atol": 1e-10, "start": "U=0", "l2": "inputs larger than L2 (CSR values 0.76 GB + geometry factors 2.1 GB per solve)"}
    if disc is not None:
        d["dofs"] = disc.N
        d["nnz"] = disc.nnz
    return d


# ------------------------------------------------------ replica timing -----
def max_over_ranks(value, world, device):
    """The job's time is its slowest rank's: MAX all-reduce of a per-rank time (the
    process group must exist when world > 1; gloo on the CPU, NCCL on GPUs)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


def job_throughput(world, steps, seconds):
    """Whole-job solves per second: every rank solves `steps` independent problems."""
    return world * steps / seconds


# ------------------------------------------------------------- our arm -----
def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_1305_4452_gb300 import build, iga, workloads as W

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    build.build()
    stream = torch.cuda.current_stream()

    t0 = time.perf_counter()
    kn, ctrl, w = W.quarter_annulus(NEL, P)
    bc = {(a, s): 0.0 for a in range(3) for s in range(2)}
    disc = iga.Discretization(3, P, knots=kn, ctrl=ctrl, weights=w, lam=LAM, dirichlet=bc)
    torch.cuda.synchronize()
    setup_ms = 1e3 * (time.perf_counter() - t0)
    N = disc.N
    U0 = torch.zeros(N, dtype=torch.float64, device="cuda")
    U = torch.empty_like(U0)
    opts = iga.newton_defaults()

    def solve():
        U.copy_(U0)
        return disc.solve_newton(U, opts)

    for _ in range(args.warmup):
        rep = solve()
    # dominant kernel classes are timed with events on the library's stream
    disc.profile_enable(["jac_stage1", "jac_stage2", "jac_final", "spmv", "residual_element", "gs_orth"])
    disc.profile_read()
    clocks = ClockSampler(local)
    clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    reps = []
    for _ in range(args.steps):
        reps.append(solve())
    ev1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    prof = disc.profile_read()
    disc.profile_enable([])
    ms = max_over_ranks(ms, world, "cuda")
    value = job_throughput(world, args.steps, ms / 1e3)
    launches = sum(v[2] for v in prof.values())

    # end to end through the host-buffer entry point (H2D of U0, D2H of the solution)
    Uh = torch.zeros(N, dtype=torch.float64).pin_memory()
    Uh_np = Uh.numpy()
    for _ in range(1):
        Uh.zero_()
        disc.solve_newton_host(Uh_np, opts)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(args.steps):
        Uh.zero_()
        disc.solve_newton_host(Uh_np, opts)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t
    e2e_s = max_over_ranks(e2e_s, world, "cuda")
    e2e = {"value": job_throughput(world, args.steps, e2e_s), "unit": UNIT, "h2d_bytes_per_step": N * 8,
           "d2h_bytes_per_step": N * 8}

    # secondary throughputs of the FP64 assembly calls (same discretisation)
    Ur = torch.tensor(W.interior_field([NEL + P] * 3, 2), device="cuda")
    F = torch.empty_like(Ur)
    J = torch.empty(disc.nnz, dtype=torch.float64, device="cuda")

    def timeit(fn, n):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(n):
            fn()
        b.record(stream)
        b.synchronize()
        return a.elapsed_time(b) / n

    t_res = timeit(lambda: disc.form_residual(Ur, F), 10)
    t_jac = timeit(lambda: disc.form_jacobian(Ur, vals=J), 3)
    # matrix-free Newton-Krylov on the same problem (exact products, no assembled Jacobian):
    # one product, and one whole solve, outside the timed region
    xr = torch.ones_like(U0)
    t_jv = timeit(lambda: disc.apply_jacobian_mf(Ur, xr, F), 5)
    o_mf = iga.newton_defaults()
    o_mf.jac = iga.IGA_JAC_NONE
    Umf = torch.zeros_like(U0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r_mf = disc.solve_newton(Umf, o_mf)
    torch.cuda.synchronize()
    mf = {"solve_ms": 1e3 * (time.perf_counter() - t0), "newton_its": r_mf.newton_its, "krylov_its": r_mf.krylov_its,
          "fnorm": r_mf.fnorm, "jv_ms": t_jv, "spmv_ms_for_comparison": prof["spmv"][0] / max(prof["spmv"][1], 1),
          "csr_bytes_avoided": disc.nnz * 8}

    # roofline of the dominant kernel class in the timed region
    hbm, hbm_src = peaks()
    dom = max(prof, key=lambda c: prof[c][0])
    dms, dn, _ = prof[dom]
    avg_ms = dms / max(dn, 1)
    roof = roofline_entry(disc, dom, avg_ms, hbm, hbm_src)

    r = reps[-1]
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config_dict(disc),
            "parallelism": "replicas" if world > 1 else "single",
            "e2e": e2e, "gpu_launches": int(launches), "clocks": clk, "roofline": roof,
            "newton": {"its": r.newton_its, "krylov_its": r.krylov_its, "fnorm0": r.fnorm0, "fnorm": r.fnorm},
            "kernel_share": {c: round(v[0] / max(ms, 1e-9), 4) for c, v in prof.items() if v[1] > 0},
            "assembly_fp64": {"jacobian_ms": t_jac, "jacobian_nnz_per_s": disc.nnz / (t_jac / 1e3),
                              "residual_ms": t_res, "residual_dofs_per_s": N / (t_res / 1e3)},
            "matrix_free_newton": mf,
            "setup_ms": setup_ms}
    if rank == 0 and world == 1 and args.cpu_seconds > 0:
        import oracle as O
        O.build()
        line["cpu_baseline"] = oracle_sample(min_seconds=args.cpu_seconds, newton_its=r.newton_its)
    if rank == 0:
        print(json.dumps(line))
    disc.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


# DRAM bytes (read + write) of one k_spmv_stencil launch on the 64^3 annulus, from one ncu
# capture of this benchmark (profiles/k_spmv_stencil_annulus64_fp64_traffic.md); valid for
# that workload and the kernel as captured.
SPMV_DRAM_BYTES_ANNULUS64 = 803.45e6 + 4.97e6


def roofline_entry(disc, cls, avg_ms, hbm_gbs, hbm_src):
    """Algorithmic work of one launch of the given kernel class on this workload."""
    N, nnz = disc.N, disc.nnz
    nq = (P + 1) ** 3
    nel1 = NEL
    npair = nel1 * (P + 1) ** 2 * (P + 1)  # sum over 1D pairs of their Gauss points: nel (p+1)^2 q
    X = NEL * (P + 1)
    P1 = sum(min(i, P) + min(NEL + P - 1 - i, P) + 1 for i in range(NEL + P))  # 1D pairs
    if cls == "spmv":
        # values (columns follow from the stencil), rowptr, x read, y written; one FP64 FMA per
        # stored value.  At 8 B per FMA this product is bound by GB300's FP64 pipe, not by HBM.
        bytes_ = nnz * 8 + (N + 1) * 8 + 2 * N * 8
        flops = 2.0 * nnz
        t = avg_ms * 1e-3
        hbm_frac = bytes_ / t / 1e9 / hbm_gbs
        fp_frac = flops / t / 1e12 / FP64_PEAK_TFLOPS
        traffic = SPMV_DRAM_BYTES_ANNULUS64 if NEL == 64 else None
        return {"kernel": "k_spmv_stencil (FP64 values, stencil columns)", "bound": "alu", "achieved": flops / t / 1e12,
                "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": fp_frac, "traffic": traffic,
                "peak_source": "derived: 152 SM x 2 DFMA/clk x 2.07 GHz",
                "algorithmic_flops_per_launch": flops, "algorithmic_bytes_per_launch": bytes_,
                "hbm": {"achieved_gbs": bytes_ / t / 1e9, "peak_gbs": hbm_gbs, "frac": hbm_frac, "peak_source": hbm_src}}
    if cls == "jac_stage1":
        flops = 2.0 * 16 * npair * X * X  # 16 terms x sum of pair points per line x lines (stiffness launch)
    elif cls == "jac_stage2":
        flops = 2.0 * 9 * P1 * X * npair
    elif cls == "jac_final":
        flops = 2.0 * 4 * P1 * P1 * npair
    elif cls == "residual_element":
        n1, q = P + 1, P + 1
        fwd = 2 * n1 * n1 * q * n1 + 3 * n1 * q * q * n1 + 4 * q ** 3 * n1
        flops = 2.0 * NEL ** 3 * (2 * fwd + 14 * nq)
    else:
        return {"kernel": cls, "bound": "alu", "achieved": None, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": None, "traffic": None}
    ach = flops / (avg_ms * 1e-3) / 1e12
    return {"kernel": cls, "bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": ach / FP64_PEAK_TFLOPS, "traffic": None, "peak_source": "derived: 152 SM x 2 DFMA/clk x 2.07 GHz",
            "algorithmic_flops_per_launch": flops}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--nel", type=int, default=64, help="elements per direction (64 is the benchmark workload)")
    ap.add_argument("--cpu-seconds", type=float, default=10.0, help="CPU-baseline sampling time (0: skip)")
    ap.add_argument("--workload", default="annulus64",
                    choices=["annulus64", "bratu16", "cube_mixed", "batch512", "learned64", "nn64", "fdjac", "genalpha", "periodic64", "mixed64"],
                    help="annulus64 is the benchmark line; the others print their configuration's line")
    args = ap.parse_args()
    if args.workload != "annulus64" and args.impl == "ours":
        import torch
        import bench_workloads as BW
        from paper_1305_4452_gb300 import build, iga, workloads as W
        build.build()
        torch.cuda.set_device(0)
        print(BW.WORKLOADS[args.workload](torch, iga, W, ClockSampler(0)))
        return 0
    global NEL
    NEL = args.nel
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
