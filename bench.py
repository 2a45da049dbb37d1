"""Benchmark: Newton solves/s of the 3D Bratu problem on the NURBS quarter annulus.

Workload (default, one GPU): -lap u - 2 e^u = 0 on the quarter annulus extruded in z
(radii 1 and 2, height 1; rational quadratic in theta raised to cubic C2), 64^3
elements, 4^3 Gauss points, homogeneous Dirichlet on all faces, FP64 throughout;
one step = one Newton-GMRES(Jacobi) solve from U = 0 to ||F||_2 <= 1e-10 through
the C ABI (residual assembly, Jacobian assembly, Krylov, line search).
The discretisation (knots, tables, CSR pattern, geometry factors) is set up once
per process, outside the timed region; its time is reported as setup_ms.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--no-extras]

Under torchrun (N > 1) every rank solves its own replica (weak scaling); rank 0
prints one JSON line.  The value is timed with the library's per-launch profiler
off; a second, profiled pass over the same solves gives the kernel shares and the
roofline of the dominant kernel, against FP64/FP32/copy peaks measured in the same
process (iga_measure_peaks).  Extra keys (skipped with --no-extras) carry the
other half of the metric: Newton solves/s of the 128^3 quadratic cube with the
FP64 Jacobian against the reduced-precision ones (same Krylov method each), and
the learned initial guess against the zero start on held-out kappa fields.
--impl reference times the oracle (plain C, colour-loop timing mode on all host
cores) on a bounded sample of the same workload and prints the same metric.
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


def hbm_peak():
    """The measured copy bandwidth of the GB300s, else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured (copy, MEASURED_PEAKS.json)"
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
def _oracle_problem(nel, p=P):
    import oracle as O
    from paper_1305_4452_gb300 import workloads as W
    kn, ctrl, w = W.quarter_annulus(nel, p)
    prob = O.Problem(kn, [p] * 3, ctrl=ctrl, weights=w, lam=LAM, dirichlet={(a, s): 0.0 for a in range(3) for s in range(2)})
    n = [len(k) - p - 1 for k in kn]
    return prob, W.interior_field(n, 2)


def oracle_whole_mesh(newton_its):
    """The oracle's residual and Jacobian assembly of the whole benchmark mesh, each timed
    once, in its colour-loop timing mode on every OpenMP thread of this host (the same
    element arithmetic as the serial oracle, elements of one colour spread over the
    threads).  Solves/s counts (newton_its + 1) residuals and newton_its Jacobians per
    solve, as the GPU's Newton takes; the oracle's linear solves are not counted, so the
    figure favours the CPU."""
    import oracle as O
    O.build()
    prob, U = _oracle_problem(NEL)
    t0 = time.perf_counter()
    prob.pattern()
    t_pat = time.perf_counter() - t0
    t = time.perf_counter(); prob.residual_colored(U); tr = time.perf_counter() - t
    t = time.perf_counter(); prob.jacobian_colored(U); tj = time.perf_counter() - t
    t_solve = newton_its * (tr + tj) + tr
    return {"value": 1.0 / t_solve, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
            "sample": "oracle residual and Jacobian of the whole %d^3 annulus mesh (p=3, 4^3 Gauss points, lambda=2), "
                      "each timed once in the colour-loop timing mode on %d OpenMP threads: %.2f s + %.2f s; solve = "
                      "%d Jacobians + %d residuals (the GPU solve's Newton steps); linear solves not counted"
                      % (NEL, O.num_threads(), tr, tj, newton_its, newton_its + 1),
            "residual_s": tr, "jacobian_s": tj, "pattern_s": t_pat}


SLAB = 8


def oracle_step(newton_its, prob, U, sl, Us):
    """One step of the reference arm: the oracle's residual of the whole mesh (prob, U)
    and its Jacobian on a slab of nel x nel x SLAB elements of the same discretisation
    (sl, Us; the Jacobian's cost per element does not depend on the slab), both in the
    colour-loop timing mode.  Returns (solves/s for the whole mesh, seconds of the step)."""
    t0 = time.perf_counter()
    prob.residual_colored(U)
    tr = time.perf_counter() - t0
    t = time.perf_counter()
    sl.jacobian_colored(Us)
    tj = (time.perf_counter() - t) * NEL / float(SLAB)
    return 1.0 / (newton_its * (tr + tj) + tr), time.perf_counter() - t0


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle as O
    O.build()
    its = 3  # Newton steps of the GPU's solve of this workload (its JSON line reports them)
    prob, U = _oracle_problem(NEL)
    sl, Us = _oracle_problem((NEL, NEL, SLAB))
    sl.pattern()
    for _ in range(args.warmup):
        oracle_step(its, prob, U, sl, Us)
    vals, secs = [], []
    for _ in range(args.steps):
        v, s = oracle_step(its, prob, U, sl, Us)
        vals.append(v)
        secs.append(s)
    value = len(vals) / sum(1.0 / v for v in vals)
    cb = {"value": value, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
          "sample": "per step: the oracle's residual of the whole %d^3 annulus mesh and its Jacobian on a %dx%dx8-element "
                    "slab (scaled x%d), colour-loop timing mode on %d OpenMP threads; solve = %d Jacobians + %d residuals; "
                    "linear solves not counted" % (NEL, NEL, NEL, NEL // SLAB, O.num_threads(), its, its + 1)}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(secs) / len(secs),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(None), "cpu_baseline": cb,
            "note": "ms_per_step is the wall time of one sampled step; value is the whole-mesh solve rate it implies",
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
    pk = iga.measure_peaks()  # FP64/FP32 FMA and copy rates of this GPU, measured now

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
    # timed region: the library's event profiler is off (launches are still counted)
    disc.profile_enable([])
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
    launches = sum(v[2] for v in disc.profile_read().values())
    ms = max_over_ranks(ms, world, "cuda")
    value = job_throughput(world, args.steps, ms / 1e3)

    # profiled pass over the same solves: per-class device times (CUDA events on the
    # library's stream, around each launch) for the kernel shares and the roofline
    disc.profile_enable(["jac_stage1", "jac_stage2", "jac_final", "spmv", "residual_element", "residual_gather", "q00",
                         "gs_orth", "vector", "gmres_scalar"])
    disc.profile_read()
    torch.cuda.synchronize()
    p0 = time.perf_counter()
    for _ in range(args.steps):
        solve()
    torch.cuda.synchronize()
    prof_ms = 1e3 * (time.perf_counter() - p0)
    prof = disc.profile_read()
    disc.profile_enable([])

    # end to end through the host-buffer entry point (H2D of U0, D2H of the solution)
    Uh = torch.zeros(N, dtype=torch.float64).pin_memory()
    Uh_np = Uh.numpy()
    Uh.zero_()
    disc.solve_newton_host(Uh_np, opts)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t = time.perf_counter()
    step_s = []
    for _ in range(args.steps):
        t1 = time.perf_counter()
        Uh.zero_()
        disc.solve_newton_host(Uh_np, opts)
        step_s.append(time.perf_counter() - t1)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t
    e2e_s = max_over_ranks(e2e_s, world, "cuda")
    e2e = {"value": job_throughput(world, args.steps, e2e_s), "unit": UNIT, "h2d_bytes_per_step": N * 8,
           "d2h_bytes_per_step": N * 8,
           "step_ms": {"min": 1e3 * min(step_s), "median": 1e3 * statistics.median(step_s), "max": 1e3 * max(step_s)}}

    # the same solve with classical Gram-Schmidt applied twice in every GMRES step (the
    # IGA_CGS_REFINE_ALWAYS option; the default is one pass, PETSc's refinement type)
    o2 = iga.newton_defaults()
    o2.gmres_cgs_refine = iga.IGA_CGS_REFINE_ALWAYS
    U.copy_(U0)
    disc.solve_newton(U, o2)
    torch.cuda.synchronize()
    c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n2 = min(args.steps, 3)
    c0.record(stream)
    for _ in range(n2):
        U.copy_(U0)
        r2 = disc.solve_newton(U, o2)
    c1.record(stream)
    c1.synchronize()
    cgs2 = {"ms_per_solve": c0.elapsed_time(c1) / n2, "krylov_its": r2.krylov_its, "newton_its": r2.newton_its,
            "fnorm": r2.fnorm, "solutions_max_abs_diff": (U - Uh.to(U.device)).abs().max().item()}

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
    del J
    # matrix-free Newton-Krylov on the same problem (exact products, no assembled Jacobian)
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

    # roofline of the dominant kernel class of the profiled pass
    hbm, hbm_src = hbm_peak()
    dom = max(prof, key=lambda c: prof[c][0])
    dms, dn, _ = prof[dom]
    used = None
    if dom == "spmv":
        used = fixed_product_entries(torch, disc, [len(k) - P - 1 for k in kn], list(bc))
        torch.cuda.empty_cache()
    roof = roofline_entry(disc, dom, dms / max(dn, 1), hbm, hbm_src, pk, used)

    r = reps[-1]
    solve_s = ms / args.steps / 1e3
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config_dict(disc),
            "parallelism": "replicas" if world > 1 else "single",
            "e2e": e2e, "gpu_launches": int(launches), "clocks": clk, "roofline": roof,
            "peaks_measured": {"fp64_tflops": pk["fp64_tflops"], "fp32_tflops": pk["fp32_tflops"],
                               "copy_gbs": pk["copy_gbs"], "sms": pk["sms"],
                               "how": "iga_measure_peaks: DFMA/FFMA chains on every SM, 512 MiB copy; best of 5-10"},
            "newton": {"its": r.newton_its, "krylov_its": r.krylov_its, "fnorm0": r.fnorm0, "fnorm": r.fnorm},
            "kernel_share": {c: round(v[0] / max(prof_ms, 1e-9), 4) for c, v in prof.items() if v[1] > 0},
            "profiled_pass_ms_per_step": prof_ms / args.steps,
            "assembly_fp64": {"jacobian_ms": t_jac, "jacobian_nnz_per_s": disc.nnz / (t_jac / 1e3),
                              "residual_ms": t_res, "residual_dofs_per_s": N / (t_res / 1e3)},
            "matrix_free_newton": mf,
            "gmres_cgs_refine_always": cgs2,
            "setup_ms": setup_ms,
            # a solve on a mesh not seen before: set-up (tables, pattern, geometry factors) plus the solve
            "new_mesh": {"solves_per_s": 1.0 / (setup_ms / 1e3 + solve_s), "setup_ms": setup_ms,
                         "solve_ms": solve_s * 1e3}}
    disc.close()
    del Ur, F, xr, Umf, U, U0
    torch.cuda.empty_cache()
    if rank == 0 and world == 1 and not args.no_extras:
        line["fp64_vs_mixed"] = mixed_comparison(torch, iga, W)
        torch.cuda.empty_cache()
        line["learned_start"] = learned_comparison(torch, iga, W)
        torch.cuda.empty_cache()
    if rank == 0 and world == 1 and args.cpu_seconds > 0:
        line["cpu_baseline"] = oracle_whole_mesh(r.newton_its)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


# ------------------------------------------- the metric's second half ------
def mixed_comparison(torch, iga, W, nel=128, p=2, reps=3):
    """3D Bratu, lambda = 2, on the unit cube, 128^3 quadratic (2.2M dofs, 267M nnz): Newton
    solves from U = 0 to ||F||_2 <= 1e-10 with the FP64 Jacobian and with the reduced-precision
    ones (FP32 sum factorisation, BF16 and TF32 tensor-core element matrices), each with GMRES
    and with CG (the same Krylov method on both sides of every ratio); residual, norms and
    orthogonalisation are FP64 in every run.  Best of `reps` solves after one warm-up.
    Jacobian errors: relative Frobenius distance to the FP64 Jacobian at seeded U ~ U[-0.1,
    0.1] (the FP64 Jacobian equals the oracle's to 1e-12 in the parity tests)."""
    bc = {(a, s): 0.0 for a in range(3) for s in range(2)}
    d = iga.Discretization(3, p, nel=nel, lam=2.0, dirichlet=bc)
    out = {"workload": "bratu3d_cube_%dcubed_p%d_lambda2_from_zero" % (nel, p), "dofs": d.N, "nnz": d.nnz}
    Ur = torch.tensor(W.interior_field([nel + p] * 3, 3), device="cuda")
    J = torch.empty(d.nnz, dtype=torch.float64, device="cuda")
    J32 = torch.empty(d.nnz, dtype=torch.float32, device="cuda")
    d.form_jacobian(Ur, vals=J)
    nJ = torch.linalg.norm(J).item()
    modes = [("fp64", iga.IGA_FP64), ("fp32", iga.IGA_JAC_FP32), ("bf16", iga.IGA_JAC_BF16), ("tf32", iga.IGA_JAC_TF32)]
    jac = {}
    for name, code in modes:
        if code == iga.IGA_FP64:
            t = _best_ms(torch, lambda: d.form_jacobian(Ur, vals=J), 3)
            jac[name] = {"ms": t, "nnz_per_s": d.nnz / (t * 1e-3), "rel_frobenius_error_vs_fp64": 0.0}
            continue
        t = _best_ms(torch, lambda: d.form_jacobian(Ur, prec=code, vals=J32), 3)
        err = (torch.linalg.norm(J32.double() - J) / nJ).item()
        jac[name] = {"ms": t, "nnz_per_s": d.nnz / (t * 1e-3), "rel_frobenius_error_vs_fp64": err}
    out["jacobian"] = jac
    del J, J32
    torch.cuda.empty_cache()
    U = torch.zeros(d.N, dtype=torch.float64, device="cuda")
    solves = {}
    for ksp_name, ksp in (("gmres", iga.IGA_KSP_GMRES), ("cg", iga.IGA_KSP_CG)):
        for name, code in modes:
            o = iga.newton_defaults()
            o.jac, o.ksp = code, ksp
            U.zero_()
            d.solve_newton(U, o)
            best, rep = 1e30, None
            for _ in range(reps):
                U.zero_()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                rep = d.solve_newton(U, o)
                torch.cuda.synchronize()
                best = min(best, time.perf_counter() - t0)
            solves["%s_%s" % (name, ksp_name)] = {"solves_per_s": 1.0 / best, "ms": best * 1e3, "newton_its": rep.newton_its,
                                                  "krylov_its": rep.krylov_its, "fnorm": rep.fnorm}
        base = solves["fp64_%s" % ksp_name]["solves_per_s"]
        for name, _ in modes:
            solves["%s_%s" % (name, ksp_name)]["speedup_vs_fp64_same_krylov"] = solves["%s_%s" % (name, ksp_name)]["solves_per_s"] / base
    out["newton"] = solves
    d.close()
    return out


def learned_comparison(torch, iga, W):
    """kappa-Bratu on 64^2 quadratic elements: the convolutional initial guess (trained in this
    process on 20k seeded solves of the batched solver) against the zero start, 2,000
    held-out fields, batched Newton; the network start's wall time includes inference."""
    import bench_workloads as BW
    res, _, _ = BW.learned_core(torch, iga, W)
    return res


def _best_ms(torch, fn, reps):
    fn()
    torch.cuda.synchronize()
    best = 1e30
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        b.synchronize()
        best = min(best, a.elapsed_time(b))
    return best


# DRAM bytes (read + write) of one Krylov operator product (k_spmv_fixed, FP64 values) on
# the 64^3 annulus, from one ncu capture of this benchmark's command (named in the JSON
# line); valid for that workload while the kernel is unchanged (None: not captured).
SPMV_DRAM_BYTES_ANNULUS64 = 751.96e6 + 2.00e6
SPMV_TRAFFIC_CAPTURE = ("profiles/k_spmv_fixed_annulus64_fp64_traffic.md: ncu --metrics "
                        "dram__bytes_read.sum,dram__bytes_write.sum --clock-control none -k regex:k_spmv_fixed")


def fixed_product_entries(torch, disc, n, faces):
    """Stored CSR entries that the product with the Dirichlet-fixed Newton Jacobian
    (k_spmv_fixed) multiplies: those of rows off the Dirichlet faces, less the columns on
    a Dirichlet face of the last axis (a contiguous part of each row, which the kernel
    skips); the Dirichlet rows are copied.  Returns (entries, Dirichlet rows)."""
    rp, ci = disc.pattern()
    idx = torch.arange(disc.N, device="cuda")
    ijk = [idx % n[0], (idx // n[0]) % n[1], idx // (n[0] * n[1])]
    dmask = torch.zeros(disc.N, dtype=torch.bool, device="cuda")
    last = torch.zeros(disc.N, dtype=torch.bool, device="cuda")
    for ax, side in faces:
        on = ijk[ax] == (0 if side == 0 else n[ax] - 1)
        dmask |= on
        if ax == len(n) - 1:
            last |= on
    rows = torch.repeat_interleave(idx, rp[1:] - rp[:-1])
    keep = ~dmask[rows]
    del rows
    keep &= ~last[ci.long()]
    return int(keep.sum().item()), int(dmask.sum().item())


def roofline_entry(disc, cls, avg_ms, hbm_gbs, hbm_src, pk, used=None):
    """Algorithmic work of one launch of the given kernel class on this workload, against the
    FP64 FMA peak measured in this process (the operator product and the assembly stages
    are bound by GB300's FP64 pipe, not by HBM: one DFMA per 8-byte value).  used: for the
    Krylov product, (entries it multiplies, Dirichlet rows it copies)."""
    N, nnz = disc.N, disc.nnz
    fp64 = pk["fp64_tflops"]
    src = "measured in this run (iga_measure_peaks, DFMA chains)"
    t = avg_ms * 1e-3
    if cls == "spmv":
        # the product with the Dirichlet-fixed Jacobian: one FP64 FMA and one 8-byte value per
        # entry off the Dirichlet rows and columns; rowptr, x read, y written
        ent, ndir = used if used else (nnz, 0)
        bytes_ = ent * 8 + (N + 1) * 8 + 2 * N * 8
        flops = 2.0 * ent
        traffic = SPMV_DRAM_BYTES_ANNULUS64 if NEL == 64 else None
        return {"kernel": "k_spmv_fixed (FP64 values, stencil columns, Dirichlet rows copied, zero columns of the last axis's Dirichlet faces skipped)",
                "bound": "alu", "achieved": flops / t / 1e12, "entries_multiplied": ent, "stored_entries": nnz,
                "dirichlet_rows": ndir,
                "peak": fp64, "unit": "TFLOP/s", "frac": flops / t / 1e12 / fp64, "traffic": traffic,
                "traffic_capture": SPMV_TRAFFIC_CAPTURE if traffic else None, "peak_source": src,
                "avg_launch_ms": avg_ms, "algorithmic_flops_per_launch": flops, "algorithmic_bytes_per_launch": bytes_,
                "hbm": {"achieved_gbs": bytes_ / t / 1e9, "peak_gbs": hbm_gbs, "frac": bytes_ / t / 1e9 / hbm_gbs,
                        "peak_source": hbm_src}}
    return {"kernel": cls, "bound": "alu", "achieved": None, "peak": fp64, "unit": "TFLOP/s", "frac": None,
            "traffic": None, "peak_source": src, "avg_launch_ms": avg_ms}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--nel", type=int, default=64, help="elements per direction (64 is the benchmark workload)")
    ap.add_argument("--cpu-seconds", type=float, default=10.0, help="0 skips the CPU baseline (the oracle on all host cores)")
    ap.add_argument("--no-extras", action="store_true", help="skip the FP64-vs-mixed and learned-start comparisons")
    ap.add_argument("--workload", default="annulus64",
                    choices=["annulus64", "bratu16", "cube_mixed", "batch512", "learned64", "nn64", "fdjac", "genalpha", "periodic64",
                             "mixed64", "newton64_mixed"],
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
