"""Benchmark lines for the configurations other than the headline one.

    python bench.py --workload {bratu16, cube_mixed, batch512, learned64, nn64, fdjac, genalpha, periodic64, mixed64,
                                newton64_mixed}

Each prints one JSON line with the keys of the headline line (metric, value,
unit, config, clocks, e2e-style extras) for one configuration:

  bratu16     2D Bratu, lambda = 1, 16x16 quadratic C1: one residual + Jacobian
              assembly at seeded interior values U ~ U[-0.1, 0.1], then a full
              Newton solve (the smallest case: launch-latency bound).
  cube_mixed  3D unit cube, lambda = 2, 128^3 quadratic and 48^3 quartic:
              Jacobian assembly in FP64, FP32 (sum factorisation) and, for
              p <= 3, BF16/TF32 tensor-core element matrices; relative Frobenius
              error against the FP64 Jacobian; Newton solves with each.
  batch512    512 independent 2D instances (n ~ U{16..128}, p ~ U{2,3},
              lambda ~ U[0.5, 6]) in one persistent, graph-captured launch.
  fdjac       Appendix C / Table 3: explicit versus local numerical differentiation
              Jacobians of 3D Bratu on the unit cube (32^3-128^3, p = 1-3).
  nn64        the learned-guess network alone: forward and training step on a batch
              of 64 synthetic 66 x 66 inputs, against the BF16 tensor peak.
  genalpha    Sec. 4.2: generalized-alpha time steps (rho_inf = 0.5, dt = 0.01) of the
              transient Bratu problem u_t = div grad u + 2 e^u on the 64^3 cubic NURBS
              quarter annulus from u = 0, each step a Newton-Krylov solve to 1e-10.
  periodic64  Sec. 2.4: 3D Bratu, lambda = 2, on the unit cube 64^3 cubic, C^2 periodic in
              x and y, Dirichlet faces in z: residual and Jacobian assembly (unwrapped
              space plus the fold onto the wrapped functions) and Newton solves.
  newton64_mixed  Newton on the 64^3 quadratic cube with the FP64 and the reduced-precision
              Jacobians, GMRES and CG (the main line's 128^3 comparison at a profiler size).
  mixed64     the reduced-precision Jacobians alone on the 64^3 quadratic cube (lambda = 2,
              U ~ U[-0.1, 0.1]): BF16 and TF32 element matrices (tcgen05 GEMM across
              elements) and the FP32 sum factorisation, per-kernel-class times, error
              against the FP64 Jacobian; sized for a profiler capture.
  learned64   kappa-Bratu on 64^2 quadratic (66 x 66 control grid): training
              data from the batched solver, the convolutional guess trained on
              the GPU, evaluation on held-out fields against the zero start and
              against one-at-a-time FP64 Newton.
"""
import json
import time

import numpy as np

METRIC = "assembled Jacobian nnz/s & Newton solves/s to ||F||≤1e-10, FP64 vs mixed/NN"


def _ev(torch, fn, reps):
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


# ------------------------------------------------------------------ oracle legs ---
# Each line carries "cpu_baseline": the oracle (plain C / numpy, one thread) timed on this
# host on a bounded sample of the line's workload, scaled to the line's unit; it is a
# reported baseline, not a target.

def _oracle_loop(fn, min_seconds):
    import oracle as O
    O.build()
    fn()  # first call outside the clock (pattern caches, page-in)
    t0, n = time.perf_counter(), 0
    while n == 0 or time.perf_counter() - t0 < min_seconds:
        fn()
        n += 1
    return (time.perf_counter() - t0) / n, n


def _baseline(value, unit, sample, reps, seconds):
    return {"value": value, "unit": unit, "cores": 1, "kind": "oracle",
            "sample": "%s; %d repetitions in %.1f s" % (sample, reps, seconds)}


def _oracle_assembly_block(W, dim, p, sub, periodic=None, geom=None, lam=2.0, min_seconds=3.0):
    """Seconds per element of the oracle's residual and of its Jacobian on a sub^dim block
    (uniform cube, or the annulus with geom='annulus'; periodic axes as given)."""
    import oracle as O
    if geom == "annulus":
        kn, ctrl, w = W.quarter_annulus(sub, p)
    else:
        kn, ctrl, w = [O.open_uniform_knots(sub, p)] * dim, None, None
    per = periodic or {}
    bc = {(a, s): 0.0 for a in range(dim) if a not in per for s in range(2)}
    prob = O.Problem(kn, [p] * dim, ctrl=ctrl, weights=w, lam=lam, dirichlet=bc, periodic=per)
    U = np.where(prob.dirichlet_mask(), 0.0, W.uniform(2, prob.N, -0.1, 0.1))
    prob.pattern()
    tr, nr = _oracle_loop(lambda: prob.residual(U), min_seconds / 2)
    tj, nj = _oracle_loop(lambda: prob.jacobian(U), min_seconds / 2)
    ne = float(sub ** dim)
    return tr / ne, tj / ne, nr + nj, (tr * nr + tj * nj)


def _line(metric_value, unit, workload, extra, clocks, hib=True, dtype="f64"):
    d = {"metric": METRIC, "value": metric_value, "unit": unit, "n_gpus": 1, "higher_is_better": hib,
         "scaling": "weak", "vs_baseline": None, "dtype": dtype, "data": "synthetic", "config": {"workload": workload}}
    d.update(extra)
    d["clocks"] = clocks
    return json.dumps(d)


def bratu16(torch, iga, W, clock):
    bc = {(a, s): 0.0 for a in range(2) for s in range(2)}
    d = iga.Discretization(2, 2, nel=16, lam=1.0, dirichlet=bc)
    U = torch.tensor(W.interior_field([18, 18], 1), device="cuda")
    F = torch.empty_like(U)
    J = torch.empty(d.nnz, dtype=torch.float64, device="cuda")
    clock.start()
    tr = _ev(torch, lambda: d.form_residual(U, F), 50)
    tj = _ev(torch, lambda: d.form_jacobian(U, vals=J), 50)
    o = iga.newton_defaults()
    times, rep = [], None
    for _ in range(20):
        Us = U.clone()
        torch.cuda.synchronize()
        t = time.perf_counter()
        rep = d.solve_newton(Us, o)
        times.append(time.perf_counter() - t)
    # the same problem as a one-instance batch: the persistent solver runs the whole Newton
    # solve in one graph-captured launch (FP64 residual, FP32 Jacobian), so the 16x16 solve
    # is no longer bound by launch latency and host synchronisations
    B = iga.Batch([{"nel": 16, "p": 2, "lam": 1.0}])
    Ub = torch.empty(B.total, dtype=torch.float64, device="cuda")
    btimes, brep = [], None
    for _ in range(23):
        Ub.copy_(U)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        brep = B.solve(Ub)
        btimes.append(time.perf_counter() - t0)
    btimes = btimes[3:]
    Us = U.clone()
    d.solve_newton(Us, o)
    batch1 = {"solves_per_s": 1.0 / min(btimes), "ms_per_solve": 1e3 * min(btimes),
              "ms_median": 1e3 * float(np.median(btimes)), "newton_its": int(brep["newton_its"][0]),
              "krylov_its": int(brep["krylov_its"][0]), "fnorm": float(brep["fnorm"][0]),
              "max_abs_diff_vs_fp64_newton": (Ub - Us).abs().max().item(),
              "how": "iga_batch_solve on one instance (wall time of the call, copy of the reports included)"}
    B.close()
    ck = clock.stop()
    t = min(times)
    import oracle as O
    kn = O.open_uniform_knots(16, 2)
    prob = O.Problem([kn, kn], [2, 2], lam=1.0, dirichlet=bc)
    U0 = W.interior_field([18, 18], 1)
    to, no = _oracle_loop(lambda: O.newton(prob, U0, atol=1e-10), 3.0)
    cb = _baseline(1.0 / to, "solves/s", "oracle Newton (sparse LU per step) on the same 16x16 problem from the same U", no,
                   to * no)
    return _line(1.0 / t, "solves/s", "bratu2d_16x16_p2_lambda1_fp64", {
        "residual_us": tr * 1e3, "jacobian_us": tj * 1e3, "jacobian_nnz_per_s": d.nnz / (tj * 1e-3),
        "newton": {"its": rep.newton_its, "krylov_its": rep.krylov_its, "fnorm": rep.fnorm},
        "ms_per_solve": t * 1e3, "dofs": d.N, "nnz": d.nnz, "one_instance_batch": batch1, "cpu_baseline": cb}, ck)


def cube_mixed(torch, iga, W, clock):
    out = {}
    clock.start()
    for name, p, nel in (("cube128_p2", 2, 128), ("cube48_p4", 4, 48)):
        bc = {(a, s): 0.0 for a in range(3) for s in range(2)}
        d = iga.Discretization(3, p, nel=nel, lam=2.0, dirichlet=bc)
        U = torch.tensor(W.interior_field([nel + p] * 3, 3), device="cuda")
        J = torch.empty(d.nnz, dtype=torch.float64, device="cuda")
        J32 = torch.empty(d.nnz, dtype=torch.float32, device="cuda")
        res = {"dofs": d.N, "nnz": d.nnz}
        t = _ev(torch, lambda: d.form_jacobian(U, vals=J), 3)
        res["fp64"] = {"ms": t, "nnz_per_s": d.nnz / (t * 1e-3)}
        modes = [("fp32_sumfact", iga.IGA_JAC_FP32), ("bf16_tensor", iga.IGA_JAC_BF16)]
        if p <= 3:
            modes += [("tf32_tensor", iga.IGA_JAC_TF32)]
        d.form_jacobian(U, vals=J)
        nJ = torch.linalg.norm(J).item()
        for mname, code in modes:
            t = _ev(torch, lambda: d.form_jacobian(U, prec=code, vals=J32), 3)
            err = (torch.linalg.norm(J32.double() - J) / nJ).item()
            res[mname] = {"ms": t, "nnz_per_s": d.nnz / (t * 1e-3), "rel_frobenius_error_vs_fp64": err}
        del J32
        solves = {}
        for label, jac, ksp in (("fp64_gmres", iga.IGA_FP64, iga.IGA_KSP_GMRES), ("fp32_gmres", iga.IGA_JAC_FP32, iga.IGA_KSP_GMRES),
                                ("fp32_cg", iga.IGA_JAC_FP32, iga.IGA_KSP_CG), ("bf16_gmres", iga.IGA_JAC_BF16, iga.IGA_KSP_GMRES)):
            o = iga.newton_defaults()
            o.jac, o.ksp = jac, ksp
            best, rep = 1e30, None
            for _ in range(2):
                Us = torch.zeros(d.N, dtype=torch.float64, device="cuda")
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                rep = d.solve_newton(Us, o)
                best = min(best, time.perf_counter() - t0)
            solves[label] = {"ms": best * 1e3, "newton_its": rep.newton_its, "krylov_its": rep.krylov_its, "fnorm": rep.fnorm}
        res["newton"] = solves
        out[name] = res
        d.close()
        del J
        torch.cuda.empty_cache()
    ck = clock.stop()
    v = out["cube128_p2"]["fp32_sumfact"]["nnz_per_s"]
    _, tj, nr, sec = _oracle_assembly_block(W, 3, 2, 8)
    cb = _baseline(out["cube128_p2"]["nnz"] / (tj * 128 ** 3), "nnz/s",
                   "oracle FP64 Jacobian of an 8^3-element block of the p=2 cube, per element x 128^3", nr, sec)
    return _line(v, "nnz/s", "cube_128cubed_p2_and_48cubed_p4_lambda2_mixed_jacobian", {"cases": out, "cpu_baseline": cb}, ck,
                 dtype="f32")


def batch512(torch, iga, W, clock):
    ins = W.batch_instances(512, seed=0)
    t0 = time.perf_counter()
    b = iga.Batch(ins)
    setup = time.perf_counter() - t0
    U = torch.zeros(b.total, dtype=torch.float64, device="cuda")
    from paper_1305_4452_gb300 import autotune
    res = {"autotune": {}}
    clock.start()
    for label, ksp in (("cg", iga.IGA_KSP_CG), ("gmres30", iga.IGA_KSP_GMRES)):
        o = iga.newton_defaults()
        o.ksp = ksp
        o.gmres_restart = 30
        # launch shape, and for GMRES the work unit of its Gram-Schmidt dots, for this mix
        # (timed from the zero start, as the solves below)
        U.zero_()
        res["autotune"][label] = autotune.tune(b, ins, U, o, retime=True)
        best, r = 1e30, None
        for _ in range(3):
            U.zero_()
            torch.cuda.synchronize()
            t = time.perf_counter()
            r = b.solve(U, o)
            best = min(best, time.perf_counter() - t)
        us = r["solve_us"]
        big = int(np.argmax(us))
        res[label] = {"ms": best * 1e3, "solves_per_s": 512 / best, "solved": int(r["solved"]),
                      "newton_its_total": int(r["newton_its"].sum()), "krylov_its_total": int(r["krylov_its"].sum()),
                      "max_fnorm": float(r["fnorm"].max()),
                      # load balance: the longest instance against the sum of all over the SMs
                      "instance_ms": {"max": float(us[big]) / 1e3, "sum": float(us.sum()) / 1e3,
                                      "sum_over_sms": float(us.sum()) / 1e3 / torch.cuda.get_device_properties(0).multi_processor_count,
                                      "longest": {"n": int(ins[big]["nel"]), "p": int(ins[big]["p"]),
                                                  "newton_its": int(r["newton_its"][big]),
                                                  "krylov_its": int(r["krylov_its"][big])}}}
    ck = clock.stop()
    b.close()
    res["jacobian_2d_tensor_vs_sumfact"] = jacobian_2d_comparison(torch, iga, W)
    import oracle as O
    done, t_or, k = 0, 0.0, 0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < 6.0 and k < len(ins):  # the seeded instances in order
        x = ins[k]
        kn = O.open_uniform_knots(x["nel"], x["p"])
        prob = O.Problem([kn, kn], [x["p"]] * 2, lam=x["lam"], dirichlet={(a, s): 0.0 for a in range(2) for s in range(2)})
        t = time.perf_counter()
        O.newton(prob, np.zeros(prob.N), atol=1e-10)
        t_or += time.perf_counter() - t
        done, k = done + 1, k + 1
    cb = _baseline(done / t_or, "solves/s", "oracle Newton (sparse LU) on the first %d of the 512 seeded instances, "
                   "one at a time" % done, done, t_or)
    return _line(res["cg"]["solves_per_s"], "solves/s", "batch512_2d_n16to128_p2or3_lambda0.5to6_fp64res_fp32jac",
                 {"results": res, "setup_s": setup, "total_dofs": int(b.total), "cpu_baseline": cb}, ck)


def jacobian_2d_comparison(torch, iga, W, reps=5):
    """The reduced-precision Jacobians the batched instances could use, on single 2D meshes
    of the batch's range (identity map, lambda = 3, U ~ U[-0.1, 0.1]): FP32 global sum
    factorisation on the CUDA cores (the batch's own kind) against the BF16 and TF32
    tensor-core element matrices, best of `reps`; errors against the FP64 Jacobian."""
    out = []
    bc = {(a, s): 0.0 for a in range(2) for s in range(2)}
    for nel, p in ((32, 2), (64, 2), (128, 2), (32, 3), (64, 3), (128, 3)):
        d = iga.Discretization(2, p, nel=nel, lam=3.0, dirichlet=bc)
        U = torch.tensor(W.interior_field([nel + p] * 2, 3), device="cuda")
        J = d.form_jacobian(U)
        nJ = torch.linalg.norm(J).item()
        row = {"nel": nel, "p": p, "nnz": d.nnz}
        J32 = torch.empty(d.nnz, dtype=torch.float32, device="cuda")
        for name, code in (("fp32_sumfact", iga.IGA_JAC_FP32), ("bf16_tensor", iga.IGA_JAC_BF16), ("tf32_tensor", iga.IGA_JAC_TF32)):
            t = _ev(torch, lambda: d.form_jacobian(U, prec=code, vals=J32), reps)
            row[name] = {"us": t * 1e3, "rel_frobenius_error_vs_fp64": (torch.linalg.norm(J32.double() - J) / nJ).item()}
        row["fastest"] = min(("fp32_sumfact", "bf16_tensor", "tf32_tensor"), key=lambda k: row[k]["us"])
        out.append(row)
        d.close()
    return out


def learned_core(torch, iga, W, n_train=20000, n_test=2000, steps=16000, clock=None):
    """Training data from the batched solver (seeds 0..n_train-1), the convolutional guess
    trained on the GPU, and the held-out comparison (seeds 1,000,000...): batched Newton from
    the zero start against batched Newton from the network's guess (inference included in
    its wall time), plus plain one-at-a-time FP64 Newton on a sample.  Returns the results
    and the clock record of the held-out phase."""
    from paper_1305_4452_gb300 import nn
    nel = 64
    t0 = time.perf_counter()
    train = nn.kappa_instances(range(0, n_train), nel=nel)
    test = nn.kappa_instances(range(1_000_000, 1_000_000 + n_test), nel=nel)
    Utr, rtr, gen_s = nn.solve_batch(train)
    keep = rtr["status"] == 0
    train = [x for x, k in zip(train, keep) if k]
    Utr = Utr[keep]
    x, mask = nn.features(train)
    tgt = torch.tensor(Utr.reshape(len(train), nel + 2, nel + 2), dtype=torch.float32, device="cuda")
    net = nn.Net(nel + 2, nel + 2, hidden=64, max_batch=64, seed=0)
    net.set_h1_weight(64.0)  # discrete H1 term: penalise the oscillatory error Newton's residual sees
    rng = np.random.default_rng(0)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    losses = []
    for step in range(steps):
        idx = torch.as_tensor(rng.choice(len(train), 64, replace=False), device="cuda")
        lr = 2e-3 * (0.5 * (1 + np.cos(np.pi * step / steps))) + 1e-5
        losses.append(net.loss_grad(x[idx], tgt[idx], mask))
        net.adam_step(lr)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t1
    del x, tgt, Utr
    if clock is not None:
        clock.start()
    # held-out: batched Newton from zero and from the network's guess (inference timed).
    # Inference runs the trained weights on all held-out fields in one call (a network
    # handle sized for the whole set), one launch per layer instead of one per 64 fields.
    U0, r0, s0 = nn.solve_batch(test)
    xt, _ = nn.features(test)
    inf = nn.Net(nel + 2, nel + 2, hidden=64, max_batch=len(test), seed=0)
    inf.set_params(net.get_params())
    inf.forward(xt[:64], mask)  # first call outside the clock (module load, tensor maps)
    torch.cuda.synchronize()
    ti = time.perf_counter()
    guess = inf.forward(xt, mask)
    torch.cuda.synchronize()
    infer_s = time.perf_counter() - ti
    # the guess does not depend on the call's batch size (a field's convolutions read only
    # its own pixels); checked against 64-field calls on the first 256 fields
    g64 = torch.cat([net.forward(xt[a:a + 64], mask) for a in range(0, min(len(test), 256), 64)])
    guess_batch_check = float(torch.abs(g64 - guess[:g64.shape[0]]).max().item())
    inf.close()
    U1, r1, s1 = nn.solve_batch(test, U0=guess.double().cpu().numpy().reshape(len(test), -1))
    ok = (r0["status"] == 0) & (r1["status"] == 0)
    # one-at-a-time plain FP64 Newton (GMRES + Jacobi, zero start) on a sample of the test fields
    bc = {(a, s): 0.0 for a in range(2) for s in range(2)}
    nsamp = 64
    tp = 0.0
    its_plain = []
    for ins in test[:nsamp]:
        d = iga.Discretization(2, 2, nel=nel, lam=ins["lam"], log_kappa=ins["log_kappa"], dirichlet=bc)
        Us = torch.zeros(d.N, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        t = time.perf_counter()
        rep = d.solve_newton(Us, iga.newton_defaults(), check=False)
        tp += time.perf_counter() - t
        its_plain.append(rep.newton_its)
        d.close()
    ck = clock.stop() if clock is not None else None
    rel_err = float(np.median(np.linalg.norm(U1[ok] - guess.double().cpu().numpy().reshape(len(test), -1)[ok], axis=1)
                              / np.maximum(np.linalg.norm(U1[ok], axis=1), 1e-30)))
    zero = n_test / s0
    nn_start = n_test / (s1 + infer_s)
    res = {
        "workload": "kappa_bratu_64x64_p2_grf_logkappa_lambda0.5to4_heldout%d" % n_test,
        "train_solves": int(keep.sum()), "train_skipped_no_convergence": int((~keep).sum()), "data_gen_s": gen_s,
        "train_steps": steps, "train_s": train_s, "loss_first": losses[0], "loss_last": float(np.mean(losses[-50:])),
        "params": net.nparams, "test": n_test, "test_both_converged": int(ok.sum()),
        "guess_median_rel_error": rel_err,
        "zero_start": {"solves_per_s": zero, "newton_its_mean": float(r0["newton_its"][ok].mean()),
                       "krylov_its_mean": float(r0["krylov_its"][ok].mean())},
        "nn_start": {"solves_per_s": nn_start, "inference_s": infer_s, "solve_s": s1,
                     "inference": "one forward call over all %d fields" % n_test,
                     "max_abs_diff_vs_64_field_calls": guess_batch_check,
                     "newton_its_mean": float(r1["newton_its"][ok].mean()), "krylov_its_mean": float(r1["krylov_its"][ok].mean())},
        "speedup_nn_vs_zero_start": nn_start / zero,
        "plain_fp64_single": {"solves_per_s": nsamp / tp, "newton_its_mean": float(np.mean(its_plain)), "sample": nsamp},
        "total_s": time.perf_counter() - t0,
    }
    net.close()
    return res, ck, test


def learned64(torch, iga, W, clock, n_train=20000, n_test=2000, steps=16000):
    res, ck, test = learned_core(torch, iga, W, n_train, n_test, steps, clock)
    import oracle as O
    nel = 64
    bc = {(a, s): 0.0 for a in range(2) for s in range(2)}
    kn = O.open_uniform_knots(nel, 2)
    t_or, done = 0.0, 0
    for ins in test[:64]:
        prob = O.Problem([kn, kn], [2, 2], lam=ins["lam"], log_kappa=ins["log_kappa"], dirichlet=bc)
        t = time.perf_counter()
        O.newton(prob, np.zeros(prob.N), atol=1e-10)
        t_or += time.perf_counter() - t
        done += 1
        if t_or > 6.0:
            break
    res["cpu_baseline"] = _baseline(done / t_or, "solves/s", "oracle Newton (sparse LU) from the zero start on the first "
                                    "%d held-out fields" % done, done, t_or)
    return _line(res["nn_start"]["solves_per_s"], "solves/s", "kappa_bratu_64x64_p2_learned_initial_guess", {"results": res}, ck)


def nn64(torch, iga, W, clock, batch=64, reps=10):
    """The learned-guess network alone (random weights, synthetic inputs of the
    66 x 66 control grid): inference and training-step throughput against the
    measured dense BF16 tensor peak."""
    import json as _json
    import os as _os
    from paper_1305_4452_gb300 import nn
    H = Wd = 66
    net = nn.Net(H, Wd, hidden=64, max_batch=batch, seed=0)
    g = torch.Generator(device="cuda").manual_seed(0)
    x = torch.randn(batch, H, Wd, 4, device="cuda", generator=g)
    tgt = 0.1 * torch.randn(batch, H, Wd, device="cuda", generator=g)
    mask = torch.ones(H, Wd, device="cuda")
    shapes, _ = nn.layer_shapes(4, 64, nn.DILATIONS)
    P = batch * H * Wd
    fwd_flops = sum(2.0 * P * 9 * cin * cout for cin, cout, _, _, _ in shapes)
    tc_flops = sum(2.0 * P * 9 * (16 if i == 0 else cin) * (16 if i == len(shapes) - 1 else cout)
                   for i, (cin, cout, _, _, _) in enumerate(shapes))
    clock.start()
    t_fwd = _ev(torch, lambda: net.forward(x, mask), reps)
    t_step = _ev(torch, lambda: (net.loss_grad(x, tgt, mask), net.adam_step(1e-4)), reps)
    ck = clock.stop()
    try:
        with open(_os.path.join(_os.path.dirname(_os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            peak, src = float(_json.load(f)["bf16_tflops"]), "measured burst"
    except Exception:
        peak, src = 1900.0, "fallback"
    ach = fwd_flops / (t_fwd * 1e-3) / 1e12
    from oracle import nn_ref as R
    shapes_r, _ = R.layer_shapes(4, 64, nn.DILATIONS)
    params = net.get_params().astype(np.float64)
    xs, ms = x[:2].double().cpu().numpy(), mask.double().cpu().numpy()
    to, no = _oracle_loop(lambda: R.forward(params, shapes_r, xs, ms), 3.0)
    cb = _baseline(2 / to, "fields/s", "numpy reference forward (FP64) of the same network on 2 of the fields", no, to * no)
    net.close()
    return _line(batch / (t_fwd * 1e-3), "fields/s", "neural_operator_66x66_6layers_64ch_batch%d_bf16" % batch, {
        "forward_ms": t_fwd, "train_step_ms": t_step, "forward_flops": fwd_flops,
        "forward_flops_on_tensor_cores": tc_flops,
        "roofline": {"kernel": "k_conv_tc (forward, 6 launches)", "bound": "tensor", "achieved": ach, "peak": peak,
                     "unit": "TFLOP/s", "frac": ach / peak, "peak_source": src,
                     "note": "achieved = unpadded network FLOPs / forward time; the padded first and last layers run "
                             "%.1f%% more tensor-core FLOPs" % (100 * (tc_flops / fwd_flops - 1))},
        "train_step_tflops": 3 * fwd_flops / (t_step * 1e-3) / 1e12, "cpu_baseline": cb}, ck, dtype="bf16")


def fdjac(torch, iga, W, clock):
    """Sec. 2.10 / Appendix C (Table 3): the 3D Bratu Jacobian on the unit cube computed
    explicitly (global sum factorisation, FP64) and by local numerical differentiation
    (Eq. fdjac: per Gauss point and element value, FP64), best of 3 each, for the
    table's cases that run on one GPU; the paper's CPU times are context."""
    # (nel, p, k, paper explicit s, paper local ND s, paper cores)
    cases = [(32, 2, 0, 0.31, 1.21, 8), (32, 2, 1, 0.33, 1.24, 8), (32, 3, 2, 3.71, 15.27, 8),
             (64, 2, 0, 1.31, 5.15, 16), (64, 2, 1, 1.35, 5.26, 16), (64, 3, 2, 15.41, 64.93, 16),
             (128, 1, 0, 0.52, 1.72, 16), (128, 2, 1, 10.74, 41.46, 16)]
    out = []
    clock.start()
    for nel, p, k, pe, pn, cores in cases:
        bc = {(a, s): 0.0 for a in range(3) for s in range(2)}
        d = iga.Discretization(3, p, nel=nel, continuity=k, lam=2.0, dirichlet=bc)
        U = torch.tensor(W.uniform(4, d.N, -0.1, 0.1), device="cuda")
        J = torch.empty(d.nnz, dtype=torch.float64, device="cuda")
        t_exp = _ev(torch, lambda: d.form_jacobian(U, vals=J), 3)
        Jx = J.clone()
        t_fd = _ev(torch, lambda: d.form_jacobian(U, prec=iga.IGA_JAC_FD, vals=J), 3)
        err = (torch.linalg.norm(J - Jx) / torch.linalg.norm(Jx)).item()
        out.append({"nel": nel, "p": p, "k": k, "nnz": d.nnz, "explicit_ms": t_exp, "local_nd_ms": t_fd,
                    "ratio": t_fd / t_exp, "rel_frobenius_fd_vs_explicit": err,
                    "paper_cpu_s": {"explicit": pe, "local_nd": pn, "ratio": pn / pe, "cores": cores}})
        d.close()
        del J, Jx
        torch.cuda.empty_cache()
    ck = clock.stop()
    big = out[5]
    import oracle as O
    kn = O.open_uniform_knots(8, 3)
    prob = O.Problem([kn] * 3, [3] * 3, lam=2.0, dirichlet={(a, s): 0.0 for a in range(3) for s in range(2)})
    U = np.where(prob.dirichlet_mask(), 0.0, W.uniform(4, prob.N, -0.1, 0.1))
    prob.pattern()
    to, no = _oracle_loop(lambda: prob.jacobian_fd(U), 4.0)
    cb = _baseline(big["nnz"] / (to / 8 ** 3 * 64 ** 3), "nnz/s", "oracle local-ND Jacobian of an 8^3-element block of the "
                   "p=3 cube, per element x 64^3 (the 64^3 p=3 case)", no, to * no)
    return _line(big["nnz"] / (big["local_nd_ms"] * 1e-3), "nnz/s", "bratu3d_cube_table3_cases_local_numerical_differentiation",
                 {"cases": out, "cpu_baseline": cb}, ck)


def genalpha(torch, iga, W, clock, nel=64, steps=10, dt=0.01, rho=0.5):
    kn, ctrl, w = W.quarter_annulus(nel, 3)
    bc = {(a, s): 0.0 for a in range(3) for s in range(2)}
    d = iga.Discretization(3, 3, knots=kn, ctrl=ctrl, weights=w, lam=2.0, dirichlet=bc)
    out = {}
    clock.start()
    for label, jac, ksp in (("fp64_gmres", iga.IGA_FP64, iga.IGA_KSP_GMRES), ("fp32_cg", iga.IGA_JAC_FP32, iga.IGA_KSP_CG)):
        o = iga.newton_defaults()
        o.jac, o.ksp = jac, ksp
        U = torch.zeros(d.N, dtype=torch.float64, device="cuda")
        V = torch.zeros_like(U)
        d.ts_alpha_step(U.clone(), V.clone(), dt, rho, o)  # warm-up (also assembles the stiffness once)
        its, kits = [], []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            rep = d.ts_alpha_step(U, V, dt, rho, o)
            its.append(rep.newton_its)
            kits.append(rep.krylov_its)
        t = time.perf_counter() - t0
        out[label] = {"ms_per_step": 1e3 * t / steps, "steps_per_s": steps / t, "newton_its": its, "krylov_its": kits,
                      "u_max_at_end": U.max().item(), "t_end": steps * dt}
    ck = clock.stop()
    d.close()
    tr, tj, nr, sec = _oracle_assembly_block(W, 3, 3, 8, geom="annulus")
    its = float(np.mean(out["fp64_gmres"]["newton_its"]))
    t_step = (its * (tr + tj) + tr) * nel ** 3
    cb = _baseline(1.0 / t_step, "time steps/s", "oracle residual+Jacobian of an 8^3-element annulus block, per element "
                   "x 64^3, times the GPU's mean Newton steps per time step (%.1f); linear solves not counted" % its, nr, sec)
    return _line(out["fp64_gmres"]["steps_per_s"], "time steps/s",
                 "transient_bratu_annulus64_p3_lambda2_genalpha_rho0.5_dt0.01", {"cases": out, "dofs": d.N,
                                                                                "cpu_baseline": cb}, ck)


def periodic64(torch, iga, W, clock, nel=64, p=3):
    per = {0: p - 1, 1: p - 1}
    bc = {(2, 0): 0.0, (2, 1): 0.0}
    d = iga.Discretization(3, p, nel=nel, lam=2.0, dirichlet=bc, periodic=per)
    n = [nel, nel, nel + p]
    U = torch.tensor(W.interior_field(n, 3), device="cuda")
    F = torch.empty_like(U)
    J = torch.empty(d.nnz, dtype=torch.float64, device="cuda")
    clock.start()
    tr = _ev(torch, lambda: d.form_residual(U, F), 5)
    tj = _ev(torch, lambda: d.form_jacobian(U, vals=J), 3)
    d.profile_enable(iga.KERNEL_CLASSES)
    d.form_jacobian(U, vals=J)
    torch.cuda.synchronize()
    prof = d.profile_read()
    d.profile_enable(())
    solves = {}
    for label, jac, ksp in (("fp64_gmres", iga.IGA_FP64, iga.IGA_KSP_GMRES), ("fp32_cg", iga.IGA_JAC_FP32, iga.IGA_KSP_CG)):
        o = iga.newton_defaults()
        o.jac, o.ksp = jac, ksp
        best, rep = 1e30, None
        for _ in range(2):
            Us = torch.zeros(d.N, dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rep = d.solve_newton(Us, o)
            best = min(best, time.perf_counter() - t0)
        solves[label] = {"ms": best * 1e3, "newton_its": rep.newton_its, "krylov_its": rep.krylov_its, "fnorm": rep.fnorm}
    ck = clock.stop()
    d.close()
    otr, otj, nr, sec = _oracle_assembly_block(W, 3, p, 8, periodic=per)
    its = solves["fp64_gmres"]["newton_its"]
    cb = _baseline(1.0 / ((its * (otr + otj) + otr) * nel ** 3), "solves/s", "oracle residual+Jacobian of an 8^3-element block "
                   "periodic in x and y, per element x 64^3, times %d Newton steps; linear solves not counted" % its, nr, sec)
    return _line(1e3 / solves["fp64_gmres"]["ms"], "solves/s", "bratu3d_cube64_p3_periodic_xy_C2_lambda2_fp64", {
        "cpu_baseline": cb,
        "dofs": d.N, "nnz": d.nnz, "residual_ms": tr, "jacobian_ms": tj, "jacobian_nnz_per_s": d.nnz / (tj * 1e-3),
        "jacobian_fold_ms": prof["combine"][0], "jacobian_unwrapped_stages_ms": prof["jac_stage1"][0] + prof["jac_stage2"][0] + prof["jac_final"][0],
        "newton": solves}, ck)


def mixed64(torch, iga, W, clock, nel=64, p=2):
    bc = {(a, s): 0.0 for a in range(3) for s in range(2)}
    d = iga.Discretization(3, p, nel=nel, lam=2.0, dirichlet=bc)
    U = torch.tensor(W.interior_field([nel + p] * 3, 3), device="cuda")
    J = torch.empty(d.nnz, dtype=torch.float64, device="cuda")
    J32 = torch.empty(d.nnz, dtype=torch.float32, device="cuda")
    clock.start()
    d.form_jacobian(U, vals=J)
    nJ = torch.linalg.norm(J).item()
    res = {"dofs": d.N, "nnz": d.nnz, "fp64_ms": _ev(torch, lambda: d.form_jacobian(U, vals=J), 3)}
    for name, code in (("bf16_tensor", iga.IGA_JAC_BF16), ("tf32_tensor", iga.IGA_JAC_TF32), ("fp32_sumfact", iga.IGA_JAC_FP32)):
        t = _ev(torch, lambda: d.form_jacobian(U, prec=code, vals=J32), 3)
        d.profile_enable(iga.KERNEL_CLASSES)
        d.form_jacobian(U, prec=code, vals=J32)
        torch.cuda.synchronize()
        prof = d.profile_read()
        d.profile_enable(())
        err = (torch.linalg.norm(J32.double() - J) / nJ).item()
        res[name] = {"ms": t, "nnz_per_s": d.nnz / (t * 1e-3), "rel_frobenius_error_vs_fp64": err,
                     "classes_ms": {k: round(v[0], 4) for k, v in prof.items() if v[0] > 0}}
    ck = clock.stop()
    d.close()
    _, tj, nr, sec = _oracle_assembly_block(W, 3, p, 8)
    res["cpu_baseline"] = _baseline(res["nnz"] / (tj * nel ** 3), "nnz/s", "oracle FP64 Jacobian of an 8^3-element block of "
                                    "the p=2 cube, per element x 64^3", nr, sec)
    return _line(res["bf16_tensor"]["nnz_per_s"], "nnz/s", "cube_64cubed_p2_lambda2_reduced_precision_jacobian", {"cases": res}, ck,
                 dtype="bf16")


def newton64_mixed(torch, iga, W, clock, nel=64, p=2, reps=3):
    """Newton solves (lambda = 2, U = 0 to ||F|| <= 1e-10) of the 64^3 quadratic cube with the
    FP64 Jacobian and with the FP32 / BF16 reduced-precision ones, GMRES and CG: the
    128^3 comparison of the main line at a size a profiler capture can take (CSR values
    136 MB FP32, above the 126 MB L2)."""
    bc = {(a, s): 0.0 for a in range(3) for s in range(2)}
    d = iga.Discretization(3, p, nel=nel, lam=2.0, dirichlet=bc)
    U = torch.zeros(d.N, dtype=torch.float64, device="cuda")
    out = {"dofs": d.N, "nnz": d.nnz}
    clock.start()
    for ksp_name, ksp in (("gmres", iga.IGA_KSP_GMRES), ("cg", iga.IGA_KSP_CG)):
        for name, code in (("fp64", iga.IGA_FP64), ("fp32", iga.IGA_JAC_FP32), ("bf16", iga.IGA_JAC_BF16)):
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
                best = min(best, time.perf_counter() - t0)
            out["%s_%s" % (name, ksp_name)] = {"ms": best * 1e3, "solves_per_s": 1.0 / best, "newton_its": rep.newton_its,
                                               "krylov_its": rep.krylov_its, "fnorm": rep.fnorm}
    ck = clock.stop()
    d.close()
    for ksp_name in ("gmres", "cg"):
        for name in ("fp32", "bf16"):
            k = "%s_%s" % (name, ksp_name)
            out[k]["speedup_vs_fp64_same_krylov"] = out[k]["solves_per_s"] / out["fp64_%s" % ksp_name]["solves_per_s"]
    return _line(out["fp32_cg"]["solves_per_s"], "solves/s", "bratu3d_cube_64cubed_p2_lambda2_newton_fp64_vs_mixed",
                 {"cases": out}, ck)


WORKLOADS = {"bratu16": bratu16, "cube_mixed": cube_mixed, "batch512": batch512, "learned64": learned64, "nn64": nn64, "fdjac": fdjac,
             "genalpha": genalpha, "periodic64": periodic64, "mixed64": mixed64, "newton64_mixed": newton64_mixed}
