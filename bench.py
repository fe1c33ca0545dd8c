#!/usr/bin/env python3
"""Throughput of the VAG Darcy + transport path on GB300 (one JSON line).

One step = one realisation of the 64^3 workload pushed through the C ABI:
  vag_assemble  (symbolic phase, local VAG matrices on 24 sub-tetrahedra per
                 cell, fracture matrices, Schur row gather into CSR)
  vag_solve     (aggregation-AMG preconditioned CG to ||r|| <= 1e-10 ||b||,
                 cell recovery, fluxes)
  vag_transport (porous volumes, CFL step at CFL 0.9, upwind map, 200 explicit
                 steps)
  vag_system_destroy.
Workload: 64^3 hexahedra, interior nodes jittered by +-20% h (fracture-normal
coordinates frozen), fractures on x=.5, y=.5, z=.5 and x=.25 (y<.5),
lognormal matrix permeability (log10 std 1) with 10:1 anisotropy along a
seeded axis, fracture/matrix ratio 1e4, p = 1 - x on x = 0, 1.

`value` times steps whose inputs already sit in HBM (torch CUDA tensors);
`e2e` times the same steps from pinned host buffers with the copies in and the
pressure and concentration copies out inside the timed region.  L2 is flushed
(256 MiB write) before every timed step.  Usage:
  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
import os

for _v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import argparse  # noqa: E402
import hashlib  # noqa: E402
import json  # noqa: E402
import statistics  # noqa: E402
import subprocess  # noqa: E402
import sys  # noqa: E402
import time  # noqa: E402

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_CELLS_EDGE = 64
TRANSPORT_STEPS = 200
RTOL = 1e-10
METRIC = "Darcy solves/s (assemble + solve to 1e-10 + 200 transport steps)"
UNIT = "solves/s"
WORKLOAD = ("scale64: 64^3 jittered hex (262144 cells, 274625 nodes), 4 fractures (14336 fracture faces), "
            "lognormal anisotropic Lambda_m, Lambda_f/Lambda_m = 1e4, FP64 AMG-CG to 1e-10, 200 upwind steps at CFL 0.9")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precond", default="amg", choices=["jacobi", "chebyshev", "amg"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--n", type=int, default=N_CELLS_EDGE, help="mesh edge (profiling cases only)")
    ap.add_argument("--workload", default="scale64", choices=["scale64", "batch", "serve", "mixed128", "solvers"],
                    help="scale64: the headline line; batch / serve / mixed128 / solvers: the batched, "
                         "served and mixed-precision workloads, and the solver comparison")
    ap.add_argument("--batch-size", type=int, default=256)
    ap.add_argument("--requests", type=int, default=400)
    return ap.parse_args()


# ----------------------------------------------------------------- helpers --

def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def replica_throughput(local_ms, steps, world, device="cpu"):
    """Whole-job throughput of `world` independent replicas that each ran
    `steps` steps in `local_ms`: the slowest rank's time bounds the job (the
    maximum over ranks), and every rank processed `steps` units."""
    tot = float(local_ms)
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([tot], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        tot = float(t.item())
    return world * steps / (tot / 1e3), tot


def fp64_peak_gflops():
    """FP64 FMA peak of the GB300 from its unit counts and clock: 2 DFMA per
    clock per SM (ncu: sm__sass_thread_inst_executed_op_dfma_pred_on
    .avg.peak_sustained = 2) x 152 SMs x the maximum SM clock x 2 flops."""
    mhz = 2070.0
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            mhz = float(json.load(f).get("sm_max_mhz", mhz))
    return 2 * 2 * 152 * mhz / 1e3


class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs (rows of
    the GPU with our UUID, else of the CUDA ordinal)."""
    Q = ("uuid,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, uuid, ordinal):
        self.uuid = (uuid or "").lower()
        self.ordinal = str(ordinal)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        time.sleep(0.25)
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
            out, _ = self.p.communicate()
        rows = [[x.strip() for x in line.split(",")] for line in out.strip().splitlines()]
        rows = [r for r in rows if len(r) >= 10]
        mine = [r for r in rows if self.uuid and self.uuid in r[0].lower()]
        if not mine:
            mine = [r for r in rows if r[1] == self.ordinal]
        sm, mx, reasons = [], [], set()
        for f in mine:
            try:
                sm.append(float(f[2]))
                mx.append(float(f[3]))
            except ValueError:
                continue
            for name, v in zip(self.NAMES, f[6:10]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def source_hash(files):
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_key):
    """DRAM bytes per launch from the committed ncu summary, only if the
    kernel's source is unchanged since the capture."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f).get(kernel_key)
    if not d:
        return None
    if d.get("source_hash") != source_hash(d.get("sources", [])):
        return None
    return d.get("dram_bytes_per_launch")


# -------------------------------------------------------------- CPU oracle --

def oracle_sample():
    """The oracle end to end on the 32^3 instance of the workload recipe,
    each phase scaled to 64^3 by exact work counts (cells; nonzeros x CG
    iterations; control volumes x steps).  Returns (seconds per full-size
    solve, seconds of CPU work spent)."""
    import vag_inputs as vi
    from oracle import vag_oracle as vo
    with open(os.path.join(ROOT, "oracle", "cpu_baseline_counts.json")) as f:
        cnt = json.load(f)
    full, smp = cnt["scale64"], cnt["scale32"]
    pb = vi.config_scale64(32)
    t0 = time.perf_counter()
    m = vo.Mesh(pb)
    cms = vo._all_cell_matrices(pb, m)
    fm = vo.fracture_local_matrices(pb, m)
    A = vo.assemble_full(pb, m, cms, fm)
    S, b, R = vo.schur_system(pb, A)
    t1 = time.perf_counter()
    x, it = vo.pcg_jacobi(S, b, rtol=RTOL, maxit=100000)
    t2 = time.perf_counter()
    u = np.zeros(A.shape[0]); u[pb.dir_nodes] = pb.dir_values; u[R] = x
    u = vo.recover_cells(pb, A, u)
    Fc = [vo.cell_fluxes(cm, u) for cm in cms]
    Ff = vo.fracture_fluxes(fm, u)
    tr = vo.Transport(pb, cms, fm, Fc, Ff, omega=0.5, mesh=m)
    dt = 0.9 * tr.cfl_dt()
    t3 = time.perf_counter()
    c = pb.c0()
    for _ in range(TRANSPORT_STEPS):
        c = tr.step(c, dt)
    t4 = time.perf_counter()
    s_cells = full["n_cells"] / smp["n_cells"]
    s_pcg = (full["nnz"] * full["oracle_pcg_iterations"]) / (smp["nnz"] * max(it, 1))
    s_cv = full["n_cv"] / smp["n_cv"]
    scaled = (t1 - t0) * s_cells + (t2 - t1) * s_pcg + (t3 - t2) * s_cells + (t4 - t3) * s_cv
    return scaled, t4 - t0


def cpu_baseline_block(n_samples=5):
    tot, spent = 0.0, 0.0
    for _ in range(n_samples):
        s, w = oracle_sample()
        tot += s
        spent += w
    return {"value": n_samples / tot, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": (f"{n_samples} complete oracle runs (numpy/scipy FP64, one thread) of the same recipe at "
                       f"32^3, each phase scaled to 64^3 by exact work counts (cells; nnz x the oracle's own "
                       f"Jacobi-CG iteration count at 64^3; control volumes x 200 steps); "
                       f"{spent:.1f} s of CPU work")}


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    for _ in range(args.warmup):
        oracle_sample()
    times, spent = [], 0.0
    for _ in range(args.steps):
        s, w = oracle_sample()
        times.append(s)
        spent += w
    value = args.steps / sum(times)
    cpu = {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": (f"per step: one complete oracle run of the recipe at 32^3 scaled to 64^3 by exact work "
                      f"counts; {spent:.1f} s of CPU work over {args.steps} steps")}
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "solver": "Jacobi-CG (oracle)"},
        "cpu_baseline": cpu, "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                                     "d2h_bytes_per_step": 0}}))


# ---------------------------------------------------------------- GPU arm --

def batch_problems_cfg(count, seed=99):
    import vag_inputs as vi
    return vi.batch_problems(count, seed=seed, n_lo=16, n_hi=48)


def serve_problems(count, seed=2024):
    """Poisson arrivals (mean 200 per second); n from a lognormal (ln n ~
    N(ln 39.2, 0.45)) truncated to [16, 96]; 1-50 rectangles; ratio
    log-uniform in [1e2, 1e6]; lognormal matrix permeability."""
    import vag_inputs as vi
    rng = np.random.default_rng(seed)
    arrivals = np.cumsum(rng.exponential(1.0 / 200.0, size=count))
    pbs = []
    for _ in range(count):
        while True:
            n = int(round(np.exp(rng.normal(np.log(39.2), 0.45))))
            if 16 <= n <= 96:
                break
        pbs.append(vi.random_dfn_problem(n, int(rng.integers(1, 51)), float(10 ** rng.uniform(2, 6)),
                                         int(rng.integers(0, 2**31 - 1))))
    return arrivals, pbs


def batch_arm(args):
    """256 realisations (16^3-48^3, 1-20 fractures, ratio 1e2-1e6): one batched
    assembly + solve + 100 transport steps, against the same systems solved
    one at a time with the FP64 path, both to a 1e-8 relative residual."""
    import torch
    import __graft_entry__ as ge
    ge.build()
    import paper_1602_03641_gb300 as pkg
    torch.cuda.set_device(0)
    pbs = batch_problems_cfg(args.batch_size)
    qs = [pkg.problem_arrays(p, device=True) for p in pbs]
    ctx = pkg.Context(0)
    stream = torch.cuda.Stream()
    ctx.set_stream(stream.cuda_stream)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    phm = dev(np.concatenate([p.phi_m for p in pbs]))
    phf = dev(np.concatenate([p.phi_f for p in pbs]))
    cb = dev(np.concatenate([p.cbar for p in pbs]))
    singles = [(q, dev(p.phi_m), dev(p.phi_f), dev(p.cbar), dev(p.c0())) for q, p in zip(qs, pbs)]
    nodes = [p.c0()[:p.n_nodes] for p in pbs]
    ffs = [p.c0()[p.n_nodes:p.n_nodes + p.n_ff] for p in pbs]
    cells = [p.c0()[p.n_nodes + p.n_ff:] for p in pbs]
    c0 = dev(np.concatenate(nodes + ffs + cells))

    def batched(precision, precond):
        s = ctx.assemble_batch(qs)
        s.solve(out=torch.empty(s.info().n_cv, dtype=torch.float64, device="cuda"), precision=precision,
                precond=precond, rtol=1e-8, maxit=100000, raise_on_error=False)
        c = c0.clone()
        s.transport(c, phm, phf, cb, n_steps=100, cfl=0.9)
        infos = s.solve_infos()
        s.close()
        return infos

    def one_at_a_time():
        for q, pm, pf, cbr, cc0 in singles:
            s = ctx.assemble(q["xyz"], q["cell_nodes"], q["ff_nodes"], q["lambda_m"], q["lambda_f"], q["d_f"],
                             q["mu"], q["dir_nodes"], q["dir_values"])
            s.solve(out=torch.empty(s.info().n_cv, dtype=torch.float64, device="cuda"), rtol=1e-8, maxit=100000,
                    raise_on_error=False)
            c = cc0.clone()
            s.transport(c, pm, pf, cbr, n_steps=100, cfl=0.9)
            s.close()

    def t(fn):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1), out

    res = {}
    for name, prec, pc in (("batched_fp64_jacobi", pkg.VAG_FP64, pkg.VAG_PC_JACOBI),
                           ("batched_fp64_amg", pkg.VAG_FP64, pkg.VAG_PC_AMG),
                           ("batched_mixed_jacobi", pkg.VAG_MIXED, pkg.VAG_PC_JACOBI),
                           ("batched_mixed_amg", pkg.VAG_MIXED, pkg.VAG_PC_AMG)):
        ms, infos = t(lambda: batched(prec, pc))
        res[name] = {"solves_per_s": len(pbs) / (ms / 1e3), "ms": ms,
                     "max_rel_residual": max(i.rel_residual for i in infos),
                     "max_iterations": max(i.iterations for i in infos)}
    ms1, _ = t(one_at_a_time)
    res["one_at_a_time_fp64_jacobi"] = {"solves_per_s": len(pbs) / (ms1 / 1e3), "ms": ms1}
    best = max(v["solves_per_s"] for k, v in res.items() if k.startswith("batched"))
    print(json.dumps({"metric": "Darcy solves/s, batched realisations", "value": best, "unit": UNIT,
                      "n_gpus": 1, "higher_is_better": True, "dtype": "f64", "data": "synthetic",
                      "config": {"workload": f"batch of {len(pbs)} realisations: n ~ U{{16..48}}, 1-20 fractures, "
                                             f"ratio log-uniform 1e2-1e6, lognormal K, rtol 1e-8, 100 steps"},
                      "results": res, "speedup_vs_one_at_a_time": best / res["one_at_a_time_fp64_jacobi"]["solves_per_s"]}))
    ctx.close()


def serve_arm(args):
    import threading
    import torch
    import __graft_entry__ as ge
    ge.build()
    import paper_1602_03641_gb300 as pkg
    arrivals, pbs = serve_problems(args.requests)
    lines = {}
    for name, prec, pc in (("fp64_jacobi", pkg.VAG_FP64, pkg.VAG_PC_JACOBI), ("fp64_amg", pkg.VAG_FP64, pkg.VAG_PC_AMG),
                           ("mixed_amg", pkg.VAG_MIXED, pkg.VAG_PC_AMG)):
        srv = pkg.Server(0, budget_bytes=60 * 2**30, slots=3, max_batch=64)
        tickets = [None] * len(pbs)
        t0 = time.perf_counter()

        def producer():
            for i, (ta, pb) in enumerate(zip(arrivals, pbs)):
                dt = ta - (time.perf_counter() - t0)
                if dt > 0:
                    time.sleep(dt)
                tickets[i] = srv.submit(pb, n_steps=100, precision=prec, precond=pc, rtol=1e-8)

        th = threading.Thread(target=producer)
        th.start()
        th.join()
        res = [srv.wait(tk, timeout_ms=600000)[2] for tk in tickets]
        st = srv.stats()
        lines[name] = {"p50_ms": st.p50_ms, "p99_ms": st.p99_ms, "solves_per_s": st.solves_per_s,
                       "completed": int(st.completed), "mean_batch": float(np.mean([r.batch_size for r in res])),
                       "max_rel_residual": max(r.solve.rel_residual for r in res),
                       "failed": sum(1 for r in res if r.status != 0), "peak_reserved_gb": st.peak_bytes / 2**30}
        srv.close()
    print(json.dumps({"metric": "served Darcy+transport requests: solves/s, p50/p99 latency", "unit": UNIT,
                      "value": lines["mixed_amg"]["solves_per_s"], "n_gpus": 1, "higher_is_better": True,
                      "data": "synthetic",
                      "config": {"workload": f"{len(pbs)} Poisson arrivals at 200/s, n lognormal in [16, 96], "
                                             "1-50 fractures, 100 transport steps, rtol 1e-8, 60 GB budget, 3 slots"},
                      "results": lines}))


def mixed128_arm(args):
    """The mixed-precision workload: 128^3 jittered hex with a DFN of 50 seeded
    rectangles at fracture/matrix ratios 1e2, 1e4, 1e6.  Per ratio: the FP64
    and mixed solvers to a 1e-8 relative residual (FP64 residual in all of
    them), each pressure compared with the FP64 AMG solve to 1e-12, then 1000
    explicit transport steps; the hot kernels timed at this size (the CSR
    and the transport map no longer fit the 129 MB L2)."""
    import torch
    import __graft_entry__ as ge
    ge.build()
    import paper_1602_03641_gb300 as pkg
    import vag_inputs as vi
    torch.cuda.set_device(0)
    n = 128 if args.n == N_CELLS_EDGE else args.n
    ctx = pkg.Context(0)
    stream = torch.cuda.Stream()
    ctx.set_stream(stream.cuda_stream)
    peak, peak_kind = measured_peaks()
    fp64_peak = fp64_peak_gflops()
    out = {}
    ev = lambda: torch.cuda.Event(enable_timing=True)
    for ratio in (1e2, 1e4, 1e6):
        pb = vi.config_mixed128(n, ratio)
        a = pkg.problem_arrays(pb, device=True)
        s = ctx.assemble(a["xyz"], a["cell_nodes"], a["ff_nodes"], a["lambda_m"], a["lambda_f"], a["d_f"], a["mu"],
                         a["dir_nodes"], a["dir_values"])
        inf = s.info()
        u_ref = torch.empty(inf.n_cv, dtype=torch.float64, device="cuda")
        _, iref = s.solve(out=u_ref, precond=pkg.VAG_PC_AMG, rtol=1e-12, maxit=20000, raise_on_error=False)
        nref = float(torch.linalg.vector_norm(u_ref))
        res = {"n_rows": inf.n_rows, "nnz": inf.nnz, "n_ff": pb.n_ff, "reference_rel_residual": iref.rel_residual}
        u = torch.empty_like(u_ref)
        for name, prec, pc in (("fp64_amg", pkg.VAG_FP64, pkg.VAG_PC_AMG), ("mixed_amg", pkg.VAG_MIXED, pkg.VAG_PC_AMG),
                               ("mixed16_amg", pkg.VAG_MIXED_F16, pkg.VAG_PC_AMG),
                               ("fp64_jacobi", pkg.VAG_FP64, pkg.VAG_PC_JACOBI),
                               ("mixed_jacobi", pkg.VAG_MIXED, pkg.VAG_PC_JACOBI)):
            times = []
            for rep in range(3):
                e0, e1 = ev(), ev()
                e0.record(stream)
                _, info = s.solve(out=u, precision=prec, precond=pc, rtol=1e-8, maxit=50000, raise_on_error=False)
                e1.record(stream)
                e1.synchronize()
                times.append(e0.elapsed_time(e1))
            err = float(torch.linalg.vector_norm(u - u_ref)) / nref
            res[name] = {"ms": float(np.median(times)), "iterations": info.iterations, "refinements": info.outer,
                         "rel_residual": info.rel_residual, "status": info.status, "rel_l2_vs_fp64_1e-12": err}
        res["mixed_amg_over_fp64_amg"] = res["fp64_amg"]["ms"] / res["mixed_amg"]["ms"]
        res["mixed_amg_over_fp64_jacobi"] = res["fp64_jacobi"]["ms"] / res["mixed_amg"]["ms"]
        # 1000 transport steps on the mixed solve's fluxes
        s.solve(out=u, precision=pkg.VAG_MIXED, precond=pkg.VAG_PC_AMG, rtol=1e-8, maxit=50000, raise_on_error=False)
        c = torch.from_numpy(pb.c0()).cuda()
        phm, phf, cb = (torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in (pb.phi_m, pb.phi_f, pb.cbar))
        torch.cuda.synchronize()
        e0, e1 = ev(), ev()
        e0.record(stream)
        tinf = s.transport(c, phm, phf, cb, n_steps=1000, cfl=0.9)
        e1.record(stream)
        e1.synchronize()
        res["transport_1000_ms"] = e0.elapsed_time(e1)
        res["transport_steps_ms"] = tinf.ms
        inf = s.info()
        nr, nz, ncv, nzt = inf.n_rows, inf.nnz, inf.n_cv, inf.nnz_transport
        ks = {}
        for key, kid, nbytes, flops in (
                ("k_spmv", pkg.VAG_KERNEL_SPMV, nz * 12 + (nr + 1) * 4 + nr * 16, 2 * nz),
                ("k_step", pkg.VAG_KERNEL_TRANSPORT_STEP, ncv * 28 + nzt * 12, 2 * nzt + ncv)):
            ms = s.kernel_time(kid, 100)
            ks[key] = {"ms": ms, "bytes": nbytes, "gbs": nbytes / ms / 1e6, "frac_hbm": nbytes / ms / 1e6 / peak,
                       "frac_fp64": flops / ms / 1e6 / fp64_peak}
        s.solve(out=u, precond=pkg.VAG_PC_AMG, rtol=1e-8, maxit=50000, raise_on_error=False)
        ms = s.kernel_time(pkg.VAG_KERNEL_SMOOTH, 100)
        nbytes = nz * 12 + (nr + 1) * 4 + nr * 32
        ks["k_jac_sell<double>"] = {"ms": ms, "bytes": nbytes, "gbs": nbytes / ms / 1e6,
                                    "frac_hbm": nbytes / ms / 1e6 / peak,
                                    "frac_fp64": (2 * nz + 4 * nr) / ms / 1e6 / fp64_peak}
        res["kernels"] = ks
        out[f"{ratio:g}"] = res
        s.close()
        torch.cuda.empty_cache()
    mid = out["10000"]
    print(json.dumps({"metric": "mixed vs FP64 at 1e-8 relative residual (Darcy solve), 128^3 DFN",
                      "value": mid["mixed_amg_over_fp64_amg"], "unit": "x (FP64 AMG time / mixed AMG time, ratio 1e4)",
                      "n_gpus": 1, "higher_is_better": True, "dtype": "f64 outer / f32 inner", "data": "synthetic",
                      "config": {"workload": f"mixed128: {n}^3 jittered hex, 50 seeded rectangles, ratios 1e2/1e4/1e6, "
                                             "rtol 1e-8, 1000 transport steps", "hbm_peak_gbs": peak,
                                 "hbm_peak_kind": peak_kind, "fp64_peak_tflops": fp64_peak / 1e3},
                      "results": out}))
    ctx.close()


# Iterations of the paper's Table solver_cpg_perm (n_x = 128, N_p = 2; GMRES
# from PETSc, no restart; "-": no convergence in 1200 iterations), context only.
PAPER_SOLVER_PERM = {"GMRES + Boomer AMG": {"20": 15, "100": 15, "1000": 16},
                     "GMRES + Aggregation AMG (Trilinos)": {"20": 59, "100": None, "1000": None},
                     "GMRES + ILU(0)": {"20": 751, "100": None, "1000": None}}


def solvers_arm(args):
    """The shape of the paper's solver experiment (iterations against the
    fracture/matrix permeability ratio, §5.3) on the 128^3 DFN of 50
    rectangles: CG and BiCGStab, each with Jacobi and with the aggregation
    AMG, FP64, to a 1e-8 relative residual, at ratios 20, 100, 1000 (the
    paper's) and 1e4, 1e6."""
    import torch
    import __graft_entry__ as ge
    ge.build()
    import paper_1602_03641_gb300 as pkg
    import vag_inputs as vi
    torch.cuda.set_device(0)
    n = 128 if args.n == N_CELLS_EDGE else args.n
    ctx = pkg.Context(0)
    stream = torch.cuda.Stream()
    ctx.set_stream(stream.cuda_stream)
    ev = lambda: torch.cuda.Event(enable_timing=True)
    res = {}
    for ratio in (20.0, 100.0, 1000.0, 1e4, 1e6):
        pb = vi.config_mixed128(n, ratio)
        a = pkg.problem_arrays(pb, device=True)
        s = ctx.assemble(a["xyz"], a["cell_nodes"], a["ff_nodes"], a["lambda_m"], a["lambda_f"], a["d_f"], a["mu"],
                         a["dir_nodes"], a["dir_values"])
        u = torch.empty(s.info().n_cv, dtype=torch.float64, device="cuda")
        row = {}
        for name, kr, pc in (("CG + Jacobi", pkg.VAG_KRYLOV_CG, pkg.VAG_PC_JACOBI),
                             ("CG + Chebyshev-Jacobi", pkg.VAG_KRYLOV_CG, pkg.VAG_PC_CHEBYSHEV),
                             ("CG + aggregation AMG", pkg.VAG_KRYLOV_CG, pkg.VAG_PC_AMG),
                             ("BiCGStab + Jacobi", pkg.VAG_KRYLOV_BICGSTAB, pkg.VAG_PC_JACOBI),
                             ("BiCGStab + aggregation AMG", pkg.VAG_KRYLOV_BICGSTAB, pkg.VAG_PC_AMG),
                             ("GMRES(30) + aggregation AMG", pkg.VAG_KRYLOV_GMRES, pkg.VAG_PC_AMG)):
            s.solve(out=u, precond=pc, rtol=1e-8, maxit=50000, raise_on_error=False, krylov=kr)   # warm-up
            e0, e1 = ev(), ev()
            e0.record(stream)
            _, info = s.solve(out=u, precond=pc, rtol=1e-8, maxit=50000, raise_on_error=False, krylov=kr)
            e1.record(stream)
            e1.synchronize()
            row[name] = {"iterations": info.iterations, "ms": e0.elapsed_time(e1), "setup_ms": info.ms_setup,
                         "rel_residual": info.rel_residual, "status": info.status}
        res[f"{ratio:g}"] = row
        s.close()
        torch.cuda.empty_cache()
    print(json.dumps({"metric": "linear solver iterations and time vs fracture/matrix permeability ratio (128^3 DFN)",
                      "value": res["1000"]["CG + aggregation AMG"]["iterations"],
                      "unit": "CG + AMG iterations at ratio 1000", "n_gpus": 1, "higher_is_better": False,
                      "dtype": "f64", "data": "synthetic",
                      "config": {"workload": f"solvers: {n}^3 jittered hex, 50 seeded rectangles, rtol 1e-8, "
                                             "ratios 20/100/1000/1e4/1e6"},
                      "results": res, "paper_table_solver_cpg_perm_np2": PAPER_SOLVER_PERM}))
    ctx.close()


def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
        return
    if args.workload == "batch":
        batch_arm(args)
        return
    if args.workload == "serve":
        serve_arm(args)
        return
    if args.workload == "mixed128":
        mixed128_arm(args)
        return
    if args.workload == "solvers":
        solvers_arm(args)
        return
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import __graft_entry__ as ge
    ge.build()
    import paper_1602_03641_gb300 as pkg
    import vag_inputs as vi

    precond = {"jacobi": pkg.VAG_PC_JACOBI, "chebyshev": pkg.VAG_PC_CHEBYSHEV, "amg": pkg.VAG_PC_AMG}[args.precond]
    pb = vi.config_scale64(args.n)
    host = {
        "xyz": pb.xyz.ravel(), "cn": pb.cell_nodes.ravel(), "ffn": pb.ff_nodes.ravel(),
        "lam": pb.lambda_m.ravel(), "lamf": pb.lambda_f, "df": pb.d_f,
        "dn": pb.dir_nodes, "dv": pb.dir_values, "phm": pb.phi_m, "phf": pb.phi_f, "cb": pb.cbar, "c0": pb.c0(),
    }
    host = {k: np.ascontiguousarray(v) for k, v in host.items()}
    d = {k: torch.from_numpy(v).to(dev) for k, v in host.items()}
    # pinned host copies for the end-to-end leg
    pin = {}
    for k, v in host.items():
        t = torch.empty(v.shape, dtype=torch.from_numpy(v).dtype, pin_memory=True)
        t.copy_(torch.from_numpy(v))
        pin[k] = t.numpy()
    n_cv = pb.n_nodes + pb.n_ff + pb.n_cells
    u_pin = torch.empty(n_cv, dtype=torch.float64, pin_memory=True).numpy()
    c_pin = torch.empty(n_cv, dtype=torch.float64, pin_memory=True).numpy()

    ctx = pkg.Context(local)
    stream = torch.cuda.Stream(device=dev)
    ctx.set_stream(stream.cuda_stream)
    u_dev = torch.empty(n_cv, dtype=torch.float64, device=dev)
    c_dev = torch.empty(n_cv, dtype=torch.float64, device=dev)
    flush_buf = torch.empty(256 * 2**20 // 4, dtype=torch.float32, device=dev)

    phase_ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
    phase_ms = {"assemble": [], "solve": [], "transport": [], "destroy": []}

    def step_device():
        phase_ev[0].record(stream)
        s = ctx.assemble(d["xyz"], d["cn"], d["ffn"], d["lam"], d["lamf"], d["df"], pb.mu, d["dn"], d["dv"])
        phase_ev[1].record(stream)
        _, info = s.solve(out=u_dev, precond=precond, rtol=RTOL, maxit=100000)
        phase_ev[2].record(stream)
        with torch.cuda.stream(stream):
            c_dev.copy_(d["c0"])
        tinf = s.transport(c_dev, d["phm"], d["phf"], d["cb"], n_steps=TRANSPORT_STEPS, cfl=0.9)
        phase_ev[3].record(stream)
        s.close()
        phase_ev[4].record(stream)
        phase_ev[4].synchronize()
        for k, name in enumerate(["assemble", "solve", "transport", "destroy"]):
            phase_ms[name].append(phase_ev[k].elapsed_time(phase_ev[k + 1]))
        return info, tinf

    def step_device_prec(precision, pc, rtol):
        s = ctx.assemble(d["xyz"], d["cn"], d["ffn"], d["lam"], d["lamf"], d["df"], pb.mu, d["dn"], d["dv"])
        _, info = s.solve(out=u_dev, precision=precision, precond=pc, rtol=rtol, maxit=100000)
        with torch.cuda.stream(stream):
            c_dev.copy_(d["c0"])
        tinf = s.transport(c_dev, d["phm"], d["phf"], d["cb"], n_steps=TRANSPORT_STEPS, cfl=0.9)
        s.close()
        return info, tinf

    def step_host():
        s = ctx.assemble(pin["xyz"], pin["cn"], pin["ffn"], pin["lam"], pin["lamf"], pin["df"], pb.mu,
                         pin["dn"], pin["dv"])
        _, info = s.solve(out=u_pin, precond=precond, rtol=RTOL, maxit=100000)
        c_pin[:] = pin["c0"]
        tinf = s.transport(c_pin, pin["phm"], pin["phf"], pin["cb"], n_steps=TRANSPORT_STEPS, cfl=0.9)
        s.close()
        return info, tinf

    def flush():
        with torch.cuda.stream(stream):
            flush_buf.zero_()

    def timed(fn, k):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
        infos = []
        for i in range(k):
            flush()
            evs[i][0].record(stream)
            infos.append(fn())
            evs[i][1].record(stream)
        stream.synchronize()
        return [a.elapsed_time(b) for a, b in evs], infos

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step_device()
    barrier()
    gpu_uuid = getattr(torch.cuda.get_device_properties(dev), "uuid", None)
    sampler = ClockSampler(str(gpu_uuid) if gpu_uuid is not None else None, local)
    lc0 = pkg.launch_count()
    for v in phase_ms.values():
        v.clear()
    ms, infos = timed(step_device, args.steps)
    lc1 = pkg.launch_count()
    barrier()
    clocks = sampler.stop()
    value, tot = replica_throughput(sum(ms), args.steps, world, dev)

    # end to end from pinned host buffers
    e2e = None
    if not args.no_e2e:
        step_host()
        barrier()
        ms_h, _ = timed(step_host, args.steps)
        _, tot_h = replica_throughput(sum(ms_h), args.steps, world, dev)
        h2d = sum(pin[k].nbytes for k in ["xyz", "cn", "ffn", "lam", "lamf", "df", "dn", "dv", "phm", "phf", "cb",
                                         "c0"])
        e2e = {"value": world * args.steps / (tot_h / 1e3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(u_pin.nbytes + c_pin.nbytes), "ms_per_step": tot_h / args.steps}

    # the metric's "mixed vs FP64 at 1e-8": every solver variant to a 1e-8
    # relative residual (FP64 residual in all of them), same step otherwise.
    # mixed + jacobi = FP64 refinement around FP32 CG; mixed + amg = FP64 CG
    # preconditioned by the FP32 copy of the AMG hierarchy.
    cmp = {}
    for name, prec, pc in (("fp64_jacobi", pkg.VAG_FP64, pkg.VAG_PC_JACOBI), ("mixed_jacobi", pkg.VAG_MIXED, pkg.VAG_PC_JACOBI),
                           ("fp64_chebyshev", pkg.VAG_FP64, pkg.VAG_PC_CHEBYSHEV),
                           ("fp64_amg", pkg.VAG_FP64, pkg.VAG_PC_AMG), ("mixed_amg", pkg.VAG_MIXED, pkg.VAG_PC_AMG),
                           ("mixed16_amg", pkg.VAG_MIXED_F16, pkg.VAG_PC_AMG)):
        step_device_prec(prec, pc, 1e-8)
        ms_c, inf_c = timed(lambda: step_device_prec(prec, pc, 1e-8), max(3, args.steps // 2))
        cmp[name] = {"solves_per_s": len(ms_c) / (sum(ms_c) / 1e3), "ms_per_step": sum(ms_c) / len(ms_c),
                     "setup_ms": inf_c[-1][0].ms_setup, "solve_ms": inf_c[-1][0].ms_solve,
                     "iterations": inf_c[-1][0].iterations, "refinements": inf_c[-1][0].outer,
                     "rel_residual": inf_c[-1][0].rel_residual}
    cmp["mixed_over_fp64_jacobi"] = cmp["mixed_jacobi"]["solves_per_s"] / cmp["fp64_jacobi"]["solves_per_s"]
    cmp["mixed_over_fp64_amg"] = cmp["mixed_amg"]["solves_per_s"] / cmp["fp64_amg"]["solves_per_s"]

    # Hot kernels timed live on the workload's own data through the library's
    # measurement hook (CUDA events on the library's stream): the CG product,
    # one finest-level smoother sweep of the AMG V-cycle, one transport step.
    # Share of the step = launches per step x mean launch time / step time.
    peak, peak_kind = measured_peaks()
    fp64_peak = fp64_peak_gflops()
    s = ctx.assemble(d["xyz"], d["cn"], d["ffn"], d["lam"], d["lamf"], d["df"], pb.mu, d["dn"], d["dv"])
    _, sinf = s.solve(out=u_dev, precond=precond, rtol=RTOL, maxit=100000)
    with torch.cuda.stream(stream):
        c_dev.copy_(d["c0"])
    s.transport(c_dev, d["phm"], d["phf"], d["cb"], n_steps=TRANSPORT_STEPS, cfl=0.9)
    inf = s.info()
    reps = 400
    its = sinf.iterations
    n, nnz, ncv, nnzt = inf.n_rows, inf.nnz, inf.n_cv, inf.nnz_transport
    kern = {}
    def add(name, ms, per_step, nbytes, flops):
        kern[name] = {"ms": ms, "launches_per_step": per_step, "share_of_step": per_step * ms / (tot / args.steps),
                      "bytes": nbytes, "gbs": nbytes / ms / 1e6, "fp64_gflops": flops / ms / 1e6,
                      "frac_hbm": nbytes / ms / 1e6 / peak, "frac_fp64": flops / ms / 1e6 / fp64_peak}
    add("k_spmv (FP64 SELL q = A p)", s.kernel_time(pkg.VAG_KERNEL_SPMV, reps), its + 2,
        nnz * 12 + (n + 1) * 4 + n * 16, 2 * nnz)
    if args.precond == "amg":
        # one finest-level sweep per V-cycle with a matrix pass (the first,
        # from zero, is made by the CG update): its V-cycles + the initial one
        add("k_jac_sell<double> (finest-level l1-Jacobi sweep)", s.kernel_time(pkg.VAG_KERNEL_SMOOTH, reps),
            its + 1, nnz * 12 + (n + 1) * 4 + n * 32, 2 * nnz + 4 * n)
    add("k_step (upwind transport step)", s.kernel_time(pkg.VAG_KERNEL_TRANSPORT_STEP, reps), TRANSPORT_STEPS,
        ncv * 28 + nnzt * 12, 2 * nnzt + ncv)
    s.close()
    dom = max(kern, key=lambda k: kern[k]["share_of_step"])
    kd = kern[dom]
    # the binding resource is the one the kernel uses the larger fraction of
    if kd["frac_fp64"] >= kd["frac_hbm"]:
        roof = {"kernel": dom, "bound": "alu", "achieved": kd["fp64_gflops"] / 1e3, "peak": fp64_peak / 1e3,
                "unit": "TFLOP/s (FP64)", "frac": kd["frac_fp64"], "peak_kind": "derived: 2 DFMA/clk/SM x 152 SMs x "
                "max SM clock (ncu sm__sass_thread_inst_executed_op_dfma_pred_on peak_sustained)",
                "secondary": {"bound": "hbm", "achieved": kd["gbs"], "peak": peak, "unit": "GB/s",
                              "frac": kd["frac_hbm"], "peak_kind": peak_kind}}
    else:
        roof = {"kernel": dom, "bound": "hbm", "achieved": kd["gbs"], "peak": peak, "unit": "GB/s",
                "frac": kd["frac_hbm"], "peak_kind": peak_kind,
                "secondary": {"bound": "alu", "achieved": kd["fp64_gflops"] / 1e3, "peak": fp64_peak / 1e3,
                              "unit": "TFLOP/s (FP64)", "frac": kd["frac_fp64"]}}
    roof["traffic"] = ncu_traffic(dom)
    roof["bytes_per_launch"] = kd["bytes"]
    roof["launch_ms"] = kd["ms"]
    spmv_gbs = kern["k_spmv (FP64 SELL q = A p)"]["gbs"]
    iters = [i[0].iterations for i in infos]

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD if args.n == N_CELLS_EDGE else f"scale{args.n} (profiling case)",
                       "precond": args.precond, "rtol": RTOL,
                       "transport_steps": TRANSPORT_STEPS, "n_rows": inf.n_rows, "nnz": inf.nnz,
                       "n_cv": inf.n_cv, "l2": "flushed before every timed step (256 MiB write)",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "latency_ms": {"p50": float(np.percentile(ms, 50)), "p99": float(np.percentile(ms, 99))},
            "cg_iterations": iters[-1], "rel_residual": infos[-1][0].rel_residual,
            "phases_ms": {**{k: float(np.median(v)) for k, v in phase_ms.items()},
                          "of_which_precond_setup": infos[-1][0].ms_setup,
                          "of_which_krylov_and_recovery": infos[-1][0].ms_solve,
                          "of_which_transport_steps": infos[-1][1].ms},
            "spmv_gbs": spmv_gbs, "kernels": kern,
            "roofline": roof, "gpu_launches": int(lc1 - lc0), "clocks": clocks, "e2e": e2e,
            "solvers_at_1e-8": cmp,
        }
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline_block()
        print(json.dumps(line))
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
