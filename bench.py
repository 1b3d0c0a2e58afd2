"""Benchmark of the HBPC-DGSEM hot path on one GB300.

Workload (default): 2-D linear advection u_t + div((1, 1) u) = 0 on the periodic
unit square, 64 x 64 elements, N = 5 (Gauss-Lobatto), u0 = sin(2 pi x) sin(2 pi y),
HBPC(8, 4) (the highest order of the paper), CFL 8 -> dt = 1/96, matrix-free
Newton-GMRES with the paper's BJ_ext preconditioner, eps_Newton = 1e-12 with
the absolute test ||dW|| <= 1e-12, eps_GMRES = 1e-5, mixed precision (FP64
Newton residual, update and state; FP32 Krylov loop).  One bench step = one
HBPC time step (15 implicit stage solves).  Metric: DOF-timesteps/s = n_dof x
steps / device seconds.  The same line carries, under "learned_vs_plain", the
metric's comparison on the Euler vortex workload (learned block preconditioner
trained on the GPU from the run's own Newton-GMRES data vs plain GMRES and
BJ_ext; --no-vortex skips it).

  python bench.py [--steps K] [--warmup W] [--gpus N] [--impl reference]
  python bench.py --workload burgers_batch   (256 viscous Burgers instances, below)
  python bench.py --workload euler_vortex    (learned vs BJ_ext vs plain GMRES, below)

Under torchrun (N > 1) every rank runs an independent replica of the workload
(the path has no data-path collective), value = sum over ranks / max time.
The reference arm (--impl reference) times the FP64 CPU oracle on the host on
a bounded sample of the same workload.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DOF-timesteps/s per HBPC step at fixed L2 error; learned vs plain GMRES"
PRECISION = ["mixed"]   # set from --precision
UNIT = "DOF-timesteps/s"

WL = dict(dim=2, n=(64, 64), lo=(0.0, 0.0), hi=(1.0, 1.0), N=5, a=(1.0, 1.0), q=8, kmax=4,
          cfl=8.0, t_end=1.0, tol_newton_rel=1e-12, tol_newton_abs=1e-12, tol_gmres_rel=1e-5,
          gmres_restart=100, gmres_max_iter=7000, newton_max_iter=50)


def workload_dt():
    # dt_raw = CFL / sum_m(|a_m| p / h_m), rounded to T_end / ceil(T_end / dt_raw)
    p = WL["N"] + 1
    s = sum(abs(WL["a"][m]) * p / ((WL["hi"][m] - WL["lo"][m]) / WL["n"][m]) for m in range(WL["dim"]))
    raw = WL["cfl"] / s
    return WL["t_end"] / np.ceil(WL["t_end"] / raw - 1e-12)


def config_dict(dt, extra=None):
    c = {"workload": "2d_linear_advection_64x64_N5_HBPC(8,4)_CFL8_BJext_GMRES",
         "precision": PRECISION[0],
         "mesh": "64x64 periodic [0,1]^2", "N": 5, "nodes": "Gauss-Lobatto", "hbpc": "q=8,kmax=4",
         "dt": dt, "eps_newton": WL["tol_newton_rel"], "newton_abs_dW": WL["tol_newton_abs"],
         "eps_gmres": WL["tol_gmres_rel"],
         "gmres_restart": WL["gmres_restart"], "preconditioner": "BJ_ext (Sec. 3.2.3)",
         "l2_between_steps": "flushed (256 MB write) between timed steps",
         "launches": ("Arnoldi steps in batches of 4 replayed as one CUDA graph each"
                      if os.environ.get("HBPC_GRAPH", "1") != "0" else "one launch per kernel (HBPC_GRAPH=0)")}
    if extra:
        c.update(extra)
    return c


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                smax.append(float(f[1]))
            except ValueError:
                continue
            for k, name in enumerate(names):
                if f[4 + k].lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def exact_solution(coords, t):
    from paper_2109_04804_gb300 import inputs
    sh = [c - a * t for c, a in zip(coords, WL["a"])]
    return inputs.sine_product(sh)


# -- algorithmic work per launch (bytes, flops per W-DOF) ----------------------
def jv_work_per_dof(mixed=False):
    """Linear Jv (Eq. 24): reads dW, dS and writes the two outputs: 32 B per
    W-DOF in FP64 (16 B in FP32).  Flops: two R1 passes, each 2*d*p (volume)
    + 2*d/p face points x 7 (flux 5, lifting 2), plus 3 FMAs to combine."""
    d, p = WL["dim"], WL["N"] + 1
    r1 = 2 * d * p + (2 * d / p) * 7
    return (16.0 if mixed else 32.0), 2 * r1 + 6


def pc_work_per_dof(mixed=False):
    """BJ_ext apply on this workload: linear advection on one uniform mesh has
    the same J_i (hence M_i) in every element, so the library builds one block
    pair and the apply reads only the two input halves and writes the two
    output halves: 32 B per W-DOF in FP64, 16 B in FP32 (the 2 n_b^2 block
    values once per launch are negligible); four n_b x n_b matrix-vector
    products: 8 n_b flops per W-DOF (+ 4)."""
    nb = (WL["N"] + 1) ** WL["dim"]
    return (16.0 if mixed else 32.0), 8.0 * nb + 4.0


# DRAM bytes (read + write) per launch measured by ncu on this workload's
# kernels (summaries in profiles/: k_cgs_coop_c2_advection_64x64_N5.md, the mean
# of three captured columns; dg_operator_jv_pair_c2_advection_64x64_N5.md).
# A kernel changed after its capture must have its entry set to None (the
# shared-block apply has not been captured).
NCU_TRAFFIC = {"cgs2": 3.68e6, "pc_apply": None, "jv": 1.20e6}


def run_ours(args):
    import torch
    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    import __graft_entry__ as g
    g.build()
    from paper_2109_04804_gb300 import hbpc, inputs
    dt = workload_dt()
    stream = torch.cuda.Stream()
    ctx = hbpc.Context(WL["dim"], WL["n"], WL["lo"], WL["hi"], WL["N"], law=hbpc.LAW_ADVECTION,
                       a=WL["a"], q=WL["q"], kmax=WL["kmax"], dt=dt,
                       tol_newton_rel=WL["tol_newton_rel"], tol_newton_abs=WL["tol_newton_abs"],
                       tol_gmres_rel=WL["tol_gmres_rel"], gmres_restart=WL["gmres_restart"],
                       gmres_max_iter=WL["gmres_max_iter"], newton_max_iter=WL["newton_max_iter"],
                       pc=hbpc.PC_BJEXT, stream=stream.cuda_stream,
                       precision=hbpc.PREC_MIXED if PRECISION[0] == "mixed" else hbpc.PREC_FP64)
    coords = ctx.node_coords()
    w0 = inputs.sine_product(coords)
    ctx.set_state(w0)
    ndof = ctx.ndof
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        ctx.step(1)
    tuning = ctx.autotune()        # launch shapes of the Krylov reductions and the PC apply
    torch.cuda.synchronize()
    ctx.reset_stats()
    clocks = Clocks(local)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    total_ms = 0.0
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(1.0)             # L2 flush outside the timed window
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.step(1)
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
    torch.cuda.synchronize()
    clk = clocks.stop()
    stats = ctx.stats()
    t_sec = total_ms / 1000.0
    if world > 1:
        tt = torch.tensor([t_sec], device="cuda")
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        t_sec = float(tt.item())
        torch.distributed.barrier()
    value = ndof * args.steps * world / t_sec
    r1_per_s = (stats["r1_evals"] + stats["r2_evals"]) / t_sec
    # accuracy: L2 error vs the exact solution at the final time
    w = ctx.get_state()
    t_fin = (args.warmup + args.steps) * dt
    err = float(np.sqrt(np.mean((w - exact_solution(coords, t_fin)) ** 2)))

    # per-phase device time from a separate profiled step (events around launches)
    ctx.profile(True)
    ctx.step(1)
    prof = ctx.profile_get()
    pstats = ctx.stats()
    ctx.profile(False)
    # roofline of the dominant kernel phase (FP64 on GB300 is ALU-bound: the
    # denominator is the measured FP64 FMA throughput; HBM fraction alongside)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    fp64_peak = hbpc.fp64_fma_peak()          # measured live on this GPU
    hbm = peaks.get("hbm_gbs", 6800.0)
    mixed = PRECISION[0] == "mixed"
    # CGS2 column (one launch per Arnoldi iteration): the three passes read the
    # new vector and the j + 1 basis vectors and write the new vector twice:
    # (3 (j + 1) + 5) vectors of 2 n_dof values; 6 (j + 1) + 8 flops per value
    its_p = pstats["gmres_its"] - stats["gmres_its"]
    cols_p = pstats["arnoldi_cols"] - stats["arnoldi_cols"]
    cavg = cols_p / max(1, its_p)
    vb = 4.0 if mixed else 8.0
    cgs_b = (3.0 * cavg + 5.0) * 2.0 * vb       # bytes per W-DOF per launch
    cgs_f = (6.0 * cavg + 8.0) * 2.0            # flops per W-DOF per launch
    prof_cgs = (prof["arnoldi_dot"][0] + prof["arnoldi_update"][0], its_p)
    kernels = {"jv": ("dg_operator_kernel<advection pair,2D,P=6,JobJvLinearPair<%s>> (Eq. 24, both halves in one pass)"
                      % ("float" if mixed else "double"), jv_work_per_dof(mixed), prof["jv"]),
               "pc_apply": (("k_pc_apply_shared<float, 2> (BJ_ext, Sec. 3.2.3; one block pair for all elements)"
                             if mixed else "k_pc_apply<double> (BJ_ext, Sec. 3.2.3; one block pair for all elements)"),
                            pc_work_per_dof(mixed), prof["pc_apply"]),
               "cgs2": ("k_cgs_coop<%s> (Arnoldi CGS2 column, one cooperative launch; mean j + 1 = %.1f)"
                        % ("float" if mixed else "double", cavg), (cgs_b, cgs_f), prof_cgs)}
    entries = {}
    for ph, (name, (bpd, fpd), (ms, n)) in kernels.items():
        if n == 0:
            continue
        avg = ms / 1000.0 / n
        gf = fpd * ndof / avg / 1e9
        gb = bpd * ndof / avg / 1e9
        if mixed:   # FP32 arithmetic is 62x the FP64 rate: these kernels are HBM-bound
            entries[ph] = {"kernel": name, "bound": "hbm", "achieved": round(gb, 1), "peak": hbm,
                           "unit": "GB/s", "frac": round(gb / hbm, 4), "traffic": NCU_TRAFFIC.get(ph),
                           "algorithmic_bytes_per_launch": round(bpd * ndof),
                           "alu_tflops": round(gf / 1000.0, 3)}
        else:
            entries[ph] = {"kernel": name, "bound": "alu", "achieved": round(gf / 1000.0, 4),
                           "peak": fp64_peak / 1000.0, "unit": "TFLOP/s", "frac": round(gf / fp64_peak, 4),
                           "traffic": None, "hbm_achieved_gbs": round(gb, 1),
                           "hbm_frac_of_measured": round(gb / hbm, 4)}
        entries[ph].update({"avg_launch_us": round(avg * 1e6, 2), "launches_profiled": n,
                            "share_of_step": round(ms / sum(v[0] for v in prof.values()), 3)})
    dom = max(entries, key=lambda k: kernels[k][2][0])
    roofline = dict(entries[dom])
    roofline["peak_source"] = ("measured HBM copy bandwidth (MEASURED_PEAKS.json)" if mixed else
                               "FP64 FMA throughput measured in this run (hbpc_fp64_fma_peak)")
    roofline["phase_ms_one_step"] = {k: round(v[0], 3) for k, v in prof.items()}
    roofline["phase_launches_one_step"] = {k: v[1] for k, v in prof.items()}
    roofline["other_kernels"] = {k: v for k, v in entries.items() if k != dom}

    # e2e: the public API with host buffers, copies inside the timed region
    host_in = torch.from_numpy(w0.copy()).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ctx.set_state_host_ptr(host_in.data_ptr())
        ctx.step(1)
        ctx.get_state_host_ptr(host_out.data_ptr())
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e = {"value": ndof * args.steps * world / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": ndof * 8, "d2h_bytes_per_step": ndof * 8}
    ctx.close()
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if PRECISION[0] == "fp64" else "f64 state/Newton, f32 Krylov",
            "data": "synthetic",
            "config": config_dict(dt, {"parallelism": "replicas" if world > 1 else "single",
                                       "autotuned": tuning}),
            "r1_evals_per_s": r1_per_s, "l2_error_vs_exact": err,
            "gmres_its_per_step": stats["gmres_its"] / args.steps,
            "newton_its_per_step": stats["newton_its"] / args.steps,
            "gpu_launches": int(stats["launches"]), "roofline": roofline, "e2e": e2e, "clocks": clk}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(dt)
    if rank == 0 and world == 1 and not args.no_vortex:
        # the metric's comparison, on the Euler vortex workload (learned block
        # preconditioner trained on the run's own Newton-GMRES data vs plain
        # GMRES and BJ_ext); see --workload euler_vortex for the full line
        va = argparse.Namespace(steps=1, warmup=2)
        v = run_vortex(va, emit=False)
        ln, pl, bj = v["learned"], v["plain_gmres"], v["bjext"]
        line["learned_vs_plain"] = {
            "workload": v["config"]["workload"], "unit": UNIT,
            "learned": ln, "plain_gmres": pl, "bjext": bj,
            "speedup_learned_over_plain": (ln["value"] / pl["value"]) if pl["value"] > 0 else None,
            "speedup_learned_over_bjext": (ln["value"] / bj["value"]) if bj["value"] > 0 else None,
            "training": v["config"]["training"]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def cpu_baseline(dt, budget_s=20.0):
    """The FP64 oracle as it stands, on the host cores, on a bounded sample of
    the workload: the first predictor stage solve of one HBPC(8,4) step (one of
    its 15 stage solves), scaled to a full step."""
    from oracle import dgsem, laws, newton
    from paper_2109_04804_gb300 import inputs
    ph = laws.Physics(laws.ADVECTION, 2, a=WL["a"])
    disc = dgsem.Disc(dgsem.Mesh(2, WL["n"], WL["lo"], WL["hi"]), WL["N"], ph)
    w0 = inputs.sine_product(disc.node_coords())
    opts = newton.NewtonOptions(tol_rel=WL["tol_newton_rel"], tol_abs=WL["tol_newton_abs"],
                                gmres_tol=WL["tol_gmres_rel"], restart=WL["gmres_restart"],
                                jv="linear", pc="bjext")
    dc = 1.0 / 3.0
    a1, a2 = dc / 2.0, dc * dc / 6.0
    r1 = dgsem.R1(disc, w0)
    b = w0 + a1 * dt * r1 + (a2 * dt * dt / 2.0) * dgsem.R2(disc, w0, r1)
    t0 = time.perf_counter()
    _, _, st = newton.newton_solve(disc, b, a1, a2, dt, w0, opts)
    t1 = time.perf_counter() - t0
    solves_per_step = (4 - 1) * (1 + 4)
    step_s = t1 * solves_per_step
    threads = int(os.environ.get("OMP_NUM_THREADS", "0")) or (os.cpu_count() or 1)
    return {"value": disc.ndof / step_s, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": "first predictor stage solve of one HBPC(8,4) step on the full 64x64 N=5 "
                      "mesh (%d GMRES its, %.1f s), scaled x%d stage solves per step"
                      % (st.gmres_its, t1, solves_per_step)}


BATCH = dict(n_inst=256, n_range=(16, 96), N_range=(3, 7), nu_range=(1e-3, 1e-2), seed=2024,
             q=6, kmax=2, cfl_finest=2.0, tol_newton_rel=1e-10, tol_newton_abs=1e-12, tol_gmres_rel=1e-3,
             gmres_restart=100, gmres_max_iter=3000, newton_max_iter=50, max_per_group=0)


def batch_instances(n_inst):
    """The seeded instance list of the batched viscous Burgers workload: square
    periodic meshes n x n on [0, 1]^2 with n uniform in 16..96, N uniform in
    3..7, nu uniform in [1e-3, 1e-2]; initial data: 8 random Fourier modes,
    max |u0| = 1 (seed per instance)."""
    rng = np.random.default_rng(BATCH["seed"])
    out = []
    for i in range(n_inst):
        n = int(rng.integers(BATCH["n_range"][0], BATCH["n_range"][1] + 1))
        N = int(rng.integers(BATCH["N_range"][0], BATCH["N_range"][1] + 1))
        nu = float(rng.uniform(*BATCH["nu_range"]))
        out.append(((n, n), N, nu, 1000 + i))
    return out


def run_batch(args):
    """Batched workload: independent 2-D viscous Burgers instances
    u_t + div(u^2/2 (1, 1)) = nu Laplace(u) (BR2, Sec. 5.1.1; global LF flux), one batch
    (hbpc_batch_*) advanced by HBPC(6, 2) with a common dt (CFL 2 on the finest
    instance), mixed precision (FP32 Krylov and R1 linearisation, FP64 Newton
    residual), BJ_ext.  One step = one HBPC step of every instance."""
    import torch
    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    import __graft_entry__ as g
    g.build()
    from paper_2109_04804_gb300 import hbpc, inputs
    inst = batch_instances(args.instances)
    h_min = min(1.0 / n[0] / (N + 1) for n, N, _, _ in inst)
    dt = BATCH["cfl_finest"] * h_min        # max |u0| = 1
    b = hbpc.Batch(2, [(n, (0.0, 0.0), (1.0, 1.0)) for n, _, _, _ in inst], [N for _, N, _, _ in inst],
                   nus=[nu for _, _, nu, _ in inst], law=hbpc.LAW_BURGERS, flux=hbpc.FLUX_GLOBAL_LF,
                   q=BATCH["q"], kmax=BATCH["kmax"], dt=dt, tol_newton_rel=BATCH["tol_newton_rel"],
                   tol_newton_abs=BATCH["tol_newton_abs"], tol_gmres_rel=BATCH["tol_gmres_rel"],
                   gmres_restart=BATCH["gmres_restart"], gmres_max_iter=BATCH["gmres_max_iter"],
                   newton_max_iter=BATCH["newton_max_iter"], pc=hbpc.PC_BJEXT, precision=hbpc.PREC_MIXED,
                   max_per_group=args.max_per_group)
    ndof = 0
    w0s = []
    for i, (n, N, nu, seed) in enumerate(inst):
        w0 = inputs.burgers_fourier(b.node_coords(i), seed=seed)
        b.set_state(i, w0)
        w0s.append(w0)
        ndof += w0.size
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        b.step(1)
    tuning = b.autotune()          # launch shapes per group, on the warmed-up state
    torch.cuda.synchronize()
    st0 = b.stats()
    clocks = Clocks(local)
    if world > 1:
        torch.distributed.barrier()
    clocks.start()
    total = 0.0
    for _ in range(args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b.step(1)                 # every group's stream synchronised before it returns
        torch.cuda.synchronize()
        total += time.perf_counter() - t0
    clk = clocks.stop()
    st = b.stats()
    t_sec = total
    if world > 1:
        tt = torch.tensor([t_sec], device="cuda")
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        t_sec = float(tt.item())
    value = ndof * args.steps * world / t_sec
    d = {k: st[k] - st0[k] for k in ("newton_its", "gmres_its", "r1_evals", "r2_evals", "launches")}
    # e2e: host buffers copied in and out of every instance every step
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for i in range(len(inst)):
            b.set_state(i, w0s[i])
        b.step(1)
        for i in range(len(inst)):
            b.get_state(i)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    groups = b.groups()
    b.close()
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * t_sec / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64 state/Newton, f32 Krylov", "data": "synthetic",
            "config": {"workload": "batched_viscous_burgers_%d_instances_HBPC(6,2)_BR2_BJext" % len(inst),
                       "instances": len(inst), "groups": groups, "max_per_group": args.max_per_group,
                       "total_dof": ndof,
                       "mesh": "n x n periodic [0,1]^2, n uniform in 16..96", "N": "uniform in 3..7",
                       "nu": "uniform in [1e-3, 1e-2]", "dt": dt, "cfl_finest": BATCH["cfl_finest"],
                       "flux": "global Lax-Friedrichs (lambda = 1 = max |u0|; constant dissipation, so the "
                               "FP32 analytic Jacobian-vector product is exact)",
                       "eps_newton": BATCH["tol_newton_rel"], "eps_gmres": BATCH["tol_gmres_rel"],
                       "gmres_restart": BATCH["gmres_restart"], "precision": "mixed",
                       "timing": "host clock between device synchronisations (groups run on their own streams)",
                       "autotuned": tuning,
                       "l2_between_steps": "flushed (256 MB write) between timed steps",
                       "parallelism": "replicas" if world > 1 else "single"},
            "r1_evals_per_s": (d["r1_evals"] + d["r2_evals"]) / t_sec,
            "gmres_its_per_step": d["gmres_its"] / args.steps, "newton_its_per_step": d["newton_its"] / args.steps,
            "gpu_launches": int(d["launches"]),
            "e2e": {"value": ndof * args.steps * world / e2e_s, "unit": UNIT,
                    "h2d_bytes_per_step": ndof * 8, "d2h_bytes_per_step": ndof * 8},
            "clocks": clk}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


VORTEX = dict(n=(128, 128), lo=(-10.0, -10.0), hi=(10.0, 10.0), N=4, q=6, kmax=2, cfl=10.0,
              tol_newton_rel=1e-10, tol_newton_abs=1e-12, tol_gmres_rel=1e-3, gmres_restart=100,
              gmres_max_iter=3000, newton_max_iter=30, collect_per_newton=1024, collect_capacity=32768,
              train_inverse_its=20000, train_lr=1e-3, train_batch=256,
              train_probe=((8000, 1e-5), (8000, 1e-5), (8000, 5e-6), (8000, 2e-6)), train_probes=8)


def vortex_dt():
    """CFL / sum_m(lambda_max,m (N+1) / h_m) with lambda_max = |v| + c of the
    free stream plus the vortex's peak velocity (about 0.5 c_inf)."""
    g = 1.4
    lam = (0.5 * np.sqrt(g) + np.sqrt(g), np.sqrt(g))
    h = [(VORTEX["hi"][m] - VORTEX["lo"][m]) / VORTEX["n"][m] for m in range(2)]
    return VORTEX["cfl"] / sum(lam[m] * (VORTEX["N"] + 1) / h[m] for m in range(2))


def run_vortex(args, emit=True):
    """2-D Euler isentropic vortex (strength 5, Mach 0.5) on [-10, 10]^2, 128 x 128
    elements, N = 4, Rusanov, HBPC(6, 2), CFL 10, Newton tol 1e-10, mixed
    precision.  The learned block preconditioner is trained on the GPU on
    (features, exact block inverse) samples of the method's own BJ_ext Newton
    iterations during the warm-up steps; then the same time step is taken with
    the learned preconditioner, with BJ_ext, and with plain GMRES (no
    preconditioner), each against the FP64-state BJ_ext result."""
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__ as g
    g.build()
    from paper_2109_04804_gb300 import hbpc, inputs
    dt = vortex_dt()

    def ctx(pc):
        return hbpc.Context(2, VORTEX["n"], VORTEX["lo"], VORTEX["hi"], VORTEX["N"], law=hbpc.LAW_EULER,
                            flux=hbpc.FLUX_RUSANOV, q=VORTEX["q"], kmax=VORTEX["kmax"], dt=dt,
                            tol_newton_rel=VORTEX["tol_newton_rel"], tol_newton_abs=VORTEX["tol_newton_abs"],
                            tol_gmres_rel=VORTEX["tol_gmres_rel"], gmres_restart=VORTEX["gmres_restart"],
                            gmres_max_iter=VORTEX["gmres_max_iter"], newton_max_iter=VORTEX["newton_max_iter"],
                            pc=pc, precision=hbpc.PREC_MIXED)
    gen = ctx(hbpc.PC_BJEXT)
    gen.pc_collect(VORTEX["collect_per_newton"], VORTEX["collect_capacity"])
    gen.set_state(inputs.isentropic_vortex(gen.node_coords()))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    gen.step(max(1, args.warmup))
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    w_start = gen.get_state()
    gen.pc_collect(0, 0)
    gen.pc_model_init(seed=1, out_scale=1e-2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    l0, l1 = gen.pc_train(iters=VORTEX["train_inverse_its"], batch=VORTEX["train_batch"], probes=4,
                          lr=VORTEX["train_lr"], seed=11, loss="inverse")
    # then the probe loss |M~ S x - x|^2, what the preconditioner has to achieve
    probe_losses = []
    for k, (its, lr) in enumerate(VORTEX["train_probe"]):
        pa, pb = gen.pc_train(iters=its, batch=VORTEX["train_batch"], probes=VORTEX["train_probes"], lr=lr,
                              seed=50 + k, loss="probe")
        probe_losses.append((pa, pb))
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    params = gen.pc_model_get()
    ndof = gen.ndof
    gen.close()

    def timed(pc, steps, params=None):
        c = ctx(pc)
        if params is not None:
            c.pc_model_set(params)
        c.set_state(w_start)
        ok, ms = True, 0.0
        for _ in range(steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            try:
                c.step(1)
            except hbpc.HBPCError as e:
                ok = str(e)[:80]
            e1.record()
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
            if ok is not True:
                break
        st = c.stats()
        w = c.get_state()
        c.close()
        return {"ok": ok, "ms_per_step": ms / steps, "value": ndof * steps / (ms / 1000.0) if ok is True else 0.0,
                "gmres_its_per_step": st["gmres_its"] / steps, "newton_its_per_step": st["newton_its"] / steps,
                "launches": int(st["launches"]),
                "exact_blocks_per_build": (st["pc_exact_blocks"] / max(1, st["newton_its"])
                                           if pc == hbpc.PC_LEARNED else None)}, w

    r_bj, w_bj = timed(hbpc.PC_BJEXT, args.steps)
    r_ln, w_ln = timed(hbpc.PC_LEARNED, args.steps, params)
    r_pl, w_pl = timed(hbpc.PC_NONE, 1)
    # every result against the BJ_ext run (the same Newton tolerance fixes the answer)
    for r, w in ((r_ln, w_ln), (r_pl, w_pl)):
        if r["ok"] is True:
            ref = w_bj if r is r_ln else None
            if ref is not None:
                r["rel_l2_vs_bjext"] = float(np.linalg.norm(w - ref) / np.linalg.norm(ref))
    head = r_ln if r_ln["ok"] is True else r_bj
    line = {"metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64 state/Newton, f32 Krylov, bf16 network",
            "data": "synthetic",
            "config": {"workload": "2d_euler_isentropic_vortex_128x128_N4_HBPC(6,2)_CFL10_Rusanov",
                       "value_is": "learned preconditioner" if r_ln["ok"] is True else
                                   "BJ_ext (the learned preconditioner did not converge)",
                       "dt": dt, "eps_newton": VORTEX["tol_newton_rel"], "eps_gmres": VORTEX["tol_gmres_rel"],
                       "gmres_restart": VORTEX["gmres_restart"], "gmres_max_iter": VORTEX["gmres_max_iter"],
                       "newton_max_iter": VORTEX["newton_max_iter"], "precision": "mixed",
                       "training": {"data_steps": max(1, args.warmup), "data_s": round(t_data, 2),
                                    "samples_per_newton": VORTEX["collect_per_newton"],
                                    "inverse_regression": {"iters": VORTEX["train_inverse_its"],
                                                           "loss_first": l0, "loss_last": l1},
                                    "probe": {"rounds": [list(r) for r in VORTEX["train_probe"]],
                                              "probes": VORTEX["train_probes"],
                                              "loss_first_last": probe_losses},
                                    "train_s": round(t_train, 2)}},
            "gpu_launches": head["launches"], "learned": r_ln, "bjext": r_bj, "plain_gmres": r_pl}
    if emit:
        print(json.dumps(line), flush=True)
    return line


TGV = dict(n=32, N=5, q=4, kmax=0, cfl=20.0, eps=0.1, re=1600.0, prandtl=0.72, tol_newton_rel=1e-10,
           tol_newton_abs=1e-10, tol_gmres_rel=1e-3, gmres_restart=100, gmres_max_iter=5000, newton_max_iter=30,
           check_n=8)


def tgv_dt(n):
    """CFL / sum_m(lambda_max,m (N+1) / h_m) with lambda_max = |v|_max + c of the
    initial state (|v| <= 1, c = 1/eps with p ~ 1/gamma)."""
    h = 2.0 * np.pi / n
    lam = 1.0 + 1.0 / TGV["eps"]
    return TGV["cfl"] / (3 * lam * (TGV["N"] + 1) / h)


def run_tgv(args, emit=True):
    """3-D Navier-Stokes Taylor-Green vortex (Mach 0.1 through the reference
    Mach number eps, Re 1600, Pr 0.72) on [0, 2 pi]^3, 32^3 elements, N = 5,
    Rusanov, HBPC(4, 0), CFL 20, in the mixed mode with plain GMRES: BJ_ext
    blocks of n_b = 5 * 6^3 = 1080 do not fit (2 x 32768 x 1080^2 values), and
    a compact learned preconditioner for them is not built.  Newton stops at
    ||G|| <= 1e-10 ||G0|| or ||dW|| <= 1e-10 (the FP64 residual of 70.8 M values
    has a rounding floor near 5e-9).  The FP64-vs-mixed difference of the answer
    is measured on an 8^3 mesh at the same CFL (one step each)."""
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__ as g
    g.build()
    from paper_2109_04804_gb300 import hbpc, inputs
    L = 2.0 * np.pi

    def ctx(n, prec):
        return hbpc.Context(3, (n, n, n), (0, 0, 0), (L, L, L), TGV["N"], law=hbpc.LAW_NAVIER_STOKES,
                            flux=hbpc.FLUX_RUSANOV, mu=1.0 / TGV["re"], eps=TGV["eps"], prandtl=TGV["prandtl"],
                            q=TGV["q"], kmax=TGV["kmax"], dt=tgv_dt(n), tol_newton_rel=TGV["tol_newton_rel"],
                            tol_newton_abs=TGV["tol_newton_abs"], tol_gmres_rel=TGV["tol_gmres_rel"],
                            gmres_restart=TGV["gmres_restart"], gmres_max_iter=TGV["gmres_max_iter"],
                            newton_max_iter=TGV["newton_max_iter"], pc=hbpc.PC_NONE, precision=prec)

    def stepped(c, w0, steps):
        c.set_state(w0)
        ms = 0.0
        for _ in range(steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            c.step(1)
            e1.record()
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
        return ms

    n = args.tgv_n if args.tgv_n > 0 else TGV["n"]
    c = ctx(n, hbpc.PREC_MIXED)
    w0 = inputs.taylor_green(c.node_coords(), eps=TGV["eps"])
    ndof = c.ndof
    # R1 evaluations per second (FP64 operator, full mesh, inputs resident)
    wd = torch.from_numpy(w0).cuda()
    o = torch.empty_like(wd)
    for _ in range(3):
        c.eval_R1(wd, o)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(10):
        c.eval_R1(wd, o)
    e1.record()
    torch.cuda.synchronize()
    r1_ms = e0.elapsed_time(e1) / 10
    del wd, o
    warm = max(1, min(args.warmup, 1))
    steps = max(1, min(args.steps, 2))
    stepped(c, w0, warm)
    st0 = c.stats()
    ms = stepped(c, c.get_state(), steps)
    st = c.stats()
    c.close()
    # FP64 vs mixed on the reduced mesh, same CFL, one step each
    chk = {}
    for prec, name in (((hbpc.PREC_FP64, "fp64"), (hbpc.PREC_MIXED, "mixed")) if not args.no_check else ()):
        cc = ctx(TGV["check_n"], prec)
        w = inputs.taylor_green(cc.node_coords(), eps=TGV["eps"])
        t = stepped(cc, w, 1)
        chk[name] = (cc.get_state(), t, cc.stats())
        cc.close()
    check = None
    if chk:
        wf, wm = chk["fp64"][0], chk["mixed"][0]
        check = {"rel_l2": float(np.linalg.norm(wm - wf) / np.linalg.norm(wf)), "fp64_ms": chk["fp64"][1],
                 "mixed_ms": chk["mixed"][1], "fp64_gmres_its": int(chk["fp64"][2]["gmres_its"]),
                 "mixed_gmres_its": int(chk["mixed"][2]["gmres_its"])}
    line = {"metric": METRIC, "value": ndof * steps / (ms / 1000.0), "unit": UNIT, "n_gpus": 1, "steps": steps,
            "warmup": warm, "ms_per_step": ms / steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64 state/Newton, f32 Krylov and Jacobian-vector products",
            "data": "synthetic",
            "config": {"workload": "3d_navier_stokes_taylor_green_%dx%dx%d_N5_HBPC(4,0)_CFL20_Rusanov_Re1600_Ma0.1"
                                   % (n, n, n),
                       "dt": tgv_dt(n), "eps_newton": TGV["tol_newton_rel"], "eps_newton_abs": TGV["tol_newton_abs"],
                       "eps_gmres": TGV["tol_gmres_rel"], "gmres_restart": TGV["gmres_restart"],
                       "precision": "mixed", "preconditioner": "none (plain GMRES)",
                       "l2_flush": "inputs larger than L2 (a Krylov vector is 283 MB)"},
            "gpu_launches": int(st["launches"] - st0["launches"]),
            "gmres_its_per_step": (st["gmres_its"] - st0["gmres_its"]) / steps,
            "newton_its_per_step": (st["newton_its"] - st0["newton_its"]) / steps,
            "r1_fp64_ms": r1_ms, "r1_evals_per_s_fp64": 1000.0 / r1_ms,
            "fp64_vs_mixed_8cubed": check}
    if emit:
        print(json.dumps(line), flush=True)
    return line


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    dt = workload_dt()
    vals = []
    sample = None
    t_all = time.perf_counter()
    for _ in range(max(1, args.warmup) + max(1, args.steps)):
        cb = cpu_baseline(dt)
        vals.append(cb["value"])
        sample = cb
        if time.perf_counter() - t_all > 240:
            break
    timed = vals[-max(1, args.steps):]
    value = float(np.mean(timed))
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * 147456 / value, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(dt), "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": sample["cores"], "kind": "oracle",
                             "sample": sample["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-vortex", action="store_true",
                    help="skip the learned-vs-plain-GMRES comparison on the Euler vortex in the default line")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"],
                    help="mixed: FP32 Krylov loop, FP64 Newton residual/update; fp64: all FP64")
    ap.add_argument("--workload", default="advection2d",
                    choices=["advection2d", "burgers_batch", "euler_vortex", "taylor_green"],
                    help="advection2d: the default 64x64 N=5 HBPC(8,4) line; burgers_batch: the batched "
                         "viscous Burgers instances; euler_vortex: learned vs BJ_ext vs plain GMRES; "
                         "taylor_green: the 3-D Navier-Stokes line")
    ap.add_argument("--instances", type=int, default=BATCH["n_inst"])
    ap.add_argument("--tgv-n", type=int, default=0,
                    help="taylor_green: elements per direction (default 32; smaller for profiling)")
    ap.add_argument("--no-check", action="store_true",
                    help="taylor_green: skip the FP64-vs-mixed comparison on the 8^3 mesh")
    ap.add_argument("--max-per-group", type=int, default=BATCH["max_per_group"],
                    help="instances sharing one context and one GMRES (<= 0: all of one N)")
    args = ap.parse_args()
    PRECISION[0] = args.precision
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "burgers_batch":
        run_batch(args)
    elif args.workload == "euler_vortex":
        run_vortex(args)
    elif args.workload == "taylor_green":
        run_tgv(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
