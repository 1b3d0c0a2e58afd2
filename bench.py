"""Benchmark of the HBPC-DGSEM hot path on one GB300.

Workload (default): 2-D linear advection u_t + div((1, 1) u) = 0 on the periodic
unit square, 64 x 64 elements, N = 5 (Gauss-Lobatto), u0 = sin(2 pi x) sin(2 pi y),
HBPC(8, 4) (the highest order of the paper), CFL 8 -> dt = 1/96, FP64, matrix-free
Newton-GMRES with the paper's BJ_ext preconditioner, eps_Newton = 1e-12 with the
absolute test ||dW|| <= 1e-12, eps_GMRES = 1e-5.  One bench step = one HBPC time
step (15 implicit stage solves).  Metric: DOF-timesteps/s = n_dof x steps /
device seconds, with every result's distance to the FP64 oracle.

The same line carries (N = 1):
  mixed_precision   the same workload with the FP32 Krylov loop (FP64 Newton
                    residual, update and state), its error against the oracle
  r1_roofline       the operator pass on the Euler vortex (128^2, N = 4) and
                    Taylor-Green (32^3, N = 5) meshes: FP64 R1 against the FP64
                    ALU and HBM roofs, the FP32 Jacobian-vector pass against HBM
  learned_vs_plain  the metric's comparison on the Euler vortex: learned block
                    preconditioner (trained on the GPU from the run's own
                    Newton-GMRES data) vs plain GMRES vs BJ_ext, every arm's
                    answer against the FP64 GPU result and the FP64 oracle
  cpu_baseline      the FP64 oracle on the host cores: whole HBPC(8,4) steps on
                    a 16 x 16 mesh at the same CFL, 1 BLAS thread and all

  python bench.py [--steps K] [--warmup W] [--gpus N] [--impl reference] [--precision fp64|mixed]
  python bench.py --workload burgers_batch   (256 viscous Burgers instances)
  python bench.py --workload euler_vortex    (learned vs BJ_ext vs plain GMRES)
  python bench.py --workload taylor_green    (3-D Navier-Stokes, 32^3, N = 5)
  python bench.py --workload euler_pc        (no PC vs BJ_ext vs BJ^H_ext, Euler, eps sweep)

Under torchrun (N > 1) every rank runs an independent replica of the workload
(the path has no data-path collective), value = sum over ranks / max time.
The reference arm (--impl reference) times the FP64 CPU oracle on the host:
whole HBPC(8,4) steps of the same configuration on a 16 x 16 mesh.
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DOF-timesteps/s per HBPC step at fixed L2 error; learned vs plain GMRES"
UNIT = "DOF-timesteps/s"

WL = dict(dim=2, n=(64, 64), lo=(0.0, 0.0), hi=(1.0, 1.0), N=5, a=(1.0, 1.0), q=8, kmax=4,
          cfl=8.0, t_end=1.0, tol_newton_rel=1e-12, tol_newton_abs=1e-12, tol_gmres_rel=1e-5,
          gmres_restart=100, gmres_max_iter=7000, newton_max_iter=50)
SAMPLE_N = (16, 16)     # the oracle's sample: same CFL, whole HBPC steps


def workload_dt(n=None):
    """dt_raw = CFL / sum_m(|a_m| p / h_m), rounded to T_end / ceil(T_end / dt_raw)."""
    n = n or WL["n"]
    p = WL["N"] + 1
    s = sum(abs(WL["a"][m]) * p / ((WL["hi"][m] - WL["lo"][m]) / n[m]) for m in range(WL["dim"]))
    raw = WL["cfl"] / s
    return WL["t_end"] / np.ceil(WL["t_end"] / raw - 1e-12)


def config_dict(dt, precision):
    return {"workload": "2d_linear_advection_64x64_N5_HBPC(8,4)_CFL8_BJext_GMRES_%s" % precision,
            "precision": precision,
            "mesh": "64x64 periodic [0,1]^2", "N": 5, "nodes": "Gauss-Lobatto", "hbpc": "q=8,kmax=4",
            "dt": dt, "eps_newton": WL["tol_newton_rel"], "newton_abs_dW": WL["tol_newton_abs"],
            "eps_gmres": WL["tol_gmres_rel"], "gmres_restart": WL["gmres_restart"],
            "preconditioner": "BJ_ext (Sec. 3.2.3)",
            "l2_between_steps": "flushed (256 MB write) between timed steps"}


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


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def rel_l2(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


# -- algorithmic work per launch (bytes, flops per W-DOF) ----------------------
def jv_work_per_dof(mixed):
    """Linear Jv (Eq. 24): reads dW, dS and writes the two outputs: 32 B per
    W-DOF in FP64 (16 B in FP32).  Flops: two R1 passes, each 2*d*p (volume)
    + 2*d/p face points x 7 (flux 5, lifting 2), plus 3 FMAs to combine."""
    d, p = WL["dim"], WL["N"] + 1
    r1 = 2 * d * p + (2 * d / p) * 7
    return (16.0 if mixed else 32.0), 2 * r1 + 6


def pc_work_per_dof(mixed):
    """BJ_ext apply on this workload: linear advection on one uniform mesh has
    the same J_i (hence M_i) in every element, so the library builds one block
    pair and the apply reads only the two input halves and writes the two
    output halves: 32 B per W-DOF in FP64, 16 B in FP32 (the block values once
    per launch are negligible).  Flops: M_i w and M_i sigma, dense n_b x n_b
    (4 n_b per W-DOF), and J_i u, J_i v with J_i the Kronecker sum of its d
    one-dimensional p x p factors (4 d p per W-DOF), plus 4."""
    nb = (WL["N"] + 1) ** WL["dim"]
    return (16.0 if mixed else 32.0), 4.0 * nb + 4.0 * WL["dim"] * (WL["N"] + 1) + 4.0


def pc_tc_work_per_dof():
    """The tensor-core form of the same apply: per W-DOF the inputs and outputs
    of both halves (32 B), and the 43 digit-plane pair products of the
    2 n_b x 2 n_b block (levels 0..8 of eight balanced base-256 digits per
    operand): 43 * 2 * (2 n_b) * 2 flops per W-DOF on the BF16 tensor pipe."""
    nb = (WL["N"] + 1) ** WL["dim"]
    return 32.0, 43.0 * 2.0 * (2.0 * nb) * 2.0


def cgs_work_per_dof(mixed, cavg):
    """CGS2 column (one launch per Arnoldi iteration) at the mean column count
    cavg = j + 1: the three passes read the new vector and the j + 1 basis
    vectors and write the new vector twice, (3 cavg + 5) vectors of 2 values
    per W-DOF; 6 cavg + 8 flops per value."""
    vb = 4.0 if mixed else 8.0
    return (3.0 * cavg + 5.0) * 2.0 * vb, (6.0 * cavg + 8.0) * 2.0


# DRAM bytes (read + write) per launch measured by ncu for the kernels of this
# workload with caches as the run leaves them (--cache-control none; mean of
# ten launches inside the timed step; summaries in profiles/, one per kernel
# and precision).  An entry is None until its kernel, as committed, has been
# captured.
NCU_TRAFFIC = {
    "mixed": {"cgs2": None, "pc_apply": None, "jv": None},
    "fp64": {"cgs2": 1.411e5, "pc_apply": 8.581e4, "jv": 1.441e5},
}

KERNEL_NAMES = {
    "jv": "dg_operator_kernel<advection pair,2D,P=6,JobJvLinearPair<%s>> (Eq. 24, both halves in one pass)",
    "pc_apply_tc": ("k_pc_apply_tc (BJ_ext, Sec. 3.2.3: the shared FP64 block pair as one 2 n_b x 2 n_b product on "
                    "tcgen05, exact BF16 digit-plane products summed in FP32 tensor memory, integer recombination)"),
    "pc_apply": "k_pc_apply_shared<%s, 2> (BJ_ext, Sec. 3.2.3; one block pair for all elements, J as Kronecker factors)",
    "cgs2": "k_cgs_lowsync<%s> (Arnoldi CGS2 column, one cooperative launch, two grid barriers; mean j + 1 = %.1f)",
}


def c2_context(hbpc, n, precision, stream):
    dt = workload_dt(n)
    return hbpc.Context(WL["dim"], n, WL["lo"], WL["hi"], WL["N"], law=hbpc.LAW_ADVECTION,
                        a=WL["a"], q=WL["q"], kmax=WL["kmax"], dt=dt,
                        tol_newton_rel=WL["tol_newton_rel"], tol_newton_abs=WL["tol_newton_abs"],
                        tol_gmres_rel=WL["tol_gmres_rel"], gmres_restart=WL["gmres_restart"],
                        gmres_max_iter=WL["gmres_max_iter"], newton_max_iter=WL["newton_max_iter"],
                        pc=hbpc.PC_BJEXT, stream=stream.cuda_stream if stream is not None else None,
                        precision=hbpc.PREC_MIXED if precision == "mixed" else hbpc.PREC_FP64, t_end=WL["t_end"])


def timed_steps(torch, ctx, stream, steps, flush):
    """`steps` HBPC steps, each timed with CUDA events on the context's stream
    after an L2 flush outside the timed window; returns the summed ms."""
    total = 0.0
    for _ in range(steps):
        with torch.cuda.stream(stream):
            flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.step(1)
        e1.record(stream)
        e1.synchronize()
        total += e0.elapsed_time(e1)
    return total


def c2_roofline(hbpc, ctx, precision, stats0, fp64_peak_gf, hbm):
    """One more step with per-launch CUDA events (a separate, profiled step):
    per phase device time; the roofline entry of every measured kernel and of
    the dominant one."""
    ctx.profile(True)
    ctx.step(1)
    prof = ctx.profile_get()
    pstats = ctx.stats()
    ctx.profile(False)
    mixed = precision == "mixed"
    ndof = ctx.ndof
    its_p = pstats["gmres_its"] - stats0["gmres_its"]
    cols_p = pstats["arnoldi_cols"] - stats0["arnoldi_cols"]
    cavg = cols_p / max(1, its_p)
    tname = "float" if mixed else "double"
    pc_tc = (not mixed) and bool(pstats.get("pc_apply_tc"))
    kernels = {"jv": (KERNEL_NAMES["jv"] % tname, jv_work_per_dof(mixed), prof["jv"]),
               "pc_apply": ((KERNEL_NAMES["pc_apply_tc"], pc_tc_work_per_dof(), prof["pc_apply"]) if pc_tc else
                            (KERNEL_NAMES["pc_apply"] % tname, pc_work_per_dof(mixed), prof["pc_apply"])),
               "cgs2": (KERNEL_NAMES["cgs2"] % (tname, cavg), cgs_work_per_dof(mixed, cavg),
                        (prof["arnoldi_dot"][0] + prof["arnoldi_update"][0], its_p))}
    step_ms = sum(v[0] for v in prof.values())
    entries = {}
    for ph, (name, (bpd, fpd), (ms, n)) in kernels.items():
        if n == 0:
            continue
        avg = ms / 1000.0 / n
        gf = fpd * ndof / avg / 1e9
        gb = bpd * ndof / avg / 1e9
        e = {"kernel": name, "algorithmic_bytes_per_launch": round(bpd * ndof),
             "algorithmic_flops_per_launch": round(fpd * ndof),
             "traffic": NCU_TRAFFIC[precision].get(ph), "avg_launch_us": round(avg * 1e6, 2),
             "launches_profiled": n, "share_of_step": round(ms / step_ms, 3)}
        if ph == "pc_apply" and pc_tc:   # BF16 tensor pipe; the FP64-equivalent rate beside it
            bf16 = peaks().get("bf16_tflops", 1900.0)
            f64e = pc_work_per_dof(False)[1] * ndof / avg / 1e12
            e.update({"bound": "tensor", "achieved": round(gf / 1000.0, 2), "peak": bf16, "unit": "TFLOP/s",
                      "frac": round(gf / 1000.0 / bf16, 4), "hbm_achieved_gbs": round(gb, 1),
                      "fp64_equivalent_tflops": round(f64e, 4),
                      "fp64_equivalent_frac_of_fp64_peak": round(f64e * 1000.0 / fp64_peak_gf, 4)})
        elif mixed:   # FP32 arithmetic is 62x the FP64 rate: these kernels are bound by memory
            e.update({"bound": "hbm", "achieved": round(gb, 1), "peak": hbm, "unit": "GB/s",
                      "frac": round(gb / hbm, 4), "alu_tflops": round(gf / 1000.0, 3)})
        else:       # GB300's FP64 pipe (1/64 of FP32) binds these
            e.update({"bound": "alu", "achieved": round(gf / 1000.0, 4), "peak": round(fp64_peak_gf / 1000.0, 4),
                      "unit": "TFLOP/s", "frac": round(gf / fp64_peak_gf, 4), "hbm_achieved_gbs": round(gb, 1),
                      "hbm_frac_of_measured": round(gb / hbm, 4)})
        entries[ph] = e
    dom = max(entries, key=lambda k: kernels[k][2][0])
    roof = dict(entries[dom])
    roof["peak_source"] = ("measured HBM copy bandwidth (MEASURED_PEAKS.json)" if mixed else
                           "FP64 FMA throughput measured in this run (hbpc_fp64_fma_peak), "
                           "nominal 1.25 TFLOP/s")
    roof["phase_ms_one_step"] = {k: round(v[0], 3) for k, v in prof.items()}
    roof["phase_launches_one_step"] = {k: v[1] for k, v in prof.items()}
    roof["other_kernels"] = {k: v for k, v in entries.items() if k != dom}
    return roof


def run_c2_arm(torch, hbpc, inputs, precision, args, stream, flush, fp64_peak_gf, hbm, world, headline):
    """W warm-up steps, the launch-shape autotuner, K timed steps (CUDA events
    on the context's stream, L2 flushed between steps), one profiled step for
    the roofline; on the headline arm also the clocks during the timed region
    and the end-to-end run through host buffers."""
    dt = workload_dt()
    ctx = c2_context(hbpc, WL["n"], precision, stream)
    # corrector batching pays in the mixed mode (per-stage GMRES, latency-bound
    # kernels); the FP64 mode shares one GMRES between the stages and its
    # kernels are FP64-ALU bound, so it stays sequential unless asked
    cbatch = (precision == "mixed") if args.corrector_batch < 0 else bool(args.corrector_batch)
    if cbatch:
        ctx.set_corrector_batch(True)
    coords = ctx.node_coords()
    w0 = inputs.sine_product(coords)
    ctx.set_state(w0)
    ndof = ctx.ndof
    for _ in range(args.warmup):
        ctx.step(1)
    tuning = ctx.autotune()        # launch shapes of the Krylov reductions and the PC apply
    torch.cuda.synchronize()
    ctx.reset_stats()
    clocks = Clocks(dist_env()[2]) if headline else None
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    if clocks:
        clocks.start()
    total_ms = timed_steps(torch, ctx, stream, args.steps, flush)
    torch.cuda.synchronize()
    clk = clocks.stop() if clocks else None
    stats = ctx.stats()
    t_sec = total_ms / 1000.0
    if world > 1:
        tt = torch.tensor([t_sec], device="cuda")
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        t_sec = float(tt.item())
        torch.distributed.barrier()
    roof = c2_roofline(hbpc, ctx, precision, stats, fp64_peak_gf, hbm)
    n_steps = args.warmup + args.steps + 1
    w_fin = ctx.get_state()
    err = float(np.sqrt(np.mean((w_fin - exact_solution(coords, n_steps * dt)) ** 2)))
    res = {"value": ndof * args.steps * world / t_sec, "ms_per_step": 1000.0 * t_sec / args.steps,
           "steps_total": n_steps, "gmres_its_per_step": stats["gmres_its"] / args.steps,
           "newton_its_per_step": stats["newton_its"] / args.steps,
           "r1_evals_per_s": (stats["r1_evals"] + stats["r2_evals"]) / t_sec,
           "gpu_launches": int(stats["launches"]), "l2_error_vs_exact": err, "roofline": roof,
           "autotuned": tuning, "clocks": clk, "ndof": ndof, "w_final": w_fin,
           "corrector_batch": cbatch}
    if headline:
        # e2e: the public API with pinned host buffers, copies inside the timed
        # region, the L2 flush outside it (as in the device-timed loop)
        # the trajectory continues from the state reached: every step copies
        # the last step's host result in and its own result out
        host_in = torch.from_numpy(w_fin.copy()).pin_memory()
        host_out = torch.empty_like(host_in).pin_memory()
        e2e_s = 0.0
        for _ in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(1.0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx.set_state_host_ptr(host_in.data_ptr())
            ctx.step(1)
            ctx.get_state_host_ptr(host_out.data_ptr())
            e2e_s += time.perf_counter() - t0
            host_in, host_out = host_out, host_in
        res["e2e"] = {"value": ndof * args.steps * world / e2e_s, "unit": UNIT,
                      "h2d_bytes_per_step": ndof * 8, "d2h_bytes_per_step": ndof * 8}
    ctx.close()
    return res


def c2_sample_steps(torch, hbpc, inputs):
    """One HBPC(8,4) step of the oracle's sample (16 x 16 elements, same CFL)
    from u0 in both precisions, for the comparison with the oracle's step."""
    out = {}
    for prec in ("fp64", "mixed"):
        c = c2_context(hbpc, SAMPLE_N, prec, None)
        c.set_state(inputs.sine_product(c.node_coords()))
        c.step(1)
        out[prec] = c.get_state()
        c.close()
    return out


def r1_roofline(torch, hbpc, inputs, flush, fp64_peak_gf, hbm, launches=8):
    """The operator pass at the two large meshes: FP64 R1 (hbpc_eval_R1;
    16 B per W-DOF, FP64-ALU bound on GB300) and the FP32 Jacobian-vector pass
    of the mixed Krylov loop (hbpc_eval_Jv of a mixed context: reads the FP32
    state and direction, writes the product: 24 B per W-DOF).  Every launch
    after an L2 flush, CUDA events (R1) or the library's per-launch events (Jv).
    Flops counted for the ALU fraction: the tensor-product contractions alone,
    2 d p per W-DOF for the flux divergence and, for Navier-Stokes, 2 p d (d+1)
    per node for the gradients of (v, T): a lower bound of the work, so the
    fraction is a lower bound too."""
    L = 2.0 * np.pi
    cases = [("euler_vortex_128x128_N4", dict(dim=2, n=(128, 128), lo=(-10, -10), hi=(10, 10), N=4,
                                              law=hbpc.LAW_EULER, flux=hbpc.FLUX_RUSANOV), "vortex"),
             ("taylor_green_32x32x32_N5", dict(dim=3, n=(32, 32, 32), lo=(0, 0, 0), hi=(L, L, L), N=5,
                                               law=hbpc.LAW_NAVIER_STOKES, flux=hbpc.FLUX_RUSANOV,
                                               mu=1.0 / 1600.0, eps=0.1, prandtl=0.72), "tgv")]
    out = {}
    for name, kw, ic in cases:
        d, p = kw["dim"], kw["N"] + 1
        nv = d + 2
        flops = 2.0 * d * p + (2.0 * p * d * (d + 1) / nv if kw["law"] == hbpc.LAW_NAVIER_STOKES else 0.0)
        entry = {}
        for prec in ("fp64", "mixed"):
            ctx = hbpc.Context(kw["dim"], kw["n"], kw["lo"], kw["hi"], kw["N"], law=kw["law"], flux=kw["flux"],
                               mu=kw.get("mu"), eps=kw.get("eps", 1.0), prandtl=kw.get("prandtl", 0.72),
                               dt=0.01, gmres_restart=2, pc=hbpc.PC_NONE,
                               precision=hbpc.PREC_FP64 if prec == "fp64" else hbpc.PREC_MIXED)
            co = ctx.node_coords()
            w = inputs.isentropic_vortex(co) if ic == "vortex" else inputs.taylor_green(co, eps=0.1)
            wd = torch.from_numpy(w).cuda()
            o = torch.empty_like(wd)
            ndof = ctx.ndof
            if prec == "fp64":
                for _ in range(2):
                    ctx.eval_R1(wd, o)
                ms = []
                for _ in range(launches):
                    flush.fill_(1.0)
                    torch.cuda.synchronize()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    ctx.eval_R1(wd, o)
                    e1.record()
                    e1.synchronize()
                    ms.append(e0.elapsed_time(e1))
                avg = float(np.mean(ms)) / 1000.0
                gf = flops * ndof / avg / 1e9
                gb = 16.0 * ndof / avg / 1e9
                entry["fp64_r1"] = {"kernel": "dg_operator_kernel<JobR1<double>>", "bound": "alu",
                                    "avg_launch_us": round(avg * 1e6, 1), "launches": launches, "ndof": ndof,
                                    "r1_evals_per_s": round(1.0 / avg, 1),
                                    "alu_tflops_contractions_only": round(gf / 1000.0, 4),
                                    "alu_frac_lower_bound": round(gf / fp64_peak_gf, 4),
                                    "fp64_peak_tflops": round(fp64_peak_gf / 1000.0, 4),
                                    "hbm_achieved_gbs": round(gb, 1), "hbm_frac": round(gb / hbm, 4),
                                    "algorithmic_bytes_per_launch": 16 * ndof,
                                    "flops_counted_per_dof": round(flops, 2)}
            else:
                ctx.eval_R1(wd, o)
                X = torch.cat([wd, o])
                gen = torch.Generator(device="cuda")
                gen.manual_seed(5)
                dX = torch.randn(2 * ndof, dtype=torch.float64, device="cuda", generator=gen)
                out2 = torch.empty_like(X)
                ctx.eval_Jv(0.5, 1.0 / 6.0, X, dX, out2)
                ctx.profile(True)
                for _ in range(launches):
                    flush.fill_(1.0)
                    torch.cuda.synchronize()
                    ctx.eval_Jv(0.5, 1.0 / 6.0, X, dX, out2)
                ms, n = ctx.profile_get()["jv"]
                ctx.profile(False)
                avg = ms / 1000.0 / max(1, n)
                gb = 24.0 * ndof / avg / 1e9
                entry["fp32_jv_mixed"] = {"kernel": "dg_operator_kernel<JobJvMixed<float>> (dual numbers)",
                                          "bound": "hbm", "avg_launch_us": round(avg * 1e6, 1), "launches": n,
                                          "ndof": ndof, "achieved": round(gb, 1), "peak": hbm, "unit": "GB/s",
                                          "frac": round(gb / hbm, 4),
                                          "algorithmic_bytes_per_launch": 24 * ndof}
                del X, dX, out2
            del wd, o
            ctx.close()
            torch.cuda.empty_cache()
        out[name] = entry
    return out


# -- the oracle on the host cores (cpu_baseline leg and reference arm) ---------
def host_cpu():
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.split(":")[0].strip() in ("Model name", "Model"):
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.TimeoutExpired):
        pass
    return {"nproc": os.cpu_count(), "cpu_model": model}


ONE_THREAD = {"OMP_NUM_THREADS": "1", "OPENBLAS_NUM_THREADS": "1", "MKL_NUM_THREADS": "1"}


def oracle_task(name, outdir, steps):
    """Run in a child process (bench.py --oracle-task): the FP64 oracle as it
    stands.  c2_sample: whole HBPC(8,4) steps of the 2-D advection workload on
    the 16 x 16 sample at CFL 8, timed; c2_exact: the exact per-Fourier-mode
    HBPC(8,4) result at full size after `steps` steps (what the Newton-GMRES
    iteration converges to); vortex_sample: one HBPC(6,2) step of the Euler
    vortex on a 16 x 16 mesh at CFL 10.  Prints one JSON line; states go to
    outdir/<name>.npy."""
    from oracle import dgsem, exact, hbpc as ohbpc, laws, newton
    from paper_2109_04804_gb300 import inputs
    res = {"task": name}
    if name in ("c2_sample", "c2_exact"):
        ph = laws.Physics(laws.ADVECTION, 2, a=WL["a"])
        n = SAMPLE_N if name == "c2_sample" else WL["n"]
        disc = dgsem.Disc(dgsem.Mesh(2, n, WL["lo"], WL["hi"]), WL["N"], ph)
        w = inputs.sine_product(disc.node_coords())
        dt = workload_dt(n)
        if name == "c2_exact":
            w = exact.fourier_hbpc(disc, w, dt, WL["q"], WL["kmax"], steps)
        else:
            opts = newton.NewtonOptions(tol_rel=WL["tol_newton_rel"], tol_abs=WL["tol_newton_abs"],
                                        gmres_tol=WL["tol_gmres_rel"], restart=WL["gmres_restart"],
                                        gmres_maxiter=WL["gmres_max_iter"], newton_max=WL["newton_max_iter"],
                                        jv="linear", pc="bjext")
            st = newton.Stats()
            adv = ohbpc.dg_stepper(disc, dt, WL["q"], WL["kmax"], opts, stats=st)
            times = []
            for _ in range(steps):
                t0 = time.perf_counter()
                w = adv(w)
                times.append(time.perf_counter() - t0)
            res.update({"seconds": times, "ndof": disc.ndof, "gmres_its": st.gmres_its,
                        "newton_its": st.newton_its})
        res["ndof"] = disc.ndof
    elif name == "vortex_sample":
        ph = laws.Physics(laws.EULER, 2, flux="rusanov")
        n = (16, 16)
        disc = dgsem.Disc(dgsem.Mesh(2, n, VORTEX["lo"], VORTEX["hi"]), VORTEX["N"], ph)
        opts = newton.NewtonOptions(tol_rel=VORTEX["tol_newton_rel"], tol_abs=VORTEX["tol_newton_abs"],
                                    gmres_tol=VORTEX["tol_gmres_rel"], restart=VORTEX["gmres_restart"],
                                    gmres_maxiter=VORTEX["gmres_max_iter"], newton_max=VORTEX["newton_max_iter"],
                                    jv="fd", pc="bjext")
        t0 = time.perf_counter()
        w = ohbpc.dg_stepper(disc, vortex_dt(n), VORTEX["q"], VORTEX["kmax"], opts)(
            inputs.isentropic_vortex(disc.node_coords()))
        res.update({"seconds": [time.perf_counter() - t0], "ndof": disc.ndof})
    else:
        raise ValueError(name)
    np.save(os.path.join(outdir, name + ".npy"), w)
    print(json.dumps(res), flush=True)


class OracleRun:
    """A child process running one oracle task (subprocess: fork and exec, so
    it is independent of the parent's CUDA context)."""

    def __init__(self, name, outdir, steps=1, one_thread=True):
        env = dict(os.environ)
        if one_thread:
            env.update(ONE_THREAD)
        self.name, self.outdir = name, outdir
        self.proc = subprocess.Popen([sys.executable, os.path.abspath(__file__), "--oracle-task", name,
                                      "--oracle-out", outdir, "--oracle-steps", str(steps)],
                                     stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, env=env, cwd=ROOT)

    def result(self, timeout=1800):
        try:
            out, err = self.proc.communicate(timeout=timeout)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            return None, None
        if self.proc.returncode != 0:
            sys.stderr.write("oracle task %s failed:\n%s\n" % (self.name, err[-2000:]))
            return None, None
        info = json.loads(out.strip().splitlines()[-1])
        return info, np.load(os.path.join(self.outdir, self.name + ".npy"))


def cpu_baseline_timing(outdir):
    """The oracle's C2 sample (whole HBPC(8,4) steps on 16 x 16 elements, CFL 8)
    with BLAS pinned to one thread and with all host threads allowed, one after
    the other.  Returns (cpu_baseline dict, the one-thread run's state after
    one step)."""
    r1, w1 = OracleRun("c2_sample", outdir, steps=1, one_thread=True).result()
    alldir = os.path.join(outdir, "all")
    os.makedirs(alldir, exist_ok=True)
    ra, _ = OracleRun("c2_sample", alldir, steps=1, one_thread=False).result()
    if r1 is None:
        return None, None
    hc = host_cpu()
    ndof = r1["ndof"]
    base = {"value": ndof / r1["seconds"][0], "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": ("one whole HBPC(8,4) step (15 Newton-GMRES stage solves, %d GMRES iterations) of the "
                       "same workload on a 16x16-element mesh at the same CFL 8 (dt = 1/24, %d DOF), "
                       "numpy with BLAS pinned to 1 thread, %.1f s" % (r1["gmres_its"], ndof, r1["seconds"][0])),
            "host": hc}
    if ra is not None:
        base["all_threads"] = {"value": ndof / ra["seconds"][0], "unit": UNIT, "threads": hc["nproc"],
                               "seconds": ra["seconds"][0],
                               "note": "numpy's BLAS may use every host thread; the oracle's element "
                                       "loops are vectorised numpy, not threaded"}
    return base, w1


VORTEX = dict(n=(128, 128), lo=(-10.0, -10.0), hi=(10.0, 10.0), N=4, q=6, kmax=2, cfl=10.0,
              tol_newton_rel=1e-10, tol_newton_abs=1e-12, tol_gmres_rel=1e-3, gmres_restart=100,
              gmres_max_iter=3000, newton_max_iter=30, collect_per_newton=1024, collect_capacity=32768,
              train_inverse_its=20000, train_lr=1e-3, train_batch=256,
              train_probe=((8000, 1e-5), (8000, 1e-5), (8000, 5e-6), (8000, 2e-6)), train_probes=8,
              sample_n=(16, 16))


def vortex_dt(n=None):
    """CFL / sum_m(lambda_max,m (N+1) / h_m) with lambda_max = |v| + c of the
    free stream plus the vortex's peak velocity (about 0.5 c_inf)."""
    n = n or VORTEX["n"]
    g = 1.4
    lam = (0.5 * np.sqrt(g) + np.sqrt(g), np.sqrt(g))
    h = [(VORTEX["hi"][m] - VORTEX["lo"][m]) / n[m] for m in range(2)]
    return VORTEX["cfl"] / sum(lam[m] * (VORTEX["N"] + 1) / h[m] for m in range(2))


def run_vortex(args, emit=True, oracle_state=None):
    """2-D Euler isentropic vortex (strength 5, Mach 0.5) on [-10, 10]^2, 128 x 128
    elements, N = 4, Rusanov, HBPC(6, 2), CFL 10, Newton tol 1e-10.  The learned
    block preconditioner is trained on the GPU on (features, exact block
    inverse) samples of the method's own BJ_ext Newton iterations during the
    warm-up steps; then the same time step is taken with the learned
    preconditioner, with BJ_ext and with plain GMRES (no preconditioner), all in
    the mixed mode, and with BJ_ext in FP64.  Every answer is compared with the
    FP64 GPU result at full size and, on a 16 x 16 mesh of the same domain and
    CFL (same network), with the FP64 oracle's step (oracle_state: a callable
    returning it, or None)."""
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__ as g
    g.build()
    from paper_2109_04804_gb300 import hbpc, inputs

    def ctx(pc, n=VORTEX["n"], prec=hbpc.PREC_MIXED):
        return hbpc.Context(2, n, VORTEX["lo"], VORTEX["hi"], VORTEX["N"], law=hbpc.LAW_EULER,
                            flux=hbpc.FLUX_RUSANOV, q=VORTEX["q"], kmax=VORTEX["kmax"], dt=vortex_dt(n),
                            tol_newton_rel=VORTEX["tol_newton_rel"], tol_newton_abs=VORTEX["tol_newton_abs"],
                            tol_gmres_rel=VORTEX["tol_gmres_rel"], gmres_restart=VORTEX["gmres_restart"],
                            gmres_max_iter=VORTEX["gmres_max_iter"], newton_max_iter=VORTEX["newton_max_iter"],
                            pc=pc, precision=prec)
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

    def timed(pc, steps, params=None, prec=hbpc.PREC_MIXED, n=VORTEX["n"], w0=None):
        c = ctx(pc, n, prec)
        if params is not None:
            c.pc_model_set(params)
        c.set_state(w_start if w0 is None else w0)
        ok, ms, states = True, 0.0, []
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
            states.append(c.get_state())
        st = c.stats()
        nd = c.ndof
        c.close()
        return {"ok": ok, "ms_per_step": ms / steps, "value": nd * steps / (ms / 1000.0) if ok is True else 0.0,
                "gmres_its_per_step": st["gmres_its"] / steps, "newton_its_per_step": st["newton_its"] / steps,
                "launches": int(st["launches"]),
                "exact_blocks_per_build": (st["pc_exact_blocks"] / max(1, st["newton_its"])
                                           if pc == hbpc.PC_LEARNED else None)}, states

    r_bj, s_bj = timed(hbpc.PC_BJEXT, args.steps)
    r_ln, s_ln = timed(hbpc.PC_LEARNED, args.steps, params)
    r_pl, s_pl = timed(hbpc.PC_NONE, 1)
    r_64, s_64 = timed(hbpc.PC_BJEXT, args.steps, prec=hbpc.PREC_FP64)
    # every answer against the FP64 GPU result after the same number of steps
    for r, s in ((r_bj, s_bj), (r_ln, s_ln), (r_pl, s_pl)):
        if r["ok"] is True and r_64["ok"] is True:
            r["rel_l2_vs_fp64_gpu"] = rel_l2(s[-1], s_64[len(s) - 1])
    # the same arms on the 16 x 16 mesh, one step from the vortex, against the oracle
    small = {}
    w16 = None
    for name, pc, prec, prm in (("learned", hbpc.PC_LEARNED, hbpc.PREC_MIXED, params),
                                ("bjext", hbpc.PC_BJEXT, hbpc.PREC_MIXED, None),
                                ("plain_gmres", hbpc.PC_NONE, hbpc.PREC_MIXED, None),
                                ("fp64_bjext", hbpc.PC_BJEXT, hbpc.PREC_FP64, None)):
        c = ctx(pc, VORTEX["sample_n"], prec)
        w16 = inputs.isentropic_vortex(c.node_coords())
        c.close()
        r, s = timed(pc, 1, prm, prec, VORTEX["sample_n"], w16)
        small[name] = (r, s)
    ref16 = oracle_state() if oracle_state is not None else None
    for name, (r, s) in small.items():
        r["mesh"] = "16x16"
        if ref16 is not None and r["ok"] is True:
            r["rel_l2_vs_oracle"] = rel_l2(s[-1], ref16)
    for key, r in (("learned", r_ln), ("bjext", r_bj), ("plain_gmres", r_pl)):
        if "rel_l2_vs_oracle" in small[key][0]:
            r["rel_l2_vs_oracle_16x16"] = small[key][0]["rel_l2_vs_oracle"]
    head = r_ln if r_ln["ok"] is True else r_bj
    line = {"metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64 state/Newton, f32 Krylov, bf16 network",
            "data": "synthetic",
            "config": {"workload": "2d_euler_isentropic_vortex_128x128_N4_HBPC(6,2)_CFL10_Rusanov",
                       "value_is": "learned preconditioner" if r_ln["ok"] is True else
                                   "BJ_ext (the learned preconditioner did not converge)",
                       "dt": vortex_dt(), "eps_newton": VORTEX["tol_newton_rel"],
                       "eps_gmres": VORTEX["tol_gmres_rel"],
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
            "gpu_launches": head["launches"], "learned": r_ln, "bjext": r_bj, "plain_gmres": r_pl,
            "fp64_bjext": r_64,
            "accuracy_16x16": {k: {kk: v[0].get(kk) for kk in ("ok", "rel_l2_vs_oracle", "gmres_its_per_step",
                                                                 "exact_blocks_per_build")}
                               for k, v in small.items()},
            "oracle_16x16": "one HBPC(6,2) step of the FP64 oracle (Eq. 23 Jv, BJ_ext) on a 16x16 mesh of "
                            "the same domain at CFL 10" if ref16 is not None else None}
    if emit:
        print(json.dumps(line), flush=True)
    return line


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
    head = args.precision
    other = "mixed" if head == "fp64" else "fp64"
    extras = rank == 0 and world == 1
    dt = workload_dt()
    stream = torch.cuda.Stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    hbm = peaks().get("hbm_gbs", 6800.0)
    fp64_peak = hbpc.fp64_fma_peak()          # measured live on this GPU
    want_oracle = extras and not args.no_cpu_baseline and not args.headline_only
    tmp = tempfile.mkdtemp(prefix="hbpc_oracle_") if want_oracle else None

    res = run_c2_arm(torch, hbpc, inputs, head, args, stream, flush, fp64_peak, hbm, world, headline=True)
    line = {"metric": METRIC, "value": res["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": res["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if head == "fp64" else "f64 state/Newton, f32 Krylov", "data": "synthetic",
            "config": dict(config_dict(dt, head), parallelism="replicas" if world > 1 else "single"),
            "autotuned": res["autotuned"], "r1_evals_per_s": res["r1_evals_per_s"],
            "l2_error_vs_exact": res["l2_error_vs_exact"], "gmres_its_per_step": res["gmres_its_per_step"],
            "newton_its_per_step": res["newton_its_per_step"], "gpu_launches": res["gpu_launches"],
            "roofline": res["roofline"], "e2e": res["e2e"], "clocks": res["clocks"],
            "corrector_batch": res["corrector_batch"]}
    if not extras:
        if rank == 0:
            print(json.dumps(line), flush=True)
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return
    # oracle references that are not timed run beside the GPU work, on one host core each
    bg = {}
    if want_oracle:
        bg["c2_exact"] = OracleRun("c2_exact", tmp, steps=res["steps_total"])
        if not args.no_vortex:
            bg["vortex_sample"] = OracleRun("vortex_sample", tmp)
    if args.headline_only:
        print(json.dumps(line), flush=True)
        return
    sec = run_c2_arm(torch, hbpc, inputs, other, args, stream, flush, fp64_peak, hbm, world, headline=False)
    sample = c2_sample_steps(torch, hbpc, inputs)
    line["r1_roofline"] = None if args.no_r1_roofline else r1_roofline(torch, hbpc, inputs, flush, fp64_peak, hbm)
    if not args.no_vortex:
        def vortex_ref():
            if "vortex_sample" not in bg:
                return None
            info, w = bg["vortex_sample"].result()
            return w
        va = argparse.Namespace(steps=1, warmup=2)
        v = run_vortex(va, emit=False, oracle_state=vortex_ref)
        ln, pl, bj = v["learned"], v["plain_gmres"], v["bjext"]
        line["learned_vs_plain"] = {
            "workload": v["config"]["workload"], "unit": UNIT, "learned": ln, "plain_gmres": pl, "bjext": bj,
            "fp64_bjext": v["fp64_bjext"], "accuracy_16x16": v["accuracy_16x16"],
            "oracle_16x16": v["oracle_16x16"],
            "speedup_learned_over_plain": (ln["value"] / pl["value"]) if pl["value"] > 0 else None,
            "speedup_learned_over_bjext": (ln["value"] / bj["value"]) if bj["value"] > 0 else None,
            "training": v["config"]["training"]}
    if not args.no_batch:
        # the batched workload (256 viscous Burgers instances), one warm-up and
        # one timed step; --workload burgers_batch for the full line
        ba = argparse.Namespace(steps=1, warmup=1, instances=BATCH["n_inst"], max_per_group=BATCH["max_per_group"])
        bl = run_batch(ba, emit=False)
        line["batch"] = {k: bl[k] for k in ("value", "unit", "ms_per_step", "gmres_its_per_step",
                                            "newton_its_per_step", "gpu_launches", "e2e", "steps", "warmup")}
        line["batch"]["workload"] = bl["config"]["workload"]
        line["batch"]["total_dof"] = bl["config"]["total_dof"]
        line["batch"]["groups"] = bl["config"]["groups"]
    # the oracle: the timed CPU baseline, then the accuracy of both precisions
    acc = {"fp64" if head == "fp64" else "mixed": {"l2_error_vs_exact_solution": res["l2_error_vs_exact"]},
           other: {"l2_error_vs_exact_solution": sec["l2_error_vs_exact"]}}
    if want_oracle:
        info, w_ex = bg["c2_exact"].result()
        if w_ex is not None:
            acc[head]["rel_l2_vs_oracle_64x64"] = rel_l2(res["w_final"], w_ex)
            acc[other]["rel_l2_vs_oracle_64x64"] = rel_l2(sec["w_final"], w_ex)
            acc["oracle_64x64"] = ("exact per-Fourier-mode HBPC(8,4) result after %d steps (dense solves of "
                                   "every stage per mode: the root the Newton iterations converge to)"
                                   % res["steps_total"])
        cb, w16 = cpu_baseline_timing(tmp)
        if cb is not None:
            line["cpu_baseline"] = cb
            for prec in ("fp64", "mixed"):
                acc[prec]["rel_l2_vs_oracle_16x16_one_step"] = rel_l2(sample[prec], w16)
            acc["oracle_16x16"] = "one HBPC(8,4) step of the FP64 oracle (Newton-GMRES, BJ_ext) on 16x16, CFL 8"
    line["accuracy"] = acc
    sec.pop("w_final")
    line["mixed_precision" if head == "fp64" else "fp64_precision"] = {
        k: sec[k] for k in ("value", "ms_per_step", "gmres_its_per_step", "newton_its_per_step", "r1_evals_per_s",
                            "gpu_launches", "roofline", "autotuned", "corrector_batch")}
    line[("mixed_precision" if head == "fp64" else "fp64_precision")]["unit"] = UNIT
    line[("mixed_precision" if head == "fp64" else "fp64_precision")]["dtype"] = (
        "f64 state/Newton, f32 Krylov" if other == "mixed" else "f64")
    if not args.no_cavity:
        # the lid-driven cavity (Sec. 5.3.1): three timed steps of each arm after
        # its start-up; --workload cavity for the line alone.  A failure there is
        # recorded, not raised: the lines above stand on their own.
        try:
            ca = argparse.Namespace(steps=3, warmup=1, no_step_graph=args.no_step_graph)
            cl = run_cavity(ca, emit=False)
            line["cavity"] = {k: cl[k] for k in ("workload", "unit", "value", "best_arm", "steps", "ndof", "arms")}
        except Exception as e:   # noqa: BLE001
            line["cavity"] = {"workload": "lid_driven_cavity", "error": str(e)[:200]}
    print(json.dumps(line), flush=True)


def run_r1_only(args):
    """The default line's r1_roofline object alone (for profiling)."""
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__ as g
    g.build()
    from paper_2109_04804_gb300 import hbpc, inputs
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    out = r1_roofline(torch, hbpc, inputs, flush, hbpc.fp64_fma_peak(), peaks().get("hbm_gbs", 6800.0))
    print(json.dumps(out), flush=True)


def run_reference(args):
    """The FP64 CPU oracle as it stands, on the host cores: W + K whole
    HBPC(8,4) steps of the 2-D advection workload on the 16 x 16 sample at the
    same CFL 8 (each step continues from the last), K of them timed."""
    world, rank, _ = dist_env()
    if rank != 0:
        return
    from oracle import dgsem, hbpc as ohbpc, laws, newton
    from paper_2109_04804_gb300 import inputs
    ph = laws.Physics(laws.ADVECTION, 2, a=WL["a"])
    disc = dgsem.Disc(dgsem.Mesh(2, SAMPLE_N, WL["lo"], WL["hi"]), WL["N"], ph)
    dts = workload_dt(SAMPLE_N)
    opts = newton.NewtonOptions(tol_rel=WL["tol_newton_rel"], tol_abs=WL["tol_newton_abs"],
                                gmres_tol=WL["tol_gmres_rel"], restart=WL["gmres_restart"],
                                gmres_maxiter=WL["gmres_max_iter"], newton_max=WL["newton_max_iter"],
                                jv="linear", pc="bjext")
    st = newton.Stats()
    adv = ohbpc.dg_stepper(disc, dts, WL["q"], WL["kmax"], opts, stats=st)
    w = inputs.sine_product(disc.node_coords())
    for _ in range(args.warmup):
        w = adv(w)
    its0 = st.gmres_its
    t0 = time.perf_counter()
    for _ in range(args.steps):
        w = adv(w)
    t = time.perf_counter() - t0
    value = disc.ndof * args.steps / t
    threads = int(os.environ.get("OPENBLAS_NUM_THREADS", "0")) or (os.cpu_count() or 1)
    hc = host_cpu()
    sample = ("%d whole HBPC(8,4) steps (after %d warm-up steps) of the same workload on a 16x16-element mesh "
              "at the same CFL 8 (dt = 1/24, %d DOF), %d GMRES iterations per step, FP64 numpy oracle"
              % (args.steps, args.warmup, disc.ndof, (st.gmres_its - its0) // max(1, args.steps)))
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * t / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(config_dict(workload_dt(), "fp64"), parallelism="replicas" if world > 1 else "single"),
            "impl": "reference", "sample": sample,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample,
                             "host": hc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


BATCH = dict(n_inst=256, n_range=(16, 96), N_range=(3, 7), nu_range=(1e-3, 1e-2), seed=2024,
             q=6, kmax=2, cfl_finest=2.0, tol_newton_rel=1e-10, tol_newton_abs=1e-12, tol_gmres_rel=1e-3,
             gmres_restart=100, gmres_max_iter=3000, newton_max_iter=50, max_per_group=0)


STEP_GRAPH = True   # the batch's steps as one CUDA graph per group (--no-step-graph: host-driven)
PC_REBUILD_EVERY = False   # the batch's BJ_ext blocks: once per Newton solve (the reuse of Sec. 4.1.2)


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


def run_batch(args, emit=True):
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
    b.set_pc_rebuild(PC_REBUILD_EVERY)
    if STEP_GRAPH:
        # every group's step as one graph launch, captured here (outside the
        # timed steps) with the tuned launch shapes
        b.set_step_graph(True)
        b.step(1)
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
                       "step_graph": STEP_GRAPH,
                       "pc_rebuild": "every Newton iteration" if PC_REBUILD_EVERY else "once per Newton solve",
                       "graph_launches_per_step": groups if STEP_GRAPH else 0,
                       "l2_between_steps": "flushed (256 MB write) between timed steps",
                       "parallelism": "replicas" if world > 1 else "single"},
            "r1_evals_per_s": (d["r1_evals"] + d["r2_evals"]) / t_sec,
            "gmres_its_per_step": d["gmres_its"] / args.steps, "newton_its_per_step": d["newton_its"] / args.steps,
            "gpu_launches": int(d["launches"]),
            "e2e": {"value": ndof * args.steps * world / e2e_s, "unit": UNIT,
                    "h2d_bytes_per_step": ndof * 8, "d2h_bytes_per_step": ndof * 8},
            "clocks": clk}
    if rank == 0 and emit:
        print(json.dumps(line), flush=True)
    if world > 1 and emit:
        import torch.distributed as dist
        dist.destroy_process_group()
    return line


TGV = dict(n=32, N=5, q=4, kmax=0, cfl=20.0, eps=0.1, re=1600.0, prandtl=0.72, tol_newton_rel=1e-10,
           tol_newton_abs=1e-10, tol_gmres_rel=1e-3, gmres_restart=100, gmres_max_iter=5000, newton_max_iter=30,
           check_n=8)


EPC = dict(n=(16, 16), lo=(-1.0, -1.0), hi=(1.0, 1.0), N=5, q=4, kmax=0, tol_newton_rel=1e-8,
           tol_newton_abs=1e-10, tol_gmres_rel=1e-3, gmres_restart=700, gmres_max_iter=7000, newton_max_iter=50,
           newton_max_iter_no_pc=10,
           eps=(1.0, 0.1, 0.01), dts=(0.0125, 0.05, 0.2, 0.8))


def run_euler_pc(args, emit=True):
    """The preconditioner comparison of the paper's Euler study: the density
    wave rho = 1 + 0.3 sin(pi (x + y)), v = (0.3, 0.3), p = 1 on [-1, 1]^2, 16 x 16
    elements, N = 5, global LF with lambda = diag(1/eps, 1, 1, 1/eps), reference
    Mach numbers eps = 1, 0.1, 0.01, eps_GMRES = 1e-3, eps_Newton = 1e-8, restart
    700, at most 7000 GMRES iterations per Newton step (and the absolute
    Newton test ||dW|| <= 1e-10, at most 50 Newton steps, 10 without a
    preconditioner); one predictor step of
    HBPC(4, 0) (the J^predictor system, alpha = 1/2, 1/6) per time step size,
    in FP64, with no preconditioner, BJ_ext and BJ^H_ext (rebuilt every Newton
    iteration).  Reports GMRES iterations and device milliseconds per time step,
    and each answer's distance to the no-preconditioner one.  Without a
    preconditioner, once a time step did not converge the larger ones of the
    same eps are not run (each costs up to 70,000 GMRES iterations)."""
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__ as g
    g.build()
    from paper_2109_04804_gb300 import hbpc, inputs
    arms = (("no_pc", hbpc.PC_NONE), ("bjext", hbpc.PC_BJEXT), ("bjext_h", hbpc.PC_BJEXT_H))

    def one(eps, dt, pc):
        c = hbpc.Context(2, EPC["n"], EPC["lo"], EPC["hi"], EPC["N"], law=hbpc.LAW_EULER,
                         flux=hbpc.FLUX_GLOBAL_LF, eps=eps, q=EPC["q"], kmax=EPC["kmax"], dt=dt,
                         tol_newton_rel=EPC["tol_newton_rel"], tol_newton_abs=EPC["tol_newton_abs"],
                         tol_gmres_rel=EPC["tol_gmres_rel"], gmres_restart=EPC["gmres_restart"],
                         gmres_max_iter=EPC["gmres_max_iter"],
                         newton_max_iter=EPC["newton_max_iter"] if pc != hbpc.PC_NONE else EPC["newton_max_iter_no_pc"],
                         pc=pc, precision=hbpc.PREC_FP64)
        c.set_state(inputs.density_wave(c.node_coords(), eps=eps))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        ok = True
        try:
            c.step(1)
        except hbpc.HBPCError as e:
            ok = str(e)[:80]
        e1.record()
        torch.cuda.synchronize()
        st = c.stats()
        w = c.get_state() if ok is True else None
        c.close()
        return {"ok": ok, "ms": round(e0.elapsed_time(e1), 3), "gmres_its": int(st["gmres_its"]),
                "newton_its": int(st["newton_its"])}, w

    for pc in (hbpc.PC_BJEXT, hbpc.PC_BJEXT_H):   # kernels loaded, first-call allocations done
        one(1.0, EPC["dts"][0], pc)
    rows = []
    for eps in EPC["eps"]:
        failed = set()
        for dt in EPC["dts"]:
            row = {"eps": eps, "dt": dt}
            ref = None
            for name, pc in arms:
                if name in failed:
                    row[name] = {"ok": "not run: no convergence at a smaller dt"}
                    continue
                r, w = one(eps, dt, pc)
                if r["ok"] is not True and name == "no_pc":
                    failed.add(name)
                if name == "no_pc":
                    ref = w
                elif w is not None and ref is not None:
                    r["rel_l2_vs_no_pc"] = rel_l2(w, ref)
                row[name] = r
            rows.append(row)
    line = {"workload": "2d_euler_density_wave_16x16_N5_predictor_HBPC(4,0)_globalLF_pc_comparison",
            "unit": "GMRES iterations and device ms per time step", "n_dof": 16 * 16 * 36 * 4,
            "config": {k: v for k, v in EPC.items()}, "rows": rows}
    if emit:
        print(json.dumps(line), flush=True)
    return line


def run_pc_network(args, emit=True):
    """The learned preconditioner's build on the Euler vortex mesh (128^2, N = 4,
    16,384 elements, n_b = 100): network inference (three BF16 tcgen05 GEMMs,
    16,384 x 112 -> 256 -> 256 -> 10,000, the last one writing the FP32 blocks),
    the probe check of every block and one apply, per hbpc_eval_pc call (mixed
    precision, random network).  Reports ms per call and the GEMMs' FLOPs per
    call; the GEMM kernels' own durations come from the profile."""
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__ as g
    g.build()
    from paper_2109_04804_gb300 import hbpc, inputs
    c = hbpc.Context(2, VORTEX["n"], VORTEX["lo"], VORTEX["hi"], VORTEX["N"], law=hbpc.LAW_EULER,
                     flux=hbpc.FLUX_RUSANOV, q=VORTEX["q"], kmax=VORTEX["kmax"], dt=vortex_dt(), pc=hbpc.PC_LEARNED,
                     precision=hbpc.PREC_MIXED)
    c.pc_model_init(seed=1, out_scale=1e-2)
    info = c.pc_model_info()
    w = inputs.isentropic_vortex(c.node_coords())
    n = c.ndof
    X = torch.zeros(2 * n, dtype=torch.float64, device="cuda")
    X[:n] = torch.from_numpy(np.ascontiguousarray(w.ravel())).cuda()
    v = torch.randn(2 * n, dtype=torch.float64, device="cuda")
    out = torch.empty_like(v)
    for _ in range(max(1, args.warmup)):
        c.eval_pc(1.0, 1.0, X, v, out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        c.eval_pc(1.0, 1.0, X, v, out)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    nE = c.ndof // (4 * 25)
    H, din, dout = info["hidden"], info["d_in_padded"], 100 * 100
    flops = 2.0 * nE * H * (din + H + dout)
    c.close()
    line = {"workload": "learned_pc_build_euler_vortex_128x128_N4", "ms_per_call": ms,
            "gemm_gflop_per_call": flops / 1e9, "elements": nE,
            "gemm_shapes": [[nE, H, din], [nE, H, H], [nE, dout, H]]}
    if emit:
        print(json.dumps(line), flush=True)
    return line


CAVITY = dict(n=(16, 16), N=5, q=6, kmax=2, dt=0.02, eps=0.1, mu=0.025, tol_newton_rel=1e-3,
              tol_newton_abs=1e-10, tol_gmres_rel=1e-2, gmres_restart=200, gmres_max_iter=7000, newton_max_iter=50,
              startup=((0.002, 10), (0.005, 4), (0.01, 4)))


def run_cavity(args, emit=True):
    """The paper's lid-driven cavity (Sec. 5.3.1): Navier-Stokes on [0, 1]^2,
    16 x 16 elements, N = 5, adiabatic no-slip walls left, right and below, the
    lid state rho = 1, v = (1, 0), p = 1/gamma above, eps = 0.1, mu = 0.025
    (Re 400), HBPC(6, 2), dt = 0.02, eps_Newton = 1e-3 (or an update
    ||dW|| <= 1e-10), eps_GMRES = 1e-2; the gas at rest with the lid's density and
    pressure initially.  From the gas at rest the first dt = 0.02 step fails
    (the first Newton update of the corrector drives the pressure negative, on
    the oracle as on the GPU), so an untimed start-up of shorter steps
    (dt 0.002 x 10, 0.005 x 4, 0.01 x 4; t = 0.08) precedes the timed
    dt = 0.02 steps.  FP64, BJ_ext, one graph launch per step; two arms: the
    blocks built at every Newton iteration, and once per Newton solve.
    Reports DOF-timesteps/s, iterations per step, and the kinetic energy, the
    smallest density and the largest speed after the steps (no reference data:
    the run's own record)."""
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__ as g
    g.build()
    from paper_2109_04804_gb300 import hbpc, inputs
    C = CAVITY
    gamma, eps = 1.4, C["eps"]
    lid = inputs.euler_from_primitive(np.array([1.0]), [np.array([1.0]), np.array([0.0])], np.array([1.0 / gamma]),
                                      gamma, eps)[0]

    def ctx(dt):
        c = hbpc.Context(2, C["n"], (0.0, 0.0), (1.0, 1.0), C["N"], law=hbpc.LAW_NAVIER_STOKES,
                         flux=hbpc.FLUX_RUSANOV, mu=C["mu"], eps=eps, q=C["q"], kmax=C["kmax"], dt=dt,
                         tol_newton_rel=C["tol_newton_rel"], tol_newton_abs=C["tol_newton_abs"],
                         tol_gmres_rel=C["tol_gmres_rel"], gmres_restart=C["gmres_restart"],
                         gmres_max_iter=C["gmres_max_iter"], newton_max_iter=C["newton_max_iter"], pc=hbpc.PC_BJEXT)
        c.set_boundary(0, "noslip", "noslip")
        c.set_boundary(1, "noslip", lid)
        return c

    c = ctx(C["dt"])
    X = c.node_coords()
    ndof = c.ndof
    c.close()
    w = inputs.euler_from_primitive(np.ones_like(X[0]), [0 * X[0], 0 * X[0]], np.full_like(X[0], 1.0 / gamma),
                                    gamma, eps)
    t0 = 0.0
    for dt, n in C["startup"]:
        c = ctx(dt)
        c.set_state(w)
        c.step(n)
        w = c.get_state()
        t0 += c.stats()["t"]
        c.close()

    def arm(every):
        c = ctx(C["dt"])
        c.set_pc_rebuild(every)
        c.set_step_graph(not args.no_step_graph)
        c.set_state(w)
        ok = True
        try:
            c.step(max(1, args.warmup))
        except hbpc.HBPCError as e:
            ok = "warm-up step: " + str(e)[:100]
        st0 = c.stats()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        if ok is True:
            try:
                c.step(args.steps)
            except hbpc.HBPCError as e:
                ok = str(e)[:100]
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        st = c.stats()
        wt = c.get_state()
        c.close()
        rho, mom = wt[:, 0], wt[:, 1:3]
        out = {"ok": ok, "value": ndof * 1000.0 / ms if ok is True else 0.0, "ms_per_step": ms,
               "t": t0 + st["t"], "gmres_its_per_step": (st["gmres_its"] - st0["gmres_its"]) / args.steps,
               "newton_its_per_step": (st["newton_its"] - st0["newton_its"]) / args.steps,
               "mean_kinetic_energy_per_node": 0.5 * float((mom ** 2 / rho[:, None]).sum()) / rho.size,
               "min_density": float(rho.min()), "max_speed": float(np.sqrt(((mom / rho[:, None]) ** 2).sum(1)).max())}
        return out

    arms = {"pc_every_newton_iteration": arm(True), "pc_once_per_newton_solve": arm(False)}
    best = max(arms, key=lambda k: arms[k]["value"])
    line = {"workload": "lid_driven_cavity_16x16_N5_HBPC(6,2)_dt0.02_Re400_eps0.1", "unit": UNIT,
            "value": arms[best]["value"], "best_arm": best, "steps": args.steps, "ndof": ndof,
            "step_graph": not args.no_step_graph, "arms": arms,
            "config": {k: (list(v) if isinstance(v, tuple) else v) for k, v in C.items()}}
    if emit:
        print(json.dumps(line), flush=True)
    return line


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




def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true",
                    help="skip the oracle (timed CPU baseline and the accuracy against the oracle)")
    ap.add_argument("--no-vortex", action="store_true",
                    help="skip the learned-vs-plain-GMRES comparison on the Euler vortex in the default line")
    ap.add_argument("--corrector-batch", type=int, default=-1, choices=[-1, 0, 1],
                    help="1: the s - 1 corrector stages of every sweep solved as one batched Newton-GMRES; "
                         "0: one after the other; -1 (default): batched in the mixed mode only")
    ap.add_argument("--headline-only", action="store_true",
                    help="the headline arm alone (for profiling): no second precision, oracle or vortex")
    ap.add_argument("--no-step-graph", action="store_true",
                    help="host-driven steps (a look at the GMRES state every few columns) instead of one CUDA "
                         "graph launch per step with device-driven Newton and GMRES loops")
    ap.add_argument("--no-cavity", action="store_true",
                    help="leave the lid-driven cavity sub-line out of the default line")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the batched viscous Burgers workload in the default line")
    ap.add_argument("--no-r1-roofline", action="store_true",
                    help="skip the operator-pass roofline on the Euler vortex and Taylor-Green meshes")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"],
                    help="precision of the headline value (the other one is reported beside it): fp64, the "
                         "workload's own; mixed: FP32 Krylov loop, FP64 Newton residual/update")
    ap.add_argument("--workload", default="advection2d",
                    choices=["advection2d", "burgers_batch", "euler_vortex", "taylor_green", "r1_roofline",
                             "euler_pc", "pc_network", "cavity"],
                    help="advection2d: the default 64x64 N=5 HBPC(8,4) line; burgers_batch: the batched "
                         "viscous Burgers instances; euler_vortex: learned vs BJ_ext vs plain GMRES; "
                         "taylor_green: the 3-D Navier-Stokes line; r1_roofline: the operator-pass roofline "
                         "object of the default line alone; euler_pc: no preconditioner vs BJ_ext vs BJ^H_ext "
                         "on the Euler density wave (16x16, N=5, eps = 1, 0.1, 0.01)")
    ap.add_argument("--instances", type=int, default=BATCH["n_inst"])
    ap.add_argument("--tgv-n", type=int, default=0,
                    help="taylor_green: elements per direction (default 32; smaller for profiling)")
    ap.add_argument("--no-check", action="store_true",
                    help="taylor_green: skip the FP64-vs-mixed comparison on the 8^3 mesh")
    ap.add_argument("--max-per-group", type=int, default=BATCH["max_per_group"],
                    help="instances sharing one context and one GMRES (<= 0: all of one N)")
    ap.add_argument("--oracle-task", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--oracle-out", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--oracle-steps", type=int, default=1, help=argparse.SUPPRESS)
    args = ap.parse_args()
    global STEP_GRAPH
    STEP_GRAPH = not args.no_step_graph
    if args.oracle_task:
        oracle_task(args.oracle_task, args.oracle_out, args.oracle_steps)
    elif args.impl == "reference":
        run_reference(args)
    elif args.workload == "burgers_batch":
        run_batch(args)
    elif args.workload == "euler_vortex":
        run_vortex(args)
    elif args.workload == "taylor_green":
        run_tgv(args)
    elif args.workload == "r1_roofline":
        run_r1_only(args)
    elif args.workload == "euler_pc":
        run_euler_pc(args)
    elif args.workload == "pc_network":
        run_pc_network(args)
    elif args.workload == "cavity":
        run_cavity(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
