"""Benchmark: DOF.stages/s of one forward (primal) sweep plus one adjoint sweep
over a period of the flapping-airfoil workload on one GB300 (or N replicas).

Workload (default "c1"): 2048-triangle seeded O-grid around a 12%-thick
symmetric airfoil, degree-3 DG (40 DOF/element, 81,920 DOF), 100 DIRK3 steps
per period, motion = 6 seeded Fourier coefficients.  A step = primal sweep
(Newton per stage, stored linearization) + adjoint sweep with the QoI terms
and gradient reconstruction (Eq. uns-disc-adj-dirk2, Eq. funcl-grad-nosens-dirk)
for F = J_E, the cycle-averaged flapping energy.  Each step starts from the
previous step's final state (fixed-point iteration toward the periodic orbit).

value = N_u * Nt * 3 stages / (time per step), summed over ranks (replicas).
Multi-GPU: the path does not shard within one solve; N ranks run N independent
replicas (scaling "weak", no data-path collective).
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

# DRAM bytes (read + write) per launch of a kernel class on a workload, from one ncu
# capture of the current kernel (profiles/ names the capture); absent -> null.
MEASURED_TRAFFIC = {
    # profiles/k_stream_rows_c1.md: dram__bytes_read.sum 77.70 MB + dram__bytes_write.sum 0.99 MB
    ("stage_op", "c1"): 78.69e6,
}

METRIC = "DOF*stages/s fwd+adjoint"
UNIT = "DOF*stages/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="c1")
    ap.add_argument("--roofline-kernel", default=None,
                    help="kernel class for the roofline (default: stage_op in fp64, stage_matvec32 in mixed)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--profile-step", type=int, default=0, metavar="NT",
                    help="profiler capture mode: one primal + adjoint sweep over NT steps of the workload's "
                         "step size (period and motion amplitudes scaled by NT / Nt), no timing, no bench line")
    return ap.parse_args()


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm = [float(r[0]) for r in self.rows if r and r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if len(r) > 1 and r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for k, nm in enumerate(names):
                if len(r) > 4 + k and r[4 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------- oracle sample (CPU)
def oracle_sample(config, budget_s):
    """Times the oracle's element-local work of one stage-Newton iteration (residual and
    exact complex-step Jacobian rows) on as many elements of the workload as fit in
    budget_s, extrapolated linearly (the element loop is exactly linear) to the mesh.
    The sparse LU factorization is NOT included, so the oracle's cost is understated."""
    import numpy as np

    from oracle.dg import DG
    from pp_inputs import CONFIGS, config_mesh, config_mu, free_stream_state, state_perturbation
    c = CONFIGS[config]
    dg = DG(config_mesh(config), c["p"], kin=c["kin"])
    mu = config_mu(config)
    u = (free_stream_state(dg.Ne, c["p"]) + state_perturbation(dg.Ne, c["p"], 1, amp=1e-3)).reshape(-1)
    t0 = time.perf_counter()
    dg.residual(u, mu, 0.1)
    t_res = time.perf_counter() - t0
    done, t_jac, chunk = 0, 0.0, 32
    while done < dg.Ne and t_jac < budget_s:
        el = np.arange(done, min(done + chunk, dg.Ne))
        t0 = time.perf_counter()
        dg.jac_blocks_subset(u, mu, 0.1, el)
        t_jac += time.perf_counter() - t0
        done += len(el)
    t_jac_full = t_jac * dg.Ne / done
    # per stage the oracle's Newton evaluates about two Jacobians and a handful of residuals
    t_stage = 2.0 * t_jac_full + 5.0 * t_res
    return dict(value=dg.Nu / t_stage, t_res=t_res, t_jac_full=t_jac_full, elems=done, Ne=dg.Ne,
                seconds=t_res + t_jac, threads=_threads())


def _threads():
    try:
        from threadpoolctl import threadpool_info
        return max([i.get("num_threads", 1) for i in threadpool_info()] + [1])
    except Exception:
        return 1


# --------------------------------------------------------------------------- ours
def max_over_ranks(x, device="cpu"):
    """Largest x over the ranks of the default process group (x itself without one).
    Each rank is an independent replica; the slowest one sets the job's time."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def l2_note(res, c, precision):
    """Size of the stored linearization the sweeps stream against the 126 MB L2: per stage
    and element about 16 nb x nb blocks of 8 bytes (FP64: Jacobian 4, inverse 1, folded 6,
    transposes 5; mixed: FP64 Jacobian and transposes plus the FP32 copies, about the same)."""
    p = c["p"]
    nb = 2 * (p + 1) * (p + 2)
    word_blocks = 16 * 8
    gb = res["ne"] * nb * nb * word_blocks * 3 * res["Nt"] / 1e9
    if gb > 1.0:
        return f"working set (stored stage linearization, ~{gb:.0f} GB) far larger than L2; no flush needed"
    return f"working set ~{gb * 1e3:.0f} MB, not larger than L2: small-case timing, not a bench value"


def whole_job_value(units_per_rank, ms_max, world):
    """Units all ranks processed (the same per rank: weak scaling) per second of the slowest rank."""
    return units_per_rank * world / (ms_max * 1e-3)


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch

    from paper_1512_00616_gb300 import api as A
    from pp_inputs import CONFIGS, PHYS, config_mesh, config_mu, free_stream_state

    torch.cuda.set_device(local_rank)
    c = CONFIGS[args.config]
    mesh = config_mesh(args.config)
    mu = config_mu(args.config)
    Nt = c["Nt"]
    stream = torch.cuda.Stream()
    cfg = A.pp_config_default(p=c["p"], kin=c["kin"], T=PHYS["T"], device=local_rank, stream=stream.cuda_stream,
                              precision=A.PP_PREC_MIXED if args.precision == "mixed" else A.PP_PREC_FP64)
    ctx = A.pp_create(cfg)
    m = A.pp_mesh_create(ctx, mesh.verts, mesh.tris, mesh.ftag)
    ne, npn, nu = A.pp_mesh_info(m)
    dev = f"cuda:{local_rank}"
    u0 = torch.tensor(free_stream_state(ne, c["p"]).reshape(-1), dtype=torch.float64, device=dev)
    uN = torch.zeros_like(u0)
    lamN = torch.zeros_like(u0)
    lam0 = torch.zeros_like(u0)
    weights = np.array([-1.0 / PHYS["T"], 0.0])   # F = J_E = -W/T
    newton = []

    phase = {"primal": 0.0, "adjoint": 0.0}

    def step():
        t0 = time.perf_counter()
        A.pp_primal_period(ctx, m, mu, u0, Nt, u_final=uN)
        t1 = time.perf_counter()
        g = A.pp_adjoint_sweep(ctx, lamN, lam0, weights=weights, n_mu=len(mu))
        t2 = time.perf_counter()
        phase["primal"] += t1 - t0
        phase["adjoint"] += t2 - t1
        u0.copy_(uN)
        return g

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
        A.pp_prof_select(args.roofline_kernel)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        clk = ClockSampler(local_rank)
        clk.start()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        phase["primal"] = phase["adjoint"] = 0.0
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        clocks = clk.stop()
        launches_k, kern_ms = A.pp_prof_read()
        iters = A.pp_sweep_counts(ctx)
        counts = A.pp_prof_counts()
        ms = ev0.elapsed_time(ev1) / args.steps
        split = {k: 1e3 * v / args.steps for k, v in phase.items()}

        e2e = None
        if not args.no_e2e:
            host_u0 = torch.empty(nu, dtype=torch.float64, pin_memory=True)
            host_u0.copy_(u0.cpu())
            host_uN = torch.empty_like(host_u0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.steps):
                u0.copy_(host_u0, non_blocking=True)
                A.pp_primal_period(ctx, m, mu, u0, Nt, u_final=uN)
                A.pp_adjoint_sweep(ctx, lamN, lam0, weights=weights, n_mu=len(mu))
                host_uN.copy_(uN, non_blocking=True)
                stream.synchronize()
                host_u0.copy_(host_uN)
            e1.record(stream)
            torch.cuda.synchronize()
            e2e_ms = e0.elapsed_time(e1) / args.steps
            e2e = dict(ms_per_step=e2e_ms, h2d=nu * 8, d2h=nu * 8 + 8 * len(mu))

    ms = max_over_ranks(ms, dev)
    if e2e is not None:
        e2e["ms_per_step"] = max_over_ranks(e2e["ms_per_step"], dev)
    A.pp_mesh_destroy(m)
    A.pp_destroy(ctx)
    return dict(config=args.config, ms=ms, nu=nu, ne=ne, Nt=Nt, clocks=clocks, iters=iters, split=split, kern_launches=launches_k, kern_ms=kern_ms,
                counts=counts, e2e=e2e)


def roofline_for(kernel, res, peaks, fp64_tflops, c):
    """Algorithmic work per launch of the timed kernel class: FLOPs or bytes per element of
    the kernel's definition times the elements one launch processes."""
    p = c["p"]
    Np = (p + 1) * (p + 2) // 2
    nb = 4 * Np
    nqv, nqf = (p + 2) ** 2, p + 2
    ne = res["ne"]
    if res["kern_launches"] <= 0:
        return None
    t = res["kern_ms"] / res["kern_launches"] * 1e-3
    if kernel == "jacobian":
        # basis contraction per variable pair (16 per element): W = C T over 3 trial types at
        # 2 nqv Np volume and 2 x 3 nqf Np face entries, then J_ab = D W (Np^2 (2 nqv + 3 nqf)
        # for the diagonal block, Np^2 nqf for each face block); 2 flops per FMA.  The dual-
        # number flux derivatives are not counted.
        w_fma = 3 * (2 * nqv * Np + 2 * 3 * nqf * Np)
        j_fma = Np * Np * (2 * nqv + 3 * nqf) + 3 * Np * Np * nqf
        flops = ne * 16 * 2 * (w_fma + j_fma)
        ach = flops / t / 1e12
        return {"bound": "alu", "achieved": ach, "peak": fp64_tflops, "unit": "TFLOP/s",
                "frac": ach / fp64_tflops if fp64_tflops else None,
                "traffic": MEASURED_TRAFFIC.get((kernel, res["config"])),
                "kernel": "k_jacobian", "launches": res["kern_launches"], "avg_us": t * 1e6}
    if kernel in ("stage_matvec", "block_apply", "stage_matvec32", "block_apply32", "stage_op", "stage_op32"):
        blocks = 4 if kernel.startswith("stage_matvec") else (3 if kernel.startswith("stage_op") else 1)
        word = 4 if kernel.endswith("32") else 8
        # matrix blocks + input slices + output (stage_op: 3 neighbour slices, the element's own
        # slice for the identity term and the output)
        byts = ne * (blocks * nb * nb * word + (5 if kernel.startswith("stage_op") else 2) * nb * word)
        if word == 8:
            # GB300 issues ~2 FP64 FMA per clock per SM: the FP64 block product is FP64-ALU bound
            # (its FMA floor exceeds its HBM floor), so it is held against the measured FP64 peak
            flops = 2.0 * ne * blocks * nb * nb
            ach = flops / t / 1e12
            return {"bound": "alu", "achieved": ach, "peak": fp64_tflops, "unit": "TFLOP/s",
                    "frac": ach / fp64_tflops if fp64_tflops else None,
                    "traffic": MEASURED_TRAFFIC.get((kernel, res["config"])),
                    "kernel": ("k_stream_rows<%d,3,double> (I + B, folded block-Jacobi)" % nb if kernel == "stage_op"
                               else "k_" + kernel.replace("32", "") + "<double>"), "launches": res["kern_launches"],
                    "avg_us": t * 1e6, "hbm_gbs_equiv": byts / t / 1e9}
        ach = byts / t / 1e9
        return {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": ach / peaks["hbm_gbs"], "traffic": MEASURED_TRAFFIC.get((kernel, res["config"])),
                "kernel": ("k_stream_rows<%d,3,float> (I + B, folded block-Jacobi)" % nb if kernel == "stage_op32"
                           else "k_" + kernel.replace("32", "") + "<float>"),
                "launches": res["kern_launches"], "avg_us": t * 1e6}
    return None


def profile_step(args):
    """One primal sweep plus one adjoint sweep (F = J_E, dF/dmu) over args.profile_step steps
    of the workload's step size, from the free stream, for profiler captures.  A shorter
    period keeps the time step: T and the motion amplitudes are scaled by NT / Nt, so the
    capture runs the same kernels while holding a few GB of device memory."""
    import numpy as np
    import torch

    from paper_1512_00616_gb300 import api as A
    from pp_inputs import CONFIGS, PHYS, config_mesh, config_mu, free_stream_state
    c = CONFIGS[args.config]
    Nt = args.profile_step
    mesh = config_mesh(args.config)
    mu = config_mu(args.config)
    T = PHYS["T"] * Nt / c["Nt"]
    if Nt < c["Nt"]:
        mu = mu * (T / PHYS["T"])
    cfg = A.pp_config_default(p=c["p"], kin=c["kin"], T=T,
                              precision=A.PP_PREC_MIXED if args.precision == "mixed" else A.PP_PREC_FP64)
    ctx = A.pp_create(cfg)
    m = A.pp_mesh_create(ctx, mesh.verts, mesh.tris, mesh.ftag)
    ne, _, nu = A.pp_mesh_info(m)
    u0 = torch.tensor(free_stream_state(ne, c["p"]).reshape(-1), dtype=torch.float64, device="cuda")
    uN, lamN, lam0 = torch.zeros_like(u0), torch.zeros_like(u0), torch.zeros_like(u0)
    torch.cuda.synchronize()
    A.pp_primal_period(ctx, m, mu, u0, Nt, u_final=uN)
    A.pp_adjoint_sweep(ctx, lamN, lam0, weights=np.array([-1.0 / T, 0.0]), n_mu=len(mu))
    torch.cuda.synchronize()
    print("profile step ok", float(uN.norm()), float(lam0.norm()), A.pp_sweep_counts(ctx))
    A.pp_mesh_destroy(m)
    A.pp_destroy(ctx)


def main():
    args = parse()
    if args.profile_step > 0:
        profile_step(args)
        return
    if args.roofline_kernel is None:
        args.roofline_kernel = "stage_op32" if args.precision == "mixed" else "stage_op"
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    from pp_inputs import CONFIGS
    c = CONFIGS[args.config]
    workload = (f"{args.config}: {2 * c['n_theta'] * c['n_r']}-triangle O-grid, p={c['p']}, "
                f"{c['Nt']} DIRK3 steps/period, primal sweep + adjoint sweep (F = J_E, dF/dmu)")

    if args.impl == "reference":
        if rank != 0:
            return
        t0 = time.perf_counter()
        vals = []
        budget = max(5.0, 150.0 / max(args.steps + args.warmup, 1))
        for i in range(args.warmup + args.steps):
            s = oracle_sample(args.config, budget)
            if i >= args.warmup:
                vals.append(s["value"])
        v = statistics.mean(vals)
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": workload},
                "cpu_baseline": {"value": v, "unit": UNIT, "cores": s["threads"], "kind": "oracle",
                                 "sample": f"per step: oracle residual + complex-step Jacobian rows on "
                                           f"{s['elems']}/{s['Ne']} elements (~{budget:.0f} s), extrapolated "
                                           "linearly to one stage-Newton iteration of the mesh; sparse LU "
                                           "excluded (oracle cost understated)"},
                "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
                "wall_s": time.perf_counter() - t0}
        print(json.dumps(line))
        return

    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local_rank}"))
    res = run_ours(args, rank, world, local_rank)
    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return
    from paper_1512_00616_gb300 import api as A
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peaks = json.load(open(peaks_path)) if os.path.exists(peaks_path) else {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}
    fp64 = A.pp_measure_fp64_peak(local_rank)
    units = res["nu"] * res["Nt"] * 3
    value = whole_job_value(units, res["ms"], world)
    roof = roofline_for(args.roofline_kernel, res, peaks, fp64, c)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": res["ms"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f64+f32", "data": "synthetic",
        "config": {"workload": workload, "precision": args.precision, "dof": res["nu"], "elements": res["ne"], "Nt": res["Nt"],
                   "parallelism": f"replicas x{world}",
                   "l2": l2_note(res, c, args.precision)},
        "roofline": roof, "fp64_fma_peak_tflops_measured": fp64,
        "clocks": res["clocks"],
        "gpu_launches": int(sum(res["counts"].values())),
        "launches_by_class": res["counts"],
        "last_step_iterations": res["iters"],
        "ms_by_phase": res["split"],
    }
    if res["e2e"]:
        e = res["e2e"]
        line["e2e"] = {"value": whole_job_value(units, e["ms_per_step"], world), "unit": UNIT,
                       "h2d_bytes_per_step": e["h2d"], "d2h_bytes_per_step": e["d2h"]}
    if not args.no_cpu_baseline and world == 1:
        s = oracle_sample(args.config, args.cpu_budget)
        line["cpu_baseline"] = {"value": s["value"], "unit": UNIT, "cores": s["threads"], "kind": "oracle",
                                "sample": f"oracle residual + complex-step Jacobian rows on {s['elems']}/{s['Ne']} "
                                          f"elements ({s['seconds']:.1f} s), extrapolated linearly to one "
                                          "stage (2 Jacobians + 5 residuals); sparse LU excluded"}
    print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
