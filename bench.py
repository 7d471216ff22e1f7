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
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=3, help="steps of the end-to-end measurement (<= --steps)")
    ap.add_argument("--oracle-stage", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--out", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--profile-step", type=int, default=0, metavar="NT",
                    help="profiler capture mode: one primal + adjoint sweep over NT steps of the workload's "
                         "step size (period and motion amplitudes scaled by NT / Nt), no timing, no bench line")
    ap.add_argument("--compare-precisions", action="store_true",
                    help="one primal period + adjoint sweep of --config from the free stream in FP64 and in "
                         "mixed precision; prints wall times and the mixed arm's relative differences, no bench line")
    ap.add_argument("--gmres-maxit", type=int, default=0, help="GMRES cap per linear solve (0: the library default)")
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
def cpu_info():
    """nproc and the CPU model of this host (lscpu, else /proc/cpuinfo)."""
    import platform
    model = None
    try:
        out = subprocess.run(["lscpu"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True,
                             timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.TimeoutExpired):
        pass
    return {"nproc": os.cpu_count(), "model": model or platform.processor() or platform.machine()}


def oracle_stage(config, seed=1):
    """The oracle's unit of stage work on the full workload, with its own code as it stands:
    one stage-Newton iteration with a Jacobian refresh (the residual, the complex-step block
    Jacobian, the SuperLU factorization of M - a_ii dt J and the solve; the calls
    _stage_newton makes) and the matching adjoint stage (transposed solve, QoI derivatives,
    dr/dmu and dq/dmu terms of the gradient; the calls adjoint_sweep makes).  Every primal
    stage takes at least two such iterations (the first Newton iteration and the stored
    linearization of the converged stage), so a stage costs at least 2 t_iter + t_adjoint:
    DOF*stages/s = N_u / (2 t_iter + t_adjoint) is an upper bound on the oracle's speed."""
    import resource

    import numpy as np
    import scipy.sparse.linalg as spla

    from oracle.dg import DG
    from oracle.dirk import tableau
    from pp_inputs import CONFIGS, PHYS, config_mesh, config_mu, free_stream_state, state_perturbation
    c = CONFIGS[config]
    dg = DG(config_mesh(config), c["p"], kin=c["kin"])
    mu = config_mu(config)
    A, b, cc = tableau()
    dt = PHYS["T"] / c["Nt"]
    u = (free_stream_state(dg.Ne, c["p"]) + state_perturbation(dg.Ne, c["p"], seed, amp=1e-3)).reshape(-1)
    M = dg.mass()
    w = np.array([-1.0 / PHYS["T"], 0.0])           # F = J_E, as the GPU bench
    lam = np.random.default_rng(seed).standard_normal(dg.Nu) * 1e-3
    ti = cc[0] * dt
    k = np.zeros_like(u)
    r0 = resource.getrusage(resource.RUSAGE_SELF)
    t0 = time.perf_counter()
    ui = u + A[0, 0] * k
    R = M @ k - dt * dg.residual(ui, mu, ti)
    Ji = dg.jacobian(ui, mu, ti)
    lu = spla.splu((M - A[0, 0] * dt * Ji).tocsc())
    k = k - lu.solve(R)
    t1 = time.perf_counter()
    ui = u + A[0, 0] * k
    g = w @ dg.dqoi_du(ui, mu, ti)
    kap = lu.solve(b[0] * lam + dt * b[0] * A[0, 0] * g, trans="T")
    lam_prev = lam + dt * (Ji.T @ kap) + dt * b[0] * g
    grad = dt * (kap @ dg.dr_dmu(ui, mu, ti)) + dt * b[0] * (w @ dg.dqoi_dmu(ui, mu, ti))
    t2 = time.perf_counter()
    r1 = resource.getrusage(resource.RUSAGE_SELF)
    cpu = (r1.ru_utime - r0.ru_utime) + (r1.ru_stime - r0.ru_stime)
    assert np.all(np.isfinite(lam_prev)) and np.all(np.isfinite(grad))
    t_stage = 2.0 * (t1 - t0) + (t2 - t1)
    return dict(value=dg.Nu / t_stage, Nu=dg.Nu, Ne=dg.Ne, t_iter=t1 - t0, t_adjoint=t2 - t1, seconds=t2 - t0,
                cores=round(cpu / (t2 - t0), 2), stages=3 * c["Nt"], **cpu_info())


def oracle_stage_text(s, config):
    return (f"the oracle's stage unit on the full {config} mesh ({s['Ne']} elements, {s['Nu']} DOF), timed once: "
            f"one stage-Newton iteration with Jacobian refresh (residual, complex-step block Jacobian, SuperLU "
            f"factorization and solve: {s['t_iter']:.1f} s) and one adjoint stage with QoI and dF/dmu terms "
            f"({s['t_adjoint']:.1f} s); extrapolated to a stage as 2 Newton iterations + 1 adjoint stage (a "
            f"stage needs at least that, so the value is an upper bound on the oracle's speed; a period is "
            f"{s['stages']} stages); NumPy/SciPy as they stand, {s['cores']} cores busy on average (CPU time / "
            f"wall time); host: {s['nproc']} CPUs, {s['model']}")


def start_oracle_stage(config):
    """Runs oracle_stage in a fresh interpreter (started before any CUDA work) so that it
    overlaps the GPU timing; collect() returns its result."""
    import tempfile
    fd, path = tempfile.mkstemp(suffix=".json")
    os.close(fd)
    proc = subprocess.Popen([sys.executable, os.path.abspath(__file__), "--oracle-stage", config, "--out", path],
                            stdout=subprocess.DEVNULL, stderr=subprocess.PIPE, text=True)

    def collect():
        _, err = proc.communicate()
        try:
            with open(path) as fh:
                return json.load(fh)
        except (OSError, ValueError):
            return {"error": (err or "")[-400:]}
        finally:
            os.unlink(path)
    return collect


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
    """Where the timed sweeps' data lives against the 126 MB L2.  One stage solve re-applies
    the same folded stage operator (3 nb^2 words per element) and block inverse (nb^2) over
    its Krylov basis (restart + 1 vectors); successive stages stream new operators out of the
    stored linearization of the whole period (about 16 nb^2 words per element and stage)."""
    p = c["p"]
    nb = 2 * (p + 1) * (p + 2)
    word = 4 if precision == "mixed" else 8
    op_mb = res["ne"] * 4 * nb * nb * word / 1e6
    basis_mb = 41 * res["nu"] * 8 / 1e6
    period_gb = res["ne"] * nb * nb * 16 * 8 * 3 * res["Nt"] / 1e9
    where = "comparable to" if op_mb + basis_mb > 40 else "inside"
    return (f"per stage solve: operator + inverse {op_mb:.0f} MB and Krylov basis {basis_mb:.0f} MB, {where} the "
            f"126 MB L2 (re-read across the solve's Arnoldi steps, partly L2-resident); each step streams the "
            f"period's stored linearization (~{period_gb:.0f} GB) from HBM, so no flush is needed between steps")


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
        A.pp_prof_sample(PROF_STRIDE)
        A.pp_prof_select(KERNELS[args.precision][0])
        A.pp_prof_also(KERNELS[args.precision][1])
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
        kern = {k: A.pp_prof_read_class(k) for k in KERNELS[args.precision]}
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
            n_e2e = max(1, min(args.e2e_steps, args.steps))
            e0.record(stream)
            for _ in range(n_e2e):
                u0.copy_(host_u0, non_blocking=True)
                A.pp_primal_period(ctx, m, mu, u0, Nt, u_final=uN)
                A.pp_adjoint_sweep(ctx, lamN, lam0, weights=weights, n_mu=len(mu))
                host_uN.copy_(uN, non_blocking=True)
                stream.synchronize()
                host_u0.copy_(host_uN)
            e1.record(stream)
            torch.cuda.synchronize()
            e2e_ms = e0.elapsed_time(e1) / n_e2e
            e2e = dict(ms_per_step=e2e_ms, h2d=nu * 8, d2h=nu * 8 + 8 * len(mu))

    ms = max_over_ranks(ms, dev)
    if e2e is not None:
        e2e["ms_per_step"] = max_over_ranks(e2e["ms_per_step"], dev)
    A.pp_mesh_destroy(m)
    A.pp_destroy(ctx)
    return dict(config=args.config, ms=ms, nu=nu, ne=ne, Nt=Nt, clocks=clocks, iters=iters, split=split, kern=kern,
                counts=counts, e2e=e2e)


# kernel classes timed by the bench: (folded stage operator, fused Arnoldi step)
KERNELS = {"fp64": ("stage_op", "arnoldi"), "mixed": ("stage_op32", "arnoldi32")}
PROF_STRIDE = 8   # one launch (one Arnoldi step) in 8 is bracketed by CUDA events


def roofline_for(kernel, res, peaks, fp64_tflops, c, sustained):
    """Roofline entry of one timed kernel class.  achieved = algorithmic work per launch (the
    kernel's definition: FLOPs or bytes per element times the elements of one launch, or the
    counted bytes of the Arnoldi passes) / the launch's average CUDA-event duration."""
    p = c["p"]
    Np = (p + 1) * (p + 2) // 2
    nb = 4 * Np
    ne = res["ne"]
    launches, ms, counted = res["kern"][kernel]
    if launches <= 0:
        return None
    t = ms / launches * 1e-3
    hbm = peaks["hbm_gbs"]
    if kernel.startswith("arnoldi"):
        # bytes of one fused Arnoldi step over k basis vectors of length n, counted at launch:
        # (2k + 3) n words (projections, then the update written as the scaled new basis
        # vector; a selective second pass is not counted); one cooperative launch per step
        ach = counted / (ms * 1e-3) / 1e9
        return {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                "traffic": None, "kernel": "k_arnoldi<KB,%s> (one fused Arnoldi step: Gram-Schmidt "
                "passes, Givens update, scaling)" % ("double" if kernel == "arnoldi" else "float"),
                "launches": launches, "avg_us": t * 1e6, "algorithmic_bytes_per_launch": counted / launches,
                "note": "basis of one stage solve (<= 41 x N_u words) is L2-resident: a low fraction means "
                        "latency-bound grid reductions, not HBM"}
    word = 4 if kernel.endswith("32") else 8
    # folded operator: 3 blocks + 3 neighbour slices + own slice + output per element
    byts = ne * (3 * nb * nb * word + 5 * nb * word)
    if word == 8:
        # GB300's FP64 FMA rate is below its HBM rate for a block product (one 8-byte word per
        # FMA): the FP64 operator is held against the measured FP64 peak
        flops = 2.0 * ne * 3 * nb * nb
        ach = flops / t / 1e12
        return {"bound": "alu", "achieved": ach, "peak": fp64_tflops, "unit": "TFLOP/s",
                "frac": ach / fp64_tflops if fp64_tflops else None,
                "traffic": MEASURED_TRAFFIC.get((kernel, res["config"])),
                "kernel": "k_stream_rows<%d,3,double> (B = (M - cJ) D^-1 - I, folded block-Jacobi)" % nb,
                "launches": launches, "avg_us": t * 1e6, "hbm_gbs_equiv": byts / t / 1e9,
                "peak_source": "pp_measure_fp64_peak_clock (16-chain FMA probe, measured in this run)"}
    ach = byts / t / 1e9
    return {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
            "traffic": MEASURED_TRAFFIC.get((kernel, res["config"])),
            "kernel": "k_stream_rows<%d,3,float> (I + B, folded block-Jacobi)" % nb,
            "launches": launches, "avg_us": t * 1e6,
            "note": "operator of one stage solve (~%d MB) is re-read across its Arnoldi steps and partly "
                    "L2-resident" % (ne * 3 * nb * nb * word / 1e6)}


def compare_precisions(args):
    """One period of --config (primal sweep, then the adjoint sweep with F = J_E, dF/dmu) from
    the free stream, once in FP64 and once with PP_PREC_MIXED; prints one JSON line with the
    wall times around the public calls and the mixed arm's relative differences in u^(Nt),
    lambda^(0), the QoI rates and dF/dmu."""
    import numpy as np
    import torch

    from paper_1512_00616_gb300 import api as A
    from pp_inputs import CONFIGS, PHYS, config_mesh, config_mu, free_stream_state

    c = CONFIGS[args.config]
    mesh = config_mesh(args.config)
    mu = config_mu(args.config)
    T = PHYS["T"]
    res = {}
    for name, prec in (("fp64", A.PP_PREC_FP64), ("mixed", A.PP_PREC_MIXED)):
        over = dict(gmres_maxit=args.gmres_maxit) if args.gmres_maxit > 0 else {}
        ctx = A.pp_create(A.pp_config_default(p=c["p"], kin=c["kin"], T=T, precision=prec, **over))
        m = A.pp_mesh_create(ctx, mesh.verts, mesh.tris, mesh.ftag)
        ne, _, nu = A.pp_mesh_info(m)
        u0 = torch.tensor(free_stream_state(ne, c["p"]).reshape(-1), dtype=torch.float64, device="cuda")
        uN, lamN, lam0 = torch.zeros_like(u0), torch.zeros_like(u0), torch.zeros_like(u0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        q = A.pp_primal_period(ctx, m, mu, u0, c["Nt"], u_final=uN)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        g = A.pp_adjoint_sweep(ctx, lamN, lam0, weights=np.array([-1.0 / T, 0.0]), n_mu=len(mu))
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        res[name] = dict(uN=uN.cpu().numpy(), lam0=lam0.cpu().numpy(), q=np.asarray(q), g=np.asarray(g),
                         times=[t1 - t0, t2 - t1], counts=A.pp_sweep_counts(ctx), nu=int(nu))
        A.pp_mesh_destroy(m)
        A.pp_destroy(ctx)
    a, b = res["fp64"], res["mixed"]

    def rel(x, y):
        return float(np.linalg.norm(x - y) / np.linalg.norm(y))

    print(json.dumps(dict(config=args.config, dof=a["nu"], Nt=c["Nt"], p=c["p"],
                          u_Nt_rel=rel(b["uN"], a["uN"]), lam0_rel=rel(b["lam0"], a["lam0"]),
                          qoi_rel=float(np.max(np.abs(b["q"] - a["q"]) / np.maximum(np.abs(a["q"]), 1e-300))),
                          grad_rel=rel(b["g"], a["g"]), fp64_s=a["times"], mixed_s=b["times"],
                          counts_fp64=str(a["counts"]), counts_mixed=str(b["counts"]))))


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
    if args.oracle_stage:
        # helper mode of the cpu_baseline leg: one oracle stage, result as JSON in args.out
        r = oracle_stage(args.oracle_stage)
        with open(args.out, "w") as fh:
            json.dump(r, fh)
        return
    if args.profile_step > 0:
        profile_step(args)
        return
    if args.compare_precisions:
        compare_precisions(args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    from pp_inputs import CONFIGS
    c = CONFIGS[args.config]
    workload = (f"{args.config}: {2 * c['n_theta'] * c['n_r']}-triangle O-grid, p={c['p']}, "
                f"{c['Nt']} DIRK3 steps/period, rigid-body mesh motion (Eq. defmap), CDG viscous terms; "
                f"primal sweep + adjoint sweep (F = J_E, dF/dmu)")

    if args.impl == "reference":
        if rank != 0:
            return
        # The oracle's unit of stage work takes about two minutes on a CPU at full size, so the
        # run times it once: --steps and --warmup do not subdivide it (warm-up is the set-up).
        t0 = time.perf_counter()
        s = oracle_stage(args.config)
        v = s["value"]
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": workload},
                "cpu_baseline": {"value": v, "unit": UNIT, "cores": s["cores"], "kind": "oracle",
                                 "sample": oracle_stage_text(s, args.config)},
                "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
                "wall_s": time.perf_counter() - t0}
        print(json.dumps(line))
        return

    # the oracle's stage runs in its own process on the host cores while the GPU is timed
    collect = start_oracle_stage(args.config) if (not args.no_cpu_baseline and world == 1) else None
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
    fp64, fp64_mhz = A.pp_measure_fp64_peak_clock(local_rank)
    units = res["nu"] * res["Nt"] * 3
    value = whole_job_value(units, res["ms"], world)
    roofs = {k: roofline_for(k, res, peaks, fp64, c, False) for k in KERNELS[args.precision]}
    # the dominant kernel: the class with the larger share of the timed region (timed launches only)
    share = {k: res["kern"][k][1] for k in roofs}
    dom = max(share, key=share.get)
    other = [k for k in roofs if k != dom][0]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": res["ms"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f64+f32", "data": "synthetic",
        "config": {"workload": workload, "precision": args.precision, "dof": res["nu"], "elements": res["ne"],
                   "Nt": res["Nt"], "parallelism": f"replicas x{world}", "l2": l2_note(res, c, args.precision)},
        "roofline": roofs[dom],
        "roofline_next": roofs[other],
        "kernel_ms_timed": {k: res["kern"][k][1] for k in roofs},
        "fp64_fma_peak": {"tflops": fp64, "sm_mhz_in_probe": fp64_mhz,
                          "fma_per_clk_per_sm": (fp64 * 1e12 / 2 / (fp64_mhz * 1e6) / 152) if fp64_mhz else None},
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
    if collect is not None:
        s = collect()
        if "value" in s:
            line["cpu_baseline"] = {"value": s["value"], "unit": UNIT, "cores": s["cores"], "kind": "oracle",
                                    "sample": oracle_stage_text(s, args.config)}
        else:
            line["cpu_baseline"] = {"value": None, "unit": UNIT, "kind": "oracle", "error": s.get("error")}
    print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
