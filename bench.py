"""Benchmark: active cell-steps/s of the finite-volume solidification step.

Default workload: the 128^3 cavity (0.1 x 0.1 x 0.0125 m, 2,097,152 hex
cells) with interior nodes jittered by +-0.2 cell widths and cells, faces and
nodes randomly renumbered; Al-like alloy from 950 K at rest, x = 0 wall at
700 K, x = L wall at 950 K; dt = 1e-3 s; pressure solved to a relative
residual of 1e-8.  A step is one pass of the whole method (tags and
compaction, momentum predictor, pressure Poisson solve with AMG-Krylov, flux
and velocity correction, latent-heat energy loop, crossing times).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl fvs|reference]
                  [--precision fp64|mixed] [--n 128]

Prints one JSON line.  ``--impl reference`` times the CPU oracle (the plain
FP64 implementation written from the paper) on a bounded sample of the same
workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "active cell-steps/s at 1e-8 pressure residual (mixed vs FP64) + UQ samples/s"

# CUDA kernel behind each timed class of the solver's kernel timing (the
# coarse AMG levels run their own sweep kernels; k_jac0 serves every level)
CUDA_NAME = {"residual_vc": "k_resid<double>", "residual_vc_coarse": "k_resid_g<double>",
             "jacobi": "k_jac<double>", "jacobi_coarse": "k_jac_g<double>",
             "jacobi0": "k_jac0<double>", "jacobi0_coarse": "k_jac0<double>",
             "residual_f32": "k_resid<float>", "residual_f32_coarse": "k_resid_g<float>",
             "jacobi_f32": "k_jac<float>", "jacobi_f32_coarse": "k_jac_g<float>",
             "jacobi0_f32": "k_jac0<float>", "jacobi0_f32_coarse": "k_jac0<float>",
             "spmv": "k_spmv_dot", "residual": "k_residual"}
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum of one ncu
# capture, cold cache) per algorithmic byte of the same launches on the 96^3
# cavity, applied to the bench launch (summary under profiles/): k_spmv_dot,
# three launches, 309.46 MB on average against 307.89 MB
DRAM_PER_ALGORITHMIC = {"k_spmv_dot": 309.46 / 307.89}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="fvs", choices=["fvs", "reference"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--n", type=int, default=128, help="cells per axis of the cavity")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-n", type=int, default=20, help="cells per axis of the oracle sample")
    ap.add_argument("--cpu-steps", type=int, default=2)
    ap.add_argument("--no-uq", action="store_true")
    ap.add_argument("--no-mixed", action="store_true", help="skip the mixed-precision leg of an fp64 run")
    ap.add_argument("--prof-steps", type=int, default=3, help="steps with per-kernel event timing")
    ap.add_argument("--uq-n", type=int, default=32, help="cells per axis of the UQ cavity")
    ap.add_argument("--uq-samples", type=int, default=32)
    ap.add_argument("--uq-streams", type=int, default=16)
    ap.add_argument("--no-uq-streams", action="store_true", help="skip the independent-solves UQ baseline")
    ap.add_argument("--uq-max-steps", type=int, default=20000, help="step cap of every UQ sample")
    ap.add_argument("--uq-only", action="store_true", help="only the UQ section (for profiling the batch)")
    ap.add_argument("--uq-dt", type=float, default=2e-3)
    ap.add_argument("--uq-heldout", type=int, default=16, help="held-out plain solves judging the surrogates")
    ap.add_argument("--no-shrink", action="store_true", help="skip the active-fraction segments")
    ap.add_argument("--shrink-steps", type=int, default=10, help="timed steps per active-fraction segment")
    ap.add_argument("--uq-study", choices=["c3", "c4", "c5", "paper"], default=None,
                    help="run one study at its stated size instead of the step benchmark")
    ap.add_argument("--study-steps", type=int, default=0,
                    help="c4: timed steps (0: to full solidification); c3: step cap (0: 60000)")
    ap.add_argument("--c3-h", type=float, default=1e-3, help="c3: voxel side of the casting (m)")
    ap.add_argument("--c3-seconds", type=float, default=900.0, help="c3: wall-clock cap of the casting run (s)")
    return ap.parse_args()


def workload(n):
    from fvs_inputs import cases
    return cases.config_jittered(n=n)


def reduce_over_ranks(dist, ms, act, device):
    """Whole-job figures of a replicated run: the slowest rank's time and the
    active cell-steps of all ranks together."""
    import torch
    t = torch.tensor([float(ms)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    a = torch.tensor([float(act)], device=device, dtype=torch.float64)
    dist.all_reduce(a, op=dist.ReduceOp.SUM)
    return float(t.item()), float(a.item())


def bench_props(precision):
    from fvs_inputs import cases
    return cases.props(p_rtol=1e-8, mom_rtol=1e-10, e_rtol=1e-10, e_tol_T=1e-6, max_e_iters=40,
                       max_krylov_iters=1000, precision=1 if precision == "mixed" else 0)


# ---------------------------------------------------------------------------
# CPU oracle timing (the reference arm and the cpu_baseline key)
# ---------------------------------------------------------------------------
def _oracle_worker(n, steps, warmup, q):
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    import warnings
    warnings.filterwarnings("ignore")
    from fvs_inputs import cases
    from oracle.fv import Oracle
    c = cases.config_jittered(n=n)
    o = Oracle(c["mesh"], bench_props("fp64"))
    for _ in range(max(1, warmup)):   # untimed steps (imports, caches, AB2 history)
        o.step(c["dt"])
    t0 = time.perf_counter()
    act = 0
    for _ in range(steps):
        st = o.step(c["dt"])
        act += st["n_active"]
    dt = time.perf_counter() - t0
    q.put(dict(active_cell_steps=act, seconds=dt))


def host_cpu():
    """Core count and CPU model of this host (the oracle runs on one core)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return dict(nproc=os.cpu_count(), model=model, machine=os.uname().machine)


def cpu_oracle(n, steps, warmup=1):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    env_keep = {k: os.environ.get(k) for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in env_keep:
        os.environ[k] = "1"
    p = ctx.Process(target=_oracle_worker, args=(n, steps, warmup, q))
    p.start()
    r = q.get(timeout=1800)
    p.join()
    for k, v in env_keep.items():
        if v is None:
            os.environ.pop(k, None)
        else:
            os.environ[k] = v
    value = r["active_cell_steps"] / r["seconds"]
    return dict(value=value, unit="active cell-steps/s", cores=1, kind="oracle", host=host_cpu(),
                seconds=round(r["seconds"], 2), steps=steps,
                sample=f"{n}^3 jittered permuted cavity (same physics and dt), {steps} steps after {max(1, warmup)} "
                       f"untimed, single-threaded scipy oracle, {r['seconds']:.1f} s")


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, path):
        self.path = path
        self.proc = None

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0]],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() in ("active", "1"):
                    reasons.add(nm)
        if not sm:
            return None
        return dict(sm_mhz=statistics.median(sm), sm_max_mhz=mx, reasons=sorted(reasons), samples=len(sm))


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_gpu(args):
    import numpy as np
    import torch
    from paper_1810_08572_gb300 import LIB_PATH, build
    if not os.path.exists(LIB_PATH):
        build()
    from paper_1810_08572_gb300 import fvs

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if args.uq_only:
        print(json.dumps(dict(uq=run_uq(fvs, args))), flush=True)
        return
    if args.uq_study:
        run_study(fvs, args)
        return
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    c = workload(args.n)
    props = bench_props(args.precision)
    stream = torch.cuda.Stream()
    mesh = fvs.Mesh(c["mesh"], stream=stream)
    S = fvs.Solver(mesh, props, stream=stream)
    dt = c["dt"]
    for _ in range(args.warmup):
        S.step(dt, 1, allow_not_converged=True)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = Clocks(os.path.join(os.environ.get("TMPDIR", "/tmp"), f"fvs_clocks_{os.getpid()}.csv"))
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    act = 0
    its = []
    torch.cuda.synchronize()
    n_launch0 = fvs.fvs_launch_count()
    nvtx = getattr(torch.cuda, "nvtx", None)
    if nvtx is not None:
        nvtx.range_push("timed")   # lets ncu select the timed steps (--nvtx-include timed/)
    ev0.record(stream)
    for _ in range(args.steps):
        st = S.step(dt, 1, allow_not_converged=True)
        act += st["n_active"]
        its.append(st)
    ev1.record(stream)
    if nvtx is not None:
        nvtx.range_pop()
    torch.cuda.synchronize()
    n_launch = fvs.fvs_launch_count() - n_launch0
    ms = ev0.elapsed_time(ev1)
    ck = clocks.stop()
    ref_fields = None
    if args.precision == "fp64" and not args.no_mixed and rank == 0:
        ref_fields = {k: S.query(k) for k in ("T", "U", "P", "FS")}
    # per-kernel event timing right after the timed region, on the same
    # stream, for --prof-steps further steps (kernels run eagerly while timed)
    S.profile(True)
    for _ in range(args.prof_steps):
        S.step(dt, 1, allow_not_converged=True)
    prof = S.profile_read()
    S.profile(False)
    if dist:
        ms, act = reduce_over_ranks(dist, ms, act, "cuda")
    value = act / (ms / 1e3)

    # roofline of the CUDA kernel with the largest total time (classes that
    # run the same kernel -- several matrices, or every level for k_jac0 --
    # are summed, as the ncu launch list sums launches of one kernel)
    peak, peak_kind = load_peaks()
    groups = {}
    for r in prof:
        cls = r["name"].split("@")[0]
        kern = CUDA_NAME.get(cls, cls)
        g = groups.setdefault(kern, dict(kernel=kern, launches=0, total_ms=0.0, bytes=0.0, classes=[]))
        g["launches"] += r["launches"]
        g["total_ms"] += r["total_ms"]
        g["bytes"] += r["bytes"]
        g["classes"].append(r["name"])
    top = max(groups.values(), key=lambda g: g["total_ms"]) if groups else None
    roof = None
    if top:
        per_launch_bytes = top["bytes"] / top["launches"]
        per_launch_s = top["total_ms"] / top["launches"] / 1e3
        ach = per_launch_bytes / per_launch_s / 1e9
        ratio = DRAM_PER_ALGORITHMIC.get(top["kernel"])
        roof = dict(bound="hbm", kernel=top["kernel"], classes=top["classes"],
                    achieved=round(ach, 1), peak=peak, unit="GB/s", frac=round(ach / peak, 4),
                    traffic=round(per_launch_bytes * ratio) if ratio else None,
                    peak_source=f"{peak_kind} copy bandwidth", launches=top["launches"],
                    share_of_step=round(top["total_ms"] / max(1, args.prof_steps) / (ms / args.steps), 3),
                    bytes_per_launch=per_launch_bytes)

    # the FP64 roof next to the copy bandwidth: an ELL row does one FMA per
    # 12 bytes (8-byte value, 4-byte column), so FP64 SpMV kernels meet both
    fp64 = fvs.measure_fp64_fma()
    if roof:
        W = c_mesh_width(mesh)
        fma_bytes = 12.0 + 20.0 / max(W, 1)          # bytes per FMA of a W-slot row (vectors once per row)
        roof["fp64_fma_gflops_measured"] = round(fp64, 1)
        roof["fp64_roof_gbs"] = round(fp64 / 2.0 * fma_bytes, 1)
        roof["frac_of_fp64_roof"] = round(roof["achieved"] / (fp64 / 2.0 * fma_bytes), 4)

    mixed = None
    if ref_fields is not None:
        mixed = run_mixed(fvs, c, args, stream, torch, ref_fields)

    shrink = None
    if not args.no_shrink and rank == 0:
        shrink = run_shrink(fvs, c, args, stream, torch)

    e2e = None
    if not args.no_e2e and rank == 0:
        e2e = run_e2e(fvs, c, props, args, stream, torch)

    uq = None
    if not args.no_uq and rank == 0:
        uq = run_uq(fvs, args)

    cpu = None
    if not args.no_cpu and rank == 0 and world == 1:
        cpu = cpu_oracle(args.cpu_n, args.cpu_steps, 1)

    nkern = sum(r["launches"] for r in prof)
    line = dict(
        metric=METRIC, value=round(value, 1), unit="active cell-steps/s", n_gpus=world, steps=args.steps,
        warmup=args.warmup, ms_per_step=round(ms / args.steps, 3), higher_is_better=True, scaling="weak",
        vs_baseline=None, dtype="f64" if args.precision == "fp64" else "f64+f32",
        data="synthetic",
        config=dict(workload=f"cavity {args.n}^3 jittered+permuted, dt 1e-3 s, p_rtol 1e-8, "
                             f"{args.precision}", cells=args.n ** 3, dt=dt, p_rtol=1e-8,
                    precision=args.precision, l2="inputs larger than L2 (matrices ~1 GB)",
                    parallelism="replicas" if world > 1 else "single GPU"),
        roofline=roof, cpu_baseline=cpu, e2e=e2e, clocks=ck, uq=uq, mixed=mixed, active_fraction_segments=shrink,
        gpu_launches=int(n_launch),
        kernel_profile=sorted(prof, key=lambda r: -r["total_ms"])[:12],
        step_stats=dict(p_its=[s["p_its"] for s in its], e_its=[s["e_its"] for s in its],
                        e_lin_its=[s["e_lin_its"] for s in its], mom_its=[s["mom_its"] for s in its],
                        p_relres=max(s["p_relres"] for s in its), fallback=sum(s["fallback"] for s in its),
                        amg_levels=its[-1]["amg_levels"], n_active_last=its[-1]["n_active"],
                        p_rebuilt=[s["p_rebuilt"] for s in its], setup_ms=[round(s["setup_ms"], 2) for s in its]),
    )
    line["gpu_launches_profiled"] = nkern
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def c_mesh_width(mesh):
    return int(mesh.info["max_cell_neighbours"])


def run_shrink(fvs, c, args, stream, torch):
    """The paper's claim that work shrinks as the casting freezes (Section
    2.4), measured: segments that start from the 1-D conduction profile
    T(x) = 700 + 250 erf(x/delta) K with delta chosen so that 100, 85, 70, 55
    and 40 % of the cells are liquid or mushy; per segment and precision,
    3 untimed and --shrink-steps timed steps."""
    import numpy as np
    from scipy.special import erf, erfinv
    m = c["mesh"]
    X = np.asarray(m["nodes"])[np.asarray(m["cells"])].mean(axis=1)
    x = X[:, 0]
    L = float(np.asarray(m["nodes"])[:, 0].max())
    z = float(erfinv((833.0 - 700.0) / 250.0))      # erf(x/delta) at the solidus
    out = []
    mesh = fvs.Mesh(m, stream=stream)
    for frac in (1.0, 0.85, 0.70, 0.55, 0.40):
        T0 = np.full(len(x), 950.0) if frac >= 1.0 else 700.0 + 250.0 * erf(x / ((1.0 - frac) * L / z))
        row = dict(target_active=frac, active_at_start=round(float((T0 > 833.0).mean()), 4))
        for prec in ("fp64", "mixed"):
            S = fvs.Solver(mesh, bench_props(prec), stream=stream)
            S.set_state(T0)
            for _ in range(3):
                S.step(c["dt"], 1, allow_not_converged=True)
            torch.cuda.synchronize()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            act, p_its, setup, rebuilt = 0, [], [], []
            ev0.record(stream)
            for _ in range(args.shrink_steps):
                st = S.step(c["dt"], 1, allow_not_converged=True)
                act += st["n_active"]
                p_its.append(st["p_its"])
                setup.append(st["setup_ms"])
                rebuilt.append(st["p_rebuilt"])
            ev1.record(stream)
            torch.cuda.synchronize()
            ms = ev0.elapsed_time(ev1)
            # where the step goes: two more steps with per-kernel event timing,
            # the sparse kernels summed by the system they work on
            S.profile(True)
            for _ in range(2):
                S.step(c["dt"], 1, allow_not_converged=True)
            by = {}
            for r in S.profile_read():
                sysname = r["name"].split("@")[-1]
                by[sysname] = by.get(sysname, 0.0) + r["total_ms"] / 2.0
            S.profile(False)
            row[prec] = dict(value=round(act / (ms / 1e3), 1), ms_per_step=round(ms / args.shrink_steps, 3),
                             mean_active=round(act / args.shrink_steps), p_its=round(float(np.mean(p_its)), 1),
                             pressure_setup_ms_per_step=round(float(np.mean(setup)), 2), p_rebuilt=rebuilt,
                             sparse_kernel_ms_per_step={k: round(v, 2) for k, v in sorted(by.items())})
            S.close()
        out.append(row)
    mesh.close()
    return out


UQ_FAMILIES = (0, 1, 1)        # melt ~ normal, wall and C0 ~ uniform (fvs_pce families)
UQ_PARAMS = ((950.0, 10.0), (650.0, 750.0), (3.0, 5.0))


def judge_surrogates(fvs, X, Y, Xte, Yte, mc_n=1000000, epochs=2000, pce_degree=2):
    """MLP (BF16 tensor cores) and polynomial chaos (Eq. 27-28, least squares
    on the same training solves) judged on held-out plain solves of the same
    inputs (paired), then both on mc_n Monte Carlo inputs."""
    import numpy as np
    from fvs_inputs import cases
    out = {}
    S = fvs.Surrogate(3, 128, 4, 4, seed=1)
    S.set_scaling(X.mean(0), X.std(0), Y.mean(0), Y.std(0))
    t0 = time.perf_counter()
    S.train(X, Y, epochs, 1e-3)
    train_s = time.perf_counter() - t0
    P = fvs.Pce(UQ_FAMILIES, UQ_PARAMS, pce_degree, 4)
    P.fit(X, Y)
    Xmc = cases.uq_inputs(mc_n, seed=4)
    for name, model in (("mlp", S.predict), ("pce", P)):
        Yp = model(Xte)
        rel = np.abs(Yp - Yte) / np.abs(Yte)
        model(Xmc[:4096])
        t1 = time.perf_counter()
        Ymc = model(Xmc)
        rate = len(Xmc) / (time.perf_counter() - t1)
        out[name] = dict(heldout_mean_rel_err=[round(float(v), 5) for v in rel.mean(0)],
                         heldout_max_rel_err=[round(float(v), 5) for v in rel.max(0)],
                         heldout_paired_mean_gap=[round(float(v), 5) for v in
                                                  (Yp.mean(0) - Yte.mean(0)) / np.abs(Yte.mean(0))],
                         mc_mean=[float(v) for v in Ymc.mean(0)], mc_var=[float(v) for v in Ymc.var(0)],
                         samples_per_s=round(rate, 1))
    out["mlp"]["train_s"] = round(train_s, 2)
    _, var, total, first = P.sensitivity()
    out["pce"].update(degree=pce_degree, terms=P.num_terms(), sobol_total=total.round(4).tolist(),
                      sobol_first=first.round(4).tolist(), variance=var.tolist())
    # plain Monte Carlo reference: every plain solve, mean +- standard error
    Yall = np.concatenate([Y, Yte])
    out["plain_mc"] = dict(n=len(Yall), mean=[float(v) for v in Yall.mean(0)],
                           std_err=[float(v) for v in Yall.std(0, ddof=1) / np.sqrt(len(Yall))],
                           var=[float(v) for v in Yall.var(0, ddof=1)])
    return out


def run_uq(fvs, args):
    """UQ samples/s: plain batched solves to full solidification (lockstep,
    mixed precision), the same samples as independent FP64 and mixed solves,
    and the two surrogates trained on them, judged on held-out solves."""
    import numpy as np
    from fvs_inputs import box_mesh, cases
    n = args.uq_n
    m = box_mesh(n, n, n, cases.CAVITY)
    M = fvs.Mesh(m)
    props = bench_props("mixed")
    X = cases.uq_inputs(args.uq_samples, seed=2018)
    t0 = time.perf_counter()
    Y, steps = fvs.uq_batch(M, props, X, args.uq_dt, args.uq_max_steps, mode=fvs.UQ_LOCKSTEP)
    sec = time.perf_counter() - t0
    plain = args.uq_samples / sec
    lock64 = None
    streams = None
    if not args.no_uq_streams:
        # equal-precision comparison: lockstep FP64 against independent FP64
        # solves on streams, then independent solves with the FP32 V-cycle
        t0 = time.perf_counter()
        Yl, _ = fvs.uq_batch(M, bench_props("fp64"), X, args.uq_dt, args.uq_max_steps, mode=fvs.UQ_LOCKSTEP)
        lock64 = round(args.uq_samples / (time.perf_counter() - t0), 3)
        t0 = time.perf_counter()
        Y1, steps1 = fvs.uq_batch(M, bench_props("fp64"), X, args.uq_dt, args.uq_max_steps, n_streams=args.uq_streams,
                                  mode=fvs.UQ_STREAMS)
        s64 = args.uq_samples / (time.perf_counter() - t0)
        t0 = time.perf_counter()
        fvs.uq_batch(M, props, X, args.uq_dt, args.uq_max_steps, n_streams=args.uq_streams, mode=fvs.UQ_STREAMS)
        s32 = args.uq_samples / (time.perf_counter() - t0)
        streams = dict(fp64_samples_per_s=round(s64, 3), mixed_samples_per_s=round(s32, 3), streams=args.uq_streams,
                       max_rel_qoi_diff_vs_lockstep=float(np.nanmax(np.abs(Y1 - Yl) / np.abs(Y1))),
                       steps_equal=bool(np.array_equal(steps1, steps)))
    sur = None
    if args.uq_heldout > 0 and np.all(np.isfinite(Y)):
        Xte = cases.uq_inputs(args.uq_heldout, seed=2019)
        Yte, _ = fvs.uq_batch(M, props, Xte, args.uq_dt, args.uq_max_steps, mode=fvs.UQ_LOCKSTEP)
        sur = judge_surrogates(fvs, X, Y, Xte, Yte)
    return dict(plain_samples_per_s=round(plain, 3), unit="samples/s", samples=args.uq_samples,
                mesh=f"cavity {n}^3, all walls at the sampled temperature", dt=args.uq_dt,
                mean_steps=float(np.mean(steps)),
                mode="lockstep (one launch per phase for all samples), mixed precision",
                lockstep_fp64_samples_per_s=lock64, independent_solves=streams,
                batching_gain_fp64=round(lock64 / streams["fp64_samples_per_s"], 3) if streams else None,
                surrogates=sur,
                note="plain: fvs_uq_batch to full solidification; surrogates trained on those solves, judged on "
                     f"{args.uq_heldout} held-out plain solves (paired) and on 1e6 Monte Carlo inputs")


def run_study(fvs, args):
    """One UQ study at its stated size (not part of the step benchmark).
    c4: 256 samples on the 64^3 cavity, lockstep, mixed precision, to full
    solidification or for --study-steps timed steps (then extrapolated by
    the step count of a 32^3 run of the same samples, stated).
    c5: 512 training and 64 held-out plain solves of the 48^3 cavity; the
    MLP and the polynomial chaos judged on the held-out ones (paired) and on
    1e6 Monte Carlo inputs.
    paper: the study of Section 5 (Al-Si, its input distributions,
    convection off, grain growth, the four domain outputs) on the 64^3
    cavity with 216 tensor collocation points (Table 2's level 6) and 60
    Latin-hypercube test solves."""
    import numpy as np
    from fvs_inputs import box_mesh, cases
    t_start = time.perf_counter()
    out = dict(study=args.uq_study)
    if args.uq_study == "c3":
        out.update(run_casting(fvs, args))
    elif args.uq_study == "c4":
        m = box_mesh(64, 64, 64, cases.CAVITY)
        M = fvs.Mesh(m)
        X = cases.uq_inputs(256, seed=2018)
        cap = args.study_steps if args.study_steps > 0 else args.uq_max_steps
        t0 = time.perf_counter()
        Y, steps = fvs.uq_batch(M, bench_props("mixed"), X, args.uq_dt, cap, mode=fvs.UQ_LOCKSTEP)
        sec = time.perf_counter() - t0
        out.update(samples=256, mesh="cavity 64^3", dt=args.uq_dt, seconds=round(sec, 2),
                   steps_max=int(steps.max()), steps_mean=float(steps.mean()))
        if args.study_steps > 0:
            m32 = box_mesh(32, 32, 32, cases.CAVITY)
            _, s32 = fvs.uq_batch(fvs.Mesh(m32), bench_props("mixed"), X, args.uq_dt, args.uq_max_steps,
                                  mode=fvs.UQ_LOCKSTEP)
            full = float(s32.max())
            out.update(extrapolated=True, steps_to_solidify_32=full,
                       samples_per_s=round(256 / (sec * full / cap), 4),
                       note=f"{cap} timed steps of all 256 samples, scaled to the {full:.0f} steps the last sample "
                            "of the same inputs needs on the 32^3 cavity")
        else:
            out.update(extrapolated=False, samples_per_s=round(256 / sec, 4), qoi_mean=Y.mean(0).tolist())
    elif args.uq_study == "c5":
        m = box_mesh(48, 48, 48, cases.CAVITY)
        M = fvs.Mesh(m)
        props = bench_props("mixed")
        X = cases.uq_inputs(512, seed=1)
        t0 = time.perf_counter()
        Y, steps = fvs.uq_batch(M, props, X, args.uq_dt, args.uq_max_steps, mode=fvs.UQ_LOCKSTEP)
        sec = time.perf_counter() - t0
        Xte = cases.uq_inputs(64, seed=2)
        Yte, _ = fvs.uq_batch(M, props, Xte, args.uq_dt, args.uq_max_steps, mode=fvs.UQ_LOCKSTEP)
        out.update(train=512, heldout=64, mesh="cavity 48^3", plain_samples_per_s=round(512 / sec, 4),
                   mean_steps=float(steps.mean()), surrogates=judge_surrogates(fvs, X, Y, Xte, Yte, pce_degree=3))
    else:
        m = box_mesh(64, 64, 64, cases.CAVITY)
        M = fvs.Mesh(m)
        props = bench_props("mixed")
        props["material"] = dict(cases.AL_SI_PAPER)
        props["no_flow"] = True
        fam = (0, 0, 0)
        par = ((1000.0, 10.0), (500.0, 5.0), (10.0, 0.2))
        kw = dict(qoi_kind=fvs.QOI_EXTREMES, liquidus=(cases.AL_SI_T_F, cases.AL_SI_SLOPE),
                  grain=dict(kp=cases.AL_SI_PAPER["kp"], D_s=3e-9, r0=1e-6))
        res = {}
        for level, deg in ((3, 2), (6, 4)):
            P = fvs.Pce(fam, par, deg, 4)
            Xc = P.nodes(level)
            t0 = time.perf_counter()
            Yc, st, _ = fvs.uq_run(M, props, Xc, args.uq_dt, args.uq_max_steps, mode=fvs.UQ_LOCKSTEP, **kw)
            sec = time.perf_counter() - t0
            P.fit(Xc, Yc)
            res[level] = (P, len(Xc), sec, float(st.mean()))
        Xt = cases.latin_hypercube_normal([p[0] for p in par], [p[1] for p in par], 60, seed=7)
        Yt, _, _ = fvs.uq_run(M, props, Xt, args.uq_dt, args.uq_max_steps, mode=fvs.UQ_LOCKSTEP, **kw)
        rows = []
        for level, (P, npts, sec, mst) in res.items():
            err = np.sqrt(np.mean((P(Xt) - Yt) ** 2, axis=0)) / np.abs(Yt.mean(0))
            mean, var, total, first = P.sensitivity()
            rows.append(dict(level=level, points=npts, plain_seconds=round(sec, 2), mean_steps=mst,
                             rms_error_over_mean=[float(v) for v in err], sobol_total=total.round(4).tolist(),
                             mean=mean.tolist(), std=np.sqrt(var).tolist()))
        out.update(mesh="cavity 64^3, Al-Si (Scheil), convection off, grain growth", levels=rows,
                   outputs=["total solidification time (s)", "max SDAS (um)", "min yield (MPa)", "max grain (m)"],
                   inputs=["T_init ~ N(1000, 10) K", "T_wall ~ N(500, 5) K", "C0 ~ N(10, 0.2) wt%"])
    out["wall_seconds"] = round(time.perf_counter() - t_start, 1)
    print(json.dumps(out), flush=True)


def run_casting(fvs, args):
    """C3: the plate casting in its steel mold (fvs_inputs.cases.config_casting
    at voxel side --c3-h), mixed precision, stepped until no metal cell is
    liquid or mushy (or the step / wall-clock cap).  Each step is timed on
    the host around a synchronising step call; the steps are binned by the
    share of metal cells still liquid or mushy at the step, which is how the
    paper's claim that the work shrinks as the casting freezes shows on a
    casting rather than on a prepared profile."""
    import numpy as np
    import torch
    from fvs_inputs import cases
    c = cases.config_casting(args.c3_h)
    m = c["mesh"]
    zone = np.asarray(m["cell_zone"])
    n_metal = int((zone == 0).sum())
    M = fvs.Mesh(m)
    S = fvs.Solver(M, c["props"])
    dt = c["dt"]
    cap = args.study_steps if args.study_steps > 0 else 60000
    rows = []
    S.step(dt, 1, allow_not_converged=True)    # first step: set-up of every system
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(cap):
        a = time.perf_counter()
        st = S.step(dt, 1, allow_not_converged=True)
        b = time.perf_counter()
        rows.append((b - a, st["n_active"], st["p_its"], st["p_rebuilt"]))
        if st["n_active"] == 0 or b - t0 > args.c3_seconds:
            break
    total = time.perf_counter() - t0
    S.close()
    M.close()
    act = np.array([r[1] for r in rows], dtype=np.float64)
    return dict(mesh=f"plate casting in a steel mold, voxels of {args.c3_h * 1e3:.2f} mm", cells=len(zone),
                metal_cells=n_metal, dt=dt, precision="mixed", steps=len(rows),
                solidified=bool(act[-1] == 0), physical_seconds=round(len(rows) * dt, 3),
                seconds=round(total, 2), value=round(float(act.sum() / total), 1), unit="active cell-steps/s",
                bands=active_share_bands(rows, n_metal))


def active_share_bands(rows, n_metal):
    """Steps (seconds, active cells, pressure iterations, p_rebuilt) binned by
    the share of metal cells still liquid or mushy: 0.8-1.0, 0.6-0.8, ...,
    0.0-0.2 (steps with no active cell left out); per band the step count,
    mean ms a step, mean iterations, full AMG setups and active cell-steps/s."""
    import numpy as np
    sec = np.array([r[0] for r in rows], dtype=np.float64)
    act = np.array([r[1] for r in rows], dtype=np.float64)
    its = np.array([r[2] for r in rows], dtype=np.float64)
    full = np.array([r[3] == 1 for r in rows])
    frac = act / n_metal
    bands = []
    for hi, lo in ((1.01, 0.8), (0.8, 0.6), (0.6, 0.4), (0.4, 0.2), (0.2, 0.0)):
        sel = (frac < hi) & (frac >= lo) & (act > 0)
        if sel.any():
            bands.append(dict(active_share=f"{lo:.1f}-{min(hi, 1.0):.1f}", steps=int(sel.sum()),
                              ms_per_step=round(float(sec[sel].mean() * 1e3), 3),
                              p_its=round(float(its[sel].mean()), 1), rebuilds=int(full[sel].sum()),
                              active_cell_steps_per_s=round(float(act[sel].sum() / sec[sel].sum()), 1)))
    return bands


def run_mixed(fvs, c, args, stream, torch, ref):
    """The same steps with the FP32 V-cycle inside the FP64 Krylov method:
    throughput timed like the FP64 run (same warm-up and step count, CUDA
    events on the solver stream) and the difference of each field from the
    FP64 run after those steps."""
    import numpy as np
    mesh = fvs.Mesh(c["mesh"], stream=stream)
    S = fvs.Solver(mesh, bench_props("mixed"), stream=stream)
    dt = c["dt"]
    for _ in range(args.warmup):
        S.step(dt, 1, allow_not_converged=True)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    act, p_its = 0, []
    ev0.record(stream)
    for _ in range(args.steps):
        st = S.step(dt, 1, allow_not_converged=True)
        act += st["n_active"]
        p_its.append(st["p_its"])
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    got = {k: S.query(k) for k in ref}
    S.close()
    mesh.close()

    def rel(a, b):
        return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))

    return dict(value=round(act / (ms / 1e3), 1), unit="active cell-steps/s",
                ms_per_step=round(ms / args.steps, 3), p_its=p_its,
                err_vs_fp64=dict(T_max_abs_K=float(np.abs(got["T"] - ref["T"]).max()),
                                 fs_max_abs=float(np.abs(got["FS"] - ref["FS"]).max()),
                                 u_rel=rel(got["U"], ref["U"]), p_rel=rel(got["P"], ref["P"])),
                note="FP32 V-cycle inside FP64 BiCGStab, same 1e-8 pressure residual; errors after "
                     f"{args.warmup + args.steps} steps, max over cells, relative to the largest FP64 value")


def run_e2e(fvs, c, props, args, stream, torch):
    """Same metric through the public API from host buffers: mesh upload and
    set-up, the steps, and the fields read back, all inside the timed region."""
    import numpy as np
    m = c["mesh"]
    h2d = sum(np.asarray(m[k]).nbytes for k in ("nodes", "cells", "faces", "face_cells", "patch"))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    mesh = fvs.Mesh(m, stream=stream)
    S = fvs.Solver(mesh, props, stream=stream)
    act = 0
    k = max(1, args.steps)
    for _ in range(k):
        act += S.step(c["dt"], 1, allow_not_converged=True)["n_active"]
    T = S.query("T")
    U = S.query("U")
    P = S.query("P")
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    d2h = T.nbytes + U.nbytes + P.nbytes
    S.close()
    mesh.close()
    return dict(value=round(act / sec, 1), unit="active cell-steps/s", h2d_bytes_per_step=int(h2d / k),
                d2h_bytes_per_step=int(d2h / k), steps=k,
                note="mesh upload, renumbering and geometry, solver set-up, steps, T/u/p read back")


def run_reference(args):
    """The oracle as it stands on the host cores: --warmup untimed and
    --steps timed steps of a bounded sample (--cpu-n^3 cells) of the bench
    workload; ms_per_step is per sample step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    steps = max(1, args.steps)
    cpu = cpu_oracle(args.cpu_n, steps, args.warmup)
    line = dict(impl="reference", metric=METRIC, value=round(cpu["value"], 2), unit="active cell-steps/s",
                n_gpus=args.gpus, steps=steps, warmup=args.warmup,
                ms_per_step=round(1e3 * cpu["seconds"] / steps, 3), higher_is_better=True,
                scaling="weak", vs_baseline=None, dtype="f64", data="synthetic",
                config=dict(workload=f"cavity {args.n}^3 jittered+permuted, dt 1e-3 s, p_rtol 1e-8, "
                                     f"{args.precision}", cpu_sample_cells=args.cpu_n ** 3,
                            sample="each step is one oracle step on the sample, not on the full mesh"),
                cpu_baseline=cpu,
                e2e=dict(value=round(cpu["value"], 2), unit="active cell-steps/s", h2d_bytes_per_step=0,
                         d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
