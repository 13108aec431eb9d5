"""Benchmark: factor + solve throughput of the direct DD solver on one GB300.

A step is one pass of the whole hot path over the workload: dd_factor (every
domain's LDL^T with its Schur contribution, auxiliary assembly, block LDL^T
of the auxiliary matrix) followed by dd_solve of one right-hand side (with
FP64 refinement in the mixed form).  Metric: DoF/s = global edge unknowns /
step time (and algorithmic TFLOP/s).  Default workload: the 512-domain box
(n = 41, 497,699 DoFs, jittered bisection, 500..2,477 unknowns per domain),
mixed form; the FP64 form is timed on the same workload beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload batched|plain|large] [--precision mixed|fp64]

With N > 1 (torchrun) every rank solves its own replica (the method has no
exchange step on one problem that this build shards), scaling "weak".
"""
from __future__ import annotations

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

MEASURED = os.path.join(ROOT, "MEASURED_PEAKS.json")
# FP64 FMA throughput of this GB300, measured with an FMA-chain probe (152 SMs, 2.07 GHz)
FP64_DFMA_TFLOPS = 1.196
METRIC = "factor+solve DoF/s & TFLOP/s, mixed vs FP64 GPU form at rel. err <=1e-10"

WORKLOADS = {
    "batched": ("batched_c2", "box n=41 Kuhn tets, 512 jittered-RCB domains (500..2477 unknowns), "
                "per-domain eps_r, 1 edge-current RHS"),
    "medium": ("medium", "box n=24 Kuhn tets, 64 jittered-RCB domains, per-domain eps_r, 1 edge-current RHS"),
    "many": ("multi_rhs_c5", "box n=8 Kuhn tets, 8 equal domains, eps_r=2-0.1j, 64 RHS: 56 edge currents "
             "+ 8 plane waves, factor once"),
    "plain": ("plain_c1", "box n=8 Kuhn tets, 8 equal domains, eps_r=2-0.1j, 1 edge-current RHS"),
    "large": ("large_c4", "box n=65 Kuhn tets, 2048 jittered-RCB domains, per-domain eps_r, 1 edge-current RHS"),
}


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def load_peaks():
    try:
        with open(MEASURED) as fh:
            return json.load(fh), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.device)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle leg (the only place bench.py runs oracle/): one thread, bounded
# ---------------------------------------------------------------------------
def oracle_sample_worker(workload: str, budget_s: float, max_domains: int, out_path: str, with_skyline: bool = False):
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    import femgen
    import oracle
    p = getattr(femgen, WORKLOADS[workload][0])()
    order = np.random.default_rng(7).permutation(p.n_sub)
    t0 = time.perf_counter()
    done = []
    for i in order[:max_domains]:
        sub = p.subs[i]
        fac = oracle.dd.factor_subdomain(sub)                         # A_i = L D L^T
        Fi, duals = oracle.subdomain_schur(sub, fac)                  # F_i
        oracle.ldlt_solve(*fac, sub.f)                                # y_i = A_i^{-1} f_i
        Bt, _ = oracle.local_B(sub)
        lam_i = np.zeros((Bt.shape[1], sub.f.shape[1]), dtype=np.complex128)
        oracle.ldlt_solve(*fac, sub.f - Bt @ lam_i)                   # u_i = A_i^{-1}(f_i - B_i^T lam)
        done.append(int(i))
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    # O2's factor memory: skyline (envelope) of the undecomposed RCM-ordered system (untimed)
    sky = oracle.envelope_entries(p.A_indptr, p.A_indices) if with_skyline else None
    n3_all = float(sum(float(s.n) ** 3 for s in p.subs))
    n3_s = float(sum(float(p.subs[i].n) ** 3 for i in done))
    t_est = dt * n3_all / n3_s
    with open(out_path, "w") as fh:
        json.dump({"seconds": dt, "domains": done, "n_global": p.n, "t_est": t_est,
                   "value": p.n / t_est, "n3_fraction": n3_s / n3_all, "skyline_entries": sky}, fh)


def run_oracle_sample(workload: str, budget_s: float, max_domains: int = 10 ** 9, with_skyline: bool = False):
    import tempfile
    fd, path = tempfile.mkstemp(suffix=".json")
    os.close(fd)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ("import sys; sys.path.insert(0, %r); import bench; bench.oracle_sample_worker(%r, %r, %r, %r, %r)"
            % (ROOT, workload, budget_s, max_domains, path, with_skyline))
    subprocess.run([sys.executable, "-c", code], env=env, check=True)
    with open(path) as fh:
        r = json.load(fh)
    os.unlink(path)
    return r


def cpu_baseline_entry(r, workload):
    return {"value": r["value"], "unit": "DoF/s", "cores": 1, "kind": "oracle",
            "sample": (f"oracle domain eliminations (LDL^T, F_i, two local solves) of {len(r['domains'])} seeded "
                       f"random domains of the {workload} workload in {r['seconds']:.1f} s on 1 host thread, "
                       f"extrapolated by sum n_i^3 ({100 * r['n3_fraction']:.2f}% sampled) to all domains; "
                       f"the auxiliary-matrix factorization is not in the sample, so this overstates the "
                       f"oracle's throughput")}


# ---------------------------------------------------------------------------
def max_over_ranks(value: float, device: str) -> float:
    """The slowest rank's time: every rank gets the maximum (replicas are timed as one job)."""
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank: int, ranks: int, seconds: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return units_per_rank * ranks / seconds


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reference_arm(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return 0
    values, secs = [], []
    for step in range(args.warmup + args.steps):
        r = run_oracle_sample(args.workload, budget_s=4.0, max_domains=2)
        if step >= args.warmup:
            values.append(r["value"])
            secs.append(r["t_est"])
    v = float(np.median(values))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "DoF/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": float(np.median(secs)) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
            "data": "synthetic", "config": {"workload": WORKLOADS[args.workload][1], "form": "cpu-oracle-fp64"},
            "cpu_baseline": cpu_baseline_entry(r, args.workload),
            "e2e": {"value": v, "unit": "DoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def backward_error(p, u):
    import scipy.sparse as sp
    x = np.zeros(p.n, dtype=np.complex128)
    off = 0
    for s in p.subs:
        x[s.l2g] = u[off:off + s.n, 0]
        off += s.n
    A = p.A_csr()
    r = p.b[:, 0] - A @ x
    return float(np.linalg.norm(r) / (sp.linalg.norm(A) * np.linalg.norm(x) + np.linalg.norm(p.b)))


def time_form(p, precision, args, torch, stream):
    import paper_2002_05019_gb300 as dd
    s = dd.Solver.from_problem(p, precision=precision, stream=stream.cuda_stream, device=torch.cuda.current_device(),
                               time_kernels={"all": 1, "update": 2, "none": 0}[args.kernel_timing],
                               refine_tol=args.refine_tol,
                               pivoting=args.pivoting, update_panels=args.update_panels)
    sched = None
    if precision == "mixed" and not args.no_autotune:
        sched = s.autotune(repeats=2)      # untimed: picks the factor schedule for this workload
    f_host = dd.stacked_loads(p)
    f_dev = torch.from_numpy(f_host).cuda()
    for _ in range(args.warmup):
        s.factor()
        s.solve(f_dev)
    torch.cuda.synchronize()
    if args.ws > 1:
        torch.distributed.barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    kms, kl, kfl = {}, {}, {}
    launches = 0
    iters = []
    with ClockSampler(torch.cuda.current_device()) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            s.factor()
            u, lam = s.solve(f_dev)
            st = s.stats()
            for c in st["kernel_ms"]:
                kms[c] = kms.get(c, 0.0) + st["kernel_ms"][c]
                kl[c] = kl.get(c, 0) + st["kernel_launches"][c]
                kfl[c] = kfl.get(c, 0.0) + st["kernel_flops"][c]
            launches += st["launches_factor"] + st["launches_solve"]
            iters.append(st["refine_iters"])
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    if args.ws > 1:
        ms = max_over_ranks(ms, "cuda")
    st = s.stats()
    u_host = u.cpu().numpy()
    res = {"ms_per_step": ms / args.steps, "stats": st, "kernel_ms": kms, "kernel_launches": kl,
           "kernel_flops": kfl, "launches": launches, "refine_iters": iters,
           "backward_error": backward_error(p, u_host), "clocks": clk.summary(), "schedule": sched}

    # end to end through the C ABI with host buffers: new values + factor + solve
    if not args.no_e2e:
        vals = np.concatenate([sub.data for sub in p.subs])
        vals_pin = torch.from_numpy(vals).pin_memory()
        f_pin = torch.from_numpy(np.ascontiguousarray(f_host.T)).pin_memory()   # column-major f
        u_pin = torch.empty_like(f_pin).pin_memory()
        import ctypes as C
        lib = dd.load()
        n_loc = f_host.shape[0]
        nrhs = f_host.shape[1]
        lam_pin = torch.empty((max(p.n_dual, 1) * nrhs,), dtype=torch.complex128).pin_memory()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            lib.dd_set_values(s._h, C.c_void_p(vals_pin.data_ptr()))
            lib.dd_factor(s._h)
            lib.dd_solve(s._h, nrhs, C.c_void_p(f_pin.data_ptr()), n_loc, C.c_void_p(u_pin.data_ptr()), n_loc,
                         C.c_void_p(lam_pin.data_ptr()), max(p.n_dual, 1))
        torch.cuda.synchronize()
        e2e_ms = (time.perf_counter() - t0) * 1e3 / args.steps
        res["e2e"] = {"value": p.n / (e2e_ms * 1e-3), "unit": "DoF/s",
                      "h2d_bytes_per_step": int(vals.nbytes + f_host.nbytes),
                      "d2h_bytes_per_step": int(f_host.nbytes + 16 * p.n_dual * f_host.shape[1]),
                      "ms_per_step": e2e_ms}
    s.free()
    return res


def ours_arm(args):
    import torch
    ws, rank, local = dist_env()
    args.ws = ws
    if ws > 1:
        torch.cuda.set_device(local)
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local))
    import femgen
    import paper_2002_05019_gb300 as dd
    dd.load()
    t0 = time.perf_counter()
    p = getattr(femgen, WORKLOADS[args.workload][0])()
    log(f"[bench] workload {args.workload}: n={p.n} domains={p.n_sub} duals={p.n_dual} "
        f"(generated in {time.perf_counter() - t0:.1f} s)")
    stream = torch.cuda.current_stream()
    forms = {}
    for prec in ([args.precision, "fp64" if args.precision == "mixed" else "mixed"] if not args.single_form
                 else [args.precision]):
        forms[prec] = time_form(p, prec, args, torch, stream)
        log(f"[bench] {prec}: {forms[prec]['ms_per_step']:.2f} ms/step, refine {forms[prec]['refine_iters']}, "
            f"backward err {forms[prec]['backward_error']:.2e}, kernel ms {forms[prec]['kernel_ms']}")
    main = forms[args.precision]
    st = main["stats"]
    t_step = main["ms_per_step"] * 1e-3
    n_dof_total = p.n * ws   # replicas: every rank solves the whole workload
    iters = max(main["refine_iters"]) if main["refine_iters"] else 0
    flops_step = st["flops_factor"] + st["flops_solve"] * (1 + iters) * p.nrhs
    peaks, peaks_src = load_peaks()
    # roofline of the dominant kernel: the trailing update
    upd_ms = main["kernel_ms"].get("update", 0.0)
    upd_n = max(main["kernel_launches"].get("update", 0), 1)
    upd_fl = main["kernel_flops"].get("update", 0.0)
    achieved = upd_fl / (upd_ms * 1e-3) / 1e12 if upd_ms > 0 else None
    if args.precision == "mixed":
        # tcgen05 kind::tf32: dense TF32 peak = measured bf16 peak x nominal TF32/BF16 ratio (1.1 / 2.25);
        # the 3xTF32 split issues 3 tensor passes per algorithmic product
        tf32 = peaks["bf16_tflops"] * (1.1 / 2.25)
        kernel = ("k_update_tc (tcgen05 3xTF32, M=128 N=256 MMAs on 64x128 complex blocks; two-panel K=128 "
                  "passes, one-panel passes for the next column)" if args.update_panels == 2 else
                  "k_update_tc (tcgen05 3xTF32, M=128 N=256 MMAs on 64x128 complex blocks, one panel per pass)")
        bound, peak = "tensor", tf32 / 3.0
        src = (f"TF32 dense {tf32:.0f} TFLOP/s = measured bf16 {peaks['bf16_tflops']:.0f} x 1.1/2.25 "
               f"({peaks_src}); effective complex64 peak = TF32 / 3 split passes")
    else:
        bound, peak, kernel = "alu", FP64_DFMA_TFLOPS, "k_update<double2> (DFMA, 64x64 tiles)"
        src = "measured GB300 DFMA rate (FMA-chain probe, 1.196 TFLOP/s)"
    roofline = {"bound": bound, "kernel": kernel, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": (achieved / peak) if achieved else None, "traffic": None,
                "avg_launch_ms": upd_ms / upd_n, "launches_per_step": upd_n / args.steps,
                "share_of_step": upd_ms / args.steps / main["ms_per_step"], "peak_source": src}
    line = {
        "metric": METRIC, "value": job_value(p.n, ws, t_step), "unit": "DoF/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": main["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c64+f64" if args.precision == "mixed" else "c128", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload][1], "form": args.precision, "n_dofs": p.n,
                   "n_domains": p.n_sub, "n_duals": p.n_dual, "nrhs": p.nrhs, "pivoting": args.pivoting,
                   "update_panels": args.update_panels,
                   "schedule": main.get("schedule"),
                   "l2": "working set (front pool) far larger than the 129 MB L2",
                   "parallelism": f"replicas x{ws}"},
        "tflops": flops_step / t_step / 1e12,
        "refine_iters": iters, "refine_tol": args.refine_tol, "backward_error": main["backward_error"],
        # setup (validation, symbolic analysis, device uploads) is outside the timed step
        "setup_ms": st["t_setup_ms"],
        "roofline": roofline,
        "gpu_launches": main["launches"],
        "clocks": main["clocks"],
        # factor memory (the paper's headline comparison): stored L and D of every front
        "memory": {"factor_bytes": st["bytes_factor"], "device_bytes": st["bytes_device"],
                   "skyline_factor_bytes_c128": None},
    }
    if "e2e" in main:
        line["e2e"] = {k: main["e2e"][k] for k in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step")}
        line["e2e"]["value"] *= ws
    other = [k for k in forms if k != args.precision]
    for k in other:
        f = forms[k]
        line[f"{k}_form"] = {"value": n_dof_total / (f["ms_per_step"] * 1e-3), "ms_per_step": f["ms_per_step"],
                             "tflops": (f["stats"]["flops_factor"] + f["stats"]["flops_solve"] * p.nrhs *
                                        (1 + max(f["refine_iters"] or [0]))) / (f["ms_per_step"] * 1e-3) / 1e12,
                             "backward_error": f["backward_error"], "refine_iters": max(f["refine_iters"] or [0]),
                             "kernel_ms_per_step": {c: v / args.steps for c, v in f["kernel_ms"].items()}}
    line["kernel_ms_per_step"] = {c: v / args.steps for c, v in main["kernel_ms"].items()}
    if rank == 0 and not args.no_cpu_baseline:
        r = run_oracle_sample(args.workload, budget_s=args.cpu_budget, with_skyline=True)
        line["cpu_baseline"] = cpu_baseline_entry(r, args.workload)
        if r.get("skyline_entries"):
            line["memory"]["skyline_factor_bytes_c128"] = 16 * int(r["skyline_entries"])
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="batched", choices=list(WORKLOADS))
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--single-form", action="store_true", help="time only --precision")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--pivoting", type=int, default=0, choices=[0, 1, 2],
                    help="restricted Bunch-Kaufman: 0 none, 1 auxiliary fronts, 2 every front")
    ap.add_argument("--update-panels", type=int, default=2, choices=[1, 2],
                    help="mixed form: panels fused per tensor-core trailing-update pass")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default factor schedule")
    ap.add_argument("--kernel-timing", default="update", choices=["update", "all", "none"],
                    help="CUDA events in the timed factorizations: around the trailing-update launches "
                         "(the roofline kernel; default), around every launch (per-class breakdown, slower), "
                         "or none (no roofline)")
    ap.add_argument("--refine-tol", type=float, default=1e-11,
                    help="mixed form: stop refinement at this relative correction (1e-11 keeps the error <= 1e-10)")
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_arm(args)
    return ours_arm(args)


if __name__ == "__main__":
    sys.exit(main())
