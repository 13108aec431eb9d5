"""Benchmark: factor + solve throughput of the direct DD solver on one GB300.

A step is one pass of the whole hot path over the workload: dd_factor (every
domain's LDL^T with its Schur contribution, auxiliary assembly, block LDL^T
of the auxiliary matrix) followed by dd_solve of one right-hand side (with
FP64 refinement in the mixed form).  Metric: DoF/s = global edge unknowns /
step time (and algorithmic TFLOP/s).

Default headline workload: the largest single-GPU machine, n = 65 (1,960,595
DoFs, 2,048 jittered-bisection domains of 500..2,500 unknowns, about 0.5 M
duals), mixed form.  Beside it ("compare"), the 512-domain box (n = 41,
497,699 DoFs) in both the mixed and the FP64 form: the mixed-vs-FP64
comparison on one mesh.  Every result carries its relative error (2-norm and
max-norm) against the exact discrete solution of the linear field a + b x r,
solved with the same factors, and the pivot growth of the factorization.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload large|batched|plain|medium|many] [--precision mixed|fp64]

With N > 1 (torchrun) every rank solves its own replica (the library runs one
problem on one GPU; its subtree shard plan, dd_shard_plan, has no GPU
multi-rank engine), scaling "weak".
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
# nominal FP64 rate of GB300 (the FP64 form is bound by its DFMA pipe; no measured figure exists)
FP64_DFMA_TFLOPS = 1.25
METRIC = "factor+solve DoF/s & TFLOP/s, mixed vs FP64 GPU form at rel. err <=1e-10"

WORKLOADS = {
    "large": ("large_c4", "box n=65 Kuhn tets, 2048 jittered-RCB domains (500..2500 unknowns), per-domain eps_r, "
              "1 edge-current RHS"),
    "batched": ("batched_c2", "box n=41 Kuhn tets, 512 jittered-RCB domains (500..2477 unknowns), "
                "per-domain eps_r, 1 edge-current RHS"),
    "medium": ("medium", "box n=24 Kuhn tets, 64 jittered-RCB domains, per-domain eps_r, 1 edge-current RHS"),
    "many": ("multi_rhs_c5", "box n=8 Kuhn tets, 8 equal domains, eps_r=2-0.1j, 64 RHS: 56 edge currents "
             "+ 8 plane waves, factor once"),
    "plain": ("plain_c1", "box n=8 Kuhn tets, 8 equal domains, eps_r=2-0.1j, 1 edge-current RHS"),
    "big": ("big_domains", "box n=24 Kuhn tets, 8 equal domains of 13,428 unknowns, eps_r=2-0.1j, 1 edge-current RHS"),
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
# CPU oracle leg (the only place bench.py runs oracle/), in a spawned process
# so that its BLAS thread count is fixed before numpy loads
# ---------------------------------------------------------------------------
def pick_subtree(parent, n_sub: int, n_domains: int) -> int:
    """The first (lowest-id) tree node whose subtree holds about n_domains domains."""
    parent = np.asarray(parent)
    count = np.zeros(parent.size, dtype=np.int64)
    count[:n_sub] = 1
    for x in range(parent.size - 1):             # parents carry larger ids than children
        if parent[x] >= 0:
            count[parent[x]] += count[x]
    cand = np.nonzero(count >= min(n_domains, n_sub))[0]
    return int(cand[np.argmin(count[cand])])


def skyline_worker(workload: str, out_path: str, repeats: int = 1):
    """Time the oracle's undecomposed route O2 (RCM + band LDL^T of the global
    system, then the solve) on the whole workload, `repeats` times."""
    import femgen
    import oracle
    p = getattr(femgen, WORKLOADS[workload][0])()
    runs = []
    for _ in range(repeats):
        t0 = time.perf_counter()
        o = oracle.BandLDLT(p.A_indptr, p.A_indices, p.A_data).factor()
        t1 = time.perf_counter()
        o.solve(p.b)
        t2 = time.perf_counter()
        runs.append((t2 - t0, t1 - t0, t2 - t1))
    sec, fac, sol = runs[-1]
    with open(out_path, "w") as fh:
        json.dump({"seconds": sec, "factor_s": fac, "solve_s": sol, "runs": [r[0] for r in runs],
                   "domains": p.n_sub, "fronts": 0, "n_global": p.n, "n_sub": p.n_sub, "dofs": p.n,
                   "value": p.n / sec, "skyline_entries": None, "route": "skyline"}, fh)


def oracle_sample_worker(workload: str, n_domains: int, out_path: str, with_skyline: bool = False,
                         repeats: int = 1):
    """Time the oracle's complete DD route (oracle.TreeDDOracle: domain LU,
    F_i, block elimination of F over the front tree, forward and backward
    substitution, primal recovery) restricted to the domains and separator
    fronts of one subtree of the workload's domain tree, `repeats` times."""
    import femgen
    import oracle
    p = getattr(femgen, WORKLOADS[workload][0])()
    node = pick_subtree(p.rcb.parent, p.n_sub, n_domains)
    runs = []
    for _ in range(repeats):
        t0 = time.perf_counter()
        o = oracle.TreeDDOracle(p, subtree=node)
        t1 = time.perf_counter()
        o.solve([s.f for s in p.subs])
        t2 = time.perf_counter()
        runs.append((t2 - t0, t1 - t0, t2 - t1))
    dofs = int(np.unique(np.concatenate([p.subs[i].l2g for i in o.domains])).size)
    sky = oracle.envelope_entries(p.A_indptr, p.A_indices) if with_skyline else None   # untimed
    sec, fac, sol = runs[-1]
    with open(out_path, "w") as fh:
        json.dump({"seconds": sec, "factor_s": fac, "solve_s": sol, "runs": [r[0] for r in runs],
                   "domains": len(o.domains), "fronts": len(o.fronts), "n_global": p.n, "n_sub": p.n_sub,
                   "dofs": dofs, "value": dofs / sec, "skyline_entries": sky}, fh)


def run_oracle_sample(workload: str, n_domains: int, threads: int, with_skyline: bool = False, repeats: int = 1,
                      route: str = "tree"):
    """Run oracle_sample_worker (or skyline_worker) in a fresh interpreter with `threads` BLAS threads."""
    import tempfile
    fd, path = tempfile.mkstemp(suffix=".json")
    os.close(fd)
    t = str(threads)
    env = dict(os.environ, OMP_NUM_THREADS=t, OPENBLAS_NUM_THREADS=t, MKL_NUM_THREADS=t)
    if route == "skyline":
        code = ("import sys; sys.path.insert(0, %r); import bench; bench.skyline_worker(%r, %r, %r)"
                % (ROOT, workload, path, repeats))
    else:
        code = ("import sys; sys.path.insert(0, %r); import bench; bench.oracle_sample_worker(%r, %r, %r, %r, %r)"
                % (ROOT, workload, n_domains, path, with_skyline, repeats))
    subprocess.run([sys.executable, "-c", code], env=env, check=True)
    with open(path) as fh:
        r = json.load(fh)
    os.unlink(path)
    r["threads"] = threads
    return r


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline_entry(r, workload):
    if r.get("route") == "skyline":
        return {"value": r["value"], "unit": "DoF/s", "cores": r["threads"], "kind": "oracle",
                "sample": (f"oracle undecomposed route O2 (RCM + band LDL^T of the global system, solve) on the "
                           f"whole {workload} workload ({r['dofs']} DoFs): {r['seconds']:.1f} s (factor "
                           f"{r['factor_s']:.1f} s, solve {r['solve_s']:.2f} s) on {r['threads']} host threads "
                           f"of {host_cores()}")}
    return {"value": r["value"], "unit": "DoF/s", "cores": r["threads"], "kind": "oracle",
            "sample": (f"oracle tree route (domain LU, F_i, block elimination of F over the domain tree, "
                       f"forward/backward substitution, primal recovery) on the {r['domains']} domains and "
                       f"{r['fronts']} separator fronts of one subtree of the {workload} workload "
                       f"({r['dofs']} distinct DoFs of {r['n_global']}), timed in full: {r['seconds']:.1f} s "
                       f"(factor {r['factor_s']:.1f} s, solve {r['solve_s']:.2f} s) on {r['threads']} host "
                       f"threads of {host_cores()}" + ("; the whole workload" if r["domains"] == r["n_sub"] else
                                                          "; the separators above the subtree are not in the sample"))}


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
    """The oracle as it stands, timed on the host cores: each step is one full
    run of the oracle's tree route on a subtree sample of the workload."""
    ws, rank, local = dist_env()
    if rank != 0:
        return 0
    threads = args.ref_threads or host_cores()
    t_run = time.perf_counter()
    r = run_oracle_sample(args.workload, args.ref_domains, threads, repeats=args.warmup + args.steps,
                          route=args.ref_route)
    secs = r["runs"][args.warmup:]
    log(f"[bench] reference arm: {args.warmup + args.steps} oracle runs in {time.perf_counter() - t_run:.1f} s")
    v = r["dofs"] / float(np.mean(secs))
    base = cpu_baseline_entry(r, args.workload)
    base["value"] = v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "DoF/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": float(np.mean(secs)) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
            "data": "synthetic", "config": {"workload": WORKLOADS[args.workload][1], "form": "cpu-oracle-fp64",
                                            "sample_domains": r["domains"], "sample_dofs": r["dofs"]},
            "cpu_baseline": base,
            "e2e": {"value": v, "unit": "DoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def gather_x(p, u):
    """Global vector from stacked local copies (lowest-index domain's copy)."""
    x = np.zeros((p.n,) + u.shape[1:], dtype=np.complex128)
    seen = np.zeros(p.n, dtype=bool)
    off = 0
    for s in p.subs:
        new = ~seen[s.l2g]
        x[s.l2g[new]] = u[off:off + s.n][new]
        seen[s.l2g] = True
        off += s.n
    return x


def backward_error(p, u):
    import scipy.sparse as sp
    x = gather_x(p, u[:, :1])[:, 0]
    A = p.A_csr()
    r = p.b[:, 0] - A @ x
    return float(np.linalg.norm(r) / (sp.linalg.norm(A) * np.linalg.norm(x) + np.linalg.norm(p.b)))


def accuracy(p, s, torch):
    """Error of a solve with the factors in place against an exact discrete
    solution: the linear field a + b x r on the same mesh and materials."""
    import femgen
    import paper_2002_05019_gb300 as dd
    f_lin, x_lin = femgen.linear_field_loads(p)
    u, _ = s.solve(torch.from_numpy(np.concatenate(f_lin, axis=0)).cuda())
    x = gather_x(p, u.cpu().numpy())
    st = s.stats()
    return {"rel_err": float(np.linalg.norm(x - x_lin) / np.linalg.norm(x_lin)),
            "rel_err_max": float(np.abs(x - x_lin).max() / np.abs(x_lin).max()),
            "against": "exact discrete solution (edge interpolant of E = a + b x r), same factors",
            "refine_iters": int(st["refine_iters"]), "growth": float(st["growth"]),
            "min_pivot": float(st["min_pivot"])}


def time_form(p, precision, args, torch, stream, steps, warmup, e2e=True, autotune=True):
    import paper_2002_05019_gb300 as dd
    s = dd.Solver.from_problem(p, precision=precision, stream=stream.cuda_stream, device=torch.cuda.current_device(),
                               time_kernels={"all": 1, "update": 2, "none": 0}[args.kernel_timing],
                               refine_tol=args.refine_tol,
                               pivoting=args.pivoting, update_panels=args.update_panels,
                               sparse_min=args.sparse_min)
    sched = None
    if precision == "mixed" and args.schedule:
        vals = [int(x) for x in args.schedule.split(",")]
        panels, ahead, reserve = vals[:3]
        split = vals[3] if len(vals) > 3 else 0
        s.set_schedule(panels, ahead, reserve, split)
        sched = {"update_panels": panels, "ahead_fronts": ahead, "reserve_sms": reserve, "split_sms": split,
                 "set": True}
    elif precision == "mixed" and autotune and not args.no_autotune:
        sched = s.autotune(repeats=2)      # untimed: picks the factor schedule for this workload
    f_host = dd.stacked_loads(p)
    f_dev = torch.from_numpy(f_host).cuda()
    for _ in range(warmup):
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
        for _ in range(steps):
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
    res = {"ms_per_step": ms / steps, "steps": steps, "warmup": warmup, "stats": st, "kernel_ms": kms,
           "kernel_launches": kl, "kernel_flops": kfl, "launches": launches, "refine_iters": iters,
           "backward_error": backward_error(p, u_host), "clocks": clk.summary(), "schedule": sched}
    res["accuracy"] = accuracy(p, s, torch)

    # end to end through the C ABI with host buffers: new values + factor + solve
    if e2e and not args.no_e2e:
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
        for _ in range(steps):
            lib.dd_set_values(s._h, C.c_void_p(vals_pin.data_ptr()))
            lib.dd_factor(s._h)
            lib.dd_solve(s._h, nrhs, C.c_void_p(f_pin.data_ptr()), n_loc, C.c_void_p(u_pin.data_ptr()), n_loc,
                         C.c_void_p(lam_pin.data_ptr()), max(p.n_dual, 1))
        torch.cuda.synchronize()
        e2e_ms = (time.perf_counter() - t0) * 1e3 / steps
        res["e2e"] = {"value": p.n / (e2e_ms * 1e-3), "unit": "DoF/s",
                      "h2d_bytes_per_step": int(vals.nbytes + f_host.nbytes),
                      "d2h_bytes_per_step": int(f_host.nbytes + 16 * p.n_dual * f_host.shape[1]),
                      "ms_per_step": e2e_ms}
    s.free()
    return res


def form_summary(p, f, ws):
    """Throughput, accuracy and growth of one timed form."""
    st = f["stats"]
    it = max(f["refine_iters"] or [0])
    flops = st["flops_factor"] + st["flops_solve"] * p.nrhs * (1 + it)
    return {"value": p.n * ws / (f["ms_per_step"] * 1e-3), "unit": "DoF/s", "ms_per_step": f["ms_per_step"],
            "steps": f["steps"], "warmup": f["warmup"], "tflops": flops / (f["ms_per_step"] * 1e-3) / 1e12,
            "refine_iters": it, "backward_error": f["backward_error"], "accuracy": f["accuracy"],
            "growth": f["accuracy"]["growth"], "factor_bytes": st["bytes_factor"], "clocks": f["clocks"],
            "schedule": f.get("schedule"),
            "kernel_ms_per_step": {c: v / f["steps"] for c, v in f["kernel_ms"].items()}}


TRAFFIC_FILE = os.path.join(ROOT, "profiles", "k_update_tc_traffic.md")


def kernel_sources_sha() -> str:
    """Hash of the sources that decide the update kernel's memory traffic: the
    kernel (kernels_tc.cu) and the panel kernels writing its operand images
    (kernels_factor.cu)."""
    import hashlib
    h = hashlib.sha256()
    for name in ("kernels_tc.cu", "kernels_factor.cu"):
        with open(os.path.join(ROOT, "paper_2002_05019_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def update_traffic(flops_per_launch: float):
    """DRAM bytes per launch of the tensor-core update, scaled from the ncu
    counters in profiles/ (bytes per algorithmic flop, over every launch of one
    factorization) by the launch's algorithmic flops; None when no summary
    exists or the kernel sources changed since the counters were taken."""
    try:
        with open(TRAFFIC_FILE) as fh:
            txt = fh.read()
    except OSError:
        return None, None
    vals = {}
    for ln in txt.splitlines():
        parts = ln.strip().strip("`").split()
        if len(parts) == 2 and parts[0] in ("bytes_per_flop", "kernels_sha256"):
            vals[parts[0]] = parts[1]
    if "bytes_per_flop" not in vals or vals.get("kernels_sha256") != kernel_sources_sha():
        return None, None
    return float(vals["bytes_per_flop"]) * flops_per_launch, float(vals["bytes_per_flop"])


def roofline_entry(main, args, steps):
    peaks, peaks_src = load_peaks()
    upd_ms = main["kernel_ms"].get("update", 0.0)
    upd_n = max(main["kernel_launches"].get("update", 0), 1)
    upd_fl = main["kernel_flops"].get("update", 0.0)
    achieved = upd_fl / (upd_ms * 1e-3) / 1e12 if upd_ms > 0 else None
    traffic, bpf = (None, None)
    if args.precision == "mixed":
        # tcgen05 kind::tf32: TF32 dense peak = measured bf16 peak x nominal TF32/BF16 ratio (1.1 / 2.25),
        # the sustained figure (the kernel runs inside a long step); the 3xTF32 split issues 3 tensor
        # passes per algorithmic product
        bf16 = peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"])
        tf32 = bf16 * (1.1 / 2.25)
        kernel = "k_update_tc (tcgen05 kind::tf32 3xTF32, M=128 N=256, complex 64x128 blocks)"
        bound, peak = "tensor", tf32 / 3.0
        src = (f"TF32 dense {tf32:.0f} TFLOP/s = {peaks_src} sustained bf16 {bf16:.0f} x 1.1/2.25; "
               f"effective complex64 peak = TF32 / 3 split passes")
        traffic, bpf = update_traffic(upd_fl / upd_n)
    else:
        bound, peak, kernel = "alu", FP64_DFMA_TFLOPS, "k_update<double2> (DFMA, 64x64 tiles)"
        src = f"GB300 FP64 DFMA rate {FP64_DFMA_TFLOPS} TFLOP/s (nominal FP64 of this part)"
    return {"bound": bound, "kernel": kernel, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": (achieved / peak) if achieved else None, "traffic": traffic,
            "traffic_bytes_per_flop": bpf,
            "flops_per_launch": upd_fl / upd_n, "avg_launch_ms": upd_ms / upd_n, "launches_per_step": upd_n / steps,
            "share_of_step": upd_ms / steps / main["ms_per_step"],
            "flops_counted": "exact front sizes (no tile padding), 8 real flops per complex multiply-add",
            "peak_source": src}


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
    t_all = time.perf_counter()
    t0 = time.perf_counter()
    p = getattr(femgen, WORKLOADS[args.workload][0])()
    log(f"[bench] workload {args.workload}: n={p.n} domains={p.n_sub} duals={p.n_dual} "
        f"(generated in {time.perf_counter() - t0:.1f} s)")
    stream = torch.cuda.current_stream()
    main = time_form(p, args.precision, args, torch, stream, args.steps, args.warmup)
    log(f"[bench] {args.workload} {args.precision}: {main['ms_per_step']:.2f} ms/step, accuracy {main['accuracy']}, "
        f"kernel ms {main['kernel_ms']}")
    st = main["stats"]
    t_step = main["ms_per_step"] * 1e-3
    iters = max(main["refine_iters"]) if main["refine_iters"] else 0
    flops_step = st["flops_factor"] + st["flops_solve"] * (1 + iters) * p.nrhs
    line = {
        "metric": METRIC, "value": job_value(p.n, ws, t_step), "unit": "DoF/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": main["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c64+f64" if args.precision == "mixed" else "c128", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload][1], "form": args.precision, "n_dofs": p.n,
                   "n_domains": p.n_sub, "n_duals": p.n_dual, "nrhs": p.nrhs, "pivoting": args.pivoting,
                   "update_panels": (main.get("schedule") or {}).get("update_panels", args.update_panels),
                   "schedule": main.get("schedule"),
                   "sparse_min": args.sparse_min,
                   "refine_tol": args.refine_tol,
                   "l2": "inputs larger than L2: the front pool is far larger than the 129 MB L2",
                   "parallelism": f"replicas x{ws}"},
        "tflops": flops_step / t_step / 1e12,
        "rel_err": main["accuracy"]["rel_err"], "rel_err_max": main["accuracy"]["rel_err_max"],
        "growth": main["accuracy"]["growth"], "accuracy": main["accuracy"],
        "refine_iters": iters, "backward_error": main["backward_error"],
        # setup (validation, symbolic analysis, device uploads) is outside the timed step
        "setup_ms": st["t_setup_ms"],
        "roofline": roofline_entry(main, args, args.steps),
        "gpu_launches": main["launches"],
        "clocks": main["clocks"],
        # factor memory (the paper's headline comparison): stored L and D of every front
        "memory": {"factor_bytes": st["bytes_factor"], "device_bytes": st["bytes_device"],
                   "skyline_factor_bytes_c128": None},
        "kernel_ms_per_step": {c: v / args.steps for c, v in main["kernel_ms"].items()},
    }
    if "e2e" in main:
        line["e2e"] = {k: main["e2e"][k] for k in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step")}
        line["e2e"]["value"] *= ws
    del p
    # the mixed-vs-FP64 comparison on one mesh (the 512-domain box by default)
    if args.compare != "none":
        pc = getattr(femgen, WORKLOADS[args.compare][0])()
        cmp = {"workload": WORKLOADS[args.compare][1], "n_dofs": pc.n, "n_domains": pc.n_sub, "n_duals": pc.n_dual}
        for prec, steps, warm in (("mixed", args.steps, args.warmup), ("fp64", args.fp64_steps, args.fp64_warmup)):
            f = time_form(pc, prec, args, torch, stream, steps, warm, e2e=False)
            cmp[prec] = form_summary(pc, f, ws)
            log(f"[bench] compare {args.compare} {prec}: {f['ms_per_step']:.2f} ms/step, accuracy {f['accuracy']}")
        cmp["mixed_over_fp64"] = cmp["mixed"]["value"] / cmp["fp64"]["value"]
        line["compare"] = cmp
        del pc
    if rank == 0 and not args.no_cpu_baseline:
        r = run_oracle_sample(args.workload, args.cpu_domains, host_cores(), with_skyline=True)
        line["cpu_baseline"] = cpu_baseline_entry(r, args.workload)
        if r.get("skyline_entries"):
            line["memory"]["skyline_factor_bytes_c128"] = 16 * int(r["skyline_entries"])
    log(f"[bench] total {time.perf_counter() - t_all:.1f} s")
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="large", choices=list(WORKLOADS))
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--compare", default="batched", choices=["none"] + list(WORKLOADS),
                    help="workload timed in both forms beside the headline (none: skip)")
    ap.add_argument("--fp64-steps", type=int, default=2, help="timed steps of the FP64 form in the comparison")
    ap.add_argument("--fp64-warmup", type=int, default=1)
    ap.add_argument("--single-form", action="store_true", help="the same as --compare none (kept for the commands "
                                                                "recorded with earlier profiles)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-domains", type=int, default=64,
                    help="domains in the subtree sample the CPU oracle baseline solves")
    ap.add_argument("--ref-domains", type=int, default=8,
                    help="domains in the subtree sample of each reference-arm step")
    ap.add_argument("--ref-route", default="tree", choices=["tree", "skyline"],
                    help="reference arm: the oracle's DD tree route on a subtree sample, or its undecomposed "
                         "skyline route on the whole workload")
    ap.add_argument("--ref-threads", type=int, default=0, help="reference arm: host threads (0: all)")
    ap.add_argument("--pivoting", type=int, default=0, choices=[0, 1, 2],
                    help="restricted Bunch-Kaufman: 0 none, 1 auxiliary fronts, 2 every front")
    ap.add_argument("--update-panels", type=int, default=2, choices=[1, 2, 4],
                    help="mixed form: panels fused per tensor-core trailing-update pass")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default factor schedule")
    ap.add_argument("--schedule", default="", help="PANELS,AHEAD_FRONTS,RESERVE_SMS[,SPLIT_SMS]: set this factor "
                                                   "schedule instead of autotuning")
    ap.add_argument("--sparse-min", type=int, default=0,
                    help="domains of at least this many unknowns are factored as nested-dissection front trees "
                         "(0: every domain one dense front)")
    ap.add_argument("--kernel-timing", default="update", choices=["update", "all", "none"],
                    help="CUDA events in the timed factorizations: around the trailing-update launches "
                         "(the roofline kernel; default), around every launch (per-class breakdown, slower), "
                         "or none (no roofline)")
    ap.add_argument("--refine-tol", type=float, default=1e-11,
                    help="mixed form: stop refinement at this relative correction (1e-11 keeps the error <= 1e-10)")
    args = ap.parse_args()
    if args.single_form:
        args.compare = "none"
    if args.impl == "reference":
        return reference_arm(args)
    return ours_arm(args)


if __name__ == "__main__":
    sys.exit(main())
