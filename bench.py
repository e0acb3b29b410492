"""Benchmark: HDG trace apply and nested-GMG solve on one GB300.

Workload (the paper's headline configuration): 512 x 512 quads on the unit
square, degree k = 4, per-element kappa = exp(g), g a seeded Gaussian field
(variance 1, squared-exponential correlation length 0.05, seed 0), f = 1,
element Schur blocks stored in FP64. One step is one pass of the hot path on
one right-hand side: condensed right-hand side, multigrid-preconditioned CG
with FP64 V-cycles to relative residual 1e-10, and local recovery of (u, q).
The solver set-up (local solvers, hierarchy) runs once before timing and is
reported separately.

Printed JSON line (rank 0):
  value          whole-job solves per second (all ranks, replicas)
  ms_per_step    FP64 GMG-CG solve time to 1e-10 (incl. condense + recovery)
  roofline       the trace-apply kernel (the dominant kernel of the step),
                 timed alone with CUDA events over repeated launches
  trace_apply    GB/s and fraction of the measured HBM copy peak per precision
  mixed          the same solve with FP32 / BF16 V-cycles in FP64 flexible CG
  e2e            the same step through the public API with the source samples
                 copied host -> device and lambda, u copied back each step
  cpu_baseline   the FP64 oracle (condense + sparse direct solve + recovery)
                 on a bounded sub-mesh, one core, scaled per element

--impl reference times that oracle alone (the reference arm of this repo).
Multi-GPU: one replica per rank (the solve has no data-parallel split on one
box); value sums the ranks' solves.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_DEFAULT, K_DEFAULT, SEED = 512, 4, 0
METRIC = "trace-apply GB/s and %HBM peak; GMG solve time to 1e-10 rel residual, mixed vs FP64 on GPU"


def rank_env():
    """(world, rank, local rank) from the launcher's environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(value, world, device):
    """The largest of the ranks' values (every rank gets it); the step time of a
    replica job is its slowest rank's."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], device=device, dtype=torch.float64)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, ms_per_step):
    """Whole-job solves per second: every rank solves one system per step."""
    return world * 1000.0 / ms_per_step


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return {"hbm_gbs": float(p["hbm_gbs"]), "bf16_tflops": float(p["bf16_tflops"]), "source": "measured"}
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "source": "fallback"}


# ---------------------------------------------------------------------------
# CPU baseline: the oracle as it stands on a bounded sample of the workload
def _oracle_sample(n_sub, N, k, seed):
    from oracle import hdg as ohdg, mesh as omesh
    from paper_1705_09907_gb300 import inputs
    g = inputs.gaussian_field(N, seed).reshape(N, N)
    kap = np.exp(g[:n_sub, :n_sub]).ravel()
    h = 1.0 / N
    m = omesh.Mesh(n_sub, n_sub, 0.0, 0.0, n_sub * h, n_sub * h)
    fq = np.ones((m.nel, k + 2, k + 2))
    t0 = time.perf_counter()
    prob = ohdg.HDGProblem(m, k, kap)
    b = prob.condense_rhs(fq)
    lam = prob.solve_direct(b)
    prob.recover(lam, fq)
    return time.perf_counter() - t0, m.nel


def _oracle_extras(n_sub, N, k, seed):
    """On the same sub-mesh: the assembled interior matrix's scipy CSR matvec
    (the paper's matrix-based baseline) and the oracle's GMG-preconditioned CG
    to 1e-10 (its set-up excluded)."""
    from oracle import gmg as ogmg, hdg as ohdg, mesh as omesh
    from paper_1705_09907_gb300 import inputs
    g = inputs.gaussian_field(N, seed).reshape(N, N)
    kap = np.exp(g[:n_sub, :n_sub]).ravel()
    h = 1.0 / N
    m = omesh.Mesh(n_sub, n_sub, 0.0, 0.0, n_sub * h, n_sub * h)
    prob = ohdg.HDGProblem(m, k, kap)
    A, _ = prob.assemble_interior()
    A = A.tocsr()
    x = np.random.default_rng(seed).normal(size=A.shape[0])
    reps = 100
    t0 = time.perf_counter()
    for _ in range(reps):
        A @ x
    t_mv = (time.perf_counter() - t0) / reps
    G = ogmg.NestedGMG(m, k, kap)
    b = prob.condense_rhs(np.ones((m.nel, k + 2, k + 2)))
    t0 = time.perf_counter()
    _, its, _ = G.pcg(b, rtol=1e-10)
    t_pcg = time.perf_counter() - t0
    csr_bytes = A.nnz * 12 + (A.shape[0] + 1) * 4 + 2 * A.shape[0] * 8
    return {"csr_matvec_s": t_mv, "csr_bytes": csr_bytes, "nnz": int(A.nnz), "gmg_pcg_s": t_pcg,
            "gmg_pcg_iterations": int(its)}


def cpu_baseline_worker(n_sub, N, k, seed, reps):
    times = []
    nel = None
    for _ in range(reps):
        t, nel = _oracle_sample(n_sub, N, k, seed)
        times.append(t)
    try:
        extras = _oracle_extras(n_sub, N, k, seed)
    except Exception as ex:  # reported, not fatal
        extras = {"error": str(ex)[:200]}
    print(json.dumps({"times": times, "nel": nel, "extras": extras}))


def host_cpu():
    """The host's core count and CPU model (the oracle baseline runs there)."""
    import platform
    model = None
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "hardware"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if model is None:
        try:   # aarch64 /proc/cpuinfo has no model line; lscpu names the core
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    return {"cpu_count": os.cpu_count(), "model": model or platform.machine(), "arch": platform.machine()}


def run_cpu_baseline(N, k, n_sub=48, reps=1):
    n_sub = min(n_sub, N)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    cmd = [sys.executable, "-c",
           "import bench; bench.cpu_baseline_worker(%d, %d, %d, %d, %d)" % (n_sub, N, k, SEED, reps)]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    if r.returncode != 0:
        raise RuntimeError("oracle baseline failed: " + r.stderr[-2000:])
    out = json.loads(r.stdout.strip().splitlines()[-1])
    t = statistics.median(out["times"])
    per_elem = t / out["nel"]
    full = per_elem * N * N
    line = {
        "value": 1.0 / full, "unit": "solve/s", "cores": 1, "kind": "oracle",
        "sample": "%dx%d sub-mesh of the %dx%d k=%d lognormal workload (same h and kappa), oracle condense + "
                  "scipy SuperLU direct solve + recovery, %.2f s, scaled linearly by element count"
                  % (n_sub, n_sub, N, N, k, t),
        "sample_seconds": t, "host": host_cpu(),
        "threads": "one core (BLAS/OpenMP pinned to 1; SuperLU and the oracle's per-element loops are "
                   "single-threaded, so more cores would not shorten them)",
    }
    ex = out.get("extras", {})
    if "csr_matvec_s" in ex:
        scale = N * N / out["nel"]
        line["csr_matvec"] = {
            "what": "scipy CSR matvec of the assembled interior operator on the same sub-mesh, one core; time "
                    "scaled by element count to the full mesh (the sub-mesh matrix fits in the CPU caches, so this "
                    "overstates a full-size matvec)",
            "ms_full_mesh": ex["csr_matvec_s"] * scale * 1e3, "GBps": ex["csr_bytes"] / ex["csr_matvec_s"] / 1e9,
            "nnz_sub_mesh": ex["nnz"]}
        line["gmg_pcg"] = {
            "what": "oracle GMG-preconditioned CG to 1e-10 on the same sub-mesh (set-up excluded), one core",
            "seconds_sub_mesh": ex["gmg_pcg_s"], "iterations": ex["gmg_pcg_iterations"]}
    elif ex:
        line["extras_error"] = ex.get("error")
    return line


# ---------------------------------------------------------------------------
class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during timing."""

    def __init__(self, path, index):
        self.path = path
        self.index = index
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        try:
            rows = [l.split(",") for l in open(self.path).read().strip().splitlines() if l.strip()]
        except Exception:
            rows = []
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows]
        mx = max(float(r[2]) for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[j] for r in rows for j in range(4) if r[5 + j].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": reasons, "samples": len(rows)}


def timed_events(fn, reps, torch):
    s = torch.cuda.Event(enable_timing=True)
    e = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    s.record()
    for _ in range(reps):
        fn()
    e.record()
    torch.cuda.synchronize()
    return s.elapsed_time(e) / reps


def flushed_time(fn, torch, n=8, reps=3):
    """Device time of fn with a cold L2: one CUDA graph of n x (L2 flush, fn)
    and one of n x (L2 flush) alone, each replayed `reps` times between CUDA
    events; the difference per call. The flush writes twice the L2 size, so no
    input of fn is served from L2 (used where fn's data is smaller than L2)."""
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    l2 = int(getattr(props, "L2_cache_size", 0) or (132 << 20))
    buf = torch.empty(2 * l2 // 4, dtype=torch.float32, device="cuda")

    def flush():
        buf.fill_(1.0)

    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):          # warm-up outside the capture
        flush()
        fn()
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    graphs = []
    for with_fn in (True, False):
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, capture_error_mode="thread_local"):
            for _ in range(n):
                flush()
                if with_fn:
                    fn()
        graphs.append(g)
    times = []
    for g in graphs:
        g.replay()
        torch.cuda.synchronize()
        times.append(timed_events(g.replay, reps, torch))
    del graphs
    return max(times[0] - times[1], 0.0) / n


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_1705_09907_gb300 import hdg, inputs

    world, rank, local = rank_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    N, k = args.n, args.k
    peaks = load_peaks()
    kap = inputs.lognormal_kappa(N, SEED)
    fq_h = inputs.constant_f(N, k)
    kap_d = torch.as_tensor(kap, device="cuda")
    fq_d = torch.as_tensor(fq_h, device="cuda")
    # a profiling run launches the CG loop from the host (use_graphs = 0: the
    # same kernels, launched directly): profilers do not see the kernels of a
    # conditional graph node's body
    solver = hdg.HDGSolver(N, N, k, kap_d, use_graphs=0 if args.profile else 1)
    info = solver.info
    rtol = 1e-10
    u = torch.empty((solver.nel, (k + 1) ** 2), dtype=torch.float64, device="cuda")
    lam = torch.empty(solver.ndof, dtype=torch.float64, device="cuda")

    last = {}

    def step(inner="fp64"):
        b = solver.condense_rhs(fq_d)
        lam_, inf = solver.solve(b, rtol=rtol, maxit=200, inner=inner, out=lam)
        uu, qq = solver.recover(lam_, fq_d)
        last["info"] = inf
        return uu

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if args.profile:
        # short fixed sequence for profiler launch lists: one solve step (NVTX
        # range fp64_step), then three trace applies per precision, then the
        # batched work below
        torch.cuda.nvtx.range_push("fp64_step")
        step()
        torch.cuda.nvtx.range_pop()
        # the same step with the FP32 V-cycle (outer CG in FP64)
        step("fp32")
        torch.cuda.nvtx.range_push("fp32_step")
        step("fp32")
        torch.cuda.nvtx.range_pop()
        x64 = torch.as_tensor(inputs.random_trace(solver.n_edges, k, seed=1), device="cuda")
        x32 = x64.float()
        # each precision's applies inside an NVTX range named apply_<prec>
        # (profilers can select one with --nvtx-include "apply_<prec>/")
        for p_, xx in (("fp64", x64), ("fp32", x32), ("bf16", x32), ("f32x2", x64)):
            torch.cuda.nvtx.range_push("apply_" + p_)
            for _ in range(3):
                solver.apply(xx, p_)
            torch.cuda.nvtx.range_pop()
        # tensor-core batched apply, same mesh with kappa = 1, 64 right-hand sides
        sbs = hdg.HDGSolver(N, N, k, torch.ones(N * N, dtype=torch.float64, device="cuda"), mixed=0, autotune=0)
        X4 = torch.randn((sbs.ndof, 64), device="cuda").to(torch.bfloat16)
        torch.cuda.nvtx.range_push("apply_batched")
        for _ in range(3):
            sbs.apply_shared_batched(X4)
        torch.cuda.nvtx.range_pop()
        sbs.close()
        # column-batched applies and one batched solve: 256 x 256, k = 5, kappa = 1,
        # 64 Fourier right-hand sides; NVTX ranges cols_<prec> and batched_solve
        sbm = hdg.HDGSolver(256, 256, 5, torch.ones(256 * 256, dtype=torch.float64, device="cuda"), autotune=0)
        B = sbm.condense_rhs(torch.as_tensor(inputs.fourier_rhs(256, 5, 64, seed=3), device="cuda"))
        B32 = B.float()
        for p_, xx in (("fp64", B), ("f32x2", B), ("fp32", B32), ("bf16", B32)):
            torch.cuda.nvtx.range_push("cols_" + p_)
            for _ in range(3):
                sbm.apply(xx, p_)
            torch.cuda.nvtx.range_pop()
        sbm.solve(B, rtol=1e-10, maxit=400, inner="fp32")
        torch.cuda.nvtx.range_push("batched_solve")
        sbm.solve(B, rtol=1e-10, maxit=400, inner="fp32")
        torch.cuda.nvtx.range_pop()
        sbm.close()
        # the FP64 step with the FSAI smoother (NVTX range fsai_fp64_step)
        sfs = hdg.HDGSolver(N, N, k, kap_d, smoother=1, use_graphs=0)
        bf = sfs.condense_rhs(fq_d)
        sfs.solve(bf, rtol=rtol, maxit=200)
        torch.cuda.nvtx.range_push("fsai_fp64_step")
        sfs.solve(bf, rtol=rtol, maxit=200)
        torch.cuda.nvtx.range_pop()
        sfs.close()
        torch.cuda.synchronize()
        print(json.dumps({"profile_run": True, "iterations": last["info"]["iterations"],
                          "relres": last["info"]["relres"], "vcycle_kernels": solver.get_info()["vcycle_kernels"]}))
        solver.close()
        return
    if world > 1:
        dist.barrier()
    if args.clocks_log:
        clock_path = args.clocks_log % {"rank": rank} if "%(rank)" in args.clocks_log else args.clocks_log
    else:
        fd, clock_path = tempfile.mkstemp(prefix="hdg_bench_clocks_r%d_" % rank, suffix=".csv")
        os.close(fd)
    clocks = Clocks(clock_path, local)
    # end to end through the public API with host buffers: the step's source
    # samples copied in from pinned host memory, lambda and u copied back
    fq_pin = torch.as_tensor(fq_h).pin_memory()
    lam_pin = torch.empty(solver.ndof, dtype=torch.float64).pin_memory()
    u_pin = torch.empty(tuple(u.shape), dtype=torch.float64).pin_memory()

    def e2e_step():
        fd_ = fq_pin.to("cuda", non_blocking=True)
        b = solver.condense_rhs(fd_)
        lam_, _ = solver.solve(b, rtol=rtol, maxit=200, out=lam)
        uu, _ = solver.recover(lam_, fd_)
        lam_pin.copy_(lam_, non_blocking=True)
        u_pin.copy_(uu, non_blocking=True)

    e2e_step()
    with clocks:
        torch.cuda.synchronize()
        t_ms = timed_events(step, args.steps, torch)
        its = last["info"]["iterations"]
        relres = last["info"]["relres"]
        # the same number of steps end to end, in the same clock window
        e2e_ms = timed_events(e2e_step, args.steps, torch)
        # the dominant kernel: trace apply at level k, timed alone (inputs >> L2)
        x64 = torch.as_tensor(inputs.random_trace(solver.n_edges, k, seed=1), device="cuda")
        y64 = torch.empty_like(x64)
        x32 = x64.float()
        y32 = torch.empty_like(x32)
        # the reduced blocks (128 MB FP64 / 64 MB FP32 at 512^2, k = 4) are about
        # the size of L2: each apply is timed after an L2 flush, inside a CUDA
        # graph (device time only)
        apply_ms = {}
        for p_, xx, yy in (("fp64", x64, y64), ("fp32", x32, y32), ("bf16", x32, y32), ("f32x2", x64, y64)):
            apply_ms[p_] = flushed_time(lambda: solver.apply(xx, p_, out=yy), torch)
        # the dense owner-record kernels (reduced = 0): the kernel that applies the
        # Schwarz blocks in every V-cycle, here timed on the condensed blocks (the
        # same kernel and the same bytes per launch)
        dense = hdg.HDGSolver(N, N, k, kap_d, reduced=0)
        dense_ms = {}
        for p_, xx, yy in (("fp64", x64, y64), ("fp32", x32, y32), ("bf16", x32, y32), ("f32x2", x64, y64)):
            dense_ms[p_] = flushed_time(lambda: dense.apply(xx, p_, out=yy), torch)
        dense.close()
    clk = clocks.summary()
    # the element-local operations of the step, timed alone
    b_loc = solver.condense_rhs(fq_d)
    local_ms = {"condense_rhs": timed_events(lambda: solver.condense_rhs(fq_d), 10, torch),
                "recover_local": timed_events(lambda: solver.recover(lam, fq_d), 10, torch)}
    del b_loc
    # mixed-precision solves on the same mesh (outside the clock window: reported, not the headline)
    lam64 = lam.clone()
    mixed = {}
    for inner in ("fp32", "bf16", "f32x2"):
        step(inner)
        ms = timed_events(lambda: step(inner), max(1, args.steps // 2), torch)
        inf = last["info"]
        err = float(torch.linalg.norm(lam - lam64) / torch.linalg.norm(lam64))
        mixed[inner] = {"ms_per_solve": ms, "iterations": inf["iterations"], "relres": inf["relres"],
                        "rel_diff_vs_fp64_solution": err}
    # every V-cycle precision against the FP64 oracle's SuperLU solution on a
    # mesh the host can solve directly: the same lognormal generator (seed 0) at
    # 128 x 128, k = 4 (the headline degree) and k = 3 (the 1024^2 family);
    # stored by tests/golden/make_oracle_solutions.py from the oracle alone
    mvo = {}
    if not args.profile:
        for No, ko in ((128, 4), (128, 3)):
            path = os.path.join(ROOT, "tests", "golden", "oracle_lognormal_%d_k%d.npy" % (No, ko))
            if not os.path.exists(path):
                continue
            ref = torch.as_tensor(np.load(path), device="cuda")
            so = hdg.HDGSolver(No, No, ko, torch.as_tensor(inputs.lognormal_kappa(No, SEED), device="cuda"))
            bo = so.condense_rhs(torch.as_tensor(inputs.constant_f(No, ko), device="cuda"))
            ent = {"mesh": "%dx%d k=%d lognormal kappa (seed 0), f=1" % (No, No, ko),
                   "oracle": "scipy SuperLU solution (tests/golden/oracle_lognormal_%d_k%d.npy)" % (No, ko),
                   "rtol": rtol}
            for inner in ("fp64", "fp32", "bf16", "f32x2"):
                lo, info_o = so.solve(bo, rtol=rtol, maxit=400, inner=inner)
                ent[inner] = {"err_vs_oracle": float(torch.linalg.norm(lo - ref) / torch.linalg.norm(ref)),
                              "iterations": info_o["iterations"]}
            so.close()
            mvo["%d_k%d" % (No, ko)] = ent
        key4 = "128_k4"
        if key4 in mvo:
            for inner in mixed:
                mixed[inner]["err_vs_oracle"] = mvo[key4][inner]["err_vs_oracle"]
                mixed[inner]["err_vs_oracle_mesh"] = mvo[key4]["mesh"]
    # the paper's smoother (Sec. 6.4.1): FSAI on the pattern of each p-level
    # operator instead of the element-patch Schwarz blocks, same mesh and solve
    fsai = {}
    if not args.profile:
        sf = hdg.HDGSolver(N, N, k, kap_d, smoother=1)
        bf = sf.condense_rhs(fq_d)
        lf = torch.empty_like(bf)
        fsai = {"workload": "%dx%d k=%d lognormal kappa (seed 0), f=1, rtol 1e-10, FSAI V(2,2) smoothing" % (N, N, k),
                "setup_ms": sf.info["setup_ms"]}
        for inner in ("fp64", "fp32"):
            sf.solve(bf, rtol=rtol, maxit=400, inner=inner, out=lf)
            msf = timed_events(lambda: sf.solve(bf, rtol=rtol, maxit=400, inner=inner, out=lf), 2, torch)
            inf_f = sf.solve(bf, rtol=rtol, maxit=400, inner=inner, out=lf)[1]
            fsai[inner] = {"ms_per_solve": msf, "iterations": inf_f["iterations"], "relres": inf_f["relres"],
                           "rel_diff_vs_schwarz_solution": float(torch.linalg.norm(lf - lam64) /
                                                                 torch.linalg.norm(lam64))}
        sf.close()
    # full multigrid (Sec. 7) on the same problem: one FMG cycle with 1, 2, 3
    # V-cycles per level (time, relative residual), and CG started from FMG(2)
    fmg = {}
    if not args.profile:
        b_f = solver.condense_rhs(fq_d)
        x_f = torch.empty_like(b_f)
        fmg = {"workload": "%dx%d k=%d lognormal kappa (seed 0), f=1, FP64 V-cycles" % (N, N, k)}
        for cyc in (1, 2, 3):
            solver.fmg(b_f, cycles=cyc, out=x_f)
            msf = timed_events(lambda: solver.fmg(b_f, cycles=cyc, out=x_f), 2, torch)
            rr = b_f - solver.apply(x_f)
            fmg["cycles_%d" % cyc] = {"ms": msf, "relres": float(torch.linalg.norm(rr) / torch.linalg.norm(b_f))}
        sfm = hdg.HDGSolver(N, N, k, kap_d, fmg_start=2)
        lfm = torch.empty_like(b_f)
        sfm.solve(b_f, rtol=rtol, maxit=400, out=lfm)
        fmg["cg_from_fmg2"] = {"ms_per_solve": timed_events(lambda: sfm.solve(b_f, rtol=rtol, maxit=400, out=lfm), 2,
                                                            torch),
                               "iterations": sfm.solve(b_f, rtol=rtol, maxit=400, out=lfm)[1]["iterations"],
                               "iterations_zero_start": its}
        sfm.close()
    # the small manufactured problem (16 x 16, k = 1, kappa = 1, u = sin pi x
    # sin pi y): latency of one step (condense + FP64 GMG-CG to 1e-10 + recovery)
    c1 = {}
    if not args.profile:
        s1 = hdg.HDGSolver(16, 16, 1, torch.ones(256, dtype=torch.float64, device="cuda"))
        f1 = torch.as_tensor(inputs.manufactured_poisson_f(16, 1), device="cuda")
        l1 = torch.empty(s1.ndof, dtype=torch.float64, device="cuda")

        def step1():
            b1 = s1.condense_rhs(f1)
            s1.solve(b1, rtol=rtol, maxit=100, out=l1)
            s1.recover(l1, f1)

        step1()
        c1 = {"workload": "16x16 k=1 kappa=1, f from u = sin(pi x) sin(pi y), FP64 GMG-CG to 1e-10 (2x2 coarsest)",
              "ms_per_step": timed_events(step1, 20, torch),
              "iterations": s1.solve(s1.condense_rhs(f1), rtol=rtol, maxit=100, out=l1)[1]["iterations"],
              "note": "L2-resident (131 KB of blocks): latency, not bandwidth"}
        s1.close()
    # adjoint gradient (512 x 512, k = 2): log kappa = Gaussian field (seed 0),
    # lambda_obs = the solve at a second field (seed 1) + N(0, 1e-3) noise
    # (seed 2), f = 1; hdg_adjoint_grad time (adjoint multigrid CG to 1e-12 +
    # element kernel) and dJ/dlog(kappa) against central differences (step
    # 1e-3, each side a fresh set-up and a solve to 1e-13) on 20 elements (seed 5)
    adj = {}
    if not args.profile:
        Na, ka = 512, 2
        tha = inputs.gaussian_field(Na, seed=0)
        fqa = torch.as_tensor(inputs.constant_f(Na, ka), device="cuda")
        sa1 = hdg.HDGSolver(Na, Na, ka, torch.as_tensor(np.exp(inputs.gaussian_field(Na, seed=1)), device="cuda"))
        la1, _ = sa1.solve(sa1.condense_rhs(fqa), rtol=1e-13, maxit=400)
        lobs = (la1 + torch.as_tensor(inputs.observation_noise(sa1.ndof, seed=2), device="cuda")).contiguous()
        _, ela, _ = sa1.maps()
        inter = ((ela[:, 0] >= 0) & (ela[:, 1] >= 0)).repeat_interleave(ka + 1)
        sa1.close()
        sa = hdg.HDGSolver(Na, Na, ka, torch.as_tensor(np.exp(tha), device="cuda"))
        la, _ = sa.solve(sa.condense_rhs(fqa), rtol=1e-13, maxit=400)
        sa.adjoint_grad(fqa, la, lobs, rtol=1e-12)
        ms_adj = timed_events(lambda: sa.adjoint_grad(fqa, la, lobs, rtol=1e-12), 3, torch)
        Jv, dth, _, _ = sa.adjoint_grad(fqa, la, lobs, rtol=1e-12)
        dth_h = dth.cpu().numpy()
        sa.close()

        def J_of(theta):
            st_ = hdg.HDGSolver(Na, Na, ka, torch.as_tensor(np.exp(theta), device="cuda"), mixed=0, autotune=0)
            lj, _ = st_.solve(st_.condense_rhs(fqa), rtol=1e-13, maxit=400)
            st_.close()
            d_ = (lj - lobs)[inter]
            return 0.5 * float((d_ * d_).sum())

        els = np.random.default_rng(5).choice(Na * Na, size=20, replace=False)
        hfd = 1e-3
        errs = []
        for e_ in els:
            tp, tm = tha.copy(), tha.copy()
            tp[e_] += hfd
            tm[e_] -= hfd
            fd = (J_of(tp) - J_of(tm)) / (2 * hfd)
            errs.append(abs(fd - dth_h[e_]) / max(abs(fd), 1e-300))
        adj = {"workload": "512x512 k=2, log kappa seed 0, lambda_obs from seed 1 + N(0,1e-3) noise (seed 2), f=1",
               "adjoint_grad_ms": ms_adj, "J": float(Jv.item()),
               "fd_max_rel_err": float(max(errs)), "fd_median_rel_err": float(statistics.median(errs)),
               "fd": "central differences, step 1e-3 in log kappa, 20 elements (seed 5)"}
    # measured FP64 rate of this GPU: cuBLAS DGEMM through torch (4096^3, best of
    # 5), the FP64 counterpart of the driver's bf16 GEMM peak
    a64 = torch.randn(4096, 4096, dtype=torch.float64, device="cuda")
    b64 = torch.randn(4096, 4096, dtype=torch.float64, device="cuda")
    torch.matmul(a64, b64)
    fp64_tf = max(2 * 4096 ** 3 / (timed_events(lambda: torch.matmul(a64, b64), 3, torch) * 1e-3) / 1e12
                  for _ in range(5))
    del a64, b64
    # the tau_K = kappa_K variant on the same mesh and coefficient (a different
    # discretisation: solutions are not compared with the tau = 1 ones)
    tk = {}
    if not args.profile:
        stk = hdg.HDGSolver(N, N, k, kap_d, tau_kappa=1)
        btk = stk.condense_rhs(fq_d)
        ltk = torch.empty_like(btk)
        tk = {"workload": "%dx%d k=%d lognormal kappa (seed 0), f=1, tau_K = kappa_K, rtol 1e-10" % (N, N, k),
              "setup_ms": stk.info["setup_ms"]}
        for inner in ("fp64", "fp32"):
            stk.solve(btk, rtol=rtol, maxit=400, inner=inner, out=ltk)
            mtk = timed_events(lambda: stk.solve(btk, rtol=rtol, maxit=400, inner=inner, out=ltk), 2, torch)
            itk = stk.solve(btk, rtol=rtol, maxit=400, inner=inner, out=ltk)[1]
            tk[inner] = {"ms_per_solve": mtk, "iterations": itk["iterations"], "relres": itk["relres"]}
        stk.close()
    # tensor-core batched apply: uniform kappa, 256 x 256, k = 5, 64 right-hand sides
    # (Fourier sources, seed 3); BF16 inputs, FP32 outputs
    sb = {}
    if not args.profile:
        Nb, kb, nr = 256, 5, 64
        sbs = hdg.HDGSolver(Nb, Nb, kb, torch.ones(Nb * Nb, dtype=torch.float64, device="cuda"), mixed=0)
        fq4 = torch.as_tensor(inputs.fourier_rhs(Nb, kb, nr, seed=3), device="cuda")
        B4 = sbs.condense_rhs(fq4)                       # [ndof, 64] FP64
        X4 = B4.to(torch.bfloat16).contiguous()
        Y4 = torch.empty(X4.shape, dtype=torch.float32, device="cuda")
        sbs.apply_shared_batched(X4, out=Y4)
        ms4 = timed_events(lambda: sbs.apply_shared_batched(X4, out=Y4), args.apply_reps, torch)
        algo4 = X4.numel() * 2 + Y4.numel() * 4 + 2 * 16 * 48 * 2
        fl4 = 2.0 * Nb * Nb * 16 * (kb + 1) ** 2 * nr
        # the FP64 apply of the same columns on the tensor cores (exact slice
        # splitting) against the CUDA-core FP64 column kernel of the same context
        B4c = B4.contiguous()
        Y64 = torch.empty_like(B4c)
        sbs.apply_shared_fp64(B4c, out=Y64)
        ms64 = timed_events(lambda: sbs.apply_shared_fp64(B4c, out=Y64), args.apply_reps, torch)
        Yc = sbs.apply(B4c)
        msc64 = timed_events(lambda: sbs.apply(B4c, out=Yc), args.apply_reps, torch)
        algo64 = B4c.numel() * 8 * 2                       # X read once, Y written once (FP64)
        oz = {"ms": ms64, "GBps": algo64 / (ms64 * 1e-3) / 1e9,
              "frac_hbm": algo64 / (ms64 * 1e-3) / 1e9 / peaks["hbm_gbs"],
              "cuda_core_fp64_column_ms": msc64, "speedup_vs_cuda_core": msc64 / ms64,
              "rel_diff_vs_cuda_core": float(torch.linalg.norm(Y64 - Yc) / torch.linalg.norm(Yc)),
              "kernels": "ozaki_exp_kernel + ozaki_split_kernel + ozaki_apply_kernel (tcgen05, 8 BF16 slices)",
              "bytes_note": "algorithmic bytes 16 per entry; the slices add 16 written + 16 read per entry"}
        sb = {"workload": "256x256 k=5 kappa=1, 64 Fourier right-hand sides (seed 3)", "ms": ms4,
              "GBps": algo4 / (ms4 * 1e-3) / 1e9, "frac_hbm": algo4 / (ms4 * 1e-3) / 1e9 / peaks["hbm_gbs"],
              "TFLOPs": fl4 / (ms4 * 1e-3) / 1e12, "algorithmic_bytes": algo4, "flops": fl4,
              "kernel": "batched_apply_kernel (tcgen05.mma kind::f16, BF16 x BF16 -> FP32 TMEM)",
              "fp64_exact_split": oz}
        sbs.close()
    # many right-hand sides in one solve: 256 x 256, k = 5, kappa = 1, 64 Fourier
    # sources (seed 3); batched CG (one batched apply and V-cycle per iteration)
    # against plain FP64 solves one right-hand side at a time on the same mesh
    bs = {}
    if not args.profile:
        Nb, kb, nr = 256, 5, 64
        sbm = hdg.HDGSolver(Nb, Nb, kb, torch.ones(Nb * Nb, dtype=torch.float64, device="cuda"))
        B = sbm.condense_rhs(torch.as_tensor(inputs.fourier_rhs(Nb, kb, nr, seed=3), device="cuda"))
        LB = torch.empty_like(B)
        lam1 = torch.empty(sbm.ndof, dtype=torch.float64, device="cuda")
        b0 = B[:, 0].contiguous()
        sbm.solve(b0, rtol=rtol, maxit=400, out=lam1)
        single = timed_events(lambda: sbm.solve(b0, rtol=rtol, maxit=400, out=lam1), 3, torch)
        its1 = sbm.solve(b0, rtol=rtol, maxit=400, out=lam1)[1]["iterations"]
        bs = {"workload": "256x256 k=5 kappa=1, 64 Fourier right-hand sides (seed 3), rtol 1e-10",
              "plain_fp64_ms_per_rhs": single, "plain_fp64_iterations": its1}
        for inner in ("fp32", "fp64"):
            sbm.solve(B, rtol=rtol, maxit=400, inner=inner, out=LB)
            msb = timed_events(lambda: sbm.solve(B, rtol=rtol, maxit=400, inner=inner, out=LB), 1 if inner == "fp64" else 3, torch)
            inf = sbm.solve(B, rtol=rtol, maxit=400, inner=inner, out=LB)[1]
            bs["batched_" + inner] = {"ms_per_batch": msb, "ms_per_rhs": msb / nr, "iterations": inf["iterations"],
                                      "max_relres": inf["relres"], "speedup_per_rhs_vs_plain_fp64": single / (msb / nr),
                                      "rel_diff_col0_vs_plain_fp64": float(torch.linalg.norm(LB[:, 0] - lam1) /
                                                                            torch.linalg.norm(lam1))}
        # the column-batched record apply at level k (S read once for all 64 columns)
        X64 = B.clone()
        Y64 = torch.empty_like(X64)
        X32 = B.float()
        Y32 = torch.empty_like(X32)
        nelb, neb, n1b = sbm.nel, sbm.n_edges, kb + 1
        cols = {}
        for p_, xx, yy, bs_, bx_ in (("fp64", X64, Y64, 8, 8), ("f32x2", X64, Y64, 8, 8), ("fp32", X32, Y32, 4, 4),
                                     ("bf16", X32, Y32, 2, 4)):
            sbm.apply(xx, p_, out=yy)
            msc = timed_events(lambda: sbm.apply(xx, p_, out=yy), args.apply_reps, torch)
            if p_ in ("fp64", "f32x2"):
                # double vectors on reduced blocks (the default): the reduced
                # column kernels, FP64 packed blocks (Q per element) and their own
                # operations (block products + the +-1 transforms + face sums)
                a_, b_ = n1b // 2 + n1b % 2, n1b // 2
                dims_b = (2 * a_, a_ + b_, a_ + b_, 2 * b_)
                qb = sum(d * (d + 1) // 2 for d in dims_b)
                algo = nelb * qb * 8 + 2 * neb * n1b * nr * 8
                fl = nelb * nr * (2.0 * sum(d * d for d in dims_b) + 8 * n1b + 16 * b_ + 2 * n1b)
                kern = "reduced_cols_elem_kernel + reduced_cols_face_kernel"
            else:
                algo = nelb * 16 * n1b * n1b * bs_ + 2 * neb * n1b * nr * bx_
                fl = 2.0 * nelb * 16 * n1b * n1b * nr
                kern = "apply_cols_kernel (dense owner records)"
            cols[p_] = {"ms": msc, "kernel": kern, "GBps": algo / (msc * 1e-3) / 1e9,
                        "frac_hbm": algo / (msc * 1e-3) / 1e9 / peaks["hbm_gbs"], "TFLOPs": fl / (msc * 1e-3) / 1e12,
                        "algorithmic_bytes": algo}
        bs["column_apply_64rhs"] = cols
        sbm.close()
    # mixed precision at 1024 x 1024, k = 3 (lognormal kappa, seed 0, f = 1):
    # solve time to 1e-10 per V-cycle precision against plain FP64
    m3 = {}
    if not args.profile:
        N3, k3 = 1024, 3
        s3 = hdg.HDGSolver(N3, N3, k3, torch.as_tensor(inputs.lognormal_kappa(N3, SEED), device="cuda"))
        b3 = s3.condense_rhs(torch.as_tensor(inputs.constant_f(N3, k3), device="cuda"))
        l3 = torch.empty_like(b3)
        l64 = None
        m3 = {"workload": "1024x1024 k=3 lognormal kappa (seed 0), f=1, rtol 1e-10", "setup_ms": s3.info["setup_ms"]}
        for inner in ("fp64", "fp32", "bf16", "f32x2"):
            s3.solve(b3, rtol=rtol, maxit=400, inner=inner, out=l3)
            ms3 = timed_events(lambda: s3.solve(b3, rtol=rtol, maxit=400, inner=inner, out=l3), 2, torch)
            inf = s3.solve(b3, rtol=rtol, maxit=400, inner=inner, out=l3)[1]
            if l64 is None:
                l64 = l3.clone()
            m3[inner] = {"ms_per_solve": ms3, "iterations": inf["iterations"], "relres": inf["relres"],
                         "rel_diff_vs_fp64_solution": float(torch.linalg.norm(l3 - l64) / torch.linalg.norm(l64))}
        s3.close()
    # uneven instances in one batch: 12 meshes N in {64..512}, k in {2,3,4} (seeded
    # mix), kappa = 1, FP64 reduced blocks; one hdg_apply_multi (one launch per
    # pass for all meshes) vs 12 single applies
    mi = {}
    if not args.profile:
        mix = inputs.instance_mix(12, seed=4)
        sols = hdg.setup_batch([(Nq, Nq, kq, torch.ones(Nq * Nq, dtype=torch.float64, device="cuda"))
                                for Nq, kq in mix], mixed=0)
        xs = [torch.as_tensor(inputs.random_trace(sq.n_edges, sq.k, seed=60 + q), device="cuda")
              for q, sq in enumerate(sols)]
        ys = [torch.empty_like(x) for x in xs]
        hdg.apply_multi(sols, xs, outs=ys)
        ms_multi = flushed_time(lambda: hdg.apply_multi(sols, xs, outs=ys), torch)

        def singles():
            for sq, x, y in zip(sols, xs, ys):
                sq.apply(x, out=y)

        ms_single = flushed_time(singles, torch)
        def red_q(n1):        # entries of the reduced blocks per element
            a_, b_ = n1 // 2 + n1 % 2, n1 // 2
            return sum(d * (d + 1) // 2 for d in (2 * a_, a_ + b_, a_ + b_, 2 * b_))
        algo = sum(sq.nel * red_q(sq.k + 1) * 8 + 2 * sq.n_edges * (sq.k + 1) * 8 for sq in sols)
        mi = {"instances": [[int(a_), int(b_)] for a_, b_ in mix],
              "kernels": "multi_red_elem_kernel + multi_red_face_kernel (reduced blocks, all 12 meshes)",
              "ms_batch": ms_multi, "launches_batch": 2, "ms_separate": ms_single,
              "launches_separate": sum(sq.get_info()["apply_kernels"] for sq in sols),
              "GBps_batch": algo / (ms_multi * 1e-3) / 1e9,
              "frac_hbm_batch": algo / (ms_multi * 1e-3) / 1e9 / peaks["hbm_gbs"],
              "algorithmic_bytes": algo, "timing": "cold L2, device time (CUDA graph)"}
        # the same 12 meshes solved to 1e-10 (one Fourier source each, seed 40 + q):
        # hdg_solve_multi (each on its own stream, all at once) vs one after another
        bsm = [sq.condense_rhs(torch.as_tensor(inputs.fourier_rhs(Nq, kq, 1, seed=40 + q)[0], device="cuda"))
               for q, (sq, (Nq, kq)) in enumerate(zip(sols, mix))]
        lsm = [torch.empty_like(b_) for b_ in bsm]
        hdg.solve_multi(sols, bsm, rtol=rtol, maxit=400, outs=lsm)

        def seq_solves():
            for sq, b_, l_ in zip(sols, bsm, lsm):
                sq.solve(b_, rtol=rtol, maxit=400, out=l_)

        ms_multi_solve = timed_events(lambda: hdg.solve_multi(sols, bsm, rtol=rtol, maxit=400, outs=lsm), 3, torch)
        ms_seq_solve = timed_events(seq_solves, 3, torch)
        mi["solve"] = {"what": "12 meshes to rtol 1e-10 (FP64 V-cycles), hdg_solve_multi vs 12 hdg_solve calls",
                       "ms_multi": ms_multi_solve, "ms_sequential": ms_seq_solve,
                       "speedup": ms_seq_solve / ms_multi_solve,
                       "iterations": [sq.solve(b_, rtol=rtol, maxit=400, out=l_)[1]["iterations"]
                                      for sq, b_, l_ in zip(sols, bsm, lsm)]}
        for sq in sols:
            sq.close()
    # launches in the timed region: condense 2 + recover 1 + CG
    vk = solver.get_info()["vcycle_kernels"]
    ak = solver.get_info()["apply_kernels"]
    # per CG iteration: apply, 2 dots kernels, x/r update, 2 dots, V-cycle, 2 dots, p update, commit;
    # the last iteration stops after the convergence check (no V-cycle, dots, p, commit)
    per_it = ak + 2 + 1 + 2 + vk + 2 + 1 + 1
    launches_per_step = 3 + (2 + vk + 2) + per_it * its - (vk + 4)
    # timing max over ranks
    t_ms = max_over_ranks(t_ms, world, "cuda")
    if rank != 0:
        solver.close()
        if world > 1:
            dist.destroy_process_group()
        return
    nel, ne, n1 = solver.nel, solver.n_edges, k + 1
    bytes_S = {"fp64": 8, "fp32": 4, "bf16": 2, "f32x2": 8}
    bytes_x = {"fp64": 8, "fp32": 4, "bf16": 4, "f32x2": 8}
    # reduced blocks: packed upper triangles of the four character blocks
    hh, se_, so_ = n1 // 2, n1 // 2 + n1 % 2, n1 // 2
    dims = (2 * se_, so_ + se_, se_ + so_, 2 * so_)
    q_red = sum(d * (d + 1) // 2 for d in dims)
    red_w = {"fp64": 8, "fp32": 4, "bf16": 4, "f32x2": 8}            # float cycles use the FP32 reduced blocks
    # FP64 operations per element: F x and F^T u (8 n1 + 16 h additions), the
    # block products (sum d^2 multiply-adds), the face sums of the second pass (2 n1)
    red_add = 8 * n1 + 16 * hh + 2 * n1
    red_fma = sum(d * d for d in dims)
    tra = {}
    for p_, ms in apply_ms.items():
        algo = nel * q_red * red_w[p_] + 2 * ne * n1 * bytes_x[p_]
        dense_eq = nel * 16 * n1 * n1 * bytes_S[p_] + 2 * ne * n1 * bytes_x[p_]
        gbs = algo / (ms * 1e-3) / 1e9
        tra[p_] = {"ms": ms, "kernels": "reduced_elem_kernel + reduced_face_kernel (cold L2, device time)", "GBps": gbs,
                   "frac_hbm": gbs / peaks["hbm_gbs"], "algorithmic_bytes": algo,
                   "scratch_bytes": 2 * nel * 4 * n1 * red_w[p_],
                   "dense_equivalent_GBps": dense_eq / (ms * 1e-3) / 1e9,
                   "fp64_ops_per_element": {"fma": red_fma, "add": red_add} if p_ == "fp64" else None}
        if p_ == "f32x2":
            tra[p_]["kernels"] += "; float2 (hi, lo) blocks, double-float arithmetic on the FP32 pipe"
            tra[p_]["double_float_ops_per_element"] = {"fma": red_fma, "add": red_add}
    tra["fp64"]["fp64_pipe_frac"] = nel * (red_fma + red_add) / (apply_ms["fp64"] * 1e-3) / (1.25e12 / 2)
    trd = {}
    for p_, ms in dense_ms.items():
        algo = nel * 16 * n1 * n1 * bytes_S[p_] + 2 * ne * n1 * bytes_x[p_]
        gbs = algo / (ms * 1e-3) / 1e9
        trd[p_] = {"ms": ms, "GBps": gbs, "frac_hbm": gbs / peaks["hbm_gbs"], "algorithmic_bytes": algo,
                   "flops": 2 * nel * 16 * n1 * n1}
    fp = trd["fp64"]
    tflops = fp["flops"] / (dense_ms["fp64"] * 1e-3) / 1e12
    # The step's dominant kernel is the dense owner-record apply of the Schwarz
    # blocks (4 launches per V-cycle at each p-level, no symmetry to reduce).
    # FP64: 0.25 flop/byte needs more FP64 issue than the GPU has (1.25 TFLOP/s
    # nominal), so it is bound by the FP64 pipe, not by HBM.
    # DRAM read+write of one such FP64 level-k launch at 512 x 512, k = 4 (ncu,
    # one-pass dram__bytes_read.sum + dram__bytes_write.sum, warm launches of
    # the set-up autotuner's choice, the 4-warp segment kernel, taken after the
    # kernel's last change): 859.9 MB + 18.2 MB
    traffic = 878.1e6 if (N, k) == (512, 4) else None
    roof = {"kernel": "FP64 Schwarz-block apply at level k (autotuned; apply_seg_kernel<5,double,double,double,0,4> "
                      "on GB300), timed on the condensed blocks of a reduced=0 context (same kernel, same bytes)",
            "bound": "alu", "achieved": tflops, "peak": 1.25, "unit": "TFLOP/s", "frac": tflops / 1.25,
            "peak_source": "nominal FP64 rate of GB300 (recipe table); HBM fraction in trace_apply_dense",
            "traffic": traffic, "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of this kernel at "
                                                  "512x512 k=4 (profiles/apply_k4_512_dram.md); null at other sizes",
            "algorithmic_bytes": fp["algorithmic_bytes"]}
    roof["peak_fp64_measured"] = fp64_tf
    roof["peak_fp64_measured_source"] = "cuBLAS DGEMM through torch.matmul, 4096^3 float64, best of 5 (this run)"
    roof["frac_of_measured_fp64"] = tflops / fp64_tf if fp64_tf > 0 else None
    if "128_k3" in mvo and m3:
        for inner in ("fp64", "fp32", "bf16", "f32x2"):
            if inner in m3:
                m3[inner]["err_vs_oracle"] = mvo["128_k3"][inner]["err_vs_oracle"]
                m3[inner]["err_vs_oracle_mesh"] = mvo["128_k3"]["mesh"]
    cpu = None
    if not args.no_cpu_baseline:
        try:
            cpu = run_cpu_baseline(N, k)
        except Exception as ex:  # reported, not fatal
            cpu = {"error": str(ex)[:300]}
    line = {
        "metric": METRIC, "value": job_throughput(world, t_ms), "unit": "solve/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "hdg_trace_gmg_pcg", "mesh": "%dx%d" % (N, N), "k": k,
                   "kappa": "lognormal sigma^2=1 l=0.05 seed 0", "f": 1, "rtol": rtol,
                   "ndof": solver.ndof, "cg_iterations": its, "final_relres": relres,
                   "l2": "inputs larger than L2 (FP64 reduced S %.0f MB + Schwarz blocks %.0f MB)"
                         % (nel * q_red * 8 / 1e6, nel * 16 * n1 * n1 * 8 / 1e6),
                   "parallelism": "replicas" if world > 1 else "single"},
        "setup_ms": info["setup_ms"], "device_bytes": info["device_bytes"],
        "roofline": roof, "trace_apply": tra, "trace_apply_dense": trd,
        "paper_context": {"what": "the paper's matrix-free FP64 trace apply on a Xeon Phi KNL 7210 ran at about 80% of "
                                  "its STREAM bandwidth (about 240 of 300 GB/s); context only, not a target",
                          "this_gpu_fp64_dense_frac_hbm": trd.get("fp64", {}).get("frac_hbm")},
        "local_ops_ms": local_ms, "mixed": mixed, "mixed_1024_k3": m3,
        "batched_solve": bs, "tau_kappa_variant": tk, "mixed_vs_oracle": mvo, "fsai_smoother": fsai,
        "config1_16x16_k1": c1, "adjoint_512_k2": adj, "fmg": fmg,
        "shared_batched_apply": sb, "multi_instance_apply": mi,
        "e2e": {"value": 1000.0 / e2e_ms, "unit": "solve/s", "ms_per_step": e2e_ms,
                "h2d_bytes_per_step": int(fq_h.nbytes), "d2h_bytes_per_step": int(solver.ndof * 8 + u.numel() * 8)},
        "gpu_launches": int(launches_per_step * args.steps),
        "clocks": clk, "peaks": peaks,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line))
    solver.close()
    if world > 1:
        dist.destroy_process_group()


def run_reference(args):
    _, rank, _ = rank_env()
    if rank != 0:          # the oracle runs once, on rank 0; other ranks exit without work
        return
    N, k = args.n, args.k
    n_sub = min(48, N)         # the same sub-mesh as the cpu_baseline leg of our arm
    for _ in range(args.warmup):
        _oracle_sample(8, N, k, SEED)
    times = []
    nel = None
    for _ in range(args.steps):
        t, nel = _oracle_sample(n_sub, N, k, SEED)
        times.append(t)
    t = statistics.median(times)
    per_solve = t / nel * N * N
    value = 1.0 / per_solve
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solve/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1000.0,
        "ms_per_full_solve_extrapolated": per_solve * 1000.0, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "hdg_trace_gmg_pcg", "mesh": "%dx%d" % (N, N), "k": k},
        "cpu_baseline": {"kind": "oracle", "cores": 1, "value": value, "unit": "solve/s",
                         "sample": "%dx%d sub-mesh per step (same h, kappa), oracle condense + SuperLU + recovery, "
                                   "scaled linearly by element count; a step is one sub-mesh sample, so "
                                   "ms_per_step is its measured time" % (n_sub, n_sub), "host": host_cpu(),
                         "threads": "one core: SuperLU and the oracle's per-element loops are single-threaded"},
        "e2e": {"value": value, "unit": "solve/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def run_profile_apply(args):
    """A small fixed launch sequence for kernel captures (ncu --set full): a
    context (lognormal kappa, seed 0; FP64 only for --prec fp64, about 6 GB on
    the device at 512^2, k = 4), then 3 applies of the condensed blocks in
    --prec on the reduced blocks (NVTX range apply_reduced) and 3 on the dense
    owner records with the autotuned kernel that also applies the Schwarz
    blocks (apply_dense)."""
    import torch

    from paper_1705_09907_gb300 import hdg, inputs

    N, k, prec = args.n, args.k, args.prec
    kap = torch.as_tensor(inputs.lognormal_kappa(N, SEED), device="cuda")
    x = torch.as_tensor(inputs.random_trace(2 * N * (N + 1), k, seed=1), device="cuda")
    if prec in ("fp32", "bf16"):
        x = x.float()
    y = torch.empty_like(x)
    for name, red in (("apply_reduced", 1), ("apply_dense", 0)):
        s = hdg.HDGSolver(N, N, k, kap, mixed=0 if prec == "fp64" else 1, reduced=red)
        for _ in range(args.warmup):
            s.apply(x, prec, out=y)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push(name)
        for _ in range(3):
            s.apply(x, prec, out=y)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        s.close()
    print(json.dumps({"profile_apply": True, "n": N, "k": k, "prec": prec}))


def run_profile_small(args):
    """Small fixed launch sequences for kernel captures of the column apply and
    the V-cycle (about 2 GB on the device): the column-batched apply of 64
    Fourier right-hand sides at 256^2, k = 5, kappa = 1 in --prec (NVTX range
    cols, after --warmup untimed ones), then V-cycles in --prec on a 256^2,
    k = 2 lognormal-kappa context (NVTX range vcycle)."""
    import torch

    from paper_1705_09907_gb300 import hdg, inputs

    prec = args.prec
    dt = torch.float64 if prec in ("fp64", "f32x2") else torch.float32
    sbm = hdg.HDGSolver(256, 256, 5, torch.ones(256 * 256, dtype=torch.float64, device="cuda"), autotune=0)
    B = sbm.condense_rhs(torch.as_tensor(inputs.fourier_rhs(256, 5, 64, seed=3), device="cuda")).to(dt)
    Y = torch.empty_like(B)
    for _ in range(args.warmup):
        sbm.apply(B, prec, out=Y)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("cols")
    for _ in range(3):
        sbm.apply(B, prec, out=Y)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    sbm.close()
    s = hdg.HDGSolver(256, 256, 2, torch.as_tensor(inputs.lognormal_kappa(256, SEED), device="cuda"))
    r = torch.as_tensor(inputs.random_trace(s.n_edges, 2, seed=1), device="cuda").to(dt)
    for _ in range(args.warmup):
        s.vcycle(r, prec=prec)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("vcycle")
    for _ in range(3):
        s.vcycle(r, prec=prec)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    s.close()
    print(json.dumps({"profile_small": True, "prec": prec}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N_DEFAULT)
    ap.add_argument("--k", type=int, default=K_DEFAULT)
    ap.add_argument("--apply-reps", type=int, default=30)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile", action="store_true", help="one solve step and 3 applies per precision, then exit")
    ap.add_argument("--profile-apply", action="store_true",
                    help="3 reduced and 3 dense condensed-block applies in --prec (kernel captures)")
    ap.add_argument("--profile-small", action="store_true",
                    help="column applies (256^2, k = 5, 64 right-hand sides) and V-cycles (256^2, k = 2) in --prec")
    ap.add_argument("--prec", default="fp64", choices=["fp64", "fp32", "bf16", "f32x2"])
    ap.add_argument("--clocks-log", default=None,
                    help="CSV path for the nvidia-smi clock samples (default: a temporary file)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.profile_apply:
        run_profile_apply(args)
    elif args.profile_small:
        run_profile_small(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
