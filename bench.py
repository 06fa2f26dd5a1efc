#!/usr/bin/env python
"""Throughput of the p-multigrid-preconditioned pressure-Poisson solve on GB300.

One step = one Runge-Kutta-stage pressure solve of the synthetic sigma-mapped wave tank
(512 x 32 quads on [0, 200] x [-1, eta], P = 6, curved surface, divergence right-hand
side): set the stage geometry, assemble the weak divergence, solve to a relative residual
of 1e-10.  Inputs are resident in HBM; L2 is flushed (256 MiB write) between steps.

Prints one JSON line (rank 0):
  value      free DOF x steps / device time, all ranks (replicas) together
  plain_fp64 the same steps with the plain FP64 p-multigrid (the comparison the target is
             stated against), speedup_vs_plain_fp64 the ratio
  roofline   the dominant kernel (the finest-level FP32 Schwarz sweep), timed alone with CUDA
             events: algorithmic bytes / time against the measured HBM peak, with the DRAM
             traffic of the recorded ncu capture while the kernel's sources are unchanged;
             roofline_outer_operator: the double-float outer operator against HBM;
             roofline_graded: the operator-apply kernels on a 10.1M-node tank of the same
             family with L2 flushed before every launch
  e2e        the same metric through pmg_set_geometry + pmg_solve_host, with the inputs
             copied from pinned host memory and the pressure copied back inside the timed
             region
  cpu_baseline  the FP64 CPU oracle on a bounded slice of the same tank

--impl reference times the oracle (the CPU reference implementation of this method).
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "Poisson solves/s x free DOF (DOF/s) to rel. residual 1e-10"
UNIT = "DOF/s"
L2_FLUSH_BYTES = 256 << 20


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="cfg2", choices=["cfg2", "cfg3", "cfg4", "cfg5", "paper", "bar"])
    ap.add_argument("--kernel-scaling", action="store_true",
                    help="time the hot kernels alone on config-2 tanks of growing length and report "
                         "their HBM roofline fractions")
    ap.add_argument("--variants", action="store_true",
                    help="cfg2/cfg3: every precision variant (iterations, time, error vs FP64) and the "
                         "operator kernels (FP64, FP32, BF16 tensor cores) side by side")
    ap.add_argument("--tank-steps", type=int, default=1000, help="cfg5: RK4 steps per run")
    ap.add_argument("--train-steps", type=int, default=200, help="cfg5: steps whose solves train the warm start")
    ap.add_argument("--scheme", default="rk4", choices=["rk4", "lserk54", "lserk54_mixed"],
                    help="cfg5 time integrator: classical RK4 (4 solves/step) or LSERK(5,4) (5 solves/step)")
    ap.add_argument("--filter", default="strong", choices=["strong", "few-percent", "none"],
                    help="cfg5 spectral filter after every step: strong = (P_c 0, alpha -36, beta 8), "
                         "few-percent = (P_c P-2, S(P) 0.97, beta 8)")
    ap.add_argument("--level-costs", action="store_true",
                    help="cfg2/cfg3: mixed solves with the level sequence cut after each level (finest and "
                         "coarse kept): time per outer iteration, and with it each level's cost")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-graded", action="store_true", help="skip the roofline_graded block (large tank)")
    ap.add_argument("--oracle-one-core-child", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--ncu-step", action="store_true",
                    help="profiling aid: one warm step, then one step inside the NVTX range 'profiled_step'")
    ap.add_argument("--ncu-large", action="store_true",
                    help="profiling aid: three launches each of the finest-level FP32 sweep (slab, 256 threads) and "
                         "the tiled level operator (8 x 8 elements) on a 9.5M-node tank (8192 x 32 quads, P = 6), "
                         "no autotuning")
    return ap.parse_args()


def aggregate_over_ranks(t_local, units_per_step, steps, ws, device="cpu"):
    """Whole-job rate of `ws` independent replicas (the path has no exchange step across
    tanks): the job lasts as long as its slowest rank, so the per-rank times are reduced by
    MAX over the process group (any backend: NCCL with CUDA tensors, gloo on the CPU), and
    value = ws * units_per_step * steps / t_max.  Returns (t_max, value)."""
    t = float(t_local)
    if ws > 1:
        import torch
        import torch.distributed as dist
        tt = torch.tensor([t], dtype=torch.float64, device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t = float(tt.item())
    return t, ws * units_per_step * steps / t


def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def workload(name):
    import workloads as W
    return W.config2() if name == "cfg2" else W.config3()


def oracle_slice():
    """A 32 x 32-cell, P = 6 slice of the config-2 tank (same cell size, depth
    resolution and generator seed)."""
    import workloads as W
    return W.tank(32, 32, 6, seed=W.BASE_SEED + 2)


def oracle_solve_timed(w, hier=None):
    """FP64 oracle p-MG-PCG solve to 1e-10 (operator assembly + PCG; the multigrid
    hierarchy is setup, excluded).  Returns (wall s, cpu s, free DOF, iterations, hier)."""
    from oracle import mg
    from oracle.sem import Mesh
    m = Mesh(**w.mesh_kwargs())
    F = w.fields(m.column_x(), m.row_sigma())
    b = m.rhs_divergence(F["eta"], F["u"], F["w"])
    if hier is None:
        hier = mg.Hierarchy(m, F["eta"], overlap=1, nu=2, omega=0.8)
    t0, c0 = time.perf_counter(), time.process_time()
    _, its, hist, _ = mg.solve(m, F["eta"], b, F["pD"], hier=hier, tol=1e-10)
    t1, c1 = time.perf_counter(), time.process_time()
    assert hist[-1] <= 1e-10
    return t1 - t0, c1 - c0, int((~m.dirichlet_mask()).sum()), its, hier


def _host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_one_core_child():
    """Child process of the one-core oracle timing: pinned to one CPU, BLAS on one thread
    (set in its environment by the parent), prints one JSON line."""
    try:
        os.sched_setaffinity(0, {sorted(os.sched_getaffinity(0))[0]})
    except (AttributeError, OSError):
        pass
    wall, cpu, nfree, its, _ = oracle_solve_timed(oracle_slice())
    print(json.dumps({"wall": wall, "cpu": cpu, "nfree": nfree, "its": its}), flush=True)


def oracle_one_core():
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               NUMEXPR_NUM_THREADS="1", VECLIB_MAXIMUM_THREADS="1")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-one-core-child"], env=env,
                       capture_output=True, text=True, timeout=600)
    lines = [x for x in r.stdout.splitlines() if x.startswith("{")]
    if r.returncode != 0 or not lines:
        return None
    return json.loads(lines[-1])


def cpu_baseline_entry():
    """The FP64 oracle (as it stands) on a bounded sample of the tank: one solve of the
    32 x 32-cell, P = 6 slice on all host cores (the BLAS thread pool), and one on a
    single core (child process pinned to one CPU, one BLAS thread)."""
    w = oracle_slice()
    wall, cpu, nfree, its, _ = oracle_solve_timed(w)
    nproc = _host_cores()
    out = {"value": nfree / wall, "unit": UNIT, "cores": nproc, "kind": "oracle",
           "cpu_utilisation": round(cpu / wall, 1), "nproc": nproc,
           "sample": f"one FP64 oracle p-MG-PCG solve to 1e-10 (assembly + PCG, setup excluded) of the "
                     f"32x32-cell P=6 slice of the tank ({nfree} free DOF, {its} iterations, {wall:.1f} s) on "
                     f"all {nproc} host cores (process CPU / wall = {cpu / wall:.1f})"}
    one = oracle_one_core()
    if one is not None:
        out["one_core"] = {"value": one["nfree"] / one["wall"], "unit": UNIT, "cores": 1,
                           "wall_s": round(one["wall"], 2), "iterations": one["its"]}
    return out


def cpu_baseline_paper(w):
    """CPU baseline of the paper-shape workload: the FP64 oracle p-MG-PCG (same levels and
    smoother) on the host cores at 1e-6 and 1e-10, setup included."""
    from oracle import mg as omg
    from oracle.sem import Mesh
    m = Mesh(**w.mesh_kwargs())
    F = w.fields(m.column_x(), m.row_sigma())
    bo = m.rhs_divergence(F["eta"], F["u"], F["w"])
    out = {"kind": "oracle", "sample": f"one solve of {w.name} per tolerance"}
    for tol in (1e-6, 1e-10):
        t0, c0 = time.perf_counter(), time.process_time()
        _, its, _, _ = omg.solve(m, F["eta"], bo, F["pD"], tol=tol, overlap=1, nu=2, omega=0.8)
        wall, cpu = time.perf_counter() - t0, time.process_time() - c0
        out[f"{tol:g}"] = {"iterations": its, "s_incl_setup": wall, "cores": round(cpu / wall, 1)}
    return out


def cpu_baseline_bar(w):
    """CPU baseline of the bar workload: the FP64 oracle p-MG-PCG with the same slope-free
    levels, one solve to 1e-10, setup included."""
    from oracle import mg as omg
    from oracle.sem import Mesh
    m = Mesh(**w.mesh_kwargs(), depth=w.bathymetry)
    F = w.fields(m.column_x(), m.row_sigma())
    bo = m.rhs_divergence(F["eta"], F["u"], F["w"])
    t0, c0 = time.perf_counter(), time.process_time()
    _, its, _, _ = omg.solve(m, F["eta"], bo, F["pD"], tol=1e-10, overlap=1, nu=2, omega=0.8)
    wall, cpu = time.perf_counter() - t0, time.process_time() - c0
    return {"kind": "oracle", "sample": f"one solve of {w.name} to 1e-10", "iterations": its,
            "s_incl_setup": wall, "cores": round(cpu / wall, 1)}


# ------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.path = None
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


NCU_RECORD = os.path.join(ROOT, "profiles", "ncu_traffic.json")
CSRC = os.path.join(ROOT, "paper_2411_14977_gb300", "csrc")
FDM32_SOURCES = ("k_fdm32.cu", "k_fdm32.cuh", "pmg_common.cuh", "pmg_kernels.h")
CURVED_SOURCES = ("k_curved.cuh", "k_apply.cu", "pmg_common.cuh", "pmg_kernels.h")


def source_digest(files):
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(CSRC, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_record(key, files):
    """The ncu counters of one kernel (DRAM bytes per launch = dram__bytes_read.sum +
    dram__bytes_write.sum, pipe utilisation) recorded from one capture in
    profiles/ncu_traffic.json, returned only while the kernel's sources are byte for byte
    those the capture was taken from; otherwise (None, reason)."""
    try:
        with open(NCU_RECORD) as fh:
            rec = json.load(fh).get(key)
    except (OSError, ValueError):
        rec = None
    if not rec:
        return None, "no ncu capture recorded for this kernel and workload"
    if rec.get("source_digest") != source_digest(files):
        return None, "stale: the kernel's sources changed after the ncu capture"
    return rec, rec.get("profile", "")


def cold_launch_us(torch, fn, flush, reps=10):
    """Median device time of one launch of fn after an L2 flush (a write of `flush`, larger
    than L2), CUDA events on the current stream; a GPU-side sleep after the flush keeps the
    launch queue ahead of the device so the events bracket the kernel alone."""
    st = torch.cuda.current_stream()
    ts = []
    for k in range(reps + 2):
        flush.fill_(1.0)
        if hasattr(torch.cuda, "_sleep"):
            torch.cuda._sleep(200000)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        fn()
        e1.record(st)
        e1.synchronize()
        if k >= 2:
            ts.append(1e3 * e0.elapsed_time(e1))
    return statistics.median(ts)


GRADED_CELLS_X = 8704   # 8704 x 32 quads at P = 6: 10.1M nodes, the size of the 64-problem batch


def graded_roofline(torch, pmg, dev, hbm, flush):
    """The operator-apply kernels at a size beyond L2 (a 10.1M-node tank of the same family,
    FP32 vectors of 40 MB) with L2 flushed before every launch: algorithmic bytes (the
    vectors each launch must read and write once, plus the geometry's column factors) /
    median cold launch time, against the measured HBM copy rate."""
    import workloads as W
    w = W.tank(GRADED_CELLS_X, 32, 6)
    S = pmg.Solver(**w.mesh_kwargs(), precision=pmg.PMG_MIXED_FP32)
    xc, sr = S.node_coords()
    F = w.fields(xc, sr)
    S.set_geometry(torch.as_tensor(np.ascontiguousarray(F["eta"]), dtype=torch.float64, device=dev))
    S.autotune()
    N, P = S.n, 6
    cols = GRADED_CELLS_X * (P + 1)
    r32, x32, y32 = (torch.randn(N, dtype=torch.float32, device=dev) for _ in range(3))
    x64, y64 = (torch.randn(N, dtype=torch.float64, device=dev) for _ in range(2))
    kern = {
        "k_fdm32 finest-level Schwarz sweep (FP32; r, x in, x out)":
            (lambda: S.level_sweep(0, r32, x32), 3.0 * N * 4),
        "k_flat finest-level operator (FP32; x in, y out)":
            (lambda: S.level_apply(0, x32, y32), 2.0 * N * 4),
        "k_curved actual-geometry operator (FP32; x in, y out, 4 column factors per node column)":
            (lambda: S.apply_f32(x32, y32), 2.0 * N * 4 + cols * 4 * 4),
        "k_curved outer operator (double-float on the FP32 pipe; FP64 x in, y out, column factors)":
            (lambda: S.apply(x64, y64), 2.0 * N * 8 + cols * 4 * 8),
    }
    out = {"workload": f"{w.name} ({GRADED_CELLS_X}x32 quads, P=6)", "nodes": N,
           "l2": "flushed before every launch (256 MiB write)", "peak": hbm, "unit": "GB/s",
           "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured), burst: kernels timed alone",
           "level0_kernels": S.level_kernels(0), "kernels": {}}
    for name, (fn, by) in kern.items():
        for _ in range(3):
            fn()
        us = cold_launch_us(torch, fn, flush)
        gbs = by / (us * 1e-6) / 1e9
        out["kernels"][name] = {"bound": "hbm", "avg_launch_us": us, "algorithmic_bytes_per_launch": by,
                                "achieved": gbs, "frac": gbs / hbm}
    S.close()
    del r32, x32, y32, x64, y64
    torch.cuda.empty_cache()
    return out


# ------------------------------------------------------------------------------------
def graph_launch_us(torch, fn, reps=50):
    """Device time per launch of fn: `reps` launches captured in one CUDA graph and
    replayed (CUDA events around the replays), so host-side call overhead is excluded."""
    for _ in range(5):
        fn()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    st = torch.cuda.Stream()
    st.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(st):
        with torch.cuda.graph(g, stream=st):
            for _ in range(reps):
                fn()
    torch.cuda.synchronize()
    g.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(4):
        g.replay()
    e1.record()
    torch.cuda.synchronize()
    return 1e3 * e0.elapsed_time(e1) / (4 * reps)


def run_ours(args, ws, rank, local):
    import torch
    import paper_2411_14977_gb300.pmg as pmg

    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pmg.load(build_if_missing=True)
    w = workload(args.workload)

    def setup(**opts):
        S = pmg.Solver(**w.mesh_kwargs(), **opts)
        xc, sr = S.node_coords()
        F = w.fields(xc, sr)
        S.set_geometry(torch.as_tensor(np.ascontiguousarray(F["eta"]), dtype=torch.float64, device=dev))
        S.autotune()  # CTA sizes of this mesh's kernels, picked by timing (setup, not timed)
        host = {k: torch.from_numpy(np.ascontiguousarray(F[k])).pin_memory() for k in ("eta", "u", "w", "pD")}
        devt = {k: v.to(dev) for k, v in host.items()}
        bufs = {"b": torch.empty(S.n, dtype=torch.float64, device=dev),
                "p": torch.empty(S.n, dtype=torch.float64, device=dev)}
        return S, host, devt, bufs

    def step(S, d, bufs):
        S.set_geometry(d["eta"])
        S.assemble_rhs_div(d["u"], d["w"], out=bufs["b"])
        _, info = S.solve(bufs["b"], d["pD"], out=bufs["p"])
        return info

    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    def timed(S, d, bufs, K):
        """Per-step CUDA-event device times (L2 flushed before each step, outside the events)."""
        evs, infos = [], []
        st = torch.cuda.current_stream()
        for _ in range(K):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            infos.append(step(S, d, bufs))
            e1.record(st)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in evs) / 1e3, infos

    def all_max(x):
        return aggregate_over_ranks(x, 1, 1, ws, device=dev)[0]

    # ---- headline: mixed precision (FP32 V-cycle inside FP64 refinement)
    S, host, d, bufs = setup(precision=pmg.PMG_MIXED_FP32)
    if args.ncu_step:
        step(S, d, bufs)
        # eager launches (the kernel-timing path): ncu does not profile kernel nodes of
        # graphs that hold conditional nodes; the kernels and their order are the same
        S.profile_reset(timing=True)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("profiled_step")
        info = step(S, d, bufs)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        log("ncu step:", info)
        return
    for _ in range(max(args.warmup, 3)):
        step(S, d, bufs)
    barrier()
    S.profile_reset(timing=False)
    clk = ClockSampler(local)
    barrier()
    t_dev, infos = timed(S, d, bufs, args.steps)
    barrier()
    clocks = clk.stop()
    prof = S.profile_read(full=True)
    launches = int(sum(v[0] for v in prof.values()))
    K = args.steps
    t_dev, value = aggregate_over_ranks(t_dev, S.n_free, K, ws, device=dev)
    for inf in infos:
        assert inf["status"] == 0 and inf["rel_residual"] <= 1e-10, inf

    # ---- profiled step (CUDA-event pairs around every launch): per-class device time
    S.profile_reset(timing=True)
    flush.fill_(1.0)
    step(S, d, bufs)
    pclass = S.profile_read(full=True)
    S.profile_reset(timing=False)
    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)

    def per_launch_us(fn, reps=50):
        return graph_launch_us(torch, fn, reps)

    # ---- dominant kernel: the finest-level FP32 Schwarz sweep (one launch per call),
    # timed alone: 50 launches captured in a CUDA graph (no host overhead); its vectors
    # (7 MB) stay in L2
    N0 = S.n
    r32 = torch.randn(N0, dtype=torch.float32, device=dev)
    x32 = torch.zeros(N0, dtype=torch.float32, device=dev)
    us_sweep = per_launch_us(lambda: S.level_sweep(0, r32, x32))
    bytes_sweep = 3.0 * N0 * 4  # r and x in, x out (FP32)
    achieved = bytes_sweep / (us_sweep * 1e-6) / 1e9
    p0 = S.level_info(0)[0]
    code0 = S.level_kernels(0)["fdm32"]
    kname = f"k_fdm32z<{p0},1> (z-split, {code0 // 1000} element rows, {code0 % 1000} threads)" if code0 >= 1000 \
        else f"k_fdm32<{p0},1,0> (slab, {code0} threads)"
    key = f"{kname.split(' ')[0]} {args.workload}"
    rec, src = ncu_record(key, FDM32_SOURCES)
    roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
            # dram__bytes_read.sum + dram__bytes_write.sum per launch from one ncu capture of
            # this kernel and workload, used only while its sources are unchanged
            "traffic": rec["dram_bytes_per_launch"] if rec else None,
            "traffic_source": src,
            "kernel": f"{kname} finest-level FP32 Schwarz sweep", "avg_launch_us": us_sweep,
            "algorithmic_bytes_per_launch": bytes_sweep,
            "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured); burst peak, kernel timed alone",
            "note": "latency-bound: the working set is L2-resident; see kernel_time_shares and roofline_graded"}
    # ---- the outer operator (double-float arithmetic on the FP32 pipe, FP64 vectors):
    # against HBM; its FP32-pipe utilisation is an ncu counter (recorded capture, if current)
    x64 = torch.randn(N0, dtype=torch.float64, device=dev)
    us_ap = per_launch_us(lambda: S.apply(x64))
    cols0 = S.mesh.cells_x * (p0 + 1)
    by_ap = 2.0 * N0 * 8 + cols0 * 4 * 8
    rec_o, src_o = ncu_record(f"k_curved<{p0},df64,2> {args.workload}", CURVED_SOURCES)
    roof_outer = {"bound": "hbm", "kernel": f"k_curved<{p0},df64> outer operator (FP64 in/out, double-float "
                                            f"arithmetic on the FP32 pipe)",
                  "avg_launch_us": us_ap, "algorithmic_bytes_per_launch": by_ap,
                  "achieved": by_ap / (us_ap * 1e-6) / 1e9, "peak": hbm, "unit": "GB/s",
                  "frac": by_ap / (us_ap * 1e-6) / 1e9 / hbm,
                  "fp32_pipe_busy_pct": rec_o.get("fma_pipe_busy_pct") if rec_o else None,
                  "fp64_pipe_busy_pct": rec_o.get("fp64_pipe_busy_pct") if rec_o else None,
                  "pipe_source": src_o,
                  "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured); burst peak, kernel timed alone"}
    shares = {k: round(v[1] / sum(x[1] for x in pclass.values()), 4) for k, v in pclass.items() if v[0]}

    # ---- plain FP64 p-multigrid on the same steps
    S64, _, d64, b64 = setup(precision=pmg.PMG_FP64)
    for _ in range(2):
        step(S64, d64, b64)
    barrier()
    K64 = max(3, K // 4)
    t64, inf64 = timed(S64, d64, b64, K64)
    barrier()
    t64 = all_max(t64)
    v64 = ws * S64.n_free * K64 / t64

    # ---- end to end through the host-buffer call: per step the stage surface (pinned host
    # -> device, then pmg_set_geometry) and pmg_solve_host with the step's load vector and
    # Dirichlet data in pinned host memory and the pressure back into pinned host memory
    b_host = bufs["b"].cpu().pin_memory()
    pD_host = host["pD"]
    pout = torch.empty(S.n, dtype=torch.float64).pin_memory()
    st = torch.cuda.current_stream()
    for _ in range(2):
        d["eta"].copy_(host["eta"], non_blocking=True)
        S.set_geometry(d["eta"])
        S.solve_host(b_host, pD_host, out=pout)
    barrier()
    evs = []
    for _ in range(K):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        d["eta"].copy_(host["eta"], non_blocking=True)
        S.set_geometry(d["eta"])
        _, ie = S.solve_host(b_host, pD_host, out=pout)
        e1.record(st)
        evs.append((e0, e1))
        assert ie["status"] == 0 and ie["rel_residual"] <= 1e-10, ie
    torch.cuda.synchronize()
    te = sum(a.elapsed_time(b) for a, b in evs) / 1e3
    barrier()
    te = all_max(te)
    h2d = host["eta"].numel() * 8 + b_host.numel() * 8 + pD_host.numel() * 8

    graded = None
    if rank == 0 and not args.no_graded:
        graded = graded_roofline(torch, pmg, dev, hbm, flush)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": K, "warmup": max(args.warmup, 3),
        "ms_per_step": 1e3 * t_dev / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": w.name + " (512x32 quads, P=6, curved sigma-mapped tank, divergence RHS)"
                   if args.workload == "cfg2" else w.name,
                   "nodes": S.n, "free_dof": S.n_free, "levels": [S.level_info(l)[0] for l in range(S.nlevels)],
                   "precision": "FP64 flexible CG (outer residual, inner products) preconditioned by an FP32 "
                                "V-cycle (operator, Schwarz smoother, transfers); FP64 coarse p=1 solve",
                   "cta_sizes": "autotuned at setup (64..512 threads per column slab; fused or split sweep residual)",
                   "level_kernels": [S.level_kernels(l) for l in range(S.nlevels)],
                   "smoother": "additive Schwarz (element + 1 overlap line, fast diagonalisation), nu=2, omega=0.8",
                   "tol": 1e-10, "l2": "flushed between steps (256 MiB write, outside the timed events)",
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                   "iterations": {"outer": infos[-1]["iterations"], "inner": infos[-1]["inner_iterations"]}},
        "solves_per_s": ws * K / t_dev,
        "plain_fp64": {"value": v64, "unit": UNIT, "ms_per_step": 1e3 * t64 / K64, "steps": K64,
                       "iterations": inf64[-1]["iterations"]},
        "speedup_vs_plain_fp64": value / v64,
        "roofline": roof,
        "roofline_outer_operator": roof_outer,
        "roofline_graded": graded,
        "kernel_time_shares": shares,
        "gpu_launches": launches,
        "e2e": {"value": ws * S.n_free * K / te, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": S.n * 8,
                "path": "pmg_set_geometry + pmg_solve_host (C ABI, pinned host buffers in and out); the step's "
                        "load vector is an input here (assembled once at setup), the device-timed step "
                        "assembles it"},
        "clocks": clocks,
    }
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_entry()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def run_batch(args, ws, rank, local):
    """Config 4: 64 independent tanks of uneven size and order solved as one batch (one CUDA
    graph whose launches each cover the work items of all 64 problems); inputs exceed L2."""
    import torch
    import paper_2411_14977_gb300.pmg as pmg
    import workloads as W

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pmg.load(build_if_missing=True)
    probs = W.config4()
    t_setup = time.perf_counter()
    B = pmg.Batch([w.mesh_kwargs() for w in probs], precision=pmg.PMG_MIXED_FP32)
    t_setup = time.perf_counter() - t_setup
    inputs = []
    for w, S in zip(probs, B.members):
        xc, sr = S.node_coords()
        F = w.fields(xc, sr)
        d = {k: torch.as_tensor(np.ascontiguousarray(F[k]), dtype=torch.float64, device=dev)
             for k in ("eta", "f", "g_bottom", "g_left", "g_right", "pD")}
        d["b"] = torch.empty(S.n, dtype=torch.float64, device=dev)
        d["p"] = torch.empty(S.n, dtype=torch.float64, device=dev)
        inputs.append(d)
    nfree = sum(S.n_free for S in B.members)

    def step():
        for S, d in zip(B.members, inputs):
            S.set_geometry(d["eta"])
            S.assemble_rhs(d["f"], d["g_bottom"], d["g_left"], d["g_right"], out=d["b"])
        _, infos = B.solve([d["b"] for d in inputs], [d["pD"] for d in inputs], [d["p"] for d in inputs])
        return infos

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    if args.ncu_step:
        # the same launches with the iteration loop on the host (a profiler does not see
        # kernels inside graphs with conditional nodes)
        B.set_path(1)
        torch.cuda.nvtx.range_push("profiled_step")
        infos = step()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        log("ncu step (cfg4, eager batch):", max(i["iterations"] for i in infos), "iterations")
        return
    clk = ClockSampler(local)
    evs = []
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        infos = step()
        e1.record()
        evs.append((e0, e1))
    torch.cuda.synchronize()
    clocks = clk.stop()
    t = sum(a.elapsed_time(b) for a, b in evs) / 1e3
    assert all(i["status"] == 0 and i["rel_residual"] <= 1e-10 for i in infos), infos
    # the same steps with each problem's own device-side loop on its own stream
    B.set_path(2)
    for _ in range(2):
        step()
    torch.cuda.synchronize()
    evs2 = []
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        step()
        e1.record()
        evs2.append((e0, e1))
    torch.cuda.synchronize()
    t_streams = sum(a.elapsed_time(b) for a, b in evs2) / 1e3
    B.set_path(0)
    # the same handles solved one after another (no concurrency)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for S, d in zip(B.members, inputs):
        S.set_geometry(d["eta"])
        S.assemble_rhs(d["f"], d["g_bottom"], d["g_left"], d["g_right"], out=d["b"])
        S.solve(d["b"], d["pD"], out=d["p"])
    e1.record()
    torch.cuda.synchronize()
    t_seq = e0.elapsed_time(e1) / 1e3
    # per-problem error of the mixed-precision pressure against FP64 p-MG on the same GPU
    errs = []
    for w, S, d in zip(probs, B.members, inputs):
        S64 = pmg.Solver(**w.mesh_kwargs(), precision=pmg.PMG_FP64, tol=1e-12)
        S64.set_geometry(d["eta"])
        p64, _ = S64.solve(d["b"], d["pD"])
        errs.append((torch.linalg.norm(d["p"] - p64) / torch.linalg.norm(p64)).item())
        S64.close()
    value = nfree * args.steps / t
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": "cfg4: 64 tanks, N_x in [64,1024], N_z in [8,32], P in [4,8], h in [0.5,2]",
                   "problems": len(probs), "free_dof": nfree, "l2": "inputs larger than L2",
                   "setup_s_incl_autotune": round(t_setup, 2)},
        "batch_path": B.info(),
        "per_problem_loops_value": nfree * args.steps / t_streams,
        "sequential_value": nfree / t_seq, "batch_speedup_vs_sequential": t_seq / (t / args.steps),
        "rel_err_vs_fp64": {"max": max(errs), "median": float(np.median(errs))},
        "iterations": {"min": min(i["iterations"] for i in infos), "max": max(i["iterations"] for i in infos)},
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


def run_paper(args, ws, rank, local):
    """The paper's own solver experiments in shape (Sec. 6.3): the Table 1 case (P = 8,
    N_x = 102, N_z = 2, 17 waves of kh = 1, H/L = 0.0301) at tolerances 1e-4 ... 1e-10
    with FP64 PCG, FP64 PDC, FP64 flexible GMRES and the mixed-precision solve, the oracle on the host cores
    beside it; then the scaling sweeps at tol 1e-6 (N_x = 25 ... 800 at P = 8; P = 2 ... 10
    at N_x = 200 with equal orders, and P_x = 2 ... 10 at P_z = 8 as in the paper; ~48 points
    per wavelength).  Device time per solve: CUDA events, median
    of `steps` solves from a zero initial guess."""
    import torch
    import paper_2411_14977_gb300.pmg as pmg
    import workloads as W

    if rank != 0:
        return
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pmg.load(build_if_missing=True)
    methods = [("fp64_pcg", dict(precision=pmg.PMG_FP64, outer=pmg.PMG_PCG)),
               ("fp64_pdc", dict(precision=pmg.PMG_FP64, outer=pmg.PMG_PDC)),
               ("fp64_gmres", dict(precision=pmg.PMG_FP64, outer=pmg.PMG_GMRES)),
               ("mixed", dict(precision=pmg.PMG_MIXED_FP32))]

    def prepare(w, **opts):
        S = pmg.Solver(**w.mesh_kwargs(), **opts)
        xc, sr = S.node_coords()
        F = w.fields(xc, sr)
        d = {k: torch.as_tensor(np.ascontiguousarray(F[k]), dtype=torch.float64, device=dev)
             for k in ("eta", "u", "w", "pD")}
        S.set_geometry(d["eta"])
        b = S.assemble_rhs_div(d["u"], d["w"])
        return S, b, d["pD"]

    def time_solve(S, b, pD):
        p = torch.empty_like(b)
        info = None
        for _ in range(2):
            _, info = S.solve(b, pD, out=p, raise_on_error=False)
        ts = []
        for _ in range(max(args.steps, 3)):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            _, info = S.solve(b, pD, out=p, raise_on_error=False)
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.median(ts)), info

    clk = ClockSampler(local)
    w = W.paper_shape()
    table = {}
    for name, opts in methods:
        for tol in (1e-4, 1e-6, 1e-8, 1e-10):
            S, b, pD = prepare(w, tol=tol, **opts)
            ms, info = time_solve(S, b, pD)
            table[f"{name}@{tol:g}"] = {"iterations": info["iterations"], "ms": ms, "status": info["status"],
                                        "rel_residual": info["rel_residual"],
                                        "nodes_per_s": S.n / (ms / 1e3)}
            log(name, tol, table[f"{name}@{tol:g}"])
            nodes = S.n
            S.close()
    # the same case on the paper's mixed-stage operator: stage k-1 = the wave one time step
    # (T/100) earlier; PDC and GMRES (the nonsymmetric operator rules out CG)
    from paper_2411_14977_gb300.stepper import G as GRAV
    kk, h0 = w.surface.k, w.h
    om = float(np.sqrt(GRAV * kk * np.tanh(kk * h0)))
    shift = (om / kk) * (2 * np.pi / om / 100)
    mixed_stage = {}
    for name, opts in (methods[1], methods[2]):
        for tol in (1e-4, 1e-6, 1e-8, 1e-10):
            S, b, pD = prepare(w, tol=tol, **opts)
            xc = torch.as_tensor(S.node_coords()[0], device=dev)
            eta_k = w.surface.amp * torch.cos(kk * xc)
            eta_km1 = w.surface.amp * torch.cos(kk * (xc + shift))
            S.set_geometry_mixed(eta_k.contiguous(), eta_km1.contiguous())
            ms, info = time_solve(S, b, pD)
            mixed_stage[f"{name}@{tol:g}"] = {"iterations": info["iterations"], "ms": ms, "status": info["status"],
                                              "rel_residual": info["rel_residual"]}
            log("mixed-stage", name, tol, mixed_stage[f"{name}@{tol:g}"])
            S.close()
    oracle = cpu_baseline_paper(w)
    # scaling sweeps at tol 1e-6
    sweep = {"cells_x": [], "order": []}
    for cx in (25, 50, 102, 200, 400, 800):
        row = {"cells_x": cx, "order": 8}
        for name, opts in (methods[0], methods[3]):
            S, b, pD = prepare(W.paper_scaling(cx, 8), tol=1e-6, **opts)
            ms, info = time_solve(S, b, pD)
            row[name] = {"iterations": info["iterations"], "ms": ms, "nodes": S.n}
            S.close()
        sweep["cells_x"].append(row)
        log("cells_x", row)
    for order in (2, 3, 4, 5, 6, 7, 8, 9, 10):
        row = {"cells_x": 200, "order": order}
        for name, opts in (methods[0], methods[3]):
            S, b, pD = prepare(W.paper_scaling(200, order), tol=1e-6, **opts)
            ms, info = time_solve(S, b, pD)
            row[name] = {"iterations": info["iterations"], "ms": ms, "nodes": S.n}
            S.close()
        sweep["order"].append(row)
        log("order", row)
    # the paper's own order sweep: P_x varied at N_x = 200 with the vertical order fixed at
    # P_z = 8 (semi-coarsened hierarchy)
    sweep["order_x_at_order_z_8"] = []
    for order in (2, 3, 4, 5, 6, 7, 8, 9, 10):
        row = {"cells_x": 200, "order_x": order, "order_z": 8}
        for name, opts in (methods[0], methods[3]):
            S, b, pD = prepare(W.paper_scaling(200, order, order_z=8), tol=1e-6, **opts)
            ms, info = time_solve(S, b, pD)
            row[name] = {"iterations": info["iterations"], "ms": ms, "nodes": S.n}
            S.close()
        sweep["order_x_at_order_z_8"].append(row)
        log("order_x (P_z = 8)", row)
    clocks = clk.stop()
    print(json.dumps({"workload": w.name, "nodes": int(nodes), "table1_shape": table,
                      "table1_shape_mixed_stage": mixed_stage, "cpu_baseline": oracle,
                      "scaling_tol1e-6": sweep, "clocks": clocks,
                      "paper_table1_context": {"pdc_mg_iterations": [3, 5, 8], "gmres_mg_iterations": [1, 3, 4],
                                               "tolerances": [1e-4, 1e-6, 1e-8],
                                               "note": "mixed-stage nonsymmetric operator, MATLAB, unstated CPU"}}),
          flush=True)


def run_bar(args, ws, rank, local):
    """Solves over a varying still-water depth (the bar geometry of Sec. 6, synthetic bar):
    the paper's bar discretisation (P = 8, N_x = 100, N_z = 2) and a 1.2M-node bar tank
    (P = 6, N_x = 2048, N_z = 16), FP64 PCG and the mixed-precision solve to 1e-10, each
    beside the same mesh over a flat bottom of the off-bar depth (what the slope-free level
    operator costs in iterations), the oracle's iteration count on the paper-size case,
    and the finest Schwarz sweep alone (per-column factors vs the constant-depth kernel).
    Device time per solve: CUDA events, median of `steps` solves from a zero guess."""
    import torch
    import paper_2411_14977_gb300.pmg as pmg
    import workloads as W

    if rank != 0:
        return
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pmg.load(build_if_missing=True)

    def prepare(w, flat_bottom=False, **opts):
        S = pmg.Solver(**w.mesh_kwargs(), **opts)
        xc, sr = S.node_coords()
        F = w.fields(xc, sr)
        d = {k: torch.as_tensor(np.ascontiguousarray(F[k]), dtype=torch.float64, device=dev)
             for k in ("eta", "u", "w", "pD", "h")}
        if not flat_bottom:
            S.set_bathymetry(d["h"])
        S.set_geometry(d["eta"])
        S.autotune()
        b = S.assemble_rhs_div(d["u"], d["w"])
        return S, b, d["pD"]

    def time_solve(S, b, pD):
        p = torch.empty_like(b)
        info = None
        for _ in range(2):
            _, info = S.solve(b, pD, out=p, raise_on_error=False)
        ts = []
        for _ in range(max(args.steps, 3)):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            _, info = S.solve(b, pD, out=p, raise_on_error=False)
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.median(ts)), info, p

    clk = ClockSampler(local)
    out = {}
    for w in (W.bar(100, 2, 8), W.bar(2048, 16, 6)):
        row = {}
        ref = None
        for name, opts in (("fp64_pcg", dict(precision=pmg.PMG_FP64)), ("mixed", dict(precision=pmg.PMG_MIXED_FP32))):
            for bottom in ("bar", "flat"):
                S, b, pD = prepare(w, flat_bottom=bottom == "flat", tol=1e-10, **opts)
                ms, info, p = time_solve(S, b, pD)
                e = {"iterations": info["iterations"], "ms": ms, "status": info["status"],
                     "rel_residual": info["rel_residual"], "dof_per_s": (S.n - S.level_info(0)[1]) / (ms / 1e3)}
                if bottom == "bar":
                    if ref is None:
                        ref = p.clone()
                    else:
                        e["rel_l2_vs_fp64"] = float(torch.linalg.norm(p - ref) / torch.linalg.norm(ref))
                row[f"{name}_{bottom}"] = e
                log(w.name, name, bottom, e)
                if bottom == "bar" and name == "mixed":
                    N0 = S.n
                    r32 = torch.randn(N0, dtype=torch.float32, device=dev)
                    x32 = torch.zeros(N0, dtype=torch.float32, device=dev)
                    row["sweep_us_per_column_factors"] = graph_launch_us(torch, lambda: S.level_sweep(0, r32, x32))
                    row["flat_op_us_per_column_depth"] = graph_launch_us(torch, lambda: S.level_apply(0, r32, x32))
                    x64 = torch.randn(N0, dtype=torch.float64, device=dev)
                    y64 = torch.empty_like(x64)
                    row["outer_apply_us_bathymetry"] = graph_launch_us(torch, lambda: S.apply(x64, y64))
                if bottom == "flat" and name == "mixed":
                    N0 = S.n
                    r32 = torch.randn(N0, dtype=torch.float32, device=dev)
                    x32 = torch.zeros(N0, dtype=torch.float32, device=dev)
                    row["sweep_us_constant_depth"] = graph_launch_us(torch, lambda: S.level_sweep(0, r32, x32))
                    row["flat_op_us_constant_depth"] = graph_launch_us(torch, lambda: S.level_apply(0, r32, x32))
                    x64 = torch.randn(N0, dtype=torch.float64, device=dev)
                    y64 = torch.empty_like(x64)
                    row["outer_apply_us_flat_bottom"] = graph_launch_us(torch, lambda: S.apply(x64, y64))
                nodes = S.n
                S.close()
        row["nodes"] = int(nodes)
        out[w.name] = row
    out["cpu_baseline"] = cpu_baseline_bar(W.bar(100, 2, 8))
    # time stepping over the bar: a surface hump (0.01 high, released at rest at x = 6) runs
    # 500 RK4 steps of 0.02 (10 s: across the bar) with one pressure solve per stage
    from paper_2411_14977_gb300.stepper import WaveTank
    wl = W.bar(100, 2, 8)
    stepping = {}
    etas = {}
    for name, opts in (("fp64_pcg", dict(precision=pmg.PMG_FP64)), ("mixed", dict(precision=pmg.PMG_MIXED_FP32))):
        tank = WaveTank(wl, filter=(0, -36.0, 8.0), scheme="rk4", dt=0.02, **opts)
        zero = np.zeros(tank.N)
        tank.set_state(0.01 * np.exp(-((tank.xc - 6.0) / 1.5) ** 2), zero, zero)
        for _ in range(10):
            tank.step()
        tank.solve_infos = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(490):
            tank.step()
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        infos = tank.solve_infos
        assert all(i["status"] == 0 for i in infos), name
        etas[name] = tank.eta.detach().cpu().numpy()
        stepping[name] = {"solves": len(infos), "solves_per_s": len(infos) / wall, "wall_s": wall,
                          "iterations_mean": float(np.mean([i["iterations"] for i in infos])),
                          "max_rel_residual": max(i["rel_residual"] for i in infos),
                          "final_max_eta": float(np.abs(etas[name]).max())}
        log("bar stepping", name, stepping[name])
    stepping["final_eta_maxdiff_mixed_vs_fp64_over_amp"] = float(np.abs(etas["mixed"] - etas["fp64_pcg"]).max() / 0.01)
    out["stepping_bar_p8_100x2"] = stepping
    print(json.dumps({"workload": "bar", "results": out, "clocks": clk.stop()}), flush=True)


def run_kernel_scaling(args, ws, rank, local):
    """The hot kernels alone (CUDA events around a CUDA graph of 50 launches) on the
    config-2 tank family (32 cells deep, P = 6) with 512 ... 16384 element columns: from an
    L2-resident working set (config 2: 2.4 MB per FP32 vector) to vectors 15x the 129 MB
    L2.  Achieved = algorithmic bytes / time against the measured HBM copy rate."""
    import torch
    import paper_2411_14977_gb300.pmg as pmg
    import workloads as W

    if rank != 0:
        return
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pmg.load(build_if_missing=True)
    hbm = measured_peaks().get("hbm_gbs", 6800.0)

    def per_launch_us(fn, reps=50):
        return graph_launch_us(torch, fn, reps)

    rows = []
    clk = ClockSampler(local)
    for cx in (512, 2048, 8192, 16384):
        w = W.tank(cx, 32, 6)
        S = pmg.Solver(**w.mesh_kwargs(), precision=pmg.PMG_MIXED_FP32)
        xc, sr = S.node_coords()
        F = w.fields(xc, sr)
        S.set_geometry(torch.as_tensor(np.ascontiguousarray(F["eta"]), dtype=torch.float64, device=dev))
        S.autotune()
        N = S.n
        f32 = lambda: torch.randn(N, dtype=torch.float32, device=dev)
        f64 = lambda: torch.randn(N, dtype=torch.float64, device=dev)
        r32, x32, y32, b32 = f32(), f32(), f32(), f32()
        x64, y64 = f64(), f64()
        P1 = 7
        E = cx * 32
        kern = {
            "k_fdm32 sweep (FP32)": (lambda: S.level_sweep(0, r32, x32), 3 * N * 4),
            "k_flat level residual (FP32)": (lambda: S.level_apply(0, x32, y32), 2 * N * 4),
            "k_curved operator (FP32)": (lambda: S.apply_f32(x32, y32), 2 * N * 4),
            "k_curved operator (double-float, FP64 vectors)": (lambda: S.apply(x64, y64), 2 * N * 8),
        }
        row = {"cells_x": cx, "nodes": N, "fp32_vector_MB": N * 4 / 1e6}
        for name, (fn, by) in kern.items():
            us = per_launch_us(fn)
            row[name] = {"us": us, "GB/s": by / (us * 1e-6) / 1e9, "frac_hbm": by / (us * 1e-6) / 1e9 / hbm}
        us = per_launch_us(lambda: S.apply(x64, y64))
        row["k_curved operator (double-float, FP64 vectors)"]["fp64_equiv_TFLOPs"] = \
            E * (8.0 * P1 ** 3 + 12.0 * P1 ** 2) / (us * 1e-6) / 1e12
        row["level0_kernels"] = S.level_kernels(0)
        # the tiled level operator forced (its best shape), beside the tuner's free choice
        St = pmg.Solver(**w.mesh_kwargs(), precision=pmg.PMG_MIXED_FP32, flat_kernel=2)
        St.set_geometry(torch.as_tensor(np.ascontiguousarray(F["eta"]), dtype=torch.float64, device=dev))
        St.autotune()
        us = per_launch_us(lambda: St.level_apply(0, x32, y32))
        row["k_flat_tile level operator (FP32, tiled forced)"] = {
            "us": us, "GB/s": 2 * N * 4 / (us * 1e-6) / 1e9, "frac_hbm": 2 * N * 4 / (us * 1e-6) / 1e9 / hbm,
            "shape": St.level_kernels(0)["flat32"]}
        St.close()
        # the bulk-staged level operator forced (its best CTA size)
        Sb = pmg.Solver(**w.mesh_kwargs(), precision=pmg.PMG_MIXED_FP32, flat_kernel=3)
        Sb.set_geometry(torch.as_tensor(np.ascontiguousarray(F["eta"]), dtype=torch.float64, device=dev))
        Sb.autotune()
        us = per_launch_us(lambda: Sb.level_apply(0, x32, y32))
        row["k_flat_bulk level operator (FP32, bulk-staged forced)"] = {
            "us": us, "GB/s": 2 * N * 4 / (us * 1e-6) / 1e9, "frac_hbm": 2 * N * 4 / (us * 1e-6) / 1e9 / hbm,
            "shape": Sb.level_kernels(0)["flat32"]}
        Sb.close()
        rows.append(row)
        log(cx, {k: (round(v["frac_hbm"], 3) if isinstance(v, dict) and "frac_hbm" in v else v) for k, v in row.items()})
        S.close()
        del r32, x32, y32, b32, x64, y64
        torch.cuda.empty_cache()
    clocks = clk.stop()
    print(json.dumps({"kernel_scaling": rows, "peak_hbm_gbs": hbm,
                      "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured), burst", "clocks": clocks}),
          flush=True)


def run_ncu_large(args, ws, rank, local):
    """Profiling aid: the finest-level FP32 sweep and the tiled level operator on a tank
    beyond L2, three launches each with fixed launch shapes, for an ncu capture of one
    launch (-s 2 -c 1) of either kernel."""
    import torch
    import paper_2411_14977_gb300.pmg as pmg
    import workloads as W

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pmg.load(build_if_missing=True)
    w = W.tank(8192, 32, 6)
    S = pmg.Solver(**w.mesh_kwargs(), precision=pmg.PMG_MIXED_FP32, flat_kernel=10808, sweep_kernel=0)
    xc, sr = S.node_coords()
    F = w.fields(xc, sr)
    S.set_geometry(torch.as_tensor(np.ascontiguousarray(F["eta"]), dtype=torch.float64, device=dev))
    g = torch.Generator(device=dev).manual_seed(W.BASE_SEED + 5)
    r32 = torch.randn(S.n, dtype=torch.float32, device=dev, generator=g)
    x32 = torch.randn(S.n, dtype=torch.float32, device=dev, generator=g)
    y32 = torch.empty(S.n, dtype=torch.float32, device=dev)
    for _ in range(3):
        S.level_sweep(0, r32, x32)
        S.level_apply(0, x32, y32)
    torch.cuda.synchronize()
    log("ncu-large:", S.n, "nodes", S.level_kernels(0))


def run_level_costs(args, ws, rank, local):
    """Cost of each multigrid level per outer iteration: the mixed solve with the level
    sequence P_0, ..., P_k, 1 for growing k (the finest and the order-1 coarse level always
    present), each autotuned; the difference of the times per outer iteration of two
    consecutive sequences is the cost of the level added, as the solve runs it (graph
    replay, L2-resident).  Also the same with the fused coarse V-cycle switched off."""
    import torch
    import paper_2411_14977_gb300.pmg as pmg

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pmg.load(build_if_missing=True)
    w = workload(args.workload)
    full = [ox for ox, _ in pmg.level_sequence(**w.mesh_kwargs())]
    rows = []
    for k in range(1, len(full)):
        seq = list(full[:k]) + [1]
        S = pmg.Solver(**w.mesh_kwargs(), precision=pmg.PMG_MIXED_FP32, level_orders=seq)
        xc, sr = S.node_coords()
        F = w.fields(xc, sr)
        d = {kk: torch.from_numpy(np.ascontiguousarray(F[kk])).to(dev) for kk in ("eta", "u", "w", "pD")}
        S.set_geometry(d["eta"])
        S.autotune()
        b = S.assemble_rhs_div(d["u"], d["w"])
        p = torch.empty_like(b)
        rec = {"levels": seq, "fused": S.fused_vcycle_info()}
        for on in ([0, 1] if rec["fused"]["first_level"] >= 0 else [0]):
            S.set_fused_vcycle(on)
            for _ in range(max(args.warmup, 3)):
                S.solve(b, d["pD"], out=p)
            torch.cuda.synchronize()
            st = torch.cuda.current_stream()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            for _ in range(args.steps):
                _, info = S.solve(b, d["pD"], out=p)
            e1.record(st)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / args.steps
            rec["fused_on" if on else "fused_off"] = {"ms_per_solve": ms, "iterations": info["iterations"],
                                                      "us_per_iteration": ms * 1e3 / info["iterations"]}
        rows.append(rec)
        log(json.dumps(rec))
        S.close()
    for a, b2 in zip(rows, rows[1:]):
        b2["added_level_us_per_iteration"] = (b2["fused_off"]["us_per_iteration"] -
                                              a["fused_off"]["us_per_iteration"])
    print(json.dumps({"metric": "us per outer iteration by level sequence (mixed solve, 1e-10)",
                      "workload": w.name, "full_sequence": list(full), "rows": rows}))


def run_variants(args, ws, rank, local):
    """Precision variants of the solve on one tank (config 3: 512 x 32, P = 8): plain FP64
    PCG, FP64 flexible CG around the FP32 V-cycle, FP64 refinement around an inner FP32
    flexible CG, and the same with the inner operator on the BF16 tensor cores.  Each:
    iterations, device time per solve (CUDA events, L2 flushed), relative L2 error against
    an FP64 solve to 1e-12.  Then the operator builds timed alone."""
    import torch
    import paper_2411_14977_gb300.pmg as pmg

    if rank != 0:
        return
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pmg.load(build_if_missing=True)
    w = workload(args.workload)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    variants = [("fp64_pcg", dict(precision=pmg.PMG_FP64)),
                ("mixed_fp32_fcg", dict(precision=pmg.PMG_MIXED_FP32)),
                ("mixed_fp32_ir", dict(precision=pmg.PMG_MIXED_FP32, outer=pmg.PMG_IR)),
                ("mixed_bf16_ir", dict(precision=pmg.PMG_MIXED_BF16, outer=pmg.PMG_IR)),
                ("mixed_fp32_fcg_dense_schwarz", dict(precision=pmg.PMG_MIXED_FP32, smoother=pmg.PMG_ASM_DENSE)),
                ("mixed_fp32_fcg_actual_levels", dict(precision=pmg.PMG_MIXED_FP32, smoother=pmg.PMG_ASM_DENSE,
                                                      precond_geom=pmg.PMG_ACTUAL)),
                # launch structure of the V-cycle: level residuals formed inside the sweeps
                # and restrictions (always, or where the autotuner times it faster), and the
                # coarse levels as one cooperative launch
                ("mixed_fp32_fcg_fused_residuals", dict(precision=pmg.PMG_MIXED_FP32, fuse_residual=1)),
                ("mixed_fp32_fcg_fused_residuals_tuned", dict(precision=pmg.PMG_MIXED_FP32, fuse_residual=-1)),
                ("mixed_fp32_fcg_fused_coarse_vcycle", dict(precision=pmg.PMG_MIXED_FP32, fuse_coarse=1))]
    ref = None
    out = {}
    clk = ClockSampler(local)
    ref_info = None
    for name, opts in [("reference_fp64_tol1e-12", dict(precision=pmg.PMG_FP64, tol=1e-12))] + variants:
        S = pmg.Solver(**w.mesh_kwargs(), **opts)
        xc, sr = S.node_coords()
        F = w.fields(xc, sr)
        d = {k: torch.as_tensor(np.ascontiguousarray(F[k]), dtype=torch.float64, device=dev)
             for k in ("eta", "u", "w", "pD")}
        S.set_geometry(d["eta"])
        S.autotune()
        b = S.assemble_rhs_div(d["u"], d["w"])
        p = torch.empty_like(b)
        if ref is None:
            _, ref_info = S.solve(b, d["pD"], out=p)
            ref = p.clone()
            S.close()
            continue
        for _ in range(max(args.warmup, 3)):
            S.solve(b, d["pD"], out=p)
        ts = []
        for _ in range(args.steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            _, info = S.solve(b, d["pD"], out=p)
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        err = (torch.linalg.norm(p - ref) / torch.linalg.norm(ref)).item()
        ms = float(np.median(ts))
        out[name] = {"ms_per_solve": ms, "dof_per_s": S.n_free / (ms / 1e3), "iterations": info["iterations"],
                     "inner_iterations": info["inner_iterations"], "rel_residual": info["rel_residual"],
                     "rel_l2_err_vs_fp64": err}
        if opts.get("smoother") == pmg.PMG_ASM_DENSE and "precond_geom" not in opts:
            # the finest dense sweep alone (block apply + per-node gather, one captured graph):
            # it streams the FP32 inverse blocks of every subdomain, far more than L2 holds
            r32 = torch.randn(S.n, dtype=torch.float32, device=dev)
            x32 = torch.zeros(S.n, dtype=torch.float32, device=dev)
            us = graph_launch_us(torch, lambda: S.level_sweep(0, r32, x32))
            p0 = S.level_info(0)[0]
            nb = (p0 + 3) ** 2
            E = w.cells_x * w.cells_z
            algo = E * nb * nb * 4.0 + E * nb * 4.0 * 2 + 3.0 * S.n * 4
            peaks = measured_peaks()
            out[name]["finest_sweep"] = {"us": us, "algorithmic_bytes": algo, "achieved_gbs": algo / (us * 1e-6) / 1e9,
                                         "hbm_frac_of_measured": algo / (us * 1e-6) / 1e9 / peaks.get("hbm_gbs", 6800.0)}
        if opts.get("precond_geom") == pmg.PMG_ACTUAL:
            # the levels follow the surface: pmg_set_geometry rebuilds them (dense inverses)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            S.set_geometry(d["eta"])
            e1.record()
            torch.cuda.synchronize()
            out[name]["set_geometry_ms"] = e0.elapsed_time(e1)
        log(name, out[name])
        if name == "mixed_bf16_ir":
            # the operator builds alone: CUDA-event time per launch (graph-free, warm)
            x32 = torch.randn(S.n, dtype=torch.float32, device=dev)
            x64 = x32.double()
            kern = {}
            for kname, fn in [("outer_fp64_vectors_double_float", lambda: S.apply(x64)),
                              ("fp32_cuda_cores", lambda: S.apply_f32(x32)),
                              ("bf16_tensor_split", lambda: S.apply_bf16(x32, split=True)),
                              ("bf16_tensor_plain", lambda: S.apply_bf16(x32, split=False))]:
                for _ in range(5):
                    fn()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                for _ in range(50):
                    fn()
                e1.record()
                torch.cuda.synchronize()
                kern[kname] = {"us_per_apply": 1e3 * e0.elapsed_time(e1) / 50}
            y64 = S.apply(x64)
            for kname, fn in [("fp32_cuda_cores", lambda: S.apply_f32(x32)),
                              ("bf16_tensor_split", lambda: S.apply_bf16(x32, split=True)),
                              ("bf16_tensor_plain", lambda: S.apply_bf16(x32, split=False))]:
                kern[kname]["rel_err_vs_fp64_apply"] = (torch.linalg.norm(fn().double() - y64) /
                                                        torch.linalg.norm(y64)).item()
            out["operator_kernels"] = kern
            log("kernels", kern)
        S.close()
    clocks = clk.stop()
    base = out["fp64_pcg"]["ms_per_solve"]
    for k, v in out.items():
        if "ms_per_solve" in v:
            v["speedup_vs_fp64"] = base / v["ms_per_solve"]
    print(json.dumps({"metric": METRIC, "workload": w.name, "nodes": int(S.n), "free_dof": int(S.n_free),
                      "tol": 1e-10, "l2": "flushed before every timed solve", "variants": out,
                      "reference": {"tol": 1e-12, "iterations": ref_info["iterations"],
                                    "rel_residual": ref_info["rel_residual"]},
                      "clocks": clocks}), flush=True)


SCHEME_NAMES = {"rk4": "RK4", "lserk54": "LSERK(5,4)",
                "lserk54_mixed": "LSERK(5,4) with the mixed-stage pressure-velocity coupling"}


def run_tank(args, ws, rank, local):
    """Config 5: a nonlinear progressive wave (eta0 = 0.05 cos(pi x), kh = pi) in the
    periodic 256 x 16, P = 6 tank, classical RK4 with dt = T/100, four pressure solves per
    step to a relative residual of 1e-10.  Three runs from the same initial state:
      plain_fp64     FP64 p-MG-PCG, x0 = previous stage's pressure
      mixed          FP64 flexible CG around the FP32 V-cycle, same x0
      mixed_learned  as mixed; the solves of the first train-steps steps train the warm
                     start network (pmg_ws_*), which then proposes x0 for the rest (kept
                     only where its residual beats the previous pressure; after 8
                     rejections in a row it is consulted on every 16th solve only)
      mixed_learned_smooth_c2 / _c3
                     as mixed_learned, predicting only the smooth part of the pressure
                     change: the training targets and the predictions pass through a
                     per-element modal low-pass keeping the modes <= 2 (or <= 3) per
                     direction (cutoff 2 or 3, alpha -36, beta 2)
      mixed_learned_always / mixed_learned_smooth_c3_always
                     the network's guess (plain, or its smooth part) used for every solve,
                     with no residual check
    Reported over the evaluation window (steps after train-steps): solves/s, iterations,
    solve time; and the final surface against the plain FP64 run."""
    import torch
    import paper_2411_14977_gb300.pmg as pmg
    import workloads as W
    from paper_2411_14977_gb300.stepper import WaveTank, G, RHO, default_filter
    from paper_2411_14977_gb300.warmstart import WarmStart

    if rank != 0:
        return
    torch.cuda.set_device(local)
    pmg.load(build_if_missing=True)
    w = W.config5()
    amp, k = 0.05, np.pi
    n_steps, n_train = args.tank_steps, min(args.train_steps, args.tank_steps)
    flt = {"strong": (0, -36.0, 8.0), "few-percent": default_filter(w.order), "none": None}[args.filter]
    clk = ClockSampler(local)

    def run(name, **kw):
        learned = kw.pop("learned", False)
        tank = WaveTank(w, record=learned, filter=flt, scheme=args.scheme, **kw)
        smooth = tank.S_smooth is not None
        om = tank.set_linear_wave(amp, k)
        tank.dt = 2 * np.pi / om / 100
        out = {"train_s": 0.0}
        windows = []
        t_start = None
        for s in range(n_steps):
            if s == n_train:
                torch.cuda.synchronize()
                if learned:
                    t0 = time.perf_counter()
                    sc = dict(s_eta=amp, s_deta=amp * om * tank.dt, s_p=RHO * G * amp,
                              s_dp=RHO * G * amp * om * tank.dt)
                    net = WarmStart(tank.NX, tank.NZ, period=w.order, hidden=128, taps=5, max_batch=32, seed=7,
                                    roughness=10.0, **sc)
                    samples = tank.samples[4:]
                    if smooth:  # learn only the smooth part of each pressure change
                        samples = [(e, ep, ex, pp, tank.smooth_change(p, pp)) for e, ep, ex, pp, p in samples]
                    hist = net.fit(samples, epochs=30, batch=32, lr=1e-3)
                    torch.cuda.synchronize()
                    out["train_s"] = time.perf_counter() - t0
                    out["train_loss"] = [hist[0], hist[-1]]
                    out["params"] = net.n_params
                    tank.samples.clear()
                    tank.record = False
                    tank.predictor = net
                tank.solve_infos, tank.guess_log = [], []
                t_start = time.perf_counter()
            tank.step()
        torch.cuda.synchronize()
        t_eval = time.perf_counter() - t_start
        infos = tank.solve_infos
        assert all(i["status"] == 0 for i in infos), name
        its = [i["iterations"] for i in infos]
        out.update({
            "solves": len(infos), "wall_s": t_eval, "solves_per_s": len(infos) / t_eval,
            "solve_s": sum(i["seconds"] for i in infos), "iterations_mean": float(np.mean(its)),
            "iterations_total": int(sum(its)), "max_rel_residual": max(i["rel_residual"] for i in infos),
        })
        if tank.guess_log:
            out["learned_guess_checked"] = len(tank.guess_log)
            out["learned_guess_kept"] = int(sum(r_nn < r_prev for r_prev, r_nn in tank.guess_log))
            out["median_residual_ratio_learned_vs_prev"] = float(
                np.median([r_nn / r_prev for r_prev, r_nn in tank.guess_log]))
        out["eta"] = tank.eta.detach().cpu().numpy()
        log(name, {k: v for k, v in out.items() if k != "eta"})
        return out

    # the mixed-stage operator is nonsymmetric: both arms iterate with flexible GMRES there
    outer64 = pmg.PMG_GMRES if args.scheme == "lserk54_mixed" else pmg.PMG_PCG
    res = {"plain_fp64": run("plain_fp64", precision=pmg.PMG_FP64, outer=outer64),
           "mixed": run("mixed", precision=pmg.PMG_MIXED_FP32),
           "mixed_learned": run("mixed_learned", learned=True, precision=pmg.PMG_MIXED_FP32)}
    if args.scheme == "rk4":
        for c in (2, 3):
            res[f"mixed_learned_smooth_c{c}"] = run(f"mixed_learned_smooth_c{c}", learned=True,
                                                    precision=pmg.PMG_MIXED_FP32, guess_smooth=(c, -36.0, 2.0))
        # the guess used for every solve (no residual check): what it does to the iterations
        res["mixed_learned_always"] = run("mixed_learned_always", learned=True, precision=pmg.PMG_MIXED_FP32,
                                          guess_policy="always")
        res["mixed_learned_smooth_c3_always"] = run("mixed_learned_smooth_c3_always", learned=True,
                                                    precision=pmg.PMG_MIXED_FP32, guess_smooth=(3, -36.0, 2.0),
                                                    guess_policy="always")
    clocks = clk.stop()
    eta64 = res["plain_fp64"]["eta"]
    for r in res.values():
        r["final_eta_maxdiff_vs_fp64_over_amp"] = float(np.abs(r.pop("eta") - eta64).max() / amp)
    best = res["mixed_learned"]
    line = {
        "metric": f"Poisson solves/s in {SCHEME_NAMES[args.scheme]} time stepping to rel. residual 1e-10 "
                  "(evaluation window)",
        "value": best["solves_per_s"], "unit": "solves/s", "n_gpus": 1, "steps": n_steps - n_train,
        "warmup": n_train, "ms_per_step": 1e3 * best["wall_s"] / max(1, n_steps - n_train),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": "cfg5: periodic tank [0,20]x[-1,eta], 256x16 cells, P=6, eta0=0.05cos(pi x), "
                               f"{SCHEME_NAMES[args.scheme]} dt=T/100",
                   "tank_steps": n_steps, "train_steps": n_train,
                   "filter": None if flt is None else {"cutoff": flt[0], "alpha": flt[1], "beta": flt[2]},
                   "free_dof": 1536 * 96},
        "runs": res,
        "speedup_vs_plain_fp64": best["solves_per_s"] / res["plain_fp64"]["solves_per_s"],
        "learned_vs_mixed_iterations": {k: r["iterations_total"] / res["mixed"]["iterations_total"]
                                        for k, r in res.items() if k.startswith("mixed_learned")},
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


def run_reference(args, ws, rank):
    if rank != 0:
        return
    w = oracle_slice()
    hier = None
    for _ in range(args.warmup):
        _, _, _, _, hier = oracle_solve_timed(w, hier)
    walls, cpus, nfree, its = [], [], 0, 0
    for _ in range(args.steps):
        wall, cpu, nfree, its, hier = oracle_solve_timed(w, hier)
        walls.append(wall)
        cpus.append(cpu)
    t = sum(walls)
    value = nfree * args.steps / t
    sample = (f"each step: one FP64 oracle p-MG-PCG solve to 1e-10 (assembly + PCG, setup excluded) of the "
              f"32x32-cell P=6 slice of the tank ({nfree} free DOF, {its} iterations)")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "cfg2_p6_512x32 tank family, 32x32-cell slice (oracle on host cores)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": round(sum(cpus) / t, 1), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    args = parse()
    if args.oracle_one_core_child:
        oracle_one_core_child()
        return
    ws, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, ws, rank)
    elif args.workload == "cfg4":
        run_batch(args, ws, rank, local)
    elif args.workload == "cfg5":
        run_tank(args, ws, rank, local)
    elif args.workload == "paper":
        run_paper(args, ws, rank, local)
    elif args.workload == "bar":
        run_bar(args, ws, rank, local)
    elif args.variants:
        run_variants(args, ws, rank, local)
    elif args.kernel_scaling:
        run_kernel_scaling(args, ws, rank, local)
    elif args.level_costs:
        run_level_costs(args, ws, rank, local)
    elif args.ncu_large:
        run_ncu_large(args, ws, rank, local)
    else:
        run_ours(args, ws, rank, local)


if __name__ == "__main__":
    main()
