#!/usr/bin/env python3
"""Served vs plain FP64 deflated block-Jacobi Schur-complement GMRES.

Default workload (the headline line): a stream of Poisson / Helmholtz solve
requests -- grids drawn uniformly from 64x2, 128x4, 256x8, 512x16 and 1024x16
elements (square elements, domain [0, mx/mz] x [0, 1]), orders uniform from
{6, 8, 12, 16}, k^2 = 0 with probability 0.1 else log-uniform on
[1e-2, 1e4], f a seeded sum of 32 cos-cos modes per request -- each solved to
a relative Schur residual of 1e-10 (Alg. seq; the Helmholtz form of Sec. 5).
A step is --requests-per-step (default 100) consecutive requests of the
stream, so --steps 20 is the 2000-request stream.  Two paths serve it:

* plain: one request at a time, smpm_setup + smpm_solve + smpm_release,
  FP64 throughout;
* served: the serving runtime (smpm_server_*: worker streams, continuous
  batching of same-grid requests, HBM-footprint admission, operator cache),
  nested mixed precision (FP64 flexible GMRES outside, FP32 inner DBJ-GMRES).

value = served solves/s with the whole stream submitted at once (inputs
resident in HBM); plain_value = the plain path's solves/s; p50/p99 latency
(completion - arrival, setup included) of both under Poisson arrivals at the
rate where the plain path saturates (its measured service rate; the plain
path's latencies follow from its measured service times by the FIFO queue
recursion, the served ones are measured live).  e2e = the served solves/s
with f and u in pinned host memory (the copies inside the library calls).
Every rank serves its own stream (weak scaling, no collective on the data
path).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                  [--workload serve|poisson2d|small|modes3d|mixed]

--workload poisson2d is the 256 x 4, order-12 batched FP64 solve (128
right-hand sides per step); small / modes3d / mixed are the 8 x 2 latency,
3-D Fourier-mode and 512 x 16 mixed-precision configurations.  --impl
reference times the CPU oracle (oracle/, numpy/scipy FP64, Alg. seq with
Householder GMRES) on the host cores on a bounded sample of the same
workload.
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
sys.path.insert(0, ROOT)

GRID = dict(mx=256, mz=4, order=12, lx=64.0, lz=1.0)
WORKLOAD = "2-D Poisson-Neumann, 256x4 elements, order 12, domain 64x1, 32 seeded cos-cos modes, g=0"
METRIC = "solves/s at 1e-10 rel. residual (plain FP64 DBJ-GMRES)"
METRIC_SERVE = "solves/s at 1e-10 rel. residual, p50/p99 latency: served vs plain FP64 GMRES"
TOL = 1e-10
FP64_NOMINAL_TFLOPS = 1.25     # GB300 FP64 (non-tensor and tensor), profiling recipe table
# FP32 CUDA-core peak from unit counts and clock: 152 SMs x 128 FP32 lanes x 2 FLOP x 2.07 GHz
FP32_SIMT_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
ORACLE_MAX_NODES = 50_000      # cpu_baseline / reference arm: requests the oracle finishes in seconds
L2_FLUSH_BYTES = 256 << 20


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--rhs", type=int, default=128, help="right-hand sides per step (one batched solve)")
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--cpu-sample", type=int, default=2, help="poisson2d: oracle right-hand sides in the cpu_baseline leg")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-secondary", action="store_true", help="serve: skip the 256x4 secondary figure")
    p.add_argument("--workload", default="serve", choices=["serve", "poisson2d", "small", "modes3d", "mixed"],
                   help="serve: the request stream, served vs plain (the default line); poisson2d / small / "
                        "modes3d / mixed: the 256x4 batched, 8x2 latency, 3-D and mixed-precision configurations")
    p.add_argument("--requests-per-step", type=int, default=100, help="serve: requests of the stream per step")
    p.add_argument("--cpu-seconds", type=float, default=20.0, help="serve: oracle time budget of the cpu_baseline leg")
    p.add_argument("--profiled-requests", type=int, default=300,
                   help="serve: requests re-run with the dense-product profile on (roofline)")
    p.add_argument("--mixed-rhs", type=int, default=16, help="mixed: right-hand sides per step")
    p.add_argument("--workers", type=int, default=4, help="serve: server worker threads (one stream each)")
    p.add_argument("--max-batch", type=int, default=16, help="serve: requests per batch at most")
    p.add_argument("--served-precision", type=int, default=2, choices=[0, 1, 2],
                   help="serve: precision of the served solves (the plain baseline is always FP64)")
    return p.parse_args()


def rank_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")), int(os.environ.get("WORLD_SIZE", "1"))


def rank_seed0(rank):
    """First seed of a rank's right-hand sides: every rank solves its own
    batch (weak scaling), seeds 1000 apart so batches never overlap."""
    from paper_1512_01756_gb300 import inputs
    return inputs.seed_for(1) + 1000 * rank


def max_over_ranks(value, device, world):
    """Max of a per-rank float over the process group (the slowest rank's
    time decides the job's throughput); the value itself when world == 1."""
    import torch
    t = torch.tensor([float(value)], device=device, dtype=torch.float64)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def make_f(x, z, nrhs, seed0):
    import numpy as np
    from paper_1512_01756_gb300 import inputs
    F = np.empty((nrhs, x.size))
    for i in range(nrhs):
        spec = inputs.cos_modes_spec(seed0 + i)
        F[i], _ = inputs.cos_modes(x, z, GRID["lx"], GRID["lz"], spec)
    return F


class Clocks:
    """nvidia-smi sampler running during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [t.strip() for t in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dense_product_source_sha():
    """sha256 (16 hex digits) of the dense-product kernels' source: the part of
    kernels.cu from the class GEMM's header comment to the deflation section."""
    text = open(os.path.join(ROOT, "paper_1512_01756_gb300", "csrc", "kernels.cu"), "rb").read()
    i, j = text.find(b"// Class GEMM:"), text.find(b"// Deflation (Sec. 3.3)")
    return hashlib.sha256(text[i:j] if 0 <= i < j else text).hexdigest()[:16]


def traffic_per_launch():
    """DRAM bytes per dense-product launch from the committed ncu summary, if it was
    taken on the current dense-product kernels (else None)."""
    path = os.path.join(ROOT, "profiles", "gemm_traffic.txt")
    if not os.path.exists(path):
        return None
    kv = {}
    for line in open(path):
        if "=" in line and not line.startswith("#"):
            k, v = line.split("=", 1)
            kv[k.strip()] = v.strip()
    if kv.get("dense_product_source_sha256_16") != dense_product_source_sha():
        return None
    try:
        return float(kv["dram_bytes_per_launch_scaled"])
    except (KeyError, ValueError):
        return None


def oracle_solves_per_s(nrhs, seed0):
    """Time the CPU oracle (setup excluded, as on the GPU side): returns
    (solves/s, effective cores, seconds)."""
    import numpy as np
    from oracle.smpm import Grid
    from oracle.schur import StripSchur
    from oracle import dbj
    g = Grid(GRID["mx"], GRID["mz"], GRID["order"], GRID["lx"], GRID["lz"])
    X, Z = g.coords()
    F = make_f(X, Z, nrhs, seed0)
    sch = StripSchur(g)
    c0, w0 = os.times(), time.perf_counter()
    for i in range(nrhs):
        _, info = dbj.solve(g, F[i], method="dbj", tol=TOL, schur=sch)
        assert info["schur_residual"] < 10 * TOL
    w1, c1 = time.perf_counter(), os.times()
    cpu = (c1.user - c0.user) + (c1.system - c0.system)
    cores = max(1, round(cpu / (w1 - w0)))
    del np
    return nrhs / (w1 - w0), cores, w1 - w0


def run_reference(args):
    rank, _, world = rank_env()
    if rank != 0:
        return 0
    from oracle.smpm import Grid
    from oracle.schur import StripSchur
    from oracle import dbj
    g = Grid(GRID["mx"], GRID["mz"], GRID["order"], GRID["lx"], GRID["lz"])
    X, Z = g.coords()
    from paper_1512_01756_gb300 import inputs
    sch = StripSchur(g)
    seed0 = inputs.seed_for(1)
    F = make_f(X, Z, args.warmup + args.steps, seed0)
    for i in range(args.warmup):
        dbj.solve(g, F[i], method="dbj", tol=TOL, schur=sch)
    c0, w0 = os.times(), time.perf_counter()
    for i in range(args.steps):
        dbj.solve(g, F[args.warmup + i], method="dbj", tol=TOL, schur=sch)
    w1, c1 = time.perf_counter(), os.times()
    el = w1 - w0
    cores = max(1, round(((c1.user - c0.user) + (c1.system - c0.system)) / el))
    val = args.steps / el
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "rhs_per_step": 1, "solver": "oracle Alg. seq, Householder GMRES"},
            "cpu_baseline": {"value": val, "unit": "solves/s", "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} right-hand sides, one per step (operator setup excluded)"},
            "e2e": {"value": val, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_poisson2d(args):
    import numpy as np
    import torch
    import torch.distributed as dist
    import __graft_entry__
    __graft_entry__.build()
    from paper_1512_01756_gb300 import smpm, inputs

    rank, local, world = rank_env()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    stream = torch.cuda.current_stream()
    R = args.rhs
    grid = smpm.make_grid(**GRID)
    solver = smpm.Solver(grid, 0.0, stream)
    x, z = solver.coords()
    F = make_f(x, z, R, rank_seed0(rank))
    Fd = torch.from_numpy(F).to(dev)
    Ud = torch.empty_like(Fd)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        st = solver.solve(Fd, Ud, tol=TOL)
    barrier()
    clocks = Clocks(local)
    clocks.start()
    l0 = smpm.kernel_launches()

    def timed_steps():
        ts, sts = [], []
        for _ in range(args.steps):
            flush.fill_(1.0)                      # evict L2 between steps (not timed)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = solver.solve(Fd, Ud, tol=TOL)
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
            sts.append(st.as_dict())
        return ts, sts
    times, stats = timed_steps()              # the value: profile off
    launches = smpm.kernel_launches() - l0
    barrier()
    clk = clocks.stop()
    # roofline: the same steps again with events around every dense-product launch
    solver.profile(True)
    solver.profile_read(reset=True)
    times_prof, _ = timed_steps()
    prof = solver.profile_read(reset=True)
    solver.profile(False)
    barrier()
    ms = sum(times) / len(times)
    ms_max = max_over_ranks(ms, dev, world)
    worst_res = max(s["rel_resid_true"] for s in stats)
    iters = [s["iters"] for s in stats]

    # end to end: pinned host buffers through the same C ABI (copies inside the call)
    Fh = torch.from_numpy(F).pin_memory()
    Uh = torch.empty_like(Fh).pin_memory()
    solver.solve(Fh.numpy(), Uh.numpy(), tol=TOL)
    barrier()
    e2e_times = []
    for _ in range(args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        solver.solve(Fh.numpy(), Uh.numpy(), tol=TOL)
        e2e_times.append(time.perf_counter() - w0)
    e2e_s = max_over_ranks(sum(e2e_times) / len(e2e_times), dev, world)
    assert np.allclose(Uh.numpy(), Ud.cpu().numpy(), rtol=0, atol=1e-9 * np.abs(Uh.numpy()).max())

    fp64_probe = smpm.probe_fp64(stream)
    peak = FP64_NOMINAL_TFLOPS
    achieved = prof["flops"] / (prof["ms"] * 1e-3) / 1e12 if prof["ms"] > 0 else None
    launches_gemm = max(prof["launches"], 1)
    tr = traffic_per_launch()
    roofline = {"bound": "alu", "kernel": "mirror_gemm_kernel + class_gemm_kernel (FP64 DFMA: Schur products, block-Jacobi, strip-solver slots)",
                "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": (achieved / peak) if achieved else None,
                "traffic": tr,
                "peak_source": "recipe FP64 1.25 TFLOP/s (GB300); measured DFMA probe %.3f TFLOP/s" % fp64_probe,
                "flops_per_launch": prof["flops"] / launches_gemm,
                "ms_per_launch": prof["ms"] / launches_gemm,
                "gemm_share_of_step": prof["ms"] / sum(times_prof),
                "profiled_ms_per_step": sum(times_prof) / len(times_prof)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, cores, secs = oracle_solves_per_s(args.cpu_sample, inputs.seed_for(1))
        cpu = {"value": v, "unit": "solves/s", "cores": cores, "kind": "oracle",
               "sample": f"{args.cpu_sample} right-hand sides of the same workload ({secs:.1f} s; operator setup excluded)"}

    nb_in = F.nbytes
    line = {"metric": METRIC, "value": R * world / (ms_max * 1e-3), "unit": "solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "rhs_per_step": R, "tol": TOL, "restart": 64,
                       "l2": "flushed between timed steps (256 MiB write, untimed)",
                       "parallelism": f"independent rhs batches per GPU x{world}"},
            "e2e": {"value": R * world / e2e_s, "unit": "solves/s", "h2d_bytes_per_step": nb_in,
                    "d2h_bytes_per_step": nb_in},
            "gpu_launches": launches,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "clocks": clk,
            "solver": {"iters_per_step": iters, "worst_rel_resid": worst_res, "setup_ms": stats[0]["setup_ms"],
                       "device_bytes": solver.device_bytes()}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    solver.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_other(args):
    """Separate measurements: the 8x2 latency case, the 3-D mode batch and the
    mixed-precision solves (one JSON line each; the default line is the
    serving workload)."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1512_01756_gb300 import smpm, inputs
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    lines = []

    def timed(fn, solver=None):
        for _ in range(args.warmup):
            fn()
        if solver is not None:
            solver.profile_read(reset=True)      # count only the timed solves
        ts = []
        for _ in range(args.steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = fn()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return sum(ts) / len(ts), st

    def gemm_roofline(s, ms_total, peak, dtype):
        p = s.profile_read(reset=True)
        if p["ms"] <= 0:
            return None
        ach = p["flops"] / (p["ms"] * 1e-3) / 1e12
        return {"bound": "alu", "kernel": f"mirror_gemm_kernel + class_gemm_kernel ({dtype})", "achieved": ach, "peak": peak,
                "unit": "TFLOP/s", "frac": ach / peak if peak else None, "launches": p["launches"],
                "gemm_share_of_step": p["ms"] / ms_total}

    if args.workload == "small":
        # 4 x 1 manufactured case, 8 x 2 elements, order 8: latency of one solve
        for groups in (0, 1):
            s = smpm.Solver(smpm.make_grid(8, 2, 8, 4.0, 1.0, deflation_groups=groups), 0.0, stream)
            x, z = s.coords()
            f, _ = inputs.manufactured_cos(x, z, 4.0, 1.0)
            Fd = torch.from_numpy(f).to(dev)
            Ud = torch.empty_like(Fd)
            ms, st = timed(lambda: s.solve(Fd, Ud, tol=TOL))
            lines.append({"workload": "2-D Poisson-Neumann 8x2 elements, order 8, domain 4x1, manufactured "
                                      "u = cos(pi x/4) cos(pi z), one right-hand side",
                          "deflation": "one vector per interface" if groups == 0 else "one per interface and element row",
                          "metric": "us per solve at 1e-10 rel. residual", "value": ms * 1e3,
                          "iters": st.iters, "worst_rel_resid": st.rel_resid_true, "setup_ms": st.setup_ms})
            s.close()
    elif args.workload == "modes3d":
        s = smpm.Solver3D(smpm.make_grid(128, 8, 10, 32.0, 1.0), 128, 2 * np.pi, stream)
        f3 = inputs.uniform((s.r, 128), inputs.seed_for(2))
        fh = np.fft.rfft(f3, axis=1) / 128
        F = torch.from_numpy(np.ascontiguousarray(np.stack([fh.real.T, fh.imag.T], axis=1))).to(dev)
        U = torch.empty_like(F)
        s.profile(True)
        ms, st = timed(lambda: s.solve_3d(F, U, tol=TOL), s)
        roof = gemm_roofline(s, ms * args.steps, FP64_NOMINAL_TFLOPS, "FP64")
        lines.append({"roofline": roof, "workload": "3-D via Fourier: 128x8 elements, order 10, domain 32x1, m_y = 128 (65 modes, "
                                  "k_j = j), U[0,1] right-hand side, all modes in one batched solve",
                      "metric": "3-D solves/s at 1e-10 rel. residual (every mode)", "value": 1e3 / ms,
                      "ms_per_solve": ms, "iters": st.iters, "worst_rel_resid": st.rel_resid_true,
                      "setup_ms": st.setup_ms, "device_bytes": s.device_bytes()})
        # the same solve in physical space (y-DFTs on the GPU around the mode solve)
        F3 = torch.from_numpy(np.ascontiguousarray(f3.T)).to(dev)
        U3 = torch.empty_like(F3)
        msp, stp = timed(lambda: s.solve_3d_physical(F3, U3, tol=TOL))
        lines.append({"workload": "3-D via Fourier, physical space: the same 128x8, order 10, m_y = 128 problem "
                                  "given as 128 y-planes; y-DFTs on the GPU around the batched mode solve",
                      "metric": "3-D solves/s at 1e-10 rel. residual (every mode)", "value": 1e3 / msp,
                      "ms_per_solve": msp, "iters": stp.iters, "worst_rel_resid": stp.rel_resid_true})
        s.close()
        # Alg. 3d as printed: one concatenated GMRES over every mode (dot
        # products summed over the modes, one convergence test on the whole
        # residual) against the per-mode Krylov spaces above
        sc = smpm.Solver3D(smpm.make_grid(128, 8, 10, 32.0, 1.0, krylov=1), 128, 2 * np.pi, stream)
        Uc = torch.empty_like(F)
        msc, stc = timed(lambda: sc.solve_3d(F, Uc, tol=TOL))
        diff = float((Uc - U).abs().max() / U.abs().max())
        lines.append({"workload": "3-D via Fourier: the same 128x8, order 10, m_y = 128 problem, one concatenated "
                                  "Krylov space over all 65 modes (Sec. 5, Alg. 3d)",
                      "metric": "3-D solves/s at 1e-10 rel. residual (concatenated residual)", "value": 1e3 / msc,
                      "ms_per_solve": msc, "iters": stc.iters, "per_mode_iters": st.iters,
                      "rel_resid_concatenated": stc.rel_resid_true,
                      "max_abs_diff_vs_per_mode_rel_to_max": diff})
        sc.close()
    else:
        shape = dict(mx=512, mz=16, order=16, lx=32.0, lz=1.0, z_ratio=1.2)
        R = args.mixed_rhs
        # (precision, SMPM_OZAKI): FP64, the two mixed forms with FP32
        # CUDA-core products, and the same with the FP32 products on the
        # tensor cores (24-bit digit splits)
        for prec, oz in ((0, 0), (1, 0), (2, 0), (1, 2), (2, 2)):
            os.environ["SMPM_OZAKI"] = str(oz)
            s = smpm.Solver(smpm.make_grid(**shape, precision=prec), 0.0, stream)
            os.environ.pop("SMPM_OZAKI")
            x, z = s.coords()
            F = np.stack([inputs.cos_modes(x, z, 32.0, 1.0, inputs.cos_modes_spec(inputs.seed_for(3) + i))[0]
                          for i in range(R)])
            Fd = torch.from_numpy(F).to(dev)
            Ud = torch.empty_like(Fd)
            s.profile(True)
            ms, st = timed(lambda: s.solve(Fd, Ud, tol=TOL), s)
            # mixed: FP64 and FP32 launches together, so no single peak applies
            roof = gemm_roofline(s, ms * args.steps, None if prec else FP64_NOMINAL_TFLOPS,
                                 "FP64 and FP32 launches" if prec else "FP64")
            lines.append({"roofline": roof, "workload": "2-D Poisson-Neumann 512x16 elements, order 16, domain 32x1, z stretched "
                                      "geometrically (ratio 1.2), cos-cos modes, %d right-hand sides per step" % R,
                          "precision": ["FP64", "mixed: FP64 FGMRES, FP32 block-Jacobi",
                                        "nested mixed: FP64 FGMRES, inner DBJ-GMRES with FP32 Schur "
                                        "and block-Jacobi blocks"][prec]
                                       + (" (FP32 products on the tcgen05 tensor cores, 24-bit digit splits)" if oz else ""),
                          "metric": "solves/s at 1e-10 rel. residual", "value": R * 1e3 / ms, "ms_per_step": ms,
                          "iters": st.iters, "worst_rel_resid": st.rel_resid_true, "setup_ms": st.setup_ms,
                          "device_bytes": s.device_bytes()})
            if prec == 0:
                U64 = Ud.clone()
            else:
                lines[-1]["rel_diff_vs_fp64"] = float(torch.linalg.norm(Ud - U64) / torch.linalg.norm(U64))
            s.close()
    for ln in lines:
        print(json.dumps(ln), flush=True)
    return 0


SERVE_GRIDS = [(64, 2), (128, 4), (256, 8), (512, 16), (1024, 16)]
SERVE_ORDERS = [6, 8, 12, 16]


def serve_seed(rank):
    """First seed of a rank's request stream: every rank serves its own stream
    (weak scaling), seeds 100,000 apart so streams never overlap."""
    from paper_1512_01756_gb300 import inputs
    return inputs.seed_for(5) + 100_000 * rank


def serve_stream(n, seed):
    """The request stream: grid uniform from SERVE_GRIDS on [0, mx/mz] x [0, 1],
    order uniform from SERVE_ORDERS, k^2 = 0 with probability 0.1 else
    log-uniform on [1e-2, 1e4], f a seeded sum of 32 cos-cos modes (per-request
    seed)."""
    from paper_1512_01756_gb300 import inputs
    r = inputs.rng(seed)
    out = []
    for i in range(n):
        mx, mz = SERVE_GRIDS[int(r.integers(len(SERVE_GRIDS)))]
        order = SERVE_ORDERS[int(r.integers(len(SERVE_ORDERS)))]
        k2 = 0.0 if r.random() < 0.1 else float(10.0 ** r.uniform(-2.0, 4.0))
        out.append({"mx": mx, "mz": mz, "order": order, "k2": k2, "seed": seed + 1 + i})
    return out


def serve_rhs(smpm, grid, lx, seed):
    """f = sum_m c_m cos(a_m pi x / lx) cos(b_m pi z) at the grid's nodes, as
    the product of per-column and per-row cosine tables (node order X*fz + Z)."""
    import numpy as np
    from paper_1512_01756_gb300 import inputs
    x, z = smpm.grid_coords(grid)
    fz = (grid.order + 1) * grid.mz
    xs, zs = x[::fz], z[:fz]
    c, a, b = inputs.cos_modes_spec(seed)
    Cx = np.cos(np.outer(xs, a * np.pi / lx))
    Cz = np.cos(np.outer(zs, b * np.pi))
    return ((Cx * c) @ Cz.T).reshape(-1)


def serve_requests(n, seed, smpm=None, precision=2):
    """The stream's requests with their grids (plain FP64 and served form)."""
    reqs = serve_stream(n, seed)
    for q in reqs:
        q["lx"] = q["mx"] / q["mz"]
        q["r"] = (q["order"] + 1) ** 2 * q["mx"] * q["mz"]
        if smpm is not None:
            q["grid"] = smpm.make_grid(q["mx"], q["mz"], q["order"], q["lx"], 1.0)
            q["grid_served"] = smpm.make_grid(q["mx"], q["mz"], q["order"], q["lx"], 1.0, precision=precision)
    return reqs


def oracle_serve_sample(reqs, seconds, max_nodes=ORACLE_MAX_NODES, max_count=None):
    """The CPU oracle (setup + Alg. seq solve per request) on the stream's
    requests in order, skipping grids above max_nodes nodes, until `seconds`
    of wall time (at least two requests) or max_count requests.  Returns
    (requests solved, wall seconds, effective cores, largest grid)."""
    from oracle.smpm import Grid
    from oracle.schur import StripSchur
    from oracle import dbj
    from paper_1512_01756_gb300 import inputs
    done, biggest, big_r, worst = 0, "", 0, 0.0
    c0, w0 = os.times(), time.perf_counter()
    for q in reqs:
        if q["r"] > max_nodes:
            continue
        g = Grid(q["mx"], q["mz"], q["order"], q["lx"], 1.0)
        X, Z = g.coords()
        f, _ = inputs.cos_modes(X, Z, q["lx"], 1.0, inputs.cos_modes_spec(q["seed"]))
        _, info = dbj.solve(g, f, k2=q["k2"], method="dbj", tol=TOL, schur=StripSchur(g, q["k2"]))
        worst = max(worst, info["schur_residual"])
        done += 1
        if q["r"] > big_r:
            big_r, biggest = q["r"], f'{q["mx"]}x{q["mz"]} order {q["order"]}'
        if max_count is not None and done >= max_count:
            break
        if max_count is None and done >= 2 and time.perf_counter() - w0 > seconds:
            break
    w1, c1 = time.perf_counter(), os.times()
    cores = max(1, round(((c1.user - c0.user) + (c1.system - c0.system)) / (w1 - w0)))
    return done, w1 - w0, cores, biggest + f"; worst oracle Schur residual {worst:.1e}"


def _pct(v, p):
    import numpy as np
    return float(np.percentile(np.asarray(v) * 1e3, p))


def _served_pass(srv, reqs, f_of, u_of, arrivals=None, poll_sleep=0.0002):
    """Serve reqs through srv: all at once (arrivals None) or at the given
    arrival offsets (seconds from the call).  Returns (wall span s,
    latencies s, batch sizes, worst residual)."""
    tickets, lat, batch, worst = {}, [], [], 0.0
    sub = [0.0] * len(reqs)
    t0 = time.perf_counter()
    nxt = 0
    while nxt < len(reqs) or tickets:
        now = time.perf_counter() - t0
        while nxt < len(reqs) and (arrivals is None or arrivals[nxt] <= now):
            q = reqs[nxt]
            sub[nxt] = time.perf_counter() - t0
            tickets[srv.submit(q["grid_served"], q["k2"], f_of(nxt), u_of(nxt), tol=TOL)] = nxt
            nxt += 1
        for tk in list(tickets):
            st = srv.poll(tk)
            if st is not None:
                i = tickets[tk]
                # completion - arrival: the wait before the submit call plus
                # the server's own submit-to-completion time
                lat.append(st.solve_ms * 1e-3 + (sub[i] - arrivals[i] if arrivals is not None else 0.0))
                batch.append(st.restarts)
                worst = max(worst, st.rel_resid_true)
                del tickets[tk]
        time.sleep(poll_sleep)
    span = time.perf_counter() - t0
    return span, lat, batch, worst


def run_serve(args):
    """The headline line: the request stream served one at a time by the
    plain FP64 path and by the serving runtime (module docstring)."""
    import numpy as np
    import torch
    import torch.distributed as dist
    import __graft_entry__
    __graft_entry__.build()
    from paper_1512_01756_gb300 import smpm, inputs

    rank, local, world = rank_env()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    stream = torch.cuda.current_stream()
    K, W, per = args.steps, args.warmup, args.requests_per_step
    N = K * per
    seed = serve_seed(rank)                             # every rank its own stream
    reqs = serve_requests(N, seed, smpm, args.served_precision)
    offs = np.concatenate([[0], np.cumsum([q["r"] for q in reqs])])
    total = int(offs[-1])
    # f of every request in one pinned host buffer (the e2e pass reads it
    # there); the device-resident passes read a device copy
    Fh = torch.empty(total, dtype=torch.float64, pin_memory=True)
    Fn = Fh.numpy()
    for i, q in enumerate(reqs):
        Fn[offs[i]:offs[i + 1]] = serve_rhs(smpm, q["grid"], q["lx"], q["seed"])
    Fd = Fh.to(dev)
    Up = torch.zeros(total, dtype=torch.float64, device=dev)
    Us = torch.zeros_like(Up)
    Ub = torch.zeros_like(Up)
    Uh = torch.zeros(total, dtype=torch.float64, pin_memory=True)
    view = lambda T, i: T[int(offs[i]):int(offs[i + 1])]
    srv_args = dict(nworkers=args.workers, max_batch=args.max_batch)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # warm-up steps: one request of every grid and order of the stream (k^2
    # drawn as in the stream, its own seed), plain and served, so that neither
    # timed pass pays a first-use cost (library load, cuSOLVER kernels of every
    # matrix size, allocator pools, GEMM tile tuning)
    wr = inputs.rng(seed + 55_555)
    for w in range(W):
        warm = []
        for mx, mz in SERVE_GRIDS:
            for order in SERVE_ORDERS:
                k2 = 0.0 if w == 0 else (0.0 if wr.random() < 0.1 else float(10.0 ** wr.uniform(-2, 4)))
                q = {"mx": mx, "mz": mz, "order": order, "k2": k2, "lx": mx / mz, "seed": seed + 77_777 + len(warm)}
                q["grid"] = smpm.make_grid(mx, mz, order, q["lx"], 1.0)
                q["grid_served"] = smpm.make_grid(mx, mz, order, q["lx"], 1.0, precision=args.served_precision)
                q["f"] = torch.from_numpy(serve_rhs(smpm, q["grid"], q["lx"], q["seed"])).to(dev)
                q["u"] = torch.zeros_like(q["f"])
                warm.append(q)
        for q in warm:
            s = smpm.Solver(q["grid"], q["k2"], stream)
            s.solve(q["f"], q["u"], tol=TOL)
            s.close()
        srv = smpm.Server(**srv_args)
        _served_pass(srv, warm, lambda i: warm[i]["f"], lambda i: warm[i]["u"])
        srv.close()
        del warm
    barrier()

    clocks = Clocks(local)
    clocks.start()
    l0 = smpm.kernel_launches()
    # 1. plain FP64, one request at a time (setup + solve + release each)
    service, res_plain, it_plain = [], [], []
    for i, q in enumerate(reqs):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s = smpm.Solver(q["grid"], q["k2"], stream)
        st = s.solve(view(Fd, i), view(Up, i), tol=TOL)
        s.close()
        e1.record(stream)
        e1.synchronize()
        service.append(e0.elapsed_time(e1) * 1e-3)
        res_plain.append(st.rel_resid_true)
        it_plain.append(st.iters)
        q["setup_ms"] = st.setup_ms
    plain_span = sum(service)
    lam = N / plain_span                               # the plain path's saturation rate
    arrivals = np.cumsum(inputs.rng(seed + 7).exponential(1.0 / lam, N))
    arrivals -= arrivals[0]
    end, lat_plain = 0.0, []
    for a, sv in zip(arrivals, service):               # FIFO single server
        end = max(end, a) + sv
        lat_plain.append(end - a)
    barrier()

    # 2. served, Poisson arrivals at that rate (latency)
    srv = smpm.Server(**srv_args)
    arr_span, lat_served, batch_arr, worst_arr = _served_pass(srv, reqs, lambda i: view(Fd, i), lambda i: view(Us, i),
                                                              arrivals)
    torch.cuda.synchronize()
    srv.close()
    barrier()

    # 3. served capacity: the whole stream submitted at once (the value)
    srv = smpm.Server(**srv_args)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    burst_wall, _, batch_burst, worst_burst = _served_pass(srv, reqs, lambda i: view(Fd, i), lambda i: view(Ub, i))
    torch.cuda.synchronize()
    e1.record(stream)
    e1.synchronize()
    burst_span = e0.elapsed_time(e1) * 1e-3
    srv.close()
    launches = smpm.kernel_launches() - l0
    barrier()

    # 4. e2e: the same burst with f and u in pinned host memory
    srv = smpm.Server(**srv_args)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    _, _, _, worst_e2e = _served_pass(srv, reqs, lambda i: view(Fh, i), lambda i: view(Uh, i))
    torch.cuda.synchronize()
    e1.record(stream)
    e1.synchronize()
    e2e_span = e0.elapsed_time(e1) * 1e-3
    srv.close()
    barrier()
    clk = clocks.stop()

    # results: every served result against the plain FP64 one (relative 2-norm
    # and max-norm), the host-buffer results against the device ones
    def diffs(U):
        d2, dm = 0.0, 0.0
        for i in range(N):
            a, b = view(U, i), view(Up, i)
            nb_ = float(torch.linalg.norm(b))
            d2 = max(d2, float(torch.linalg.norm(a - b)) / nb_)
            dm = max(dm, float((a - b).abs().max() / b.abs().max()))
        return d2, dm
    d_arr, dmax_arr = diffs(Us)
    d_burst, dmax_burst = diffs(Ub)
    d_e2e = float((Uh.to(dev) - Ub).abs().max() / Ub.abs().max())

    # 5. roofline of the dense products in this mix: the first requests re-run
    # through a server with the per-launch profile on (events around every
    # dense-product launch, so not timed above)
    P = min(N, args.profiled_requests)
    smpm.profile_all(True)
    smpm.profile_split(None, reset=True)
    srv = smpm.Server(**srv_args)
    _served_pass(srv, reqs[:P], lambda i: view(Fd, i), lambda i: view(Ub, i))
    torch.cuda.synchronize()
    srv.close()
    prof = smpm.profile_split(None, reset=True)
    smpm.profile_all(False)
    fp64, fp32 = prof["fp64"], prof["fp32"]
    ach64 = fp64["flops"] / (fp64["ms"] * 1e-3) / 1e12 if fp64["ms"] > 0 else None
    ach32 = fp32["flops"] / (fp32["ms"] * 1e-3) / 1e12 if fp32["ms"] > 0 else None
    roofline = {"bound": "alu", "kernel": "mirror_gemm_kernel + class_gemm_kernel, FP64 launches (Schur products, "
                                          "block-Jacobi, strip-solver slots) of the served mix",
                "achieved": ach64, "peak": FP64_NOMINAL_TFLOPS, "unit": "TFLOP/s",
                "frac": ach64 / FP64_NOMINAL_TFLOPS if ach64 else None, "traffic": None,
                "peak_source": "recipe FP64 1.25 TFLOP/s (GB300; MEASURED_PEAKS.json has no FP64 figure)",
                "flops_per_launch": fp64["flops"] / max(fp64["launches"], 1),
                "ms_per_launch": fp64["ms"] / max(fp64["launches"], 1), "launches": fp64["launches"],
                "sample": f"the first {P} requests of the stream re-served with the per-launch profile on",
                "fp32_launches": {"achieved": ach32, "peak": FP32_SIMT_TFLOPS, "unit": "TFLOP/s",
                                  "frac": ach32 / FP32_SIMT_TFLOPS if ach32 else None, "launches": fp32["launches"],
                                  "peak_source": "152 SMs x 128 FP32 lanes x 2 FLOP x 2.07 GHz"}}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        n_o, secs, cores, biggest = oracle_serve_sample(reqs, args.cpu_seconds)
        cpu = {"value": n_o / secs, "unit": "solves/s", "cores": cores, "kind": "oracle",
               "sample": f"the first {n_o} requests of the stream with at most {ORACLE_MAX_NODES} nodes "
                         f"(largest {biggest}; the larger grids skipped), setup + solve each, {secs:.1f} s"}

    span_max = max_over_ranks(burst_span, dev, world)
    e2e_max = max_over_ranks(e2e_span, dev, world)
    bytes_f = total * 8
    line = {"metric": METRIC_SERVE, "value": N * world / span_max, "unit": "solves/s", "n_gpus": world,
            "steps": K, "warmup": W, "ms_per_step": 1e3 * span_max / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
            "config": {"workload": f"serving: {N} Poisson/Helmholtz requests ({per} per step), grids {SERVE_GRIDS} "
                                   f"on [0, mx/mz] x [0, 1], orders {SERVE_ORDERS}, k^2 = 0 (10 %) else log-uniform "
                                   f"[1e-2, 1e4], cos-cos f",
                       "tol": TOL, "served": "smpm_server: %d workers, batches of <= %d same-grid requests, %s"
                       % (args.workers, args.max_batch, ["FP64", "mixed (FP32 block-Jacobi)",
                                                         "nested mixed (FP64 FGMRES, FP32 inner DBJ-GMRES)"][args.served_precision]),
                       "plain": "smpm_setup + smpm_solve + smpm_release per request, FP64, one at a time",
                       "arrivals": f"Poisson at the plain path's saturation rate {lam:.2f}/s",
                       "l2": f"inputs larger than L2: every request reads its own f and writes its own u "
                             f"({2 * bytes_f / 2**30:.1f} GiB per pass)",
                       "parallelism": f"independent request streams per GPU x{world}"},
            "plain_value": N / plain_span,
            "p50_ms": _pct(lat_served, 50), "p99_ms": _pct(lat_served, 99),
            "plain_p50_ms": _pct(lat_plain, 50), "plain_p99_ms": _pct(lat_plain, 99),
            "served": {"capacity_solves_per_s": N / burst_span, "solves_per_s_at_arrival_rate": N / arr_span,
                       "mean_batch_burst": float(np.mean(batch_burst)), "mean_batch_arrivals": float(np.mean(batch_arr)),
                       "worst_rel_resid": max(worst_arr, worst_burst, worst_e2e),
                       "max_rel_diff_vs_plain": max(d_arr, d_burst), "max_abs_diff_vs_plain_rel_to_max": max(dmax_arr, dmax_burst)},
            "plain_fp64": {"solves_per_s": N / plain_span, "mean_service_ms": 1e3 * plain_span / N,
                           "mean_setup_ms": float(np.mean([q["setup_ms"] for q in reqs])),
                           "worst_rel_resid": max(res_plain), "mean_iters": float(np.mean(it_plain))},
            "e2e": {"value": N * world / e2e_max, "unit": "solves/s", "h2d_bytes_per_step": bytes_f // K,
                    "d2h_bytes_per_step": bytes_f // K, "max_diff_vs_device_pass": d_e2e},
            "gpu_launches": launches, "roofline": roofline, "cpu_baseline": cpu, "clocks": clk,
            "latency": "completion - arrival, operator setup included",
            "timing": "CUDA events on the launching stream around each pass, device synchronised on both sides"}
    if rank == 0 and not args.no_secondary:
        line["secondary_poisson2d"] = poisson2d_summary(args, smpm, dev, stream)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def poisson2d_summary(args, smpm, dev, stream, steps=5, warmup=3):
    """The 256 x 4, order-12 batched FP64 solve (128 right-hand sides) as a
    secondary figure of the serving line: solves/s with the profile off, and
    the dense products' FLOP rate from a separate profiled pass."""
    import torch
    from paper_1512_01756_gb300 import inputs
    solver = smpm.Solver(smpm.make_grid(**GRID), 0.0, stream)
    x, z = solver.coords()
    F = make_f(x, z, args.rhs, inputs.seed_for(1))
    Fd = torch.from_numpy(F).to(dev)
    Ud = torch.empty_like(Fd)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def timed(n):
        ts, st = [], None
        for _ in range(n):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = solver.solve(Fd, Ud, tol=TOL)
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return sum(ts) / len(ts), st
    timed(warmup)
    ms, st = timed(steps)
    solver.profile(True)
    solver.profile_read(reset=True)
    ms_prof, _ = timed(steps)
    prof = solver.profile_read(reset=True)
    solver.profile(False)
    solver.close()
    ach = prof["flops"] / (prof["ms"] * 1e-3) / 1e12 if prof["ms"] > 0 else None
    return {"workload": WORKLOAD + f", {args.rhs} right-hand sides per step, plain FP64",
            "solves_per_s": args.rhs / (ms * 1e-3), "ms_per_step": ms, "iters": st.iters,
            "worst_rel_resid": st.rel_resid_true, "ms_per_step_profiled": ms_prof,
            "gemm_tflops": ach, "gemm_frac_of_fp64_nominal": ach / FP64_NOMINAL_TFLOPS if ach else None,
            "gemm_share_of_step": prof["ms"] / (ms_prof * steps)}


def run_reference_serve(args):
    """Reference arm of the serving line: the CPU oracle on the host cores, one
    request of the same stream per step (requests above ORACLE_MAX_NODES
    nodes skipped: the oracle takes minutes on them), setup + solve."""
    rank, _, world = rank_env()
    if rank != 0:
        return 0
    from paper_1512_01756_gb300 import inputs
    reqs = serve_requests(4 * (args.warmup + args.steps) + 64, inputs.seed_for(5))
    small = [q for q in reqs if q["r"] <= ORACLE_MAX_NODES]
    oracle_serve_sample(small[:args.warmup], 0.0, max_count=args.warmup)
    n, secs, cores, biggest = oracle_serve_sample(small[args.warmup:], 0.0, max_count=args.steps)
    val = n / secs
    line = {"impl": "reference", "metric": METRIC_SERVE, "value": val, "unit": "solves/s", "n_gpus": world,
            "steps": n, "warmup": args.warmup, "ms_per_step": 1e3 * secs / n, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "serving stream (grids %s, orders %s, k^2 = 0 (10 %%) else log-uniform "
                                   "[1e-2, 1e4]), requests with at most %d nodes" % (SERVE_GRIDS, SERVE_ORDERS,
                                                                                   ORACLE_MAX_NODES),
                       "solver": "oracle Alg. seq, Householder GMRES, one request at a time"},
            "cpu_baseline": {"value": val, "unit": "solves/s", "cores": cores, "kind": "oracle",
                             "sample": f"{n} requests of the stream, one per step, setup + solve (largest {biggest})"},
            "e2e": {"value": val, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference_serve(args) if args.workload == "serve" else run_reference(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload != "poisson2d":
        return run_other(args)
    return run_poisson2d(args)


if __name__ == "__main__":
    sys.exit(main())
