#!/usr/bin/env python3
"""Throughput of the deflated block-Jacobi Schur-complement GMRES solve.

Workload: the 2-D Poisson-Neumann long-domain problem, 256 x 4 elements of
order 12 on [0, 64] x [0, 1] (r = 173,056 nodes, k = 26,520 Schur unknowns),
f = a seeded sum of 32 random low-wavenumber cos-cos modes, g = 0, plain FP64
path (Alg. seq: block-Jacobi + deflation, CGS2 GMRES) to a relative Schur
residual of 1e-10.  A step solves one batch of --rhs (default 128)
independent right-hand sides (each with its own Krylov space) through the C
ABI; value = solved
right-hand sides per second over all ranks (each rank its own batch: weak
scaling, no collective on the data path).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--rhs R] [--impl reference]

--impl reference times the CPU oracle (oracle/, numpy/scipy FP64, Alg. seq
with Householder GMRES) on the host cores on the same workload and metric.
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
TOL = 1e-10
FP64_NOMINAL_TFLOPS = 1.25     # GB300 FP64 (non-tensor and tensor), profiling recipe table
L2_FLUSH_BYTES = 256 << 20


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--rhs", type=int, default=128, help="right-hand sides per step (one batched solve)")
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--cpu-sample", type=int, default=2, help="oracle right-hand sides in the cpu_baseline leg")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--workload", default="poisson2d", choices=["poisson2d", "small", "modes3d", "mixed", "serve"],
                   help="poisson2d: the default bench line; small / modes3d / mixed / serve: the 8x2 latency, 3-D, "
                        "mixed-precision and serving configurations, measured separately (not the driver's "
                        "bench line)")
    p.add_argument("--requests", type=int, default=200, help="serve: requests in the stream")
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


def traffic_per_launch():
    """DRAM bytes per dense-product launch from the committed ncu summary, if it was
    taken on the current kernels.cu (else None)."""
    path = os.path.join(ROOT, "profiles", "gemm_traffic.txt")
    src = os.path.join(ROOT, "paper_1512_01756_gb300", "csrc", "kernels.cu")
    if not os.path.exists(path):
        return None
    kv = {}
    for line in open(path):
        if "=" in line and not line.startswith("#"):
            k, v = line.split("=", 1)
            kv[k.strip()] = v.strip()
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    if kv.get("kernels_cu_sha256_16") != sha:
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


def run_ours(args):
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
    solver.profile(True)
    solver.profile_read(reset=True)
    times, stats = [], []
    for _ in range(args.steps):
        flush.fill_(1.0)                      # evict L2 between steps (not timed)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = solver.solve(Fd, Ud, tol=TOL)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        stats.append(st.as_dict())
    launches = smpm.kernel_launches() - l0
    prof = solver.profile_read(reset=True)
    solver.profile(False)
    barrier()
    clk = clocks.stop()
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
                "gemm_share_of_step": prof["ms"] / (ms * args.steps)}

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
    """Separate measurements of the 3-D mode batch and of the mixed-precision
    solve (one JSON line each; the default bench line is poisson2d)."""
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
    else:
        shape = dict(mx=512, mz=16, order=16, lx=32.0, lz=1.0, z_ratio=1.2)
        R = args.mixed_rhs
        for prec in (0, 1, 2):
            s = smpm.Solver(smpm.make_grid(**shape, precision=prec), 0.0, stream)
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
                                        "and block-Jacobi blocks"][prec],
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


def run_serve(args):
    """Serving: the request stream served one at a time by the plain FP64 path
    (smpm_setup + smpm_solve + smpm_release per request) and by the server
    (continuous batching over worker streams), with Poisson arrivals at the
    rate where the plain path saturates (its measured mean service rate)."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1512_01756_gb300 import smpm, inputs
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    reqs = serve_stream(args.requests, inputs.seed_for(5))
    for q in reqs:
        q["grid"] = smpm.make_grid(q["mx"], q["mz"], q["order"], q["mx"] / q["mz"], 1.0)
        # the served form may run the mixed-precision solve (same FP64 true residual)
        q["grid_served"] = smpm.make_grid(q["mx"], q["mz"], q["order"], q["mx"] / q["mz"], 1.0,
                                          precision=args.served_precision)
        q["f"] = torch.from_numpy(serve_rhs(smpm, q["grid"], q["mx"] / q["mz"], q["seed"])).to(dev)
        q["u_plain"] = torch.zeros_like(q["f"])
        q["u_served"] = torch.zeros_like(q["f"])
    # warm-up (library, cuSOLVER kernels of every matrix size, allocator, GEMM
    # tile tuning): one k^2 = 1 solve per grid and order of the stream, so that
    # neither pass below pays a first-use cost
    wg = smpm.make_grid(64, 2, 6, 32.0, 1.0)
    wf = torch.from_numpy(serve_rhs(smpm, wg, 32.0, 1)).to(dev)
    wu = torch.zeros_like(wf)
    for _ in range(max(args.warmup, 1)):
        s = smpm.Solver(wg, 1.0, stream)
        s.solve(wf, wu, tol=TOL)
        s.close()
    seen = set()
    for q in reqs:
        key = (q["mx"], q["mz"], q["order"])
        if key in seen:
            continue
        seen.add(key)
        for k2w in (1.0, 0.0):
            for gw in {id(q["grid"]): q["grid"], id(q["grid_served"]): q["grid_served"]}.values():
                s = smpm.Solver(gw, k2w, stream)
                s.solve(q["f"], q["u_plain"], tol=TOL)
                s.close()
    torch.cuda.synchronize()
    srv = smpm.Server(nworkers=args.workers, max_batch=args.max_batch)
    t = srv.submit(wg, 2.0, wf, wu, tol=TOL)
    while srv.poll(t) is None:
        time.sleep(0.001)
    torch.cuda.synchronize()

    # plain FP64, one request at a time
    clocks = Clocks(0)
    clocks.start()
    service, iters_plain, res_plain = [], [], []
    for q in reqs:
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        s = smpm.Solver(q["grid"], q["k2"], stream)
        st = s.solve(q["f"], q["u_plain"], tol=TOL)
        s.close()
        torch.cuda.synchronize()
        service.append(time.perf_counter() - w0)
        iters_plain.append(st.iters)
        res_plain.append(st.rel_resid_true)
        q["setup_ms"], q["solve_ms"] = st.setup_ms, st.solve_ms
    lam = len(reqs) / sum(service)
    arrivals = np.cumsum(inputs.rng(inputs.seed_for(5) + 7).exponential(1.0 / lam, len(reqs)))
    end, lat_plain = 0.0, []
    for a, sv in zip(arrivals, service):
        end = max(end, a) + sv
        lat_plain.append(end - a)
    plain_rate = len(reqs) / (end - arrivals[0])

    # served: submit at the arrival times, poll until every ticket is done
    l0 = smpm.kernel_launches()
    tickets, done, lat_served, batch_sizes, res_served = {}, {}, [], [], []
    t0 = time.perf_counter()
    nxt = 0
    while len(done) < len(reqs):
        now = time.perf_counter() - t0
        while nxt < len(reqs) and arrivals[nxt] - arrivals[0] <= now:
            q = reqs[nxt]
            tickets[srv.submit(q["grid_served"], q["k2"], q["f"], q["u_served"], tol=TOL)] = nxt
            nxt += 1
        for tk, i in list(tickets.items()):
            st = srv.poll(tk)
            if st is not None:
                done[i] = time.perf_counter() - t0
                lat_served.append(st.solve_ms * 1e-3)
                batch_sizes.append(st.restarts)
                res_served.append(st.rel_resid_true)
                del tickets[tk]
        time.sleep(0.0002)
    served_span = max(done.values())
    torch.cuda.synchronize()
    launches = smpm.kernel_launches() - l0

    # served capacity: the whole stream submitted at once (offered load above
    # what the server completes) to a fresh server (empty operator cache: only
    # repeats within the stream reuse operators), results checked against the
    # first pass
    srv.close()
    srv = smpm.Server(nworkers=args.workers, max_batch=args.max_batch)
    for q in reqs:
        q["u_burst"] = torch.zeros_like(q["f"])
    t0 = time.perf_counter()
    burst = [srv.submit(q["grid_served"], q["k2"], q["f"], q["u_burst"], tol=TOL) for q in reqs]
    pend = set(burst)
    res_burst = []
    while pend:
        for tk in list(pend):
            st = srv.poll(tk)
            if st is not None:
                res_burst.append(st.rel_resid_true)
                pend.discard(tk)
        time.sleep(0.0002)
    burst_span = time.perf_counter() - t0
    torch.cuda.synchronize()
    clk = clocks.stop()
    srv.close()
    diffs_burst = [float(torch.linalg.norm(q["u_burst"] - q["u_plain"]) / torch.linalg.norm(q["u_plain"]))
                   for q in reqs]
    diffs = [float(torch.linalg.norm(q["u_served"] - q["u_plain"]) / torch.linalg.norm(q["u_plain"])) for q in reqs]

    def pct(v, p):
        return float(np.percentile(np.asarray(v) * 1e3, p))

    by_grid = {}
    for q, sv in zip(reqs, service):
        key = f'{q["mx"]}x{q["mz"]} p{q["order"]}'
        e = by_grid.setdefault(key, {"n": 0, "service_ms": 0.0, "setup_ms": 0.0})
        e["n"] += 1
        e["service_ms"] += sv * 1e3
        e["setup_ms"] += q["setup_ms"]
    for e in by_grid.values():
        e["service_ms"] /= e["n"]
        e["setup_ms"] /= e["n"]
    line = {"workload": f"serving: {len(reqs)} Poisson/Helmholtz requests, grids {SERVE_GRIDS} on [0, mx/mz] x [0, 1], "
                        f"orders {SERVE_ORDERS}, k^2 = 0 (10 %) else log-uniform [1e-2, 1e4], cos-cos f; Poisson "
                        f"arrivals at the plain path's saturation rate {lam:.2f}/s",
            "metric": "solves/s at 1e-10 rel. residual, p50/p99 latency: served vs plain FP64",
            "unit": "solves/s", "value": len(reqs) / burst_span, "dtype": "f64", "data": "synthetic",
            "value_is": "served capacity: the stream submitted at once",
            "served": {"precision": ["FP64", "mixed: FP64 FGMRES, FP32 block-Jacobi",
                                     "nested mixed"][args.served_precision],
                       "capacity_solves_per_s": len(reqs) / burst_span,
                       "solves_per_s_at_arrival_rate": len(reqs) / served_span, "p50_ms": pct(lat_served, 50),
                       "p99_ms": pct(lat_served, 99), "workers": args.workers, "max_batch": args.max_batch,
                       "mean_batch": float(np.mean(batch_sizes)),
                       "worst_rel_resid": max(max(res_served), max(res_burst))},
            "plain_fp64": {"capacity_solves_per_s": lam, "solves_per_s_at_arrival_rate": plain_rate,
                           "p50_ms": pct(lat_plain, 50), "p99_ms": pct(lat_plain, 99),
                           "mean_service_ms": 1e3 * float(np.mean(service)), "worst_rel_resid": max(res_plain)},
            "served_vs_plain_max_rel_diff": max(max(diffs), max(diffs_burst)),
            "latency": "completion - arrival, operator setup included",
            "operator_cache": "each pass starts with an empty cache; a request reuses operators only when "
                              "an earlier request of the same stream had its grid options and k^2",
            "gpu_launches": launches, "clocks": clk, "per_grid_plain": by_grid}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload != "poisson2d":
        return run_other(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
