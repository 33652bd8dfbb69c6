"""Benchmark: BIE solves/s of the Hele-Shaw bubble workload (1024^2 grid, 1024 nodes).

One step = one theta-L time step of the Hele-Shaw bubble r = 1 + 0.1 cos 3a + 0.05 sin 5a
in [-4,4]^2 (sigma = 1e-3, J = 1, dt = 1e-3): reconstruct the curve, set the interface,
solve the exterior modified double-layer BIE to a 1e-8 relative residual by device GMRES,
evaluate the normal velocity, advance theta-L. Each step contains exactly one BIE solve,
so steps/s = BIE solves/s. The headline runs the mixed form (float32 grid applies inside
GMRES, float64 Arnoldi, residual and refinement); the float64 plain form is timed on the
same workload beside it, together with layer-potential applies/s of both forms.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun each rank runs an independent replica (the path does not shard).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "BIE solves/s at 1e-8 GMRES residual and layer-potential applies/s vs FP64 plain"
WORKLOAD = "hele_shaw_bubble_1024x1024_n1024"
DT, SIGMA, J, TOL = 1e-3, 1e-3, 1.0, 1e-8
L2_FLUSH_BYTES = 512 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="kfbi", choices=["kfbi", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--profile", action="store_true",
                    help="timed steps only (for short profiler runs): no e2e, applies, fp64 or cpu legs")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["nvidia-smi unavailable"], samples=0)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() in ("active", "1", "0x1"):
                    reasons.add(nm)
        return dict(sm_mhz=statistics.median(sm) if sm else None, sm_max_mhz=smax, reasons=sorted(reasons),
                    samples=len(sm))


# --------------------------------------------------------------------------- workload
def workload():
    import workloads as W

    return W.config_hele_shaw(N=1024, n=1024, box=4.0)


def make_state(K, torch, p, precision):
    alpha = [2 * math.pi * j / p.n for j in range(p.n)]
    eta = torch.tensor(p.theta - alpha_array(p.n), dtype=torch.float64, device="cuda")
    ctx = K.Context(p.N, p.box, 0.0, K.BOX_FREESPACE_DL, precision, max_nodes=p.n)
    st = K.ThetaL(ctx, eta, p.L, p.xy.mean(0), K.STEP_HELE_SHAW, tol=TOL, max_iter=600, restart=150, sigma=SIGMA,
                  J=J)
    del alpha
    return ctx, st


def alpha_array(n):
    import numpy as np

    return 2 * np.pi * np.arange(n) / n


def run_steps(torch, ctx, st, K_steps, flush):
    """Times K steps with CUDA events on the current stream (L2 flushed before each step)."""
    evs = []
    infos = []
    for _ in range(K_steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        infos.append(st.step(DT))
        e1.record()
        evs.append((e0, e1))
    torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in evs]
    return ms, infos


def time_applies(torch, K, ctx, reps=50):
    """Layer-potential applies/s of the context's precision on its current interface."""
    n = ctx.n
    dens = torch.ones(n, dtype=torch.float64, device="cuda")
    vals = torch.empty(n, dtype=torch.float64, device="cuda")
    for _ in range(5):
        ctx.apply_into(K.DOUBLE, dens, vals)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        ctx.apply_into(K.DOUBLE, dens, vals)
    e1.record()
    torch.cuda.synchronize()
    return reps / (e0.elapsed_time(e1) / 1e3)


def traffic_record(kernel_src):
    """DRAM traffic per launch from a committed ncu summary, if taken on this kernel source."""
    path = os.path.join(ROOT, "profiles", "k_col_solve_traffic.json")
    if not os.path.exists(path):
        return None
    rec = json.load(open(path))
    h = hashlib.sha256(open(kernel_src, "rb").read()).hexdigest()[:16]
    if rec.get("source_sha256_16") != h:
        return None
    return rec


def cpu_baseline(iters_per_solve, budget_s=25.0):
    """The oracle as it stands on the host cores: a bounded sample of the same workload."""
    import numpy as np

    import workloads as W
    from oracle import kfbi as OK
    from oracle import thetal as OT

    p = workload()
    st = OT.state_from_nodes(p.xy, p.theta, p.L)
    s = OK.Kfbi(p.N, p.box, 0.0, OK.BOX_FREESPACE_DL)
    t0 = time.perf_counter()
    X = OT.reconstruct(st.eta, st.L, st.Xbar)
    s.set_interface(X)
    t_set = time.perf_counter() - t0
    phi = W.random_density(3, p.n)
    t1 = time.perf_counter()
    napp = 0
    while True:
        s.bie_matvec(OK.BIE_HS_EXTERIOR_MDL, phi)
        napp += 1
        if time.perf_counter() - t1 > budget_s - t_set or napp >= 40:
            break
    t_app = (time.perf_counter() - t1) / napp
    per_solve = t_set + iters_per_solve * t_app
    del np
    return dict(value=1.0 / per_solve, unit="solves/s", cores=os.cpu_count(), kind="oracle",
                sample=(f"oracle (numpy/scipy FP64) on the host: one set_interface ({t_set:.2f} s) and {napp} "
                        f"BIE applies ({t_app:.3f} s each) of the {WORKLOAD} workload, scaled to one solve of "
                        f"{iters_per_solve:.1f} applies (the GPU run's mean GMRES count) + set_interface"),
                applies_per_s=1.0 / t_app)


# --------------------------------------------------------------------------- reference arm
def run_reference(args):
    rank, world, _ = dist_env()
    if world > 1 and rank != 0:
        return 0
    import numpy as np

    import workloads as W
    from oracle import kfbi as OK
    from oracle import thetal as OT

    p = workload()
    st = OT.state_from_nodes(p.xy, p.theta, p.L)
    s = OK.Kfbi(p.N, p.box, 0.0, OK.BOX_FREESPACE_DL)
    phi = W.random_density(3, p.n)
    iters = 90.0  # GMRES applies per solve of this workload at 1e-8 (measured on both paths)

    def sample():
        t0 = time.perf_counter()
        s.set_interface(OT.reconstruct(st.eta, st.L, st.Xbar))
        t_set = time.perf_counter() - t0
        t1 = time.perf_counter()
        s.bie_matvec(OK.BIE_HS_EXTERIOR_MDL, phi)
        t_app = time.perf_counter() - t1
        return t_set + iters * t_app, t_set, t_app

    for _ in range(args.warmup):
        sample()
    per = [sample() for _ in range(args.steps)]
    per_solve = float(np.mean([q[0] for q in per]))
    value = 1.0 / per_solve
    line = dict(impl="reference", metric=METRIC, value=value, unit="solves/s", n_gpus=args.gpus, steps=args.steps,
                warmup=args.warmup, ms_per_step=per_solve * 1e3, higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="f64", data="synthetic",
                config=dict(workload=WORKLOAD, grid=1024, nodes=1024, tol=TOL, precision="fp64"),
                cpu_baseline=dict(value=value, unit="solves/s", cores=os.cpu_count(), kind="oracle",
                                  sample=(f"each step: one oracle set_interface + one BIE apply of {WORKLOAD}, "
                                          f"scaled to {iters:.0f} applies per solve")),
                e2e=dict(value=value, unit="solves/s", h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line))
    return 0


# --------------------------------------------------------------------------- main arm
def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    rank, world, local = dist_env()
    import numpy as np
    import torch

    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist
    from paper_2309_01068_gb300 import build
    from paper_2309_01068_gb300 import kfbi as K

    build.build()
    K.load()
    p = workload()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    # ---- headline: mixed precision
    ctx, st = make_state(K, torch, p, K.MIXED)
    ckpt = st.read(T=False)
    run_steps(torch, ctx, st, args.warmup, flush)
    st.write(eta=ckpt["eta"], density=ckpt["density"], nhat=ckpt["nhat"], scalars=ckpt["scalars"])
    torch.cuda.synchronize()
    launches0 = ctx.launch_count()
    sampler = ClockSampler(local)
    sampler.start()
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    ms, infos = run_steps(torch, ctx, st, args.steps, flush)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    t_wall = time.perf_counter() - t_wall
    clocks = sampler.stop()
    launches = ctx.launch_count() - launches0
    total_s = sum(ms) / 1e3
    if pg:
        tt = torch.tensor([total_s], device="cuda")
        pg.all_reduce(tt, op=pg.ReduceOp.MAX)
        total_s = float(tt.item())
    # kernel timing pass: the same steps again from the same state with per-launch CUDA events
    # around the column kernel (event timing runs the solver's stream-launched form; the
    # kernels are the same as in the graph form timed above)
    st.write(eta=ckpt["eta"], density=ckpt["density"], nhat=ckpt["nhat"], scalars=ckpt["scalars"])
    ctx.timing(True)
    run_steps(torch, ctx, st, min(args.steps, 10), flush)
    tim = ctx.timing()
    ctx.timing(False)
    iters = [i["iterations"] for i in infos]
    value = world * args.steps / total_s
    print(f"[bench] mixed: {1e3 * total_s / args.steps:.3f} ms/step, GMRES its {np.mean(iters):.1f}, "
          f"col kernel {tim}", file=sys.stderr)
    if args.profile:
        args.no_fp64 = True
        args.no_cpu_baseline = True
    mixed_applies = None if args.profile else time_applies(torch, K, ctx)

    # ---- end to end through the public API with host buffers: the same steps as the timed
    # run, from the same checkpoint; every step uploads the state from pinned host memory,
    # steps, and downloads the new state and interface (L2 flushed before each step)
    e2e = None
    if not args.profile:
        n = p.n
        h_eta = ckpt["eta"].cpu().pin_memory()
        h_dens = ckpt["density"].cpu().pin_memory()
        h_nhat = ckpt["nhat"].cpu().pin_memory()
        sc = list(ckpt["scalars"])  # host scalars, passed by value through the C ABI
        h_xy = torch.empty((n, 2), dtype=torch.float64).pin_memory()
        d_eta = torch.empty(n, dtype=torch.float64, device="cuda")
        d_dens = torch.empty(n, dtype=torch.float64, device="cuda")
        d_nhat = torch.empty_like(ckpt["nhat"])
        e2e_ms = []
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            d_eta.copy_(h_eta, non_blocking=True)
            d_dens.copy_(h_dens, non_blocking=True)
            d_nhat.copy_(h_nhat, non_blocking=True)
            st.write(eta=d_eta, density=d_dens, nhat=d_nhat, scalars=sc)
            st.step(DT)
            r = st.read(T=False)
            h_eta.copy_(r["eta"], non_blocking=True)
            h_dens.copy_(r["density"], non_blocking=True)
            h_nhat.copy_(r["nhat"], non_blocking=True)
            h_xy.copy_(r["xy"], non_blocking=True)
            sc = r["scalars"]
            torch.cuda.synchronize()
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
        h2d = 8 * (2 * n + h_nhat.numel() + len(sc))
        d2h = 8 * (4 * n + h_nhat.numel() + len(sc))
        e2e = dict(value=world * 1e3 / float(np.mean(e2e_ms)), unit="solves/s", h2d_bytes_per_step=h2d,
                   d2h_bytes_per_step=d2h, steps=args.steps)

    # ---- roofline of the dominant grid kernel (float32 column transform pass)
    N = p.N
    bytes_per_launch = 2.0 * N * N * 4
    f32_ms = tim["fp32_ms"] / max(tim["fp32_launches"], 1)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    achieved = bytes_per_launch / (f32_ms * 1e-3) / 1e9 if tim["fp32_launches"] else None
    tr = traffic_record(os.path.join(ROOT, "paper_2309_01068_gb300", "csrc", "kfbi_apply.cu"))
    roofline = dict(kernel="k_col_solve<float> (column forward DST-II, eigen divide, inverse DST)",
                    bound="hbm", achieved=achieved, peak=hbm_peak, unit="GB/s",
                    frac=(achieved / hbm_peak) if achieved else None,
                    traffic=(tr["dram_bytes_per_launch"] if tr else None),
                    algorithmic_bytes_per_launch=bytes_per_launch, launches=tim["fp32_launches"],
                    mean_launch_us=f32_ms * 1e3,
                    peak_source="MEASURED_PEAKS.json hbm_gbs (of measured)" if peaks else "fallback 6.8 TB/s")

    # ---- float64 plain form on the same workload
    fp64 = None
    if not args.no_fp64:
        ctx64, st64 = make_state(K, torch, p, K.FP64)
        run_steps(torch, ctx64, st64, 1, flush)
        st64.write(eta=ckpt["eta"], density=ckpt["density"], nhat=ckpt["nhat"], scalars=ckpt["scalars"])
        k64 = max(3, args.steps // 3)
        ctx64.timing(True)
        ms64, infos64 = run_steps(torch, ctx64, st64, k64, flush)
        tim64 = ctx64.timing()
        fp64_applies = time_applies(torch, K, ctx64, reps=20)
        fp64 = dict(solves_per_s=k64 / (sum(ms64) / 1e3), steps=k64,
                    mean_gmres_iterations=float(np.mean([i["iterations"] for i in infos64])),
                    applies_per_s=fp64_applies,
                    col_kernel_mean_us=1e3 * tim64["fp64_ms"] / max(tim64["fp64_launches"], 1))
        st64.close()
        ctx64.close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(float(np.mean(iters)))

    if rank == 0:
        line = dict(metric=METRIC, value=value, unit="solves/s", n_gpus=world, steps=args.steps,
                    warmup=args.warmup, ms_per_step=1e3 * total_s / args.steps, higher_is_better=True,
                    scaling="weak", vs_baseline=None, dtype="f32+f64", data="synthetic",
                    config=dict(workload=WORKLOAD, grid=N, nodes=p.n, box=[-4, 4], sigma=SIGMA, J=J, dt=DT,
                                tol=TOL, precision="mixed (f32 grid applies, f64 GMRES/residual/refinement)",
                                parallelism=f"replicas{world}", l2="flushed (512 MB write) before every timed step"),
                    applies_per_s=dict(mixed_f32_grid=mixed_applies, fp64=(fp64 or {}).get("applies_per_s")),
                    fp64_plain=fp64,
                    speedup_vs_fp64=(value / world / fp64["solves_per_s"]) if fp64 else None,
                    gmres=dict(mean_iterations=float(np.mean(iters)), max_iterations=int(max(iters)),
                               max_rel_residual=float(max(i["rel_residual"] for i in infos)),
                               refinements=float(np.mean([i["refinements"] for i in infos]))),
                    wall_s=t_wall, roofline=roofline, cpu_baseline=cpu, e2e=e2e, gpu_launches=int(launches),
                    clocks=clocks)
        print(json.dumps(line))
    st.close()
    ctx.close()
    if pg:
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
