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


def slowest_rank_seconds(total_s, dist_mod=None, device="cpu"):
    """The timed region's length for the whole job: the maximum over the ranks (each rank
    timed its own replica between two barriers)."""
    if dist_mod is None:
        return float(total_s)
    import torch

    t = torch.tensor([float(total_s)], dtype=torch.float64, device=device)
    dist_mod.all_reduce(t, op=dist_mod.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, world, slowest_s):
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return world * units_per_rank / slowest_s


def shard(count, rank, world):
    """Instances of a batch owned by one rank (contiguous, sizes differ by at most one): the
    instances are independent, so ranks share no data and need no collective."""
    base, extra = divmod(count, world)
    start = rank * base + min(rank, extra)
    return list(range(start, start + base + (1 if rank < extra else 0)))


def bench_config(world=1):
    """The workload's config: the same dict in both arms' lines."""
    return dict(workload=WORKLOAD, grid=1024, nodes=1024, box=[-4, 4], sigma=SIGMA, J=J, dt=DT, tol=TOL,
                parallelism=f"replicas{world}", l2="flushed (512 MB write) before every timed step")


def host_cpu():
    """Model, cores and threads of the host CPU (lscpu when present, else /proc/cpuinfo)."""
    info = dict(logical_cpus=os.cpu_count())
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            k, _, v = ln.partition(":")
            k, v = k.strip(), v.strip()
            if k in ("Architecture", "Model name", "CPU(s)", "Thread(s) per core", "Core(s) per socket", "Socket(s)",
                     "CPU max MHz", "Vendor ID"):
                info[k] = v
    except (OSError, subprocess.SubprocessError):
        try:
            for ln in open("/proc/cpuinfo"):
                if ln.lower().startswith(("model name", "cpu part")):
                    info["model"] = ln.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    return info


def oracle_sample(budget_s, max_applies):
    """One bounded oracle sample of the workload in this process: one set_interface and up to
    max_applies BIE applies within budget_s seconds. Returns (t_set, t_app, applies)."""
    import workloads as W
    from oracle import kfbi as OK
    from oracle import thetal as OT

    p = workload()
    st = OT.state_from_nodes(p.xy, p.theta, p.L)
    s = OK.Kfbi(p.N, p.box, 0.0, OK.BOX_FREESPACE_DL)
    t0 = time.perf_counter()
    s.set_interface(OT.reconstruct(st.eta, st.L, st.Xbar))
    t_set = time.perf_counter() - t0
    phi = W.random_density(3, p.n)
    t1 = time.perf_counter()
    napp = 0
    while True:
        s.bie_matvec(OK.BIE_HS_EXTERIOR_MDL, phi)
        napp += 1
        if time.perf_counter() - t1 > budget_s - t_set or napp >= max_applies:
            break
    return t_set, (time.perf_counter() - t1) / napp, napp


THREAD_VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS")


def oracle_sample_subprocess(budget_s, max_applies, one_core):
    """oracle_sample in a fresh interpreter: with one_core, every BLAS/OpenMP pool is limited to
    one thread (scipy.fft runs one worker either way: the oracle passes no workers)."""
    env = dict(os.environ)
    if one_core:
        for v in THREAD_VARS:
            env[v] = "1"
    code = (f"import sys, json; sys.path.insert(0, {ROOT!r}); import bench; "
            f"print(json.dumps(bench.oracle_sample({budget_s}, {max_applies})))")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=600)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-500:])
    t_set, t_app, napp = json.loads(r.stdout.strip().splitlines()[-1])
    return t_set, t_app, napp


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="kfbi", choices=["kfbi", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched (256 instances), warm-start and Stefan measurements")
    ap.add_argument("--profile", action="store_true",
                    help="timed steps only (for short profiler runs): no e2e, applies, fp64 or cpu legs")
    ap.add_argument("--profile-stefan", type=int, default=0, metavar="N",
                    help="for profiler launch lists: three mixed Stefan steps on an N^2 grid with N nodes "
                         "(tol 1e-8), CUDA graphs off so that every kernel of the solve is listed; no JSON line")
    ap.add_argument("--baselines", action="store_true",
                    help="one JSON line of the per-config table: the oracle on one core and on all cores and the "
                         "GPU forms for configs 1-5 (several minutes of host time)")
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


def l2_copy_peak(torch, mib=24, reps=200):
    """L2-resident copy bandwidth (GB/s, read + write bytes): a `mib` MiB tensor copied into
    another one back to back (both fit the 129 MB L2 together), CUDA events, best of 3."""
    n = mib * (1 << 20) // 4
    a = torch.ones(n, dtype=torch.float32, device="cuda")
    b = torch.empty_like(a)
    for _ in range(20):
        b.copy_(a)
    best = 0.0
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            b.copy_(a)
        e1.record()
        torch.cuda.synchronize()
        best = max(best, 2.0 * 4 * n * reps / (e0.elapsed_time(e1) * 1e-3) / 1e9)
    return best


def traffic_record(kernel_src, name):
    """DRAM traffic per launch from a committed ncu summary, if taken on this kernel source."""
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None
    rec = json.load(open(path))
    h = hashlib.sha256(open(kernel_src, "rb").read()).hexdigest()[:16]
    if rec.get("source_sha256_16") != h:
        return None
    return rec


def batched_leg(torch, K, flush, reps=3):
    """256 uneven interior Dirichlet instances (N in {128, 256, 512}, n in [64, 512],
    kappa in {0, 10, 100}), mixed precision, tol 1e-8: autotuned (untimed), then whole-batch
    solves from zero (one graph launch each, L2 flushed before each) against the same
    instances solved one after another with kfbi_solve_bie."""
    import numpy as np

    import workloads as W

    probs = W.config_batched(256)
    descs = [dict(N=p.N, box=p.box, kappa=p.kappa, boxbc=K.BOX_DIRICHLET0, max_nodes=p.n) for p in probs]
    t0 = time.perf_counter()
    b = K.Batch(descs, K.MIXED)
    for c, p in zip(b.contexts, probs):
        c.set_interface(torch.tensor(p.xy, dtype=torch.float64, device="cuda"))
    rhs = [torch.tensor(p.rhs, dtype=torch.float64, device="cuda") for p in probs]
    dens = [torch.zeros(p.n, dtype=torch.float64, device="cuda") for p in probs]
    setup_s = time.perf_counter() - t0
    tol, max_iter, restart = 1e-8, 1000, 100
    t0 = time.perf_counter()
    tuned_ms = b.autotune(K.BIE_INTERIOR_DL, rhs, tol=tol, max_iter=max_iter, restart=restart)
    tune_s = time.perf_counter() - t0
    choice = {}
    for c in b.contexts:
        form = ("tensor_core" if c.get_option(K.OPT_COL_TC) else "register" if c.get_option(K.OPT_COL_REG)
                else "radix4" if c.get_option(K.OPT_COL_RADIX4) & 1 else "radix16")
        choice.setdefault(c.N, (c.get_option(K.OPT_CLUSTER_GMRES), c.get_option(K.OPT_CLUSTER_SIZE),
                                c.get_option(K.OPT_COL_PAIRS), form))
    b.solve(K.BIE_INTERIOR_DL, rhs, dens, tol=tol, max_iter=max_iter, restart=restart)  # graph build
    ms = []
    infos = None
    for _ in range(reps):
        for d in dens:
            d.zero_()
        flush.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        _, infos = b.solve(K.BIE_INTERIOR_DL, rhs, dens, tol=tol, max_iter=max_iter, restart=restart)
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    # the same instances one at a time (each a graph launch and a synchronisation)
    for d in dens:
        d.zero_()
    flush.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for c, r, d in zip(b.contexts, rhs, dens):
        c.solve_bie(K.BIE_INTERIOR_DL, r, density=d, tol=tol, max_iter=max_iter, restart=restart)
    torch.cuda.synchronize()
    seq_s = time.perf_counter() - t0
    its = [i["iterations"] for i in infos]
    conv = int(sum(1 for i in infos if i["status"] == 0))
    out = dict(workload="batched_256_uneven_N128-512_n64-512_kappa0-10-100", instances=len(probs),
               precision="mixed (f32 grid applies and inner Gram-Schmidt, f64 residual/refinement)", tol=tol,
               converged_solves_per_s=conv / (float(np.median(ms)) / 1e3),
               note=(f"solves that reached tol only; {len(probs) - conv} instances stop unconverged at max_iter "
                     f"(node spacing below the cell width) and are timed but not counted"),
               ms_per_batch=float(np.median(ms)),
               sequential_converged_solves_per_s=conv / seq_s,
               converged=conv,
               mean_iterations=float(np.mean(its)), max_iterations=int(max(its)),
               max_rel_residual=float(max(i["rel_residual"] for i in infos)),
               autotune=dict(seconds=tune_s, best_ms=tuned_ms,
                             choice={str(k): dict(cluster=v[0], cluster_size=v[1], col_pairs=v[2], col_form=v[3])
                                     for k, v in sorted(choice.items())}),
               setup_s=setup_s, l2="flushed before every timed batch")
    b.close()
    # the float64 form of the same batch: one untimed launch (graph building), one timed
    b64 = K.Batch(descs, K.FP64)
    for c, p in zip(b64.contexts, probs):
        c.set_interface(torch.tensor(p.xy, dtype=torch.float64, device="cuda"))
    b64.solve(K.BIE_INTERIOR_DL, rhs, dens, tol=tol, max_iter=max_iter, restart=restart)
    for d in dens:
        d.zero_()
    flush.zero_()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    _, infos64 = b64.solve(K.BIE_INTERIOR_DL, rhs, dens, tol=tol, max_iter=max_iter, restart=restart)
    e1.record()
    torch.cuda.synchronize()
    conv64 = int(sum(1 for i in infos64 if i["status"] == 0))
    out["fp64"] = dict(ms_per_batch=e0.elapsed_time(e1), converged=conv64,
                       converged_solves_per_s=conv64 / (e0.elapsed_time(e1) / 1e3),
                       mean_iterations=float(np.mean([i["iterations"] for i in infos64])))
    b64.close()
    return out


def warmstart_leg(torch, K):
    """The learned warm start: trained on 80 interior Laplace problems solved by the GPU
    method (FP64, 256^2 grid), evaluated on 12 others: initial residual and GMRES iterations
    from the network's density against the zero start."""
    import numpy as np

    import workloads as W

    ctx = K.Context(256, (-1.0, 1.0, -1.0, 1.0), 0.0, K.BOX_DIRICHLET0, K.FP64, max_nodes=512)
    feats, targets = [], []
    t0 = time.perf_counter()
    for s in range(1000, 1080):
        p = W.warmstart_problem(s)
        ctx.set_interface(torch.tensor(p.xy, dtype=torch.float64, device="cuda"))
        r = torch.tensor(p.rhs, dtype=torch.float64, device="cuda")
        phi, _ = ctx.solve_bie(K.BIE_INTERIOR_DL, r, tol=1e-12, max_iter=400, restart=100)
        f, scale = ctx.warmstart_features(r)
        feats.append(f.clone())
        targets.append((phi / scale).to(torch.float32))
    X, T = torch.cat(feats), torch.cat(targets)
    data_s = time.perf_counter() - t0
    m = K.Mlp(hidden=256, max_rows=max(X.shape[0], 512))
    m.set_params(W.mlp_init(21))
    g = torch.Generator(device="cpu").manual_seed(0)
    first, _ = m.gradients(X, T)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    steps = 2500
    for it in range(steps):
        idx = torch.randint(0, X.shape[0], (512,), generator=g, dtype=torch.int32).cuda()
        m.train_step(X, T, idx=idx, lr=1e-3 if it < 1500 else 3e-4, want_loss=False)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    last, _ = m.gradients(X, T)
    its0, its1, r1 = [], [], []
    for s in range(5000, 5012):
        p = W.warmstart_problem(s)
        ctx.set_interface(torch.tensor(p.xy, dtype=torch.float64, device="cuda"))
        r = torch.tensor(p.rhs, dtype=torch.float64, device="cuda")
        guess = ctx.warmstart_predict(m, r)
        res = r - ctx.bie_apply(K.BIE_INTERIOR_DL, guess)
        r1.append(float(torch.linalg.norm(res) / torch.linalg.norm(r)))
        _, i0 = ctx.solve_bie(K.BIE_INTERIOR_DL, r, tol=1e-10, max_iter=400, restart=100)
        _, i1 = ctx.solve_bie(K.BIE_INTERIOR_DL, r, density=guess, tol=1e-10, max_iter=400, restart=100)
        its0.append(i0["iterations"])
        its1.append(i1["iterations"])
    ctx.close()
    return dict(training_rows=int(X.shape[0]), data_s=data_s, train_steps=steps, train_s=train_s,
                loss_first=first, loss_last=last, held_out=12,
                median_initial_residual=dict(zero=1.0, network=float(np.median(r1))),
                mean_gmres_iterations=dict(zero=float(np.mean(its0)), network=float(np.mean(its1))))


def warm_start_c5_leg(torch, K, train_steps=50, eval_steps=8):
    """The learned warm start on the time step of the 4096^2 Stefan dendrite (4096 nodes,
    tol 1e-8): a network (47-256-256-1, the library's kernels) trained on the (features,
    density) pairs of 50 steps of the 2048^2 dendrite (2048 nodes each, about 1e5 rows), then
    the same 4096^2 steps from one checkpoint with the previous-step start and with the
    network attached (each step takes the start with the smaller float64 residual)."""
    import numpy as np

    import workloads as W

    def stefan(N, n):
        p = W.config_stefan(N=N, n=n)
        x = p.extra
        ctx = K.Context(p.N, p.box, p.kappa, K.BOX_NEUMANN0, K.MIXED, max_nodes=p.n)
        eta = torch.tensor(p.theta - alpha_array(p.n), dtype=torch.float64, device="cuda")
        st = K.ThetaL(ctx, eta, p.L, p.xy.mean(0), K.STEP_STEFAN, tol=1e-8, max_iter=3000, restart=150,
                      St=x["St"], eps_c=x["eps_c"], eps_aniso=x["eps_aniso"], eps_v=x["eps_v"], fold=x["fold"])
        return p, ctx, st

    t0 = time.perf_counter()
    p3, c3, s3 = stefan(2048, 2048)
    feats, targets = [], []
    for _ in range(train_steps):
        s3.step(p3.extra["dt"])
        f, t = s3.training_pair()
        feats.append(f.clone())
        targets.append(t.clone())
    s3.close()
    c3.close()
    X, T = torch.cat(feats), torch.cat(targets)
    data_s = time.perf_counter() - t0
    m = K.Mlp(hidden=256, max_rows=max(X.shape[0], 4096))
    m.set_params(W.mlp_init(21))
    g = torch.Generator(device="cpu").manual_seed(0)
    first, _ = m.gradients(X, T)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for it in range(3000):
        idx = torch.randint(0, X.shape[0], (512,), generator=g, dtype=torch.int32).cuda()
        m.train_step(X, T, idx=idx, lr=1e-3 if it < 2000 else 3e-4, want_loss=False)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    last, _ = m.gradients(X, T)
    p5, c5, s5 = stefan(4096, 4096)
    dt = p5.extra["dt"]
    for _ in range(3):
        s5.step(dt)
    ck = s5.read(T=True)
    ck = {k: (v.clone() if torch.is_tensor(v) else v) for k, v in ck.items()}
    res = {}
    for name, net in (("previous_step", None), ("network_policy", m)):
        s5.write(eta=ck["eta"], density=ck["density"], nhat=ck["nhat"], T=ck["T"], T_prev=ck["T_prev"],
                 scalars=ck["scalars"])
        s5.set_warmstart(net)
        torch.cuda.synchronize()
        its, ms = [], []
        for _ in range(eval_steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            info = s5.step(dt)
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
            its.append(info["iterations"])
        out = s5.read(T=False)
        res[name] = dict(mean_gmres_iterations=float(np.mean(its)), ms_per_step=float(np.mean(ms)),
                         density=out["density"].clone(),
                         network_starts=int(out["scalars"][14] - ck["scalars"][14]),
                         last_residual_ratio=float(out["scalars"][15]))
        s5.set_warmstart(None)
    d = float((res["network_policy"]["density"] - res["previous_step"]["density"]).abs().max()
              / res["previous_step"]["density"].abs().max())
    for r in res.values():
        r.pop("density")
    s5.close()
    c5.close()
    return dict(workload="stefan_4096x4096_n4096 (network trained on stefan_2048x2048_n2048 steps)", tol=1e-8,
                training_rows=int(X.shape[0]), data_s=data_s, train_steps=3000, train_s=train_s,
                loss_first=first, loss_last=last, eval_steps=eval_steps, **res,
                final_density_rel_diff=d)


def long_time_hs_leg(torch, K, steps=300):
    """The long-time Hele-Shaw computation of Sec. 6.1.4 in its rescaled frame: nucleus
    r = 1 + 0.1 (sin 2a + cos 3a) in (-1.7, 1.7)^2, 1024^2 grid, dt = 2e-4 (scaled time), J = 1,
    sigma = 1e-3, markers doubled whenever their spacing exceeds 1.5 h (start: 2048 nodes), mixed
    form to 1e-8. The first `steps` steps are timed; the paper's run takes 15000 steps (to scaled
    time 3) in 5 hours on one CPU core, context only."""
    import numpy as np

    import workloads as W

    shape = W.polar(1.0, [(2, 0.1, -math.pi / 2), (3, 0.1, 0.0)])  # 1 + 0.1 sin 2a + 0.1 cos 3a
    n0 = 2048
    nd = W.equal_arclength(shape, n0)
    ctx = K.Context(1024, (-1.7, 1.7, -1.7, 1.7), 0.0, K.BOX_FREESPACE_DL, K.MIXED, max_nodes=16384)
    eta = torch.tensor(nd["theta"] - alpha_array(n0), dtype=torch.float64, device="cuda")
    st = K.ThetaL(ctx, eta, nd["L"], nd["xy"].mean(0), K.STEP_HELE_SHAW, tol=1e-8, max_iter=1000, restart=150,
                  sigma=1e-3, J=1.0, refine_ratio=1.5, rescale=True)
    dt = 2e-4
    ms, its, ns = [], [], []
    for _ in range(steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        info = st.step(dt)
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
        its.append(info["iterations"])
        ns.append(st.n)
    out = st.read(T=False)
    sc = out["scalars"]
    A0, tb = sc[16], sc[3]
    R = math.exp(tb)
    st.close()
    ctx.close()
    per = float(np.mean(ms))
    return dict(workload="hele_shaw_long_time_rescaled_1024x1024 (Sec. 6.1.4 setup)", steps=steps, dt_scaled=dt,
                ms_per_step=per, mean_gmres_iterations=float(np.mean(its)), nodes_first=ns[0], nodes_last=ns[-1],
                scaled_time=tb, physical_time=(A0 / math.pi) * (math.exp(2 * tb) - 1) / 2, R=R,
                projected_s_for_15000_steps=per * 15000 / 1e3,
                projection_note=("extrapolated from the first steps' mean; node count and GMRES work grow as the "
                                 "fingers develop, so the true total is larger"),
                paper_context="5 h for the 15000-step run on one i7-10700K core (Sec. 6.1.4); not the same "
                              "workload length or hardware")


def stefan_leg(torch, K, steps=3, N=2048, n=2048, tol=1e-9, compare_fp64=True):
    """Stefan dendrite steps on the N^2 Neumann grid (seed r = 0.1 (1 + 0.2 cos 4a) in [-2,2]^2,
    undercooling -0.5, 4-fold anisotropy, dt = 5e-4), mixed precision to tol; the GMRES start
    of every step is the previous step's density."""
    import numpy as np

    import workloads as W

    p = W.config_stefan(N=N, n=n)
    x = p.extra
    ctx = K.Context(p.N, p.box, p.kappa, K.BOX_NEUMANN0, K.MIXED, max_nodes=p.n)
    eta = torch.tensor(p.theta - alpha_array(p.n), dtype=torch.float64, device="cuda")
    st = K.ThetaL(ctx, eta, p.L, p.xy.mean(0), K.STEP_STEFAN, tol=tol, max_iter=3000, restart=150,
                  St=x["St"], eps_c=x["eps_c"], eps_aniso=x["eps_aniso"], eps_v=x["eps_v"], fold=x["fold"])
    st.step(x["dt"])
    torch.cuda.synchronize()
    ms, infos = [], []
    for _ in range(steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        infos.append(st.step(x["dt"]))
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    # the float64 form from the last state: one untimed step (graph building), then one timed
    # step from the same state; with compare_fp64, the accuracy of the mixed form is one step of
    # it and of the float64 form from that state
    err, fp64 = None, None
    ck = st.read(T=True)
    ck = {k: (v.clone() if torch.is_tensor(v) else v) for k, v in ck.items()}
    ctx64 = K.Context(p.N, p.box, p.kappa, K.BOX_NEUMANN0, K.FP64, max_nodes=p.n)
    st64 = K.ThetaL(ctx64, ck["eta"].clone(), p.L, p.xy.mean(0), K.STEP_STEFAN, tol=tol, max_iter=3000, restart=150,
                    St=x["St"], eps_c=x["eps_c"], eps_aniso=x["eps_aniso"], eps_v=x["eps_v"], fold=x["fold"])
    outs = []
    for state in ((st, st64) if compare_fp64 else (st64,)):
        reps = 2 if state is st64 else 1
        for r in range(reps):
            state.write(eta=ck["eta"], density=ck["density"], nhat=ck["nhat"], T=ck["T"], T_prev=ck["T_prev"],
                        scalars=ck["scalars"])
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            info64 = state.step(x["dt"])
            e1.record()
            torch.cuda.synchronize()
        if state is st64:
            fp64 = dict(ms_per_step=e0.elapsed_time(e1), gmres_iterations=info64["iterations"],
                        status=info64["status"], note="one step from the last mixed state, after one untimed step")
        outs.append(state.read(T=True))
    if compare_fp64:
        a, b64 = outs
        err = dict(density_rel_diff=float((a["density"] - b64["density"]).abs().max() / b64["density"].abs().max()),
                   T_rel_diff=float((a["T"] - b64["T"]).abs().max() / b64["T"].abs().max()),
                   eta_max_abs_diff=float((a["eta"] - b64["eta"]).abs().max()))
    st64.close()
    ctx64.close()
    st.close()
    ctx.close()
    return dict(workload=f"stefan_{N}x{N}_n{n}", steps=steps, tol=tol, guess="previous-step density",
                ms_per_step=float(np.mean(ms)), steps_per_s=1e3 / float(np.mean(ms)),
                mean_gmres_iterations=float(np.mean([i["iterations"] for i in infos])),
                max_rel_residual=float(max(i["rel_residual"] for i in infos)),
                statuses=[i["status"] for i in infos], mixed_vs_fp64_one_step=err, fp64=fp64)


def apply_forms_leg(torch, K, reps=300):
    """Float32 apply of the Hele-Shaw 1024^2 workload with the row transform as its own kernel
    (default) and formed inside the column kernel (KFBI_OPT_FUSE_ROWS): CUDA events around
    `reps` applies back to back, warm L2."""
    import workloads as W

    p = W.config_hele_shaw()
    ctx = K.Context(p.N, p.box, p.kappa, K.BOX_FREESPACE_DL, K.MIXED, max_nodes=p.n)
    ctx.set_interface(torch.tensor(p.xy, dtype=torch.float64, device="cuda"))
    dens = torch.tensor(W.random_density(3, p.n, modes=20), dtype=torch.float64, device="cuda")
    vals = torch.empty(p.n, dtype=torch.float64, device="cuda")
    out = {}
    for name, fr in (("separate_row_kernel", 0), ("rows_in_column_kernel", 1)):
        ctx.set_option(K.OPT_FUSE_ROWS, fr)
        for _ in range(20):
            ctx.apply_into(K.DOUBLE, dens, vals)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            ctx.apply_into(K.DOUBLE, dens, vals)
        e1.record()
        torch.cuda.synchronize()
        out[name] = dict(us_per_apply=1e3 * e0.elapsed_time(e1) / reps)
    ctx.close()
    return out


# column forms of the size sweep: (name, COL_RADIX4 bits, COL_PAIRS, COL_REG, COL_TC)
COL_FORMS = (("radix16", 0, 0, 0, 0), ("radix16_p1", 0, 1, 0, 0), ("radix16_p2", 0, -2, 0, 0),
             ("radix16_16pt", 0, 0, 0, 0), ("radix4", 3, 0, 0, 0),
             ("radix4_p1", 3, 1, 0, 0), ("radix4_p4", 3, 4, 0, 0), ("register", 0, 0, 1, 0),
             ("tensor_core", 0, 0, 0, 1))


def col_kernel_sizes(torch, K, hbm_peak, reps=200):
    """Column transform time per launch by grid size for every column form (register-resident
    kernel with its pair counts, 8 points per thread up to 1024^2 by default and 16 as
    `radix16_16pt`, shared-memory radix-4 Stockham with 1, 2, 4 pairs, four-step
    register FFTs up to 1024^2, tensor-core contractions up to 256^2) in float32, and the radix-16
    and radix-4 kernels in float64: kfbi_time_column (CUDA events around `reps` launches back to
    back, warm L2) on a Neumann-box context with a 256-node star after one apply."""
    import workloads as W

    out = {}
    for N in (128, 256, 512, 1024, 2048, 4096):
        p = W.random_problem(17, N=N, n=256, kappa=30.0, boxbc=W.BOX_NEUMANN0)
        row = {}
        for prec in (K.MIXED, K.FP64):
            ctx = K.Context(N, p.box, 30.0, K.BOX_NEUMANN0, prec, max_nodes=p.n)
            ctx.set_interface(torch.tensor(p.xy, dtype=torch.float64, device="cuda"))
            dens = torch.ones(p.n, dtype=torch.float64, device="cuda")
            vals = torch.empty(p.n, dtype=torch.float64, device="cuda")
            f32 = prec == K.MIXED
            for form, r4, pairs, reg, tc in COL_FORMS:
                if (reg and N > 1024) or (tc and N > 256) or (not f32 and (reg or tc or pairs > 0)):
                    continue
                if not f32 and r4 == 0 and N > 2048:  # no float64 radix-16 kernel at 4096^2
                    continue
                if not f32 and form == "radix16_16pt":  # float64 has the 16-point form only
                    continue
                ctx.set_option(K.OPT_COL_REG, reg)
                ctx.set_option(K.OPT_COL_TC, tc)
                ctx.set_option(K.OPT_COL_RADIX4, r4)
                ctx.set_option(K.OPT_COL_PAIRS, min(16, 2 * max(1, 512 // N)) if pairs < 0 else pairs)
                ctx.set_option(K.OPT_COL_POINTS, 16 if form == "radix16_16pt" else 0)
                ctx.apply_into(K.DOUBLE, dens, vals)
                us = ctx.time_column(f32, reps if f32 else max(reps // 4, 5))
                elt = 4.0 if f32 else 8.0
                row[(form if f32 else "fp64_" + form)] = dict(
                    us=us, hbm_frac=(2 * elt * N * N) / (us * 1e-6) / 1e9 / hbm_peak)
            ctx.close()
        out[str(N)] = row
    return out


def cpu_baseline(iters_per_solve, budget_s=12.0):
    """The oracle as it stands on the host cores: a bounded sample of the same workload (one
    set_interface and a few BIE applies), on one core and on all cores, each in a fresh
    process; a solve is one set_interface plus the GPU run's mean GMRES count of applies."""
    legs = {}
    for name, one in (("one_core", True), ("all_cores", False)):
        t_set, t_app, napp = oracle_sample_subprocess(budget_s, 30, one)
        legs[name] = dict(t_set_s=t_set, t_apply_s=t_app, applies=napp,
                          solves_per_s=1.0 / (t_set + iters_per_solve * t_app), applies_per_s=1.0 / t_app)
    allc = legs["all_cores"]
    return dict(value=allc["solves_per_s"], unit="solves/s", cores=os.cpu_count(), kind="oracle",
                sample=(f"oracle (numpy/scipy FP64) on the host: one set_interface ({allc['t_set_s']:.2f} s) and "
                        f"{allc['applies']} BIE applies ({allc['t_apply_s']:.3f} s each) of the {WORKLOAD} workload, "
                        f"scaled to one solve of {iters_per_solve:.1f} applies (the GPU run's mean GMRES count) + "
                        f"set_interface; all cores = BLAS on every core, scipy.fft on one worker"),
                one_core=legs["one_core"], all_cores=allc, host=host_cpu(), basis="extrapolated from the sample")


# --------------------------------------------------------------------------- reference arm
def run_reference(args):
    """The CPU oracle on the host cores (the reference arm). Each step is a bounded sample of
    the workload, measured as it runs: one oracle set_interface and one BIE apply (about half
    a second). The line's value converts the measured sample to the metric's unit, one solve =
    one set_interface + ITERS applies; ms_per_step is the measured sample time."""
    rank, world, _ = dist_env()
    if world > 1 and rank != 0:
        return 0
    import numpy as np

    iters = 90.0  # GMRES applies per solve of this workload at 1e-8 (the GPU runs' mean)
    for _ in range(args.warmup):
        oracle_sample(0.0, 1)
    per = [oracle_sample(0.0, 1) for _ in range(args.steps)]
    t_set = float(np.mean([q[0] for q in per]))
    t_app = float(np.mean([q[1] for q in per]))
    value = 1.0 / (t_set + iters * t_app)
    line = dict(impl="reference", metric=METRIC, value=value, unit="solves/s", n_gpus=args.gpus, steps=args.steps,
                warmup=args.warmup, ms_per_step=1e3 * (t_set + t_app), higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="f64", data="synthetic", precision="fp64 (the CPU oracle)",
                config=bench_config(args.gpus),
                value_basis=(f"extrapolated: measured per step one set_interface ({t_set:.3f} s) + one BIE apply "
                             f"({t_app:.3f} s); value = 1 / (set_interface + {iters:.0f} applies), the applies a "
                             f"solve of this workload takes; ms_per_step is the measured sample"),
                applies_per_s=1.0 / t_app,
                cpu_baseline=dict(value=value, unit="solves/s", cores=os.cpu_count(), kind="oracle",
                                  sample=(f"each step: one oracle set_interface + one BIE apply of {WORKLOAD}, "
                                          f"scaled to {iters:.0f} applies per solve"), host=host_cpu()),
                e2e=dict(value=value, unit="solves/s", h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line))
    return 0


# --------------------------------------------------------------------------- per-config table
ORACLE_CONFIG_CODE = """
import sys, json, time
sys.path.insert(0, {root!r})
import numpy as np
import workloads as W
from oracle import kfbi as OK
from oracle.gmres import gmres
which = {which!r}
out = {{}}
if which == "c1":
    p = W.config_small_laplace()
    t0 = time.perf_counter()
    s = OK.Kfbi(p.N, p.box, 0.0, OK.BOX_DIRICHLET0).set_interface(p.xy)
    x, info = gmres(lambda v: s.bie_matvec(OK.BIE_INTERIOR_DL, v), p.rhs, tol=1e-10)
    out = dict(solve_s=time.perf_counter() - t0, iterations=info["iterations"])
    t0 = time.perf_counter()
    for _ in range(5):
        s.bie_matvec(OK.BIE_INTERIOR_DL, x)
    out["apply_s"] = (time.perf_counter() - t0) / 5
elif which == "c4":
    probs = W.config_batched(256)
    pick = [0, 1, 2, 3]
    t0 = time.perf_counter()
    its = []
    for i in pick:
        p = probs[i]
        s = OK.Kfbi(p.N, p.box, p.kappa, OK.BOX_DIRICHLET0).set_interface(p.xy)
        x, info = gmres(lambda v: s.bie_matvec(OK.BIE_INTERIOR_DL, v), p.rhs, tol=1e-8, max_iter=300)
        its.append(info["iterations"])
    out = dict(solve_s_per_instance=(time.perf_counter() - t0) / len(pick), instances=[int(i) for i in pick],
               iterations=its, grids=[probs[i].N for i in pick])
else:
    N, n, box, kap, bc, kind = dict(c2=(1024, 1024, 4.0, 0.0, OK.BOX_FREESPACE_DL, OK.BIE_HS_EXTERIOR_MDL),
                                    c3=(2048, 2048, 2.0, 3000.0, OK.BOX_NEUMANN0, OK.BIE_STEFAN_SL),
                                    c5=(4096, 4096, 2.0, 3000.0, OK.BOX_NEUMANN0, OK.BIE_STEFAN_SL))[which]
    p = W.config_hele_shaw(N=N, n=n, box=box) if which == "c2" else W.config_stefan(N=N, n=n, box=box)
    t0 = time.perf_counter()
    s = OK.Kfbi(N, p.box, kap, bc).set_interface(p.xy)
    t_set = time.perf_counter() - t0
    phi = W.random_density(3, n)
    ev = np.full(n, 2e-3)
    t0 = time.perf_counter()
    for _ in range(2):
        s.bie_matvec(kind, phi, eps_v=ev)
    out = dict(set_interface_s=t_set, apply_s=(time.perf_counter() - t0) / 2)
print(json.dumps(out))
"""


def oracle_config(which, one_core):
    env = dict(os.environ)
    if one_core:
        for v in THREAD_VARS:
            env[v] = "1"
    r = subprocess.run([sys.executable, "-c", ORACLE_CONFIG_CODE.format(root=ROOT, which=which)], capture_output=True,
                       text=True, env=env, timeout=3600)
    if r.returncode != 0:
        return dict(error=r.stderr[-400:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def run_baselines():
    """Per-config numbers for the baseline table: the oracle on one core and on all cores (full
    solves for configs 1 and 4, a set_interface and two applies for configs 2, 3 and 5, whose
    solves are then extrapolated by the GPU runs' iteration counts), and the GPU forms."""
    import numpy as np
    import torch

    import workloads as W
    from paper_2309_01068_gb300 import build
    from paper_2309_01068_gb300 import kfbi as K

    build.build()
    K.load()
    out = dict(host=host_cpu())
    for which in ("c1", "c2", "c3", "c4", "c5"):
        out[which] = dict(oracle_one_core=oracle_config(which, True), oracle_all_cores=oracle_config(which, False))
        print(f"[baselines] {which}: {out[which]}", file=sys.stderr)
    # GPU, config 1: solves/s and applies/s, float64 and mixed
    p = W.config_small_laplace()
    for name, prec in (("fp64", K.FP64), ("mixed", K.MIXED)):
        ctx = K.Context(p.N, p.box, 0.0, K.BOX_DIRICHLET0, prec, max_nodes=p.n)
        ctx.set_interface(torch.tensor(p.xy, dtype=torch.float64, device="cuda"))
        rhs = torch.tensor(p.rhs, dtype=torch.float64, device="cuda")
        ctx.solve_bie(K.BIE_INTERIOR_DL, rhs, tol=1e-10, max_iter=400)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        reps = 50
        for _ in range(reps):
            _, info = ctx.solve_bie(K.BIE_INTERIOR_DL, rhs, tol=1e-10, max_iter=400)
        torch.cuda.synchronize()
        out["c1"]["gpu_" + name] = dict(solves_per_s=reps / (time.perf_counter() - t0), iterations=info["iterations"],
                                        applies_per_s=time_applies(torch, K, ctx))
        ctx.close()
    print(json.dumps(out))
    return 0


# --------------------------------------------------------------------------- main arm
def profile_stefan(N):
    """Three mixed Stefan steps (seed, N^2 grid, N nodes, tol 1e-8) with the solve's CUDA graphs
    off: the subject of a profiler's launch list (kernels inside conditional graph nodes are not
    listed by it)."""
    import torch

    import workloads as W
    from paper_2309_01068_gb300 import build
    from paper_2309_01068_gb300 import kfbi as K

    build.build()
    K.load()
    p = W.config_stefan(N=N, n=N)
    x = p.extra
    ctx = K.Context(p.N, p.box, p.kappa, K.BOX_NEUMANN0, K.MIXED, max_nodes=p.n)
    ctx.set_option(K.OPT_CUDA_GRAPHS, 0)
    eta = torch.tensor(p.theta - alpha_array(p.n), dtype=torch.float64, device="cuda")
    st = K.ThetaL(ctx, eta, p.L, p.xy.mean(0), K.STEP_STEFAN, tol=1e-8, max_iter=3000, restart=150, St=x["St"],
                  eps_c=x["eps_c"], eps_aniso=x["eps_aniso"], eps_v=x["eps_v"], fold=x["fold"])
    for s in range(3):
        info = st.step(x["dt"])
        torch.cuda.synchronize()
        print(f"[bench] stefan {N}: step {s}, {info['iterations']} GMRES iterations, status {info['status']}",
              file=sys.stderr)
    st.close()
    ctx.close()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.baselines:
        return run_baselines()
    if args.profile_stefan:
        return profile_stefan(args.profile_stefan)
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
    # ALU roofs of this GPU (float32 and float64 FMA), measured by the library's probe kernel
    # (not in --profile runs, whose launch lists should hold the workload's kernels only)
    alu = {} if args.profile else dict(fp32_tflops=K.alu_peak(0), fp64_tflops=K.alu_peak(1))

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
    total_s = slowest_rank_seconds(sum(ms) / 1e3, pg, "cuda")
    # kernel timing pass: the same steps again from the same state with per-launch CUDA events
    # around the column kernel (event timing runs the solver's stream-launched form; the
    # kernels are the same as in the graph form timed above)
    st.write(eta=ckpt["eta"], density=ckpt["density"], nhat=ckpt["nhat"], scalars=ckpt["scalars"])
    ctx.timing(True)
    run_steps(torch, ctx, st, min(args.steps, 10), flush)
    tim = ctx.timing()
    ctx.timing(False)
    iters = [i["iterations"] for i in infos]
    value = job_throughput(args.steps, world, total_s)
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
    csrc = os.path.join(ROOT, "paper_2309_01068_gb300", "csrc")
    if ctx.get_option(K.OPT_COL_RADIX4) & 1:
        kname = "k_col_solve<float> (radix-4 shared-memory Stockham: column DST-II, eigen divide, inverse DST)"
        tr = traffic_record(os.path.join(csrc, "kfbi_apply.cu"), "k_col_solve_traffic.json")
    else:
        pt = ctx.get_option(K.OPT_COL_POINTS) or (8 if N <= 1024 else 16)
        kname = (f"k_col_fft<float,{int(math.log2(N))},P,0,{pt}> (register-resident column solve, {pt} points "
                 "per thread: DST-II, eigen divide, inverse DST)")
        tr = traffic_record(os.path.join(csrc, "kfbi_colfft.cu"), "k_col_fft_traffic.json")
    # the same kernel back to back (kfbi_time_column: warm L2, programmatic dependent launch as
    # in the GMRES loop, no event between launches)
    # (not in --profile runs, whose launch lists should hold the workload's kernels only)
    b2b = None
    if not args.profile:
        b2b_us = ctx.time_column(True, 400)
        b2b = dict(us=b2b_us, achieved=bytes_per_launch / (b2b_us * 1e-6) / 1e9,
                   frac=bytes_per_launch / (b2b_us * 1e-6) / 1e9 / hbm_peak, launches=400)
        # the grid is L2-resident inside GMRES: the same bytes against the L2 copy bandwidth
        l2_gbs = l2_copy_peak(torch)
        b2b["l2"] = dict(bound="l2", peak=l2_gbs, unit="GB/s", frac=b2b["achieved"] / l2_gbs,
                         peak_source="torch copy of a 24 MiB float32 tensor, L2-resident, measured in this run")
    roofline = dict(kernel=kname,
                    bound="hbm", achieved=achieved, peak=hbm_peak, unit="GB/s",
                    frac=(achieved / hbm_peak) if achieved else None,
                    traffic=(tr["dram_bytes_per_launch"] if tr else None),
                    algorithmic_bytes_per_launch=bytes_per_launch, launches=tim["fp32_launches"],
                    mean_launch_us=f32_ms * 1e3, back_to_back=b2b,
                    traffic_in_loop=(dict(dram_bytes=float(np.mean([a + b for a, b in zip(tr["in_loop"]["dram_bytes_read"],
                                                                                        tr["in_loop"]["dram_bytes_write"])])),
                                          l2_bytes=float(np.mean(tr["in_loop"]["l2_bytes"])),
                                          note="caches kept between launches, as in the GMRES loop")
                                     if tr and "in_loop" in tr else None),
                    peak_source="MEASURED_PEAKS.json hbm_gbs (of measured)" if peaks else "fallback 6.8 TB/s")
    # the same kernel against the float32 FMA roof: forward and inverse real transforms of N
    # columns of length N, 2.5 M log2 M flops each (split-radix count of a real FFT)
    flops_per_launch = 2 * N * 2.5 * N * math.log2(N)
    if achieved and alu.get("fp32_tflops"):
        a_tf = flops_per_launch / (f32_ms * 1e-3) / 1e12
        roofline["alu"] = dict(bound="alu", achieved=a_tf, peak=alu["fp32_tflops"], unit="TFLOP/s",
                               frac=a_tf / alu["fp32_tflops"], algorithmic_flops_per_launch=flops_per_launch,
                               peak_source="kfbi_alu_peak float32 FMA probe on this GPU (of measured)")

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
        col64_us = 1e3 * tim64["fp64_ms"] / max(tim64["fp64_launches"], 1)
        fp64 = dict(solves_per_s=k64 / (sum(ms64) / 1e3), steps=k64,
                    mean_gmres_iterations=float(np.mean([i["iterations"] for i in infos64])),
                    applies_per_s=fp64_applies, col_kernel_mean_us=col64_us)
        if tim64["fp64_launches"] and alu.get("fp64_tflops"):
            a64 = flops_per_launch / (col64_us * 1e-6) / 1e12
            fp64["col_kernel_roofline"] = dict(
                bound="alu", achieved=a64, peak=alu["fp64_tflops"], unit="TFLOP/s", frac=a64 / alu["fp64_tflops"],
                hbm_frac=(2.0 * N * N * 8) / (col64_us * 1e-6) / 1e9 / hbm_peak,
                peak_source="kfbi_alu_peak float64 FMA probe on this GPU (of measured)")
        # accuracy of the mixed form on this workload: one step of each form from the same
        # state; the float64 form is the one the parity tests pin to the oracle
        outs = []
        for state in (st, st64):
            state.write(eta=ckpt["eta"], density=ckpt["density"], nhat=ckpt["nhat"], scalars=ckpt["scalars"])
            state.step(DT)
            outs.append(state.read(T=False))
        dm, d64 = outs[0]["density"], outs[1]["density"]
        fp64["mixed_vs_fp64_one_step"] = dict(
            density_rel_diff=float((dm - d64).abs().max() / d64.abs().max()),
            eta_max_abs_diff=float((outs[0]["eta"] - outs[1]["eta"]).abs().max()))
        st64.close()
        ctx64.close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(float(np.mean(iters)))

    # ---- further workloads (reported beside the headline, never part of it)
    extras = {}
    if rank == 0 and not args.profile and not args.no_extras:
        for name, leg in (("col_kernel_sizes", lambda: col_kernel_sizes(torch, K, hbm_peak)),
                          ("apply_forms", lambda: apply_forms_leg(torch, K)),
                          ("batched", lambda: batched_leg(torch, K, flush)), ("warm_start", lambda: warmstart_leg(torch, K)),
                          ("stefan", lambda: stefan_leg(torch, K)),
                          ("warm_start_c5", lambda: warm_start_c5_leg(torch, K)),
                          ("long_time_hs", lambda: long_time_hs_leg(torch, K)),
                          ("stefan_4096", lambda: stefan_leg(torch, K, N=4096, n=4096, tol=1e-8, compare_fp64=False))):
            try:
                extras[name] = leg()
            except Exception as exc:  # noqa: BLE001 - a failing extra must not lose the headline
                extras[name] = dict(error=f"{type(exc).__name__}: {exc}")
            print(f"[bench] {name}: {extras[name]}", file=sys.stderr)

    if rank == 0:
        line = dict(metric=METRIC, value=value, unit="solves/s", n_gpus=world, steps=args.steps,
                    warmup=args.warmup, ms_per_step=1e3 * total_s / args.steps, higher_is_better=True,
                    scaling="weak", vs_baseline=None, dtype="f32+f64", data="synthetic",
                    precision="mixed (f32 grid applies and inner Gram-Schmidt, f64 residual/refinement)",
                    config=bench_config(world),
                    applies_per_s=dict(mixed_f32_grid=mixed_applies, fp64=(fp64 or {}).get("applies_per_s")),
                    fp64_plain=fp64,
                    speedup_vs_fp64=(value / world / fp64["solves_per_s"]) if fp64 else None,
                    gmres=dict(mean_iterations=float(np.mean(iters)), max_iterations=int(max(iters)),
                               max_rel_residual=float(max(i["rel_residual"] for i in infos)),
                               refinements=float(np.mean([i["refinements"] for i in infos]))),
                    wall_s=t_wall, roofline=roofline, alu_peaks_tflops=alu, cpu_baseline=cpu, e2e=e2e,
                    gpu_launches=int(launches),
                    clocks=clocks, **extras)
        print(json.dumps(line))
    st.close()
    ctx.close()
    if pg:
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
