"""Throughput benchmark of the batched gradient of forward dynamics.

One step = one pass of the whole path (joint transforms, RNEA(q, qd, 0), direct
M^-1, FD, RNEA at qdd, analytical RNEA derivatives, -M^-1 dID) over one batch:
B trajectories x 128 knot points of the 7-DoF chain in FP32, inputs already
resident in HBM. Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (the reference arm of this build)
on the host cores on a bounded sample of the same workload.
Under torchrun every rank processes its own B trajectories (weak scaling, no
collective on the data path); value = all knot points / max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import grid_inputs as gi  # noqa: E402

METRIC = "∇FD knot-points/sec at N=128 (FP32/mixed vs FP64 plain); serve p50/p99 ms"
UNIT = "knot-points/s"
KNOTS = 128                      # knot points per trajectory (the metric's N)
TRAJ = 16384                     # trajectories per step (2,097,152 knot points)
SM_COUNT = 152
FP32_LANES_PER_SM = 128
SM_MAX_MHZ = 2070.0
L2_BYTES = 129 * 1024 * 1024
# FP32 peak from unit counts and the maximum SM clock: 152 SMs x 128 FP32
# lanes x 2 flops (FMA) x 2.07 GHz.
FP32_PEAK_TFLOPS = SM_COUNT * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
# DRAM bytes per knot point of the gradient kernel from an ncu capture, keyed
# by a hash of the kernel sources; absent when the kernel changed since.
# (profiles/grad_fd_chain7_ncu_full.md: DRAM read + write of a 524,288-knot-point
# launch, scaled by knot points to the benchmark's launch.)
NCU_DRAM_BYTES_PER_KNOT = {"517743476c2097e0": 199.75e6 / 524288,
                           "d1f6cfa03f54f835": 199.17e6 / 524288,
                           "e04804cb5f3a6d15": 188.95e6 / 524288,
                           "59c365e8cec7dca6": 189.65e6 / 524288,
                           "c7c560789c0e9069": 189.20e6 / 524288,
                           "a032ad23a8b5e7d9": 189.45e6 / 524288,
                           "f8f85c036843ba52": 189.67e6 / 524288,
                           # kernel code identical to f8f85c036843ba52: only the host-buffer
                           # pipeline (grid_capi.cu) and a host-side model field were added
                           "3b0e48a5f622bbea": 189.67e6 / 524288,
                           "ea367adecd85eda9": 189.21e6 / 524288,
                           # 7-DoF chain kernel identical to ea367adecd85eda9: only the branch
                           # kernel's launch bounds changed
                           "afb5ee0d6c339fe3": 189.21e6 / 524288}
# FP32 (FMA) pipe utilisation of the same captures: sm__pipe_fma_cycles_active, % of
# peak sustained while active (busy cycles, so a paired FP32 instruction counts for the
# cycles it occupies), reported beside the counted-flop fraction.
NCU_FMA_PIPE = {"e04804cb5f3a6d15": 0.401, "59c365e8cec7dca6": 0.418, "c7c560789c0e9069": 0.432,
                "a032ad23a8b5e7d9": 0.418, "f8f85c036843ba52": 0.418, "3b0e48a5f622bbea": 0.418,
                "ea367adecd85eda9": 0.417, "afb5ee0d6c339fe3": 0.417}


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2109_06976_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        with open(os.path.join(d, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, v in zip(self.NAMES, parts[3:7]):
                if v.lower() in ("active", "1"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(n_gpus):
    import torch
    if n_gpus <= 1 or "RANK" not in os.environ:
        return 0, 1, 0, None
    import torch.distributed as dist
    local = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(local)
    dist.init_process_group("nccl")
    return dist.get_rank(), dist.get_world_size(), local, dist


def max_over_ranks(sec, dist=None, device="cuda"):
    """Largest elapsed time over all ranks (the whole job ends with the slowest)."""
    if dist is None:
        return sec
    import torch
    t = torch.tensor([sec], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_seed(rank):
    """Each rank draws its own trajectories (weak scaling: independent shards)."""
    return gi.workload_seed(2, KNOTS) + 7919 * rank


def aggregate_value(world, knots_per_rank, steps, sec):
    """Whole-job throughput: every rank's knot points over the slowest rank's time."""
    return world * knots_per_rank * steps / sec


def time_steps(fn, steps, warmup, stream, dist=None):
    """W untimed steps, then K steps bracketed by barrier + synchronize; CUDA
    events on the launching stream. Returns (seconds, max over ranks)."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    return max_over_ranks(e0.elapsed_time(e1) / 1e3, dist)


def traj_leg(grid, model, stream, dist, B=2048, H=64, dt=0.01):
    """One iLQR iteration on the device for B trajectories of H steps of the
    7-DoF chain (rollout, gradient of FD and M^-1 at the B (H+1) knot points,
    backward pass, policy rollout), FP32, inputs resident; and its parts."""
    import numpy as np
    import torch
    import grid_inputs as gi
    n = model.n
    s = gi.Stream(4242)
    q0, qd0, _ = (torch.from_numpy(x.astype(np.float32)).cuda() for x in gi.states(n, B, 4242))
    U = torch.from_numpy((0.3 * s.normal((B, H + 1, n))).astype(np.float32)).cuda()
    Qref = torch.zeros_like(U)
    QDref = torch.zeros_like(U)
    wq = torch.tensor([10.0] * n + [0.1] * n, device="cuda")
    wr = torch.full((n,), 1e-3, device="cuda")
    wf = 10.0 * wq
    it = lambda: model.ilqr_iteration(q0, qd0, U, Qref, QDref, wq, wr, wf, dt, 1e-6, 1.0)
    steps = 5
    sec = time_steps(it, steps, 2, stream, dist)
    Q, QD, _ = model.rollout(q0, qd0, U, dt)
    J, Mi = model.grad_fd_minv(Q, QD, U)
    parts = {
        "rollout_ms": time_steps(lambda: model.rollout(q0, qd0, U, dt), steps, 2, stream, dist) / steps * 1e3,
        "grad_fd_minv_ms": time_steps(lambda: model.grad_fd_minv(Q, QD, U, out=J, minv_out=Mi), steps, 2,
                                      stream, dist) / steps * 1e3,
        "riccati_ms": time_steps(lambda: model.riccati(Q, QD, U, J, Mi, Qref, QDref, wq, wr, wf, dt, 1e-6), steps,
                                 2, stream, dist) / steps * 1e3,
    }
    return {"trajectories": B, "horizon": H, "ms_per_iteration": sec / steps * 1e3,
            "knot_points_per_s": B * (H + 1) * steps / sec, **parts,
            "note": "one iLQR iteration = rollout + gradient of FD and M^-1 at every knot point + "
                    "backward pass + policy rollout, all on the device (7-DoF chain, FP32)"}


def n_sweep(grid, Ns=(32, 64, 128, 256, 512), reps=100):
    """One launch of a single N-knot trajectory (compute only, device time) for
    the 7- and 12-DoF robots, FP32 against the FP64-plain form."""
    import numpy as np
    import torch
    import grid_inputs as gi
    out = {}
    for name in ("chain7", "tree12"):
        r = gi.robot(name)
        m = grid.Model.from_robot(r)
        row = {}
        for N in Ns:
            for dt, tag in ((torch.float32, "f32"), (torch.float64, "f64")):
                q, qd, tau = (torch.from_numpy(x).to("cuda", dt) for x in gi.states(r.n, N, gi.workload_seed(2, N)))
                J = torch.empty((N, r.n, 2 * r.n), device="cuda", dtype=dt)
                row[f"{tag}_N{N}_us"] = device_latency_us(lambda: m.grad_fd(q, qd, tau, out=J), reps, 10)
        out[name] = row
        m.close()
    return out


def vjp_leg(grid, stream, dist, B=4096, H=64):
    """The differentiation workload: FD forward and the VJP through it for the
    12-DoF tree, B rollouts x H steps = 262,144 knot points in one batch, FP32."""
    import numpy as np
    import torch
    import grid_inputs as gi
    r = gi.tree12()
    m = grid.Model.from_robot(r)
    N = B * H
    q, qd, tau = (torch.from_numpy(x.astype(np.float32)).cuda() for x in gi.states(r.n, N, 404))
    g = torch.from_numpy(gi.upstream(r.n, N, 404).astype(np.float32)).cuda()
    qdd = torch.empty_like(q)
    outs = tuple(torch.empty_like(q) for _ in range(3))
    steps = 10
    sec_fd = time_steps(lambda: m.fd(q, qd, tau, out=qdd), steps, 3, stream, dist)
    sec_vjp = time_steps(lambda: m.fd_vjp(q, qd, tau, g, out=outs), steps, 3, stream, dist)
    m.close()
    return {"knot_points": N, "fd_knot_points_per_s": N * steps / sec_fd,
            "vjp_knot_points_per_s": N * steps / sec_vjp,
            "note": "12-DoF tree, 4096 rollouts x 64 steps in one batch, FP32: forward dynamics, and the "
                    "vector-Jacobian product (dL/dq, dL/dqd, dL/dtau) through it"}


def device_latency_us(fn, reps=200, warmup=20):
    """Median device time of one call: each call is queued behind a ~50 us
    device-side spin, so the CUDA events around it (on the launching stream)
    bracket the GPU's execution of the call and not the host's time to issue it."""
    import numpy as np
    import torch
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        fn()
    ts = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda._sleep(100_000)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1) * 1e3)
    return float(np.median(ts))


def latency_table(grid, reps=200, warmup=20):
    """Single-computation latency (one knot point, compute only, inputs resident)
    of each entry point for the three workload robots (device_latency_us)."""
    import numpy as np
    import torch
    import grid_inputs as gi
    table = {}
    for name, prec in (("chain7", "fp32"), ("tree12", "fp32"), ("tree30", "fp32"), ("tree30", "mixed")):
        r = gi.robot(name)
        m = grid.Model.from_robot(r, precision=prec)
        q, qd, tau = (torch.from_numpy(x.astype(np.float32)).cuda() for x in gi.states(r.n, 1, 77))
        outs = {"rnea": torch.empty((1, r.n), device="cuda"),
                "minv": torch.empty((1, r.n, r.n), device="cuda"),
                "fd": torch.empty((1, r.n), device="cuda"),
                "grad_id": torch.empty((1, r.n, 2 * r.n), device="cuda"),
                "grad_fd": torch.empty((1, r.n, 2 * r.n), device="cuda")}
        calls = {"rnea": lambda: m.rnea(q, qd, tau, out=outs["rnea"]),
                 "minv": lambda: m.minv(q, out=outs["minv"]),
                 "fd": lambda: m.fd(q, qd, tau, out=outs["fd"]),
                 "grad_id": lambda: m.grad_rnea(q, qd, tau, out=outs["grad_id"]),
                 "grad_fd": lambda: m.grad_fd(q, qd, tau, out=outs["grad_fd"])}
        table[name if prec == "fp32" else name + "_mixed"] = {alg: device_latency_us(fn, reps, warmup)
                                                               for alg, fn in calls.items()}
        m.close()
    return table


def cpu_oracle_rate(robot, seconds_min=10.0, seconds_max=30.0, threads=None):
    """The FP64 oracle as it stands on the host cores, on a bounded sample of the
    workload: repeated batches of 128-knot trajectories until >= seconds_min."""
    import oracle
    threads = threads or os.cpu_count() or 1
    n = robot.n
    q, qd, tau = gi.states(n, 64 * KNOTS, gi.workload_seed(2, KNOTS))
    oracle.grad_fd(robot, q[:KNOTS], qd[:KNOTS], tau[:KNOTS], nthreads=threads)   # warm
    done, t0 = 0, time.perf_counter()
    batch = 4 * KNOTS
    while True:
        s = (done // batch) % 16
        sl = slice(s * batch, (s + 1) * batch)
        oracle.grad_fd(robot, q[sl], qd[sl], tau[sl], nthreads=threads)
        done += batch
        el = time.perf_counter() - t0
        if el >= seconds_min or el >= seconds_max:
            break
    return done / el, threads, done, el


def serve_leg(grid, seconds, rate_hz=20000.0, seed=5005):
    """Serving workload: open-loop Poisson arrivals at rate_hz, robot uniform
    over the 7/12/30-DoF models, horizon uniform over {16, 32, 64, 128, 256};
    1 s warm-up, then `seconds` measured. Native producer/consumer threads."""
    names = ["chain7", "tree12", "tree30"]
    models = [grid.Model.from_robot(gi.robot(r)) for r in names]
    K = 1024
    pools = [np.stack(gi.states(m.n, K, gi.workload_seed(5, K) + i)).astype(np.float32)
             for i, m in enumerate(models)]
    horizons = [16, 32, 64, 128, 256]
    srv = grid.Server(models, ring_slots=2048, arena_bytes=1 << 30)
    srv.start()
    srv.bench(rate_hz, 1.0, seed, horizons, pools)
    st = srv.bench(rate_hz, seconds, seed + 1, horizons, pools)
    status = srv.stop()
    srv.close()
    return {"rate_hz": rate_hz, "seconds": seconds, "robots": names, "horizons": horizons,
            "completed": int(st["completed"]), "knot_points_per_s": st["knot_points"] / st["wall_s"],
            "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "p50_ms_h128": st["p50_ms_h128"],
            "p99_ms_h128": st["p99_ms_h128"], "max_ms": st["max_ms"], "refused": int(st["refused"]),
            "status": int(st["status"]), "kernel_status": int(status),
            "latency": "scheduled arrival to the host seeing the done flag"}


def run_reference(args):
    """Reference arm: the FP64 CPU oracle timed on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    robot = gi.chain7()
    threads = os.cpu_count() or 1
    per_step = 128 * KNOTS          # bounded sample: 128 trajectories x 128 knot points
    q, qd, tau = gi.states(7, per_step, gi.workload_seed(2, KNOTS))
    for _ in range(args.warmup):
        oracle.grad_fd(robot, q, qd, tau, nthreads=threads)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.grad_fd(robot, q, qd, tau, nthreads=threads)
    el = time.perf_counter() - t0
    v = per_step * args.steps / el
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded 7-DoF chain, uniform states)",
        "config": {"workload": "7-DoF chain, trajectories of 128 knot points, FP64 CPU oracle; "
                               "each step a 16,384-knot-point sample of the GPU step's batch",
                   "robot": "chain7", "knot_points_per_step": per_step},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"{per_step} knot points per step x {args.steps} steps"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    import paper_2109_06976_gb300 as grid
    from paper_2109_06976_gb300.flops import grad_fd_flops_per_knot

    rank, world, local, dist = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    robot = gi.chain7()
    model = grid.Model.from_robot(robot)
    model.set_option("specialize", args.specialize)
    n = robot.n
    Nk = args.traj * KNOTS
    seed = rank_seed(rank)
    q, qd, tau = (torch.from_numpy(x.astype(np.float32)).cuda()
                  for x in gi.states(n, Nk, seed))
    J = torch.empty((Nk, n, 2 * n), device="cuda")
    in_bytes = 3 * Nk * n * 4
    out_bytes = Nk * 2 * n * n * 4

    def step():
        model.grad_fd(q, qd, tau, out=J)

    if args.only_tree12:
        # the 12-DoF tree's step alone (half the main batch), for profiling captures
        t12 = gi.tree12()
        m12 = grid.Model.from_robot(t12)
        N12 = Nk // 2
        q12, qd12, tau12 = (torch.from_numpy(x.astype(np.float32)).cuda()
                            for x in gi.states(12, N12, seed + 1))
        J12 = torch.empty((N12, 12, 24), device="cuda")
        sec12 = time_steps(lambda: m12.grad_fd(q12, qd12, tau12, out=J12), args.steps, args.warmup, stream, dist)
        if rank == 0:
            print(json.dumps({"metric": "gradient of FD, 12-DoF tree", "value": world * N12 * args.steps / sec12,
                              "unit": UNIT, "ms_per_step": sec12 / args.steps * 1e3, "knot_points": N12}),
                  flush=True)
        if dist:
            dist.destroy_process_group()
        return

    with ClockSampler(local) as clk:
        sec = time_steps(step, args.steps, args.warmup, stream, dist)
    clocks = clk.summary()
    ms = sec / args.steps * 1e3
    value = aggregate_value(world, Nk, args.steps, sec)
    flops_knot = grad_fd_flops_per_knot(robot.parent)
    achieved_tflops = flops_knot * Nk / (ms / 1e3) / 1e12
    dram = NCU_DRAM_BYTES_PER_KNOT.get(kernel_source_hash())
    fma_pipe = NCU_FMA_PIPE.get(kernel_source_hash())
    if args.only_main:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": UNIT, "ms_per_step": ms,
                              "knot_points": Nk, "achieved_tflops": achieved_tflops,
                              "clocks": clocks}), flush=True)
        if dist:
            dist.destroy_process_group()
        return

    # End to end through the public API with pinned host buffers, every step:
    # grid_grad_fd_host copies the step's states in, runs the kernel and copies
    # the Jacobians out, in chunks whose copies overlap the kernel.
    hq, hqd, htau = (t.cpu().pin_memory() for t in (q, qd, tau))
    hJ = torch.empty(J.shape, dtype=J.dtype).pin_memory()

    def e2e_step():
        model.grad_fd_host(hq, hqd, htau, out=hJ, sync=False)

    # as many timed steps as the main leg: a transient host-side stall of 10-40 ms
    # (seen now and then in every copy path) then moves the mean by a bounded share
    e2e_steps = args.steps
    sec_e2e = time_steps(e2e_step, e2e_steps, 2, stream, dist)
    e2e_copy_value = aggregate_value(world, Nk, e2e_steps, sec_e2e)

    # For comparison: the same copies and kernel one after another on one stream.
    dq, dqd, dtau = torch.empty_like(q), torch.empty_like(qd), torch.empty_like(tau)

    def serial_step():
        dq.copy_(hq, non_blocking=True)
        dqd.copy_(hqd, non_blocking=True)
        dtau.copy_(htau, non_blocking=True)
        model.grad_fd(dq, dqd, dtau, out=J)
        hJ.copy_(J, non_blocking=True)

    sec_serial = time_steps(serial_step, e2e_steps, 2, stream, dist)
    e2e_serial_value = aggregate_value(world, Nk, e2e_steps, sec_serial)

    # Zero copy: the same call on the pinned host buffers; the kernel reads the
    # states from and writes the Jacobians to host memory over NVLink-C2C.
    def e2e_zc_step():
        model.grad_fd(hq, hqd, htau, out=hJ)

    sec_zc = time_steps(e2e_zc_step, e2e_steps, 2, stream, dist)
    e2e_zc_value = aggregate_value(world, Nk, e2e_steps, sec_zc)
    e2e_value = max(e2e_copy_value, e2e_zc_value)

    # The same step in the kernel that reads the topology at run time (the
    # chain-specialised kernel is kept only if it is the faster one).
    mgen = grid.Model.from_robot(robot)
    mgen.set_option("specialize", 1 - args.specialize)
    gen_steps = max(3, args.steps // 4)
    sec_gen = time_steps(lambda: mgen.grad_fd(q, qd, tau, out=J), gen_steps, 2, stream, dist)
    other_value = aggregate_value(world, Nk, gen_steps, sec_gen)
    mgen.close()

    # FP64 plain form on the same GPU (smaller batch, same per-knot work)
    Nd = 256 * KNOTS
    q64, qd64, tau64 = (x[:Nd].double() for x in (q, qd, tau))
    J64 = torch.empty((Nd, n, 2 * n), device="cuda", dtype=torch.float64)
    sec64 = time_steps(lambda: model.grad_fd(q64, qd64, tau64, out=J64), 5, 2, stream, dist)
    fp64_value = world * Nd * 5 / sec64

    # 12-DoF tree at the same N and batch
    t12 = gi.tree12()
    m12 = grid.Model.from_robot(t12)
    q12, qd12, tau12 = (torch.from_numpy(x.astype(np.float32)).cuda()
                        for x in gi.states(12, Nk // 2, seed + 1))
    J12 = torch.empty((Nk // 2, 12, 24), device="cuda")
    sec12 = time_steps(lambda: m12.grad_fd(q12, qd12, tau12, out=J12), max(3, args.steps // 4), 2,
                       stream, dist)
    t12_value = world * (Nk // 2) * max(3, args.steps // 4) / sec12

    # single-trajectory latency at N = 128 (compute only)
    q1, qd1, tau1 = q[:KNOTS], qd[:KNOTS], tau[:KNOTS]
    J1 = J[:KNOTS]
    lat128 = device_latency_us(lambda: model.grad_fd(q1, qd1, tau1, out=J1))
    # the same with the paper's I/O: pinned host -> device, kernel, device -> pinned host
    h1 = [t.cpu().pin_memory() for t in (q1, qd1, tau1)]
    hJ1 = torch.empty(J1.shape, dtype=J1.dtype).pin_memory()
    d1 = [torch.empty_like(t) for t in (q1, qd1, tau1)]

    def io_call():
        for dd, hh in zip(d1, h1):
            dd.copy_(hh, non_blocking=True)
        model.grad_fd(*d1, out=J1)
        hJ1.copy_(J1, non_blocking=True)

    lat128_io = device_latency_us(io_call)

    lat_table = latency_table(grid) if rank == 0 else None
    sweep = n_sweep(grid) if rank == 0 else None
    vjp = vjp_leg(grid, stream, dist) if rank == 0 and world == 1 else None
    traj = traj_leg(grid, model, stream, dist) if rank == 0 and world == 1 else None

    serve = None
    if rank == 0 and world == 1 and args.serve_seconds > 0:
        serve = serve_leg(grid, args.serve_seconds)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        rate, threads, done, el = cpu_oracle_rate(robot)
        rate1, _, done1, el1 = cpu_oracle_rate(robot, seconds_min=3.0, seconds_max=10.0, threads=1)
        cpu = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"{done} knot points of 128-knot trajectories in {el:.1f} s",
               "single_thread": {"value": rate1, "unit": UNIT, "cores": 1,
                                 "sample": f"{done1} knot points in {el1:.1f} s"}}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded 7-DoF chain, q~U[-pi,pi], qd~U[-1,1], tau~U[-5,5])",
            "config": {
                "workload": f"7-DoF chain, {args.traj} trajectories x {KNOTS} knot points per step "
                            f"({Nk} knot points), FP32, grad FD",
                "robot": "chain7", "trajectories_per_gpu": args.traj, "knot_points_per_trajectory": KNOTS,
                "l2": f"inputs {in_bytes / 1e6:.0f} MB and outputs {out_bytes / 1e6:.0f} MB per "
                      f"step, both larger than the 129 MB L2",
                "parallelism": f"dp{world}"},
            "roofline": {"bound": "alu", "achieved": achieved_tflops, "peak": FP32_PEAK_TFLOPS,
                         "unit": "TFLOP/s", "frac": achieved_tflops / FP32_PEAK_TFLOPS,
                         "traffic": None if dram is None else dram * Nk,
                         "flops_per_knot": flops_knot,
                         "fp32_pipe_util_ncu": fma_pipe,
                         "peak_note": "FP32 from 152 SMs x 128 lanes x 2 x 2070 MHz",
                         "hbm_gbs": (in_bytes + out_bytes) / (ms / 1e3) / 1e9},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": in_bytes,
                    "d2h_bytes_per_step": out_bytes,
                    "zero_copy": e2e_zc_value, "copies": e2e_copy_value,
                    "serial_copies": e2e_serial_value,
                    "note": "pinned host buffers every step; value = the faster of zero copy "
                            "(the kernel reads/writes host memory) and grid_grad_fd_host (H2D, "
                            "kernel and D2H in chunks, overlapped on three streams); "
                            "serial_copies = H2D, kernel, D2H one after another, for comparison"},
            "topology": {"kernel": "chain-specialised" if args.specialize else "run-time topology",
                         "other_kernel_value": other_value, "unit": UNIT,
                         "note": "the same step in the other kernel (run-time topology vs the chain "
                                 "compiled for its length)"},
            "fp64_plain": {"value": fp64_value, "unit": UNIT, "knot_points_per_launch": Nd},
            "tree12": {"value": t12_value, "unit": UNIT, "knot_points_per_launch": Nk // 2},
            "latency_n128_us": lat128,
            "latency_n128_with_io_us": lat128_io,
            "latency_n_sweep_us": sweep,
            "latency_n1_us": lat_table,
            "latency_n1_note": "one knot point per call, compute only: median over 200 calls of the "
                               "device time between CUDA events, each call queued behind a device spin "
                               "(RNEA at qdd = tau's values; FP32, and the 30-DoF tree also in mixed precision)",
            "traj_step": traj,
            "vjp": vjp,
            "serve": serve,
            "cpu_baseline": cpu,
            "clocks": clocks,
            "gpu_launches": args.steps,
            "gpu_launches_note": "timed region of `value`: one grid_grad_fd kernel per step",
            "kernel_source": kernel_source_hash(),
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    model.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline leg")
    ap.add_argument("--traj", type=int, default=TRAJ, help="trajectories of 128 knot points per step")
    ap.add_argument("--serve-seconds", type=float, default=10.0,
                    help="measured seconds of the serving leg (0 to skip)")
    ap.add_argument("--specialize", type=int, default=1, choices=[0, 1],
                    help="1: chain-specialised kernel for the 7-DoF chain; 0: run-time topology kernel")
    ap.add_argument("--only-main", action="store_true",
                    help="time only the main FP32 step (used for profiling captures)")
    ap.add_argument("--only-tree12", action="store_true",
                    help="time only the 12-DoF tree's step (used for profiling captures)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
