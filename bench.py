#!/usr/bin/env python3
"""Benchmark: environments per second for phi + dphi/dA through the recursive contraction graph.

Default workload: K = 810 one-particle functions (n <= 10, l <= 8), nu <= 6,
total degree <= 24 (deg = n + 2l), 213,525 basis functions, 16,384 environments,
FP32 forward + adjoint in one fused kernel per step (the largest configuration,
on which the roofline target is stated).  Inputs are synthetic (seeded draws,
see workloads/), resident in HBM; successive steps rotate over buffer sets
larger than L2.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]

N > 1 runs under torchrun, one rank per GPU; every rank processes its own full
batch (independent environments, no collective on the data path: weak scaling);
the timed region is bracketed by a barrier and a device synchronisation and the
maximum time over ranks is reported.  ``--impl reference`` times the FP64 CPU
oracle (the only reference this method has) on the host cores.
"""
from __future__ import annotations

import os

for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")   # the CPU oracle legs run single-threaded; "cores" reports 1

import argparse
import json
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

# kernel forms by their ACE_KERNEL value, named as the autotuner names them
_FORCED_NAMES = {"lon": "tile_per_lane", "loe": "env_per_lane", "loeg": "env_per_lane_global",
                 "loeg2": "env_pair_per_lane_global", "loem": "env_per_lane_multi"}

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
import workloads as W  # noqa: E402

METRIC = "env/s, phi+dphi/dA: batched FP32 vs plain FP64 (GB300, rel err<=1e-5); % roofline"
TOL32 = 1e-5


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="stress_k810", choices=sorted(W.WORKLOADS))
    ap.add_argument("--readout", default="compensated", choices=["plain", "compensated", "fp64"])
    ap.add_argument("--algo", type=int, default=1, choices=[1, 2],
                    help="graph insertion heuristic: Algorithm 1 or Algorithm 2 (section 3.3)")
    ap.add_argument("--n-split", type=int, default=2, help="parameter n of Algorithm 2")
    ap.add_argument("--no-baselines", action="store_true", help="skip the plain-FP64 GPU and CPU oracle legs")
    ap.add_argument("--n-env", type=int, default=None, help="override the environment count (small profiling cases)")
    ap.add_argument("--no-graph", action="store_true", help="launch every step directly instead of replaying "
                    "a captured CUDA graph")
    return ap.parse_args()


# ---- algorithmic work (FMA-pipe operations per environment) ---------------------------------

def algorithmic_ops(w, n_nodes_ge2: int, n_basis: int, mode: str) -> float:
    """Forward: one product per node of order >= 2 plus one readout FMA per basis function and
    channel; adjoint: two FMAs per node of order >= 2 plus the seed per basis function."""
    fwd = n_nodes_ge2 + n_basis * w.n_out
    adj = 2 * n_nodes_ge2 + n_basis * w.n_out
    return float(fwd + (adj if mode != "forward" else 0))


# ---- traffic recorded from an ncu capture ---------------------------------------------------

def recorded_traffic(workload: str):
    """DRAM bytes per launch of the workload's dominant kernel from profiles/traffic.json, or None
    when no capture exists or the kernel or plan sources changed since it was taken."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path))[workload]
    except (OSError, KeyError, ValueError):
        return None
    h = hashlib.sha256()
    for f in rec["sources"]:
        try:
            h.update(open(os.path.join(ROOT, f), "rb").read())
        except OSError:
            return None
    if h.hexdigest() != rec["sources_sha256"]:
        return None
    return rec["dram_bytes_read"] + rec["dram_bytes_write"]


# ---- ranks ----------------------------------------------------------------------------------

def max_over_ranks(x: float, dist=None, device=None) -> float:
    """Largest value over all ranks (the timed region's duration is the slowest rank's)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def min_over_ranks(x: float, dist=None, device=None) -> float:
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MIN)
    return float(t.item())


def weak_scaling_value(n_env_per_rank: int, steps: int, max_ms: float, world: int) -> float:
    """Whole-job throughput: every rank processes its own batch of n_env_per_rank environments per step."""
    return world * n_env_per_rank * steps / (max_ms / 1e3)


# ---- clocks ---------------------------------------------------------------------------------

class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons while the timed region runs."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                self.rows.append(parts)

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=5)

    def summary(self):
        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[0]) for r in self.rows if num(r[0]) is not None]
        mx = [num(r[1]) for r in self.rows if num(r[1]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[4 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


# ---- the CPU oracle legs ------------------------------------------------------------------------

def oracle_setup(w):
    from oracle.basis import workload_index_set
    t0 = time.time()
    o = workload_index_set(w)
    return o, time.time() - t0


# the recursive-graph oracle leg runs in worker processes (spawned, so no CUDA state is inherited)
_REC = {}


def _rec_init(K, n_nodes, left, right, basis_node):
    from types import SimpleNamespace
    _REC["dag"] = SimpleNamespace(K=K, n_nodes=n_nodes, left=left, right=right, basis_node=basis_node)


def _rec_work(A, c):
    from oracle.evaluate import dag_forward, dag_reverse
    d = _REC["dag"]
    AA, _ = dag_forward(d, A, c)
    dag_reverse(d, AA, c)
    return A.shape[0]


def cpu_baseline_recursive(w, o, budget_s=20.0, chunk=128):
    """The oracle's FP64 recursive graph evaluation and reverse sweep (Eq. 4 and its adjoint), one
    process per host core, on chunks of environments of the workload."""
    import multiprocessing as mp
    from oracle.dag import build_dag
    d = build_dag(o)
    cores = os.cpu_count() or 1
    c = W.round_to(W.draw_c(o.deg, w.n_out), w.dtype)
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores, initializer=_rec_init,
                  initargs=(d.K, d.n_nodes, d.left, d.right, d.basis_node)) as pool:
        A = W.round_to(W.draw_A(chunk, o.basis.K, env_scale=w.env_scale), w.dtype)
        t0 = time.perf_counter()
        pool.starmap(_rec_work, [(A, c)] * cores)            # warm-up: one chunk per worker
        per_round = time.perf_counter() - t0
        rounds = int(max(1, min(8, budget_s / max(per_round, 1e-3))))
        t0 = time.perf_counter()
        n = sum(pool.starmap(_rec_work, [(A, c)] * (cores * rounds)))
        dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": "env/s", "cores": cores, "kind": "oracle",
            "sample": f"{n} environments of {w.name} in chunks of {chunk} (recursive FP64 graph "
                      f"evaluation + reverse sweep, numpy, {cores} processes)"}


def oracle_step(o, A, c):
    from oracle.evaluate import grad_naive, phi_naive
    phi = phi_naive(A, o, c)
    dA = grad_naive(A, o, c)
    return phi, dA


def cpu_baseline(w, o, budget_s=15.0, max_envs=256):
    """Time the oracle (naive term-by-term phi + product-rule gradient) on a bounded env sample."""
    c = W.round_to(W.draw_c(o.deg, w.n_out), w.dtype)
    n = 2
    A = W.round_to(W.draw_A(n, o.basis.K, env_scale=w.env_scale), w.dtype)
    t0 = time.perf_counter()
    oracle_step(o, A, c)
    per_env = (time.perf_counter() - t0) / n
    n = int(max(2, min(max_envs, budget_s / max(per_env, 1e-6))))
    A = W.round_to(W.draw_A(n, o.basis.K, env_scale=w.env_scale), w.dtype)
    t0 = time.perf_counter()
    oracle_step(o, A, c)
    dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": "env/s", "cores": 1, "host_cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{n} environments of {w.name} (naive FP64 phi + product-rule dphi/dA, numpy, 1 thread)"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = W.WORKLOADS[args.workload]
    o, _ = oracle_setup(w)
    c = W.round_to(W.draw_c(o.deg, w.n_out), w.dtype)
    A1 = W.round_to(W.draw_A(2, o.basis.K, env_scale=w.env_scale), w.dtype)
    t0 = time.perf_counter()
    oracle_step(o, A1, c)
    per_env = (time.perf_counter() - t0) / 2
    budget = 120.0 / max(1, args.steps + args.warmup)           # whole run within about two minutes
    n = int(max(1, min(256, budget / max(per_env, 1e-6))))
    A = W.round_to(W.draw_A(n, o.basis.K, env_scale=w.env_scale), w.dtype)
    for _ in range(args.warmup):
        oracle_step(o, A, c)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_step(o, A, c)
    dt = time.perf_counter() - t0
    value = n * args.steps / dt
    line = {"metric": METRIC, "value": value, "unit": "env/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": w.name, "n_env_per_step": n, "n_env_full": w.n_env,
                       "description": w.description},
            "cpu_baseline": {"value": value, "unit": "env/s", "cores": 1, "host_cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"{n} environments per step of {w.name} (naive FP64 oracle, 1 thread)"},
            "e2e": {"value": value, "unit": "env/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---- our path ------------------------------------------------------------------------------------

class Step:
    """One step of the workload on device-resident inputs (all compute in libace)."""

    def __init__(self, w, dag, torch, dev, n_sets, readout):
        self.w, self.dag, self.torch, self.readout = w, dag, torch, readout
        t = torch
        self.c = t.tensor(W.round_to(W.draw_c(dag.spec.deg, w.n_out), "f32"), dtype=t.float32, device=dev)
        self.sets = []
        self.mu = None
        if w.pooling:
            offsets, P = W.draw_neighbours(w.n_env, rc=w.rc, j_range=w.j_range)
            self.offsets = t.tensor(offsets, device=dev)
            self.n_pairs = P.shape[0]
            if w.n_species:
                self.mu = t.tensor(W.round_to(W.draw_species(P.shape[0], w.n_species), "f32"), dtype=t.float32,
                                   device=dev)
            for i in range(n_sets):
                Pi = P if i == 0 else P[np.random.default_rng(100 + i).permutation(P.shape[0])]
                self.sets.append(t.tensor(W.round_to(Pi, "f32"), dtype=t.float32, device=dev))
            self.in_bytes = P.shape[0] * (16 if w.n_species else 12) + (w.n_env + 1) * 8
            self.out_bytes = w.n_env * 4 + P.shape[0] * 12
        else:
            A = W.round_to(W.draw_A(w.n_env, dag.K, env_scale=w.env_scale), "f32")
            for i in range(n_sets):
                Ai = A if i == 0 else A[np.random.default_rng(100 + i).permutation(A.shape[0])]
                self.sets.append(t.tensor(Ai, dtype=t.float32, device=dev))
            self.in_bytes = w.n_env * dag.K * 4
            self.out_bytes = w.n_env * w.n_out * 4 + (w.n_env * dag.K * 4 if w.grad else 0)
        self.A0 = self.sets[0]

    def __call__(self, i):
        from paper_2202_04140_gb300.torch_api import energy_and_forces
        x = self.sets[i % len(self.sets)]
        w = self.w
        if w.pooling:
            return energy_and_forces(self.dag, x, self.offsets, self.c, w.nmin, w.nmax, w.lmax, w.rc, self.readout,
                                     mu=self.mu, kmax=w.kmax)
        if w.grad:
            return self.dag.evaluate_grad(x, self.c, None, self.readout)
        return self.dag.evaluate(x, self.c, self.readout), None

    def forces_form(self):
        """'fused' (one kernel per tile) or 'three kernels': the form ace_energy_forces takes here."""
        from paper_2202_04140_gb300 import ace as L
        w = self.w
        fused, _ = L.ace_energy_forces_plan(self.dag.handle, w.nmin, w.nmax, w.lmax, w.kmax)
        return "fused" if fused else "three kernels"

    def launches_per_step(self):
        if not self.w.pooling:
            return 1
        return 1 if self.forces_form() == "fused" else 3

    def capture(self):
        """One CUDA graph per buffer set (the step's launches, outputs in the graph's pool)."""
        t = self.torch
        side = t.cuda.Stream()
        side.wait_stream(t.cuda.current_stream())
        with t.cuda.stream(side):
            for i in range(len(self.sets)):
                self(i)
        t.cuda.current_stream().wait_stream(side)
        self.graphs, self.outs = [], []
        for i in range(len(self.sets)):
            g = t.cuda.CUDAGraph()
            with t.cuda.graph(g):
                out = self(i)
            self.graphs.append(g)
            self.outs.append(out)

    def run(self, i):
        graphs = getattr(self, "graphs", None)
        if graphs:
            graphs[i % len(graphs)].replay()
            return self.outs[i % len(graphs)]
        return self(i)


def capture_or_direct(torch, fn, graph: bool):
    """fn itself, or the replay of a CUDA graph captured from it (after two warm-up calls)."""
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        fn()
        fn()
    torch.cuda.current_stream().wait_stream(side)
    if not graph:
        return fn
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        fn()
    return g.replay


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    from paper_2202_04140_gb300 import ace as L
    from paper_2202_04140_gb300.torch_api import Dag, Spec

    w = W.workload(args.workload, **({"n_env": args.n_env} if args.n_env else {}))
    spec = Spec.from_workload(w)
    dag = Dag(spec, algo=args.algo, n_split=args.n_split)
    # kernel form and environments per CTA chosen by the autotuner for exactly this request
    tuned = dag.autotune(w.n_env, w.n_out, torch.float32, w.grad, args.readout)
    tuned["by"] = "autotuner"
    forced = {k: os.environ[k] for k in ("ACE_KERNEL", "ACE_TILE_E") if os.environ.get(k)}
    if forced:
        # an environment override makes every launch take the forced form, whatever the tuner kept
        tuned = {"kernel": _FORCED_NAMES.get(forced.get("ACE_KERNEL", "lon"), forced.get("ACE_KERNEL")),
                 "E": int(forced.get("ACE_TILE_E", 0)), "by": " ".join(f"{k}={v}" for k, v in forced.items())}
    n_ge2 = dag.n_nodes - dag.K
    mode = "forward" if not w.grad else "forward+adjoint"
    ops_env = algorithmic_ops(w, n_ge2, dag.n_basis, mode)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    l2 = 129e6
    step = Step(w, dag, torch, dev, 1, args.readout)
    per_set = step.in_bytes + step.out_bytes
    n_sets = max(1, int(np.ceil(2.5 * l2 / per_set)))
    step = Step(w, dag, torch, dev, n_sets, args.readout)
    if not args.no_graph:
        step.capture()

    for i in range(args.warmup):
        step.run(i)
    barrier()
    st = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        time.sleep(0.3)
        barrier()
        ev0.record(st)
        for i in range(args.steps):
            step.run(i)
        ev1.record(st)
        barrier()
    ms = max_over_ranks(ev0.elapsed_time(ev1), dist, dev)
    ms_step = ms / args.steps
    value = weak_scaling_value(w.n_env, args.steps, ms, world)

    # dominant kernel: the fused forward+adjoint kernel, timed alone on the same stream
    if w.pooling:
        A_dev = None
    kernel_ms = None
    if not w.pooling:
        barrier()
        ev0.record(st)
        for i in range(args.steps):
            step.run(i)
        ev1.record(st)
        barrier()
        kernel_ms = ev0.elapsed_time(ev1) / args.steps
    else:
        from paper_2202_04140_gb300.torch_api import pool_A
        A_dev = pool_A(step.A0, step.offsets, w.nmin, w.nmax, w.lmax, w.rc, step.mu, w.kmax)
        barrier()
        ev0.record(st)
        for i in range(args.steps):
            dag.evaluate_grad(A_dev, step.c, None, args.readout)
        ev1.record(st)
        barrier()
        kernel_ms = ev0.elapsed_time(ev1) / args.steps

    sms, smem, ccmaj, ccmin = L.ace_device_info()
    peak_clock_mhz = 2070.0                             # the part's maximum SM clock
    peak_flops = sms * 128 * 2 * peak_clock_mhz * 1e6   # FP32 lanes x FLOP per FMA x max SM clock
    achieved = 2.0 * ops_env * w.n_env / (kernel_ms / 1e3)
    probe_ms, probe_fma = L.ace_fma_peak(200000)
    probe_tflops = 2.0 * probe_fma / (probe_ms / 1e3) / 1e12

    # end to end through the public API with host buffers (pinned), copies inside the timed region
    e2e = None
    if not w.pooling:
        A_host = step.A0.cpu().pin_memory()
        dA_host = torch.empty_like(A_host).pin_memory() if w.grad else None
        phi_host = torch.empty((w.n_env, w.n_out), dtype=torch.float32).pin_memory()
        n_e2e = max(3, min(args.steps, 50))

        def e2e_step():
            # ace_eval(_grad)_host: chunked, copies in and out overlapped with the evaluation
            if w.grad:
                dag.evaluate_grad_host(A_host, step.c, None, args.readout, phi=phi_host, dA=dA_host, sync=False)
            else:
                dag.evaluate_host(A_host, step.c, args.readout, phi=phi_host, sync=False)

        run_e2e = capture_or_direct(torch, e2e_step, not args.no_graph)
        barrier()
        ev0.record(st)
        for _ in range(n_e2e):
            run_e2e()
        ev1.record(st)
        barrier()
        e_ms = ev0.elapsed_time(ev1)
        e2e = {"value": w.n_env * n_e2e / (e_ms / 1e3), "unit": "env/s", "h2d_bytes_per_step": step.in_bytes,
               "d2h_bytes_per_step": step.out_bytes, "steps": n_e2e,
               "api": "ace_eval_grad_host" if w.grad else "ace_eval_host"}
    else:
        from paper_2202_04140_gb300.torch_api import energy_and_forces_host
        P_host = step.A0.cpu().pin_memory()
        off_host = step.offsets.cpu().pin_memory()
        mu_host = step.mu.cpu().pin_memory() if step.mu is not None else None
        F_host = torch.empty_like(P_host).pin_memory()
        phi_host = torch.empty((w.n_env,), dtype=torch.float32).pin_memory()
        n_e2e = max(3, min(args.steps, 50))

        def e2e_step():
            # ace_energy_forces_host: chunked, copies in and out overlapped with the three kernels
            energy_and_forces_host(dag, P_host, off_host, step.c, w.nmin, w.nmax, w.lmax, w.rc, args.readout,
                                   mu=mu_host, kmax=w.kmax, phi=phi_host, forces=F_host, sync=False)

        run_e2e = capture_or_direct(torch, e2e_step, not args.no_graph)
        barrier()
        ev0.record(st)
        for _ in range(n_e2e):
            run_e2e()
        ev1.record(st)
        barrier()
        e_ms = ev0.elapsed_time(ev1)
        e2e = {"value": w.n_env * n_e2e / (e_ms / 1e3), "unit": "env/s", "h2d_bytes_per_step": step.in_bytes,
               "d2h_bytes_per_step": step.out_bytes, "steps": n_e2e,
               "api": "ace_energy_forces_host"}
    e2e["value"] = min_over_ranks(e2e["value"], dist, dev) * world

    extra = {}
    if rank == 0 and not args.no_baselines and not w.pooling:
        # outputs of the launch path that was timed (graph replay by default), taken before the FP64 legs
        # below bind FP64 coefficients to the same graph handle: a replay after that reads other values
        phi_t, dA_t = step.run(0)
        torch.cuda.synchronize()
        phi_t = phi_t.double().cpu().numpy()
        dA_t = dA_t.double().cpu().numpy() if dA_t is not None else None
        # plain FP64 GPU graph walk on the same environments (the comparison the method is measured against)
        A64 = step.A0.double()
        c64 = step.c.double()
        need = L.ace_eval_plain_workspace_bytes(dag.handle, w.n_env, w.grad)
        free = torch.cuda.mem_get_info(dev)[0]
        n_plain = w.n_env if need < 0.6 * free else max(1, int(w.n_env * 0.6 * free / need))
        ws = torch.empty(L.ace_eval_plain_workspace_bytes(dag.handle, n_plain, w.grad), dtype=torch.uint8,
                         device=dev)
        dag.evaluate_plain_f64(A64[:n_plain], c64, grad=w.grad, workspace=ws)
        torch.cuda.synchronize()
        reps = 3
        ev0.record(st)
        for _ in range(reps):
            dag.evaluate_plain_f64(A64[:n_plain], c64, grad=w.grad, workspace=ws)
        ev1.record(st)
        torch.cuda.synchronize()
        p_ms = ev0.elapsed_time(ev1) / reps
        del ws
        extra["plain_fp64_gpu"] = {"value": n_plain / (p_ms / 1e3), "unit": "env/s", "ms_per_call": p_ms,
                                   "n_env": n_plain}
        # the fused kernel itself in FP64 on the same environments (same graph, same plan)
        fused64 = None
        try:
            dag.evaluate_grad(A64, c64) if w.grad else dag.evaluate(A64, c64)
            torch.cuda.synchronize()
            ev0.record(st)
            for _ in range(reps):
                out64 = dag.evaluate_grad(A64, c64) if w.grad else (dag.evaluate(A64, c64), None)
            ev1.record(st)
            torch.cuda.synchronize()
            f_ms = ev0.elapsed_time(ev1) / reps
            fused64 = {"value": w.n_env / (f_ms / 1e3), "unit": "env/s", "ms_per_call": f_ms, "n_env": w.n_env}
        except Exception as exc:   # a graph whose FP64 tile does not fit reports why
            out64 = None
            fused64 = {"value": None, "why": str(exc)[:200]}
        extra["fused_fp64_gpu"] = fused64
        # accuracy of this run's configuration on 64 sampled environments, against the oracle:
        # the first and last tiles, then a seeded random sample
        o, t_setup = oracle_setup(w)
        rng = np.random.default_rng(7)
        idx = np.unique(np.concatenate([np.arange(4), w.n_env - 4 + np.arange(4),
                                        rng.choice(w.n_env, 64, replace=False)]))[:64]
        A_s = step.A0[idx].double().cpu().numpy()
        c_s = step.c.double().cpu().numpy()
        from oracle.evaluate import error_scale, grad_error_scale
        ref_phi, ref_dA = oracle_step(o, A_s, c_s)

        def gated(x, r, sc):            # |x - ref| / (the oracle with |c|, |A|): the gated measure
            d = np.abs(x - r)
            e = np.where(sc > 0, d / np.where(sc > 0, sc, 1), d)
            return {"max": float(np.max(e)), "p99": float(np.percentile(e, 99))}

        def plain(x, r):                # |x - ref| / |ref|: ill-conditioned under cancellation, not gated
            e = np.abs(x - r) / np.maximum(np.abs(r), 1e-300)
            return {"max": float(np.max(e)), "p99": float(np.percentile(e, 99))}

        s_phi = error_scale(A_s, o, c_s)
        phi_s = phi_t[idx]
        err = {"sample": int(len(idx)), "gate": TOL32,
               "phi": gated(phi_s, ref_phi, s_phi), "phi_plain_rel": plain(phi_s, ref_phi)}
        if dA_t is not None:
            s_dA = grad_error_scale(A_s, o, c_s)
            dA_s = dA_t[idx]
            err["dphi_dA"] = gated(dA_s, ref_dA, s_dA)
            err["dphi_dA_plain_rel"] = plain(dA_s, ref_dA)
        if out64 is not None:
            err["fused_fp64"] = {"phi": gated(out64[0].cpu().numpy()[idx], ref_phi, s_phi)["max"], "gate": 1e-12}
            if out64[1] is not None:
                err["fused_fp64"]["dphi_dA"] = gated(out64[1].cpu().numpy()[idx], ref_dA, s_dA)["max"]
        extra["error_vs_oracle"] = err
        extra["cpu_baseline"] = cpu_baseline(w, o)
        extra["cpu_baseline_recursive"] = cpu_baseline_recursive(w, o)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "env/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name, "description": w.description, "n_env_per_gpu": w.n_env,
                       "K": dag.K, "nu_max": w.nu_max, "deg_max": w.deg_max, "n_basis": dag.n_basis,
                       "n_nodes": dag.n_nodes, "n_aux": dag.n_aux, "n_operands": dag.n_operands,
                       "n_sinks": dag.n_sinks, "mode": mode, "readout": args.readout,
                       "graph": {"algorithm": args.algo, **({"n": args.n_split} if args.algo == 2 else {})},
                       "kernel_config": {"kernel": tuned["kernel"], "E": tuned["E"], "by": tuned["by"],
                                         **({"forces_form": step.forces_form()} if w.pooling else {})},
                       "launch": "direct" if args.no_graph else "CUDA graph replay (one graph per buffer set)",
                       "l2": f"inputs larger than L2: {n_sets} rotating buffer sets of {per_set / 1e6:.0f} MB"},
            "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_flops / 1e12, "unit": "TFLOP/s",
                         "frac": achieved / peak_flops,
                         "traffic": recorded_traffic(w.name) if w.n_env == W.WORKLOADS[w.name].n_env else None,
                         "kernel": "fused forward+adjoint (ace_eval_grad), one launch per step",
                         "kernel_ms": kernel_ms, "ops_per_env": ops_env,
                         "peak_basis": {"sm_count": sms, "fp32_lanes_per_sm": 128, "flop_per_fma": 2,
                                        "sm_clock_mhz": peak_clock_mhz, "source": "nominal (no FP32 figure is "
                                        "measured by the pool); the in-bench FMA probe is reported beside it"},
                         "fma_probe_tflops": probe_tflops, "frac_of_probe": achieved / (probe_tflops * 1e12)},
            "clocks": clk.summary(),
            "e2e": e2e,
            "gpu_launches": step.launches_per_step() * args.steps,
        }
        line.update({k: v for k, v in extra.items()})
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
