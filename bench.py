"""Benchmark of the QPINN hot path: one step = qp_loss_grad on the full-QPINN workload
(8 qubits, 6 strongly entangling layers, RFF(64) + tanh MLP(32), dielectric disk, energy
term) over a 64x64x16 collocation grid (65,536 points) plus a 64x64 initial-condition plane:
forward, exact d/dx, d/dy, d/dt by tangent states, Maxwell/IC/energy losses and the adjoint
gradient of every parameter.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line. `value` is collocation points per second over all ranks (device
time, CUDA events around each step, L2 flushed between steps). `e2e` is the same metric
through the public call with every step's inputs copied from pinned host memory and its loss
and gradient copied back inside the timed region (two device buffer sets, the copies on their
own streams beside the neighbouring steps' compute; the L2 flushes are inside it too). The reference arm times the FP64 CPU oracle
(deliberately slow, plain definition) on a bounded sample of the same workload.
"""
import argparse
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

METRIC = "collocation pts/s, fwd+d/dx,dy,dt+adjoint grad, 8q x6L"
UNIT = "colloc pts/s"
WORKLOAD = "full QPINN step: 8q/6L strongly entangling, RFF64+MLP32, dielectric, energy term"


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-graph", action="store_true",
                    help="launch the step's kernels one by one instead of replaying them as one CUDA graph")
    ap.add_argument("--path", default="auto", choices=["auto", "simt", "gemm_split"],
                    help="statevector path of the library (auto = the library's choice; with "
                         "--workload configs: every path the configuration has)")
    ap.add_argument("--operands", default=None, choices=["fp16_pairs", "tf32_pairs"],
                    help="--workload configs: only this tensor-core operand form")
    ap.add_argument("--config", default=None, choices=["C1", "C2", "C3", "C4"],
                    help="--workload configs: only this configuration")
    ap.add_argument("--grid", type=int, default=64,
                    help="--workload configs: C4 grid points per axis (64: the 64^3 grid)")
    ap.add_argument("--c3-grid", type=int, default=64,
                    help="default workload: x and y points of the collocation grid (64: the benchmark "
                         "step; smaller only for profiling captures)")
    ap.add_argument("--paper-grid", type=int, default=0,
                    help="--workload paper_net: only this grid (points per axis; 0: the 40^3 and 87^3 "
                         "grids of the paper's timing table)")
    ap.add_argument("--timeline", action="store_true",
                    help="diagnosis only, no bench line: the kernels of one graph-replayed step of the "
                         "benchmark workload with their start, duration and stream (CUPTI through "
                         "torch.profiler), one line each")
    ap.add_argument("--workload", default="c3", choices=["c3", "c5", "configs", "paper_net"],
                    help="c3: the full QPINN step (default); c5: 32 uneven instances in one "
                         "batched call against the same instances called one by one; configs: "
                         "one line per configuration (C1-C4) and compute path; paper_net: the "
                         "paper's hybrid network (7 qubits, 4 layers, RFF 128 + three tanh "
                         "layers of 128) on the 40^3 and 87^3 grids of its timing table")
    return ap.parse_args()


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def _config(world):
    return {"workload": WORKLOAD, "n_qubits": 8, "n_layers": 6, "ansatz": "strongly entangling",
            "premap": "RFF 64 freq + tanh MLP width 32", "medium": "dielectric",
            "colloc_per_gpu": 65536, "ic_per_gpu": 4096, "global_batch": 65536 * world,
            "parallelism": "dp%d" % world if world > 1 else "single",
            "l2": "flushed between timed steps (256 MiB write)"}


# ----------------------------------------------------------------------------- oracle arm

def _oracle_sample(steps_budget_s=10.0, nthreads=None):
    """Time the FP64 oracle on a bounded sample of the same workload: k collocation points of
    the grid and one initial-condition point per 16 of them (the step's ratio), with the energy
    term and slices on, loss + the gradient of every parameter. Returns (collocation points per
    second, threads, sample description)."""
    from oracle import api as oracle
    from paper_2506_23246_b300 import workloads as W
    circ, prob, params, sets = W.c3_workload(0)
    nt = nthreads or os.cpu_count() or 1
    pts, ic = sets["colloc"], sets["ic"]
    stride_c = pts.shape[0] // 64
    stride_i = ic.shape[0] // 4
    done = 0
    nic = 0
    t0 = time.perf_counter()
    while True:
        sub = {"colloc": pts[done * stride_c:done * stride_c + 1]}
        if done % 16 == 0:
            sub["ic"] = ic[(nic % 4) * stride_i:(nic % 4) * stride_i + 1]
            nic += 1
        oracle.loss(circ, prob, params, sub, nthreads=nt)
        oracle.grad(circ, prob, params, sub, nthreads=nt)
        done += 1
        el = time.perf_counter() - t0
        if el > steps_budget_s or done >= 64:
            break
    return done / el, nt, "%d collocation points spread over the 64x64x16 grid and %d initial-" \
        "condition points (the step's 16:1 ratio), energy term on: loss + all %d parameter " \
        "gradients, %d threads" % (done, nic, params.shape[0], nt)


def run_reference(a):
    rank, world, _ = _dist()
    if rank != 0:
        return 0
    from oracle import build as obuild
    obuild.build()
    per_step = max(2.0, 60.0 / max(a.steps + a.warmup, 1))
    for _ in range(a.warmup):
        _oracle_sample(per_step * 0.2)
    vals = []
    t0 = time.perf_counter()
    desc = ""
    nt = 1
    for _ in range(a.steps):
        v, nt, desc = _oracle_sample(per_step)
        vals.append(v)
    wall = time.perf_counter() - t0
    value = statistics.mean(vals)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": 1000.0 * wall / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": _config(1), "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": nt, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY,
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
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- native arm

def profiled_traffic(summary="circuit_kernel_c3_8q6l.md", source="qp_circuit.cuh"):
    """DRAM bytes per launch of the dominant kernel from the committed ncu summary, or None
    when the kernel source has changed since those counters were taken."""
    import hashlib
    try:
        md = open(os.path.join(ROOT, "profiles", summary)).read()
        src = open(os.path.join(ROOT, "paper_2506_23246_b300", "csrc", source), "rb").read()
    except OSError:
        return None
    vals = {}
    for line in md.splitlines():
        if ":" in line and line.split(":")[0] in ("kernel_source_sha1_12", "traffic_bytes_per_launch"):
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("kernel_source_sha1_12") != hashlib.sha1(src).hexdigest()[:12]:
        return None
    try:
        return int(vals["traffic_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def circuit_flops_per_point(n, L, nv):
    """Algorithmic FP32 flops of the statevector kernel for one point: 16 flops per amplitude
    per single-qubit gate per vector (complex 2x2 on amplitude pairs), forward on nv vectors,
    inverse gates on 2 nv vectors for layers 1..L-1 (layer 0 is not uncomputed), and 12 flops
    per amplitude per gate for each of the nv Pauli contractions Im<lambda|P phi>, plus the
    3 input-Jacobian contractions of layer 0 (tangent points only)."""
    dim = 1 << n
    f = 16 * dim * n * L * nv            # forward gates
    f += 16 * dim * n * (L - 1) * 2 * nv  # reverse: states and costates
    f += 12 * dim * n * L * nv            # Pauli contractions
    if nv == 4:
        f += 12 * dim * n * 3
    return f


def run_native(a):
    import torch
    rank, world, local = _dist()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2506_23246_b300 import build, qp
    from paper_2506_23246_b300 import workloads as W
    if rank == 0:
        build.build()
    if world > 1:
        torch.distributed.barrier()
    circ, prob, params, sets = W.c3_workload(0, nx=a.c3_grid, ny=a.c3_grid)
    # weak scaling: every rank owns its own 64x64x16 slab of the time axis (independent points)
    if world > 1:
        sets = dict(sets)
        sets["colloc"] = sets["colloc"].copy()
        sets["colloc"][:, 2] += 0.7 * rank
    plan = qp.Plan(circ, prob, path=a.path)
    dev = torch.device("cuda", local)
    dp = torch.tensor(params, device=dev)
    dsets = {k: torch.tensor(v, device=dev) for k, v in sets.items()}
    ncol = dsets["colloc"].shape[0]
    plan.reserve(sum(t.shape[0] for t in dsets.values()), dev)
    loss = torch.empty(9 + prob["energy_nt"], dtype=torch.float64, device=dev)
    grad = torch.empty(plan.n_params, dtype=torch.float32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    # device time of the measured kernels: the statevector kernel (SIMT path), or the three
    # tensor-core contractions (forward, weight gradient, back-projection mu)
    kinds = ["main"] if plan.path == "simt" else ["main", "wgrad", "mu"]
    kev = {k: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for k in kinds}

    # data parallelism: the union of the ranks' slabs is one loss; whole-loss normalisers are
    # gathered once (the points do not move), and each step sums loss terms and gradients
    norm = None
    if world > 1:
        from paper_2506_23246_b300 import dist as qdist
        norm = qdist.shard_norm((ncol, dsets["ic"].shape[0], 0), plan.count_dielectric(dsets["colloc"]),
                                device=dev)

    def make_step(dp_, ds_, loss_, grad_):
        def f():
            plan.loss_grad(dp_, ds_, out=(loss_, grad_), norm=norm)
            if world > 1:
                qdist.allreduce_loss_grad(loss_, grad_)
        return f

    def make_run(f):
        # the step's launches captured once into a CUDA graph and replayed (same kernels, same
        # buffers); the sharded form keeps plain launches around its collective
        if world > 1 or a.no_graph:
            return f, None
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            f()
        torch.cuda.synchronize()
        for _ in range(3):
            g.replay()
        torch.cuda.synchronize()
        return g.replay, g

    step = make_step(dp, dsets, loss, grad)
    for _ in range(max(a.warmup, 3)):
        step()
    torch.cuda.synchronize()
    launches = plan.last_launch_count()
    run, graph = make_run(step)

    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(a.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(a.steps)]
    kt = {k: [] for k in kinds}
    clk = ClockSampler(local)
    clk.start()
    time.sleep(0.3)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    for i in range(a.steps):
        flush.fill_(float(i))
        ev0[i].record(stream)
        run()
        ev1[i].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = clk.stop()
    # a second pass of the same steps with the library's profiling events around the measured
    # kernels (kept out of the timed steps above)
    for k in kinds:
        plan.set_profile_events(*kev[k], kernel=k)
    for i in range(a.steps):
        flush.fill_(float(i))
        step()
        for k in kinds:
            kev[k][1].synchronize()
            kt[k].append(kev[k][0].elapsed_time(kev[k][1]))
    for k in kinds:
        plan.set_profile_events(None, None, kernel=k)
    torch.cuda.synchronize()
    step_ms = [ev0[i].elapsed_time(ev1[i]) for i in range(a.steps)]
    ms = sum(step_ms) / a.steps
    if world > 1:
        t = torch.tensor([ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    value = world * ncol / (ms / 1000.0)

    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peaks = json.load(fh)
    except (OSError, ValueError):
        pass
    sm_max = peaks.get("sm_max_mhz", 2032.0)
    nic = dsets["ic"].shape[0]
    if plan.path == "simt":
        # statevector kernel, FP32 SIMT
        kms = statistics.mean(kt["main"])
        flops = ncol * circuit_flops_per_point(8, 6, 4) + nic * circuit_flops_per_point(8, 6, 1)
        peak = sms * 128 * 2 * sm_max * 1e6 / 1e12
        achieved = flops / (kms / 1000.0) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": profiled_traffic(),
                "kernel": "circuit_kernel<8,true>", "kernel_ms": kms,
                "peak_basis": "%d SMs x 128 FP32 FMA/clk x 2 x %.0f MHz (max SM clock of measured "
                              "peaks)" % (sms, sm_max)}
        contractions = None
        dtype = "f32"
    else:
        # the three contractions of the step on the tensor cores, each algorithmically
        # 2 x rows x 2^(n+1) x 2^n flops with rows = 4 per collocation point + 1 per IC point
        # (forward Phi = R W^T, weight gradient G = sum R Lambda^H, back-projection
        # mu = Re(U'^H Lambda)). Operands are FP16 pairs (hi + lo) with three FP16 products per
        # term, so each one's ceiling is the dense FP16 (= BF16) peak / 3. The reported
        # roofline is the one that takes the longest (all three do the same work).
        dim = 1 << 8
        flops = 2.0 * (4 * ncol + nic) * (2 * dim) * dim
        bf16 = peaks.get("bf16_tflops", 1800.0)
        peak = bf16 / 3.0
        basis = ("measured bf16 %.0f TFLOP/s (dense FP16 runs at the BF16 rate) / 3 (three FP16 "
                 "products per FP16-pair term)" % bf16)
        names = {"main": ("dense_fused_fwd_kernel<8> (forward + readout + losses + costates)",
                          "dense_fused_fwd_c3_8q6l.md", "qp_fused.cuh"),
                 "wgrad": ("dense_wgrad_gemm_kernel<FP16, 8> (weight gradient)",
                           "dense_wgrad_c3_8q6l.md", "qp_wgrad.cuh"),
                 "mu": ("dense_mu_embed_kernel<8> (back-projection + embedding gradients)",
                        "dense_mu_embed_c3_8q6l.md", "qp_mu.cuh")}
        contractions = {}
        for k in kinds:
            kms_k = statistics.mean(kt[k])
            ach = flops / (kms_k / 1000.0) / 1e12
            contractions[k] = {"kernel": names[k][0], "kernel_ms": kms_k, "achieved": ach,
                               "frac": ach / peak, "traffic": profiled_traffic(names[k][1], names[k][2])}
        top = max(kinds, key=lambda k: contractions[k]["kernel_ms"])
        c = contractions[top]
        roof = {"bound": "tensor", "achieved": c["achieved"], "peak": peak, "unit": "TFLOP/s",
                "frac": c["frac"], "traffic": c["traffic"], "kernel": c["kernel"],
                "kernel_ms": c["kernel_ms"], "peak_basis": basis}
        dtype = "fp16x2-split, fp32 accum"

    # end to end through the public call: pinned host inputs in, loss + gradient out. Two sets
    # of device buffers: step i's inputs are copied in (copy stream) while step i - 1 computes,
    # and its loss and gradient are read back (second copy stream) while step i + 1 computes.
    # The timed region runs from before the first input copy to after the last read-back, L2
    # flushes between the steps included.
    hp = torch.tensor(params).pin_memory()
    hs = {k: torch.tensor(v).pin_memory() for k, v in sets.items()}
    hl = [torch.empty(loss.shape, dtype=torch.float64).pin_memory() for _ in range(2)]
    hg = [torch.empty(grad.shape, dtype=torch.float32).pin_memory() for _ in range(2)]
    h2d = hp.numel() * 4 + sum(v.numel() * 4 for v in hs.values())
    d2h = hl[0].numel() * 8 + hg[0].numel() * 4
    bufs = [(dp, dsets, loss, grad, run)]
    dp2, ds2 = torch.empty_like(dp), {k: torch.empty_like(v) for k, v in dsets.items()}
    dp2.copy_(dp)
    for k in ds2:
        ds2[k].copy_(dsets[k])
    loss2, grad2 = torch.empty_like(loss), torch.empty_like(grad)
    step2 = make_step(dp2, ds2, loss2, grad2)
    step2()
    torch.cuda.synchronize()
    run2, graph2 = make_run(step2)
    bufs.append((dp2, ds2, loss2, grad2, run2))
    up, down = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
    ev = {n: [torch.cuda.Event() for _ in range(2)] for n in ("in", "done", "out")}

    def e2e_steps(k, i0=0):
        for i in range(i0, i0 + k):
            b = i % 2
            d_p, d_s, d_l, d_g, r = bufs[b]
            with torch.cuda.stream(up):
                if i >= 2:
                    up.wait_event(ev["done"][b])     # step i - 2 has read these inputs
                d_p.copy_(hp, non_blocking=True)
                for key in hs:
                    d_s[key].copy_(hs[key], non_blocking=True)
                ev["in"][b].record(up)
            stream.wait_event(ev["in"][b])
            if i >= 2:
                stream.wait_event(ev["out"][b])      # step i - 2's results have been read back
            flush.fill_(float(i))
            r()
            ev["done"][b].record(stream)
            with torch.cuda.stream(down):
                down.wait_event(ev["done"][b])
                hl[b].copy_(d_l, non_blocking=True)
                hg[b].copy_(d_g, non_blocking=True)
                ev["out"][b].record(down)

    e2e_steps(4)
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    up.wait_event(t0)
    e2e_steps(a.steps)
    down.wait_event(ev["out"][(a.steps - 1) % 2])
    t1.record(down)
    torch.cuda.synchronize()
    ems = t0.elapsed_time(t1) / a.steps
    if world > 1:
        t = torch.tensor([ems], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ems = float(t.item())

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
                "warmup": max(a.warmup, 3), "ms_per_step": ms, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": dtype, "data": "synthetic",
                "config": _config(world),
                "launch": ("one CUDA graph per step (the library's kernels captured once, replayed)"
                           if graph is not None else "kernels launched one by one"),
                "e2e": {"value": world * ncol / (ems / 1000.0), "unit": UNIT,
                        "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": ems,
                        "copies": "double-buffered: inputs of step i+1 in and results of step i-1 "
                                  "out on two copy streams while step i computes; L2 flush per step "
                                  "inside the timed region"},
                "gpu_launches": launches * a.steps,
                "roofline": roof,
                "contractions": contractions,
                "path": plan.path,
                "clocks": clocks}
        if not a.no_cpu_baseline and world == 1:
            v, nt, desc = _oracle_sample(10.0)
            line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": nt, "kind": "oracle",
                                    "sample": desc}
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_c5(a):
    """32 uneven instances (n ~ U{4..10}, L ~ U{2..8}, B ~ 2^U(10, 16) collocation points plus
    B/16 IC points, RFF64+MLP32 premap, strongly entangling) in one qp_batch_step per step:
    the gate-by-gate instances (n <= 7) in the multi-instance launch with the shape the tuner
    chose (tuned once before the timed region), the tensor-core instances as their own calls
    on worker streams. Against the same call without the multi-instance launch (every
    instance its own call on the worker streams) and against the instances called one after
    the other on one stream."""
    import torch
    rank, world, local = _dist()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2506_23246_b300 import build, qp
    from paper_2506_23246_b300 import workloads as W
    if rank == 0:
        build.build()
    if world > 1:
        torch.distributed.barrier()
    dev = torch.device("cuda", local)
    inst = W.c5_instances(32, seed=rank)
    plans, params, sets, outs = [], [], [], []
    for circ, prob, p, st in inst:
        pl = qp.Plan(circ, prob)
        plans.append(pl)
        params.append(torch.tensor(p, device=dev))
        sets.append({k: torch.tensor(v, device=dev) for k, v in st.items()})
        pl.reserve(sum(v.shape[0] for v in st.values()), dev)
        outs.append((torch.empty(9 + prob.get("energy_nt", 0), dtype=torch.float64, device=dev),
                     torch.empty(pl.n_params, dtype=torch.float32, device=dev)))
    ncol = sum(st["colloc"].shape[0] for _, _, _, st in inst)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def batched():
        qp.batch_step(plans, params, sets, outs=outs)

    def streams_only():
        qp.batch_step(plans, params, sets, outs=outs, grouped=False)

    def sequential():
        for pl, p, st, o in zip(plans, params, sets, outs):
            pl.loss_grad(p, st, out=o)

    def timed(fn):
        for _ in range(max(a.warmup, 3)):
            fn()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(a.steps)]
        for i in range(a.steps):
            flush.fill_(float(i))
            ev[i][0].record(stream)
            fn()
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        ms = sum(e0.elapsed_time(e1) for e0, e1 in ev) / a.steps
        if world > 1:
            t = torch.tensor([ms], device=dev)
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            ms = float(t.item())
        return ms

    tune = qp.batch_tune(plans, params, sets, outs=outs)
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    clk.start()
    time.sleep(0.3)
    ms_b = timed(batched)
    launches = sum(pl.last_launch_count() for pl in plans)
    ms_u = timed(streams_only)
    ms_s = timed(sequential)
    clocks = clk.stop()
    grouped = sum(1 for pl in plans if pl.path == "simt")
    if rank == 0:
        print(json.dumps({
            "metric": "collocation pts/s, 32 uneven QPINN instances per step (fwd+d/dx,dy,dt+adjoint grad)",
            "value": world * ncol / (ms_b / 1000.0), "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": max(a.warmup, 3), "ms_per_step": ms_b, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "32 uneven instances: n ~ U{4..10}, L ~ U{2..8}, B ~ 2^U(10,16) "
                                   "colloc + B/16 IC, RFF64+MLP32, strongly entangling, vacuum",
                       "colloc_per_gpu": ncol, "instances": len(plans),
                       "paths": sorted(set(pl.path for pl in plans)),
                       "grouped_instances": grouped,
                       "multi_launch_shape": {"warps_per_cta": tune[0], "tasks_per_warp_and_item": tune[1]},
                       "l2": "flushed between timed steps (256 MiB write)"},
            "streams_only": {"ms_per_step": ms_u, "value": world * ncol / (ms_u / 1000.0),
                             "speedup_batched": ms_u / ms_b},
            "sequential": {"ms_per_step": ms_s, "value": world * ncol / (ms_s / 1000.0),
                           "speedup_batched": ms_s / ms_b},
            "gpu_launches": launches * a.steps, "roofline": None, "clocks": clocks}))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_configs(a):
    """Every configuration on every compute path that supports it, one JSON line each:
    C1 (4q/2L, 1024 points, forward + d/dx,dy,dt), C2 (6q/4L, 16,384 + 2,048 IC + 2,048 PEC
    points, loss + gradient), C3 (the bench step) and C4 (10q/8L, 64^3 grid + 64^2 IC plane,
    RFF64 + MLP32, loss + gradient). Paths: FP32 SIMT; tensor cores with FP16 pairs and with
    3xTF32 where the configuration has them. Device time per step with L2 flushed between
    steps; the dominant kernel's device time from the library's profiling events."""
    import torch
    from paper_2506_23246_b300 import build, qp
    from paper_2506_23246_b300 import workloads as W
    build.build()
    dev = torch.device("cuda", 0)
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peaks = json.load(fh)
    except (OSError, ValueError):
        pass
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_max = peaks.get("sm_max_mhz", 2032.0)
    bf16 = peaks.get("bf16_tflops", 1800.0)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    c1c, c1p, c1x = W.c1_workload(0, 1024)
    c2c, c2pr, c2p, c2s = W.c2_workload(0)
    c3c, c3pr, c3p, c3s = W.c3_workload(0)
    c4c, c4pr, c4p, c4s = W.c4_workload(0, n=a.grid)
    cases = [("C1 4q/2L, 1024 points, forward + d/dx,dy,dt", c1c, None, c1p, {"pts": c1x},
              [("simt", "fp16_pairs")]),
             ("C2 6q/4L, 16384 colloc + 2048 IC + 2048 PEC, loss + gradient", c2c, c2pr, c2p, c2s,
              [("simt", "fp16_pairs")]),
             ("C3 8q/6L RFF64+MLP32 dielectric, 65536 colloc + 4096 IC, loss + gradient", c3c, c3pr,
              c3p, c3s, [("simt", "fp16_pairs"), ("gemm_split", "fp16_pairs")]),
             ("C4 10q/8L RFF64+MLP32, %d^3 colloc + %d IC, loss + gradient" % (a.grid, a.grid * a.grid),
              c4c, c4pr, c4p, c4s,
              [("simt", "fp16_pairs"), ("gemm_split", "fp16_pairs"), ("gemm_split", "tf32_pairs")])]
    for name, circ, prob, params, sets, paths in cases:
        if a.config and not name.startswith(a.config + " "):
            continue
        paths = [(p, o) for p, o in paths if (a.path == "auto" or p == a.path) and
                 (a.operands is None or p == "simt" or o == a.operands)]
        n, L = circ["n_qubits"], circ["n_layers"]
        dp = torch.tensor(params, device=dev)
        dsets = {k: torch.tensor(v, device=dev) for k, v in sets.items()}
        ncol = dsets["pts"].shape[0] if prob is None else dsets["colloc"].shape[0]
        rows = sum(4 * v.shape[0] if k in ("pts", "colloc") else v.shape[0] for k, v in dsets.items())
        for path, ops in paths:
            plan = qp.Plan(circ, prob, path=path, operands=ops)
            plan.reserve(sum(v.shape[0] for v in dsets.values()), dev)
            if prob is None:
                f = torch.empty(ncol, 3, device=dev)
                df = torch.empty(ncol, 3, 3, device=dev)
                fn = lambda: plan.forward(dp, dsets["pts"], out=(f, df))
            else:
                loss = torch.empty(9 + prob["energy_nt"], dtype=torch.float64, device=dev)
                grad = torch.empty(plan.n_params, dtype=torch.float32, device=dev)
                fn = lambda: plan.loss_grad(dp, dsets, out=(loss, grad))
            # measured kernels: the statevector kernel (SIMT), the forward contraction
            # (qp_forward), or all three contractions of a loss call (tensor cores)
            kinds = ["main"] if (plan.path == "simt" or prob is None) else ["main", "wgrad", "mu"]
            kev = {k: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for k in kinds}
            for k in kinds:
                plan.set_profile_events(*kev[k], kernel=k)
            for _ in range(max(a.warmup, 3)):
                fn()
            torch.cuda.synchronize()
            steps = a.steps
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(steps)]
            kt = {k: [] for k in kinds}
            for i in range(steps):
                flush.fill_(float(i))
                ev[i][0].record(stream)
                fn()
                ev[i][1].record(stream)
                for k in kinds:
                    kev[k][1].synchronize()
                    kt[k].append(kev[k][0].elapsed_time(kev[k][1]))
            torch.cuda.synchronize()
            for k in kinds:
                plan.set_profile_events(None, None, kernel=k)
            ms = sum(e0.elapsed_time(e1) for e0, e1 in ev) / steps
            top = max(kinds, key=lambda k: statistics.mean(kt[k]))
            kms = statistics.mean(kt[top])
            dim = 1 << n
            if plan.path == "simt":
                kernel = "circuit_kernel<%d,%s>" % (n, "false" if prob is None else "true")
                if prob is None:
                    flops = ncol * 16 * dim * n * L * 4
                else:
                    flops = sum(v.shape[0] * circuit_flops_per_point(n, L, 4 if k == "colloc" else 1)
                                for k, v in dsets.items())
                peak, bound = sms * 128 * 2 * sm_max * 1e6 / 1e12, "alu"
            else:
                # the longest of the contractions, 2 x rows x 2^(n+1) x 2^n algorithmic flops each
                form = "FP16" if ops == "fp16_pairs" else "TF32"
                kernel = {"main": ("dense_fused_fwd_kernel<%d>" % n) if n in (7, 8) and prob is not None
                          else "dense_row16_kernel<0>" if ops == "fp16_pairs" else "dense_row_gemm_kernel<0>",
                          "wgrad": "dense_wgrad_gemm_kernel<%s, %d>" % (form, n),
                          "mu": ("dense_mu_embed_kernel<%d>" % n) if n in (7, 8)
                          else "dense_row16_kernel<1>" if ops == "fp16_pairs" else "dense_row_gemm_kernel<1>"}[top]
                flops = 2.0 * rows * (2 * dim) * dim
                peak = bf16 / 3.0 if ops == "fp16_pairs" else bf16 * 0.5 / 3.0
                bound = "tensor"
            achieved = flops / (kms / 1000.0) / 1e12
            print(json.dumps({"config": name, "path": plan.path,
                              "operands": ops if plan.path != "simt" else "fp32",
                              "ms_per_step": ms, "colloc_pts_per_s": ncol / (ms / 1000.0),
                              "steps": steps, "warmup": max(a.warmup, 3),
                              "dominant_kernel": {"name": kernel, "ms": kms, "share": kms / ms,
                                                  "bound": bound, "achieved_tflops": achieved,
                                                  "peak_tflops": peak, "frac": achieved / peak},
                              "gpu_launches_per_step": plan.last_launch_count()}), flush=True)
            del plan
            torch.cuda.empty_cache()
    return 0


def run_paper_net(a):
    """The paper's hybrid network (Sec. 2.2-2.3, Table 1: periodic input map with a learned period,
    RFF with 128 frequencies, three tanh layers of width 128, 7 angles, 7 qubits x 4 strongly
    entangling layers, head of 3; 66,848 classical + 84 quantum parameters) on the
    grid sizes of its timing table (40^3 and 87^3 collocation points on [-1,1]^2 x [0,1.5],
    vacuum, IC plane of the grid, energy term over the grid's time slices): one step is
    qp_loss_grad (fields, input derivatives, losses, adjoint gradient of all 66,932 trainable
    parameters). Each grid runs twice: without the symmetry penalty, and with the whole loss of
    Eq. 24 (L_sym of Eq. 18 at weight 10: every collocation point also evaluated at its two
    mirrors).
    The paper's numbers (TorQ, one training epoch with second-order autograd and Adam, A100 or
    L40s) are context, not the same measurement."""
    import torch
    from paper_2506_23246_b300 import build, qp
    from paper_2506_23246_b300 import workloads as W
    build.build()
    dev = torch.device("cuda", 0)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    paper = {40: 0.145136, 87: 0.849967}
    for g, wsym in [(g, w) for g in ((a.paper_grid,) if a.paper_grid > 0 else (40, 87)) for w in (0.0, 10.0)]:
        circ = W.circuit(7, 4, 7, ansatz="strong_rot", enc="rx", scale="acos", premap="rff_mlp",
                         rff_freqs=128, mlp_width=128, mlp_depth=3, periodic=True)
        prob = W.problem("vacuum", w_energy=10.0, energy_slice=g * g, energy_nt=g, w_sym=wsym)
        sets = {"colloc": W.grid_points(g, g, g, 1.5), "ic": W.ic_grid(g, g)}
        params = W.init_params(circ, 0)
        plan = qp.Plan(circ, prob, path=a.path)
        dp = torch.tensor(params, device=dev)
        dsets = {k: torch.tensor(v, device=dev) for k, v in sets.items()}
        plan.reserve(sum(v.shape[0] for v in dsets.values()), dev)
        loss = torch.empty(9 + prob["energy_nt"] + (1 if wsym > 0 else 0), dtype=torch.float64, device=dev)
        grad = torch.empty(plan.n_params, dtype=torch.float32, device=dev)
        for _ in range(max(a.warmup, 3)):
            plan.loss_grad(dp, dsets, out=(loss, grad))
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(a.steps)]
        for i in range(a.steps):
            flush.fill_(float(i))
            ev[i][0].record(stream)
            plan.loss_grad(dp, dsets, out=(loss, grad))
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        assert plan.last_device_error() == 0
        ms = sum(e0.elapsed_time(e1) for e0, e1 in ev) / a.steps
        ncol = sets["colloc"].shape[0]
        print(json.dumps({"workload": "paper hybrid net, %d^3 grid%s" % (g, ", with L_sym (Eq. 24 in full)" if wsym > 0
                                                                         else ""), "n_params": plan.n_params,
                          "path": plan.path, "colloc_points": ncol, "ic_points": sets["ic"].shape[0],
                          "ms_per_step": ms, "colloc_pts_per_s": ncol / (ms / 1000.0),
                          "steps": a.steps, "warmup": max(a.warmup, 3),
                          "gpu_launches_per_step": plan.last_launch_count(),
                          "paper_context": {"system": "TorQ, one training epoch (backprop, Adam), A100 or L40s",
                                            "s_per_epoch": paper[g], "pts_per_s": ncol / paper[g]}
                                          if g in paper else None}),
              flush=True)
        del plan
        torch.cuda.empty_cache()
    return 0


def run_timeline(a):
    """Kernel timeline of the benchmark step (both streams of the call), replayed as one CUDA graph
    after L2 flushes, traced by CUPTI through torch.profiler. The durations come from a traced
    run: they explain the bench numbers, they are not bench numbers."""
    import tempfile
    import torch
    from torch.profiler import ProfilerActivity, profile
    from paper_2506_23246_b300 import build, qp
    from paper_2506_23246_b300 import workloads as W
    build.build()
    dev = torch.device("cuda", 0)
    circ, prob, params, sets = W.c3_workload(0, nx=a.c3_grid, ny=a.c3_grid)
    plan = qp.Plan(circ, prob, path=a.path)
    dp = torch.tensor(params, device=dev)
    dsets = {k: torch.tensor(v, device=dev) for k, v in sets.items()}
    plan.reserve(sum(t.shape[0] for t in dsets.values()), dev)
    loss = torch.empty(9 + prob["energy_nt"], dtype=torch.float64, device=dev)
    grad = torch.empty(plan.n_params, dtype=torch.float32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    for _ in range(max(a.warmup, 3)):
        plan.loss_grad(dp, dsets, out=(loss, grad))
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        plan.loss_grad(dp, dsets, out=(loss, grad))
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    nsteps = max(a.steps, 2)
    with profile(activities=[ProfilerActivity.CUDA]) as prof:
        for i in range(nsteps):
            flush.fill_(float(i))
            g.replay()
        torch.cuda.synchronize()
    with tempfile.TemporaryDirectory() as td:
        fn = os.path.join(td, "trace.json")
        prof.export_chrome_trace(fn)
        with open(fn) as fh:
            events = json.load(fh)["traceEvents"]
    ks = sorted((e["ts"], e["dur"], e.get("args", {}).get("stream"), e["name"]) for e in events
                if e.get("cat") == "kernel")
    # steps begin at the flush kernels; print the last whole step
    starts = [i for i, k in enumerate(ks) if "FillFunctor" in k[3]]
    i0, i1 = starts[-1], len(ks)
    t0 = ks[i0][0] + ks[i0][1]
    print("# start_us dur_us end_us stream kernel (t = 0 at the end of the L2 flush)")
    for ts, d, st, name in ks[i0 + 1:i1]:
        print("%9.1f %8.1f %9.1f  %s  %s" % (ts - t0, d, ts - t0 + d, st, name.split("(")[0]))
    return 0


def main():
    a = _args()
    if a.timeline:
        return run_timeline(a)
    if a.impl == "reference":
        return run_reference(a)
    if a.workload == "c5":
        return run_c5(a)
    if a.workload == "configs":
        return run_configs(a)
    if a.workload == "paper_net":
        return run_paper_net(a)
    return run_native(a)


if __name__ == "__main__":
    sys.exit(main())
