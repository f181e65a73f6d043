#!/usr/bin/env python
"""Throughput benchmark of the IDBF associated Legendre transform on GB300.

One step = the forward ALT of a batch of F fields over every order
|m| <= 2N-1 (gather, IDBF / low-rank / dense block products, parity fold)
followed by the inverse ALT of its output (weighted fold, transposed
products, scatter): every step of the apply path, on inputs resident in HBM.
Metric: fields per second (F x ranks / seconds per step).

Also reported: forward-only and inverse-only kernel times, the dominant
kernel's roofline fraction, an end-to-end number through the public API
with the batch copied from pinned host memory and the result read back
every step, and the dense FP64 CPU oracle timed on the host cores.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
    python bench.py --impl reference ...   (the oracle as the reference arm)
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2004_11346_gb300 import inputs  # noqa: E402

METRIC = "SHT fields/s at N=1024 vs FP64 IDBF & dense ALT on 1 GB300, rel err<=1e-6"
DEFAULT_WORKLOAD = "mixed_N1024_F64"
EXTRA_WORKLOADS = {
    # smaller cases used for profiling captures
    "fp64_N512": dict(N=512, F=1, seed=0, decay=1.0, real_m0=False, eps=1e-12, precision="fp64"),
    "mixed_N512_F16": dict(N=512, F=16, seed=0, decay=0.0, real_m0=False, eps=1e-7, precision="mixed"),
    "mixed_N512_F32": dict(N=512, F=32, seed=0, decay=0.0, real_m0=False, eps=1e-7, precision="mixed"),
    # the same with the headline plan's shape scaled to N=512 (n0 = N/4, leaves 4x the default)
    "mixed_N512_F32_tuned": dict(N=512, F=32, seed=0, decay=0.0, real_m0=False, eps=1e-7, precision="mixed",
                                 plan=dict(n0=128, n_leaf=128)),
    # the same with two field groups per order, as the 64-field headline
    "mixed_N512_F64_tuned": dict(N=512, F=64, seed=0, decay=0.0, real_m0=False, eps=1e-7, precision="mixed",
                                 plan=dict(n0=128, n_leaf=128)),
    # single components (--only): the FP32 phi transform of 8 fields at the
    # headline's N (1.07 GB per array), the on-the-fly dense FP64 ALT
    "mixed_N1024_F8": dict(N=1024, F=8, seed=0, decay=0.0, real_m0=False, eps=1e-7, precision="mixed"),
    "fp64_N512_F16": dict(N=512, F=16, seed=0, decay=0.0, real_m0=False, eps=1e-12, precision="fp64"),
}
# the ncu capture whose traffic a workload's roofline scales (same kernel, same plan shape, smaller case)
TRAFFIC_REF = {"mixed_N1024_F64": "mixed_N512_F64_tuned"}
FP64_PEAK_GFLOPS = 1250.0  # GB300 nominal FP64 (vector) rate


def workload(name, n0=None, n_leaf=None):
    w = dict(inputs.WORKLOADS.get(name) or EXTRA_WORKLOADS[name])
    w["name"] = name
    plan = dict(w.get("plan", {}))
    if n0:
        plan["n0"] = n0
    if n_leaf:
        plan["n_leaf"] = n_leaf
    if plan:
        w["plan"] = plan
    return w


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def reduce_max(vals, world, device="cpu"):
    """Element-wise max of per-rank timings over all ranks (identity for one rank)."""
    if world == 1:
        return list(vals)
    import torch
    import torch.distributed as dist
    t = torch.tensor(vals, device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def rank_fields(N, F, w, rank):
    """The F coefficient fields rank `rank` processes: fields rank*F .. rank*F+F-1 of the seeded stream."""
    return inputs.coefficients(N, F, w["seed"], decay=w["decay"], real_m0=w["real_m0"], field_offset=rank * F)


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(device_index)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- work accounting
def program_flops(plan, F):
    """Algorithmic FLOPs of one forward (or inverse) launch: 2 x entries x RHS.

    Each stored factor entry multiplies 4 real right-hand sides per field
    (Re/Im of +m and -m); order m = 0 has 2.
    """
    prog = plan.program(parts=("units", "ops"))
    ops, units = prog["ops"], prog["units"]
    entries = (ops["mo"].astype(np.int64) * ops["ni"].astype(np.int64))
    total = 0
    for u in units:
        e = int(entries[u["op_begin"]: u["op_end"]].sum())
        total += e * (2 if u["am"] == 0 else 4)
    return 2 * total * F, int(entries.sum())


# ---------------------------------------------------------------- reference arm
def sample_orders(N, stride):
    return list(range(0, 2 * N, stride))


def oracle_sample(N, beta_field, stride, g_check=None):
    """Forward + inverse ALT by the oracle for every stride-th order |m| (both
    signs); returns (seconds, fraction of the full transform's work), plus,
    when g_check (one field's ALT values, (4N-1, 2N, 2)) is given, the
    per-order relative errors of g_check against the oracle's forward values
    (compared after the timed loop)."""
    import oracle
    x, w = oracle.gl_rule(2 * N)
    ams = sample_orders(N, stride)
    keep = {}
    t0 = time.perf_counter()
    for am in ams:
        for m in ([am, -am] if am else [0]):
            off = oracle.coef_offset(N, m)
            gm = oracle.alt_forward_m(N, m, beta_field[off: off + 2 * N - am], x)
            oracle.alt_inverse_m(N, m, gm, x, w)
            if g_check is not None:
                keep[m] = gm
    dt = time.perf_counter() - t0
    work_s = sum((2 * N - am) * (1 if am == 0 else 2) for am in ams)
    if g_check is None:
        return dt, work_s / (4.0 * N * N)
    errs = [float(np.linalg.norm(g_check[oracle.order_slot(m)] - ref) / np.linalg.norm(ref))
            for m, ref in keep.items()]
    return dt, work_s / (4.0 * N * N), errs


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    if args.workload.startswith(UNEVEN_PREFIX):
        print(json.dumps({"impl": "reference", "unavailable": "the oracle arm times the single-N workloads; "
                          "an uneven batch is the sum of its sizes' single-N transforms"}), flush=True)
        return
    w = workload(args.workload)
    N = w["N"]
    beta = inputs.workload_coefficients(w["name"], F=1)[0]
    stride = max(1, args.ref_stride)
    for _ in range(args.warmup):
        oracle_sample(N, beta, stride * 4)
    times, frac = [], 1.0
    for _ in range(args.steps):
        dt, frac = oracle_sample(N, beta, stride)
        times.append(dt)
    import oracle
    cores = oracle.num_threads()
    sec_per_field = float(np.mean(times)) / frac
    value = 1.0 / sec_per_field
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "fields/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": float(np.mean(times)) * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config_of(w, world),
        "cpu_baseline": {"kind": "oracle", "value": value, "unit": "fields/s", "cores": cores,
                         "sample": f"forward+inverse ALT of every {stride}th order |m| of 1 field "
                                   f"({frac:.3f} of the transform), scaled to one field"},
        "e2e": {"value": value, "unit": "fields/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# The tensor-core kernel's tile (compile-time in csrc/apply_tc.cuh and apply_tc.cu): 128 right-hand
# sides (MMA M) x 128 block rows (MMA N) per accumulator pair, K chunks of 32 per pipeline stage
TC_TILE = {"M_rhs": 128, "N": 128, "K_chunk": 32, "stages": 4}


def config_of(w, world):
    cfg = {"workload": w["name"], "N": w["N"], "fields_per_rank": w["F"], "global_batch": w["F"] * world,
           "eps": w["eps"], "precision": w["precision"], "orders": 4 * w["N"] - 1,
           "step": "forward ALT + inverse ALT", "parallelism": f"replicas{world}",
           "l2": "inputs and factor store larger than L2", "plan": w.get("plan", "library defaults")}
    if w["precision"] == "mixed":
        cfg["tile"] = TC_TILE
    return cfg


# ---------------------------------------------------------------- our arm
FP32_PEAK_GFLOPS = 128 * 2 * 152 * 2.07  # FP32 lanes x 2 x SMs x max SM clock (GHz)


def plan_for(sht, w, **kw):
    """The workload's plan; its partition/leaf sizes where the workload fixes them."""
    from paper_2004_11346_gb300 import _lib
    prec = {"fp64": _lib.SHT_FP64, "mixed": _lib.SHT_MIXED, "fp32": _lib.SHT_FP32}[w["precision"]]
    return sht.Plan(w["N"], w["eps"], precision=prec, **{**w.get("plan", {}), **kw})


def time_steps(torch, plan, beta, g, back, K, W, stream):
    """W untimed then K timed (forward, inverse) steps; per-step and per-kernel ms."""
    for _ in range(W):
        plan.forward(beta, out=g)
        plan.inverse(g, out=back)
    torch.cuda.synchronize()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(K)]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(K):
        ev[i][0].record(stream)
        plan.forward(beta, out=g)
        ev[i][1].record(stream)
        plan.inverse(g, out=back)
        ev[i][2].record(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / K
    fwd = float(np.mean([ev[i][0].elapsed_time(ev[i][1]) for i in range(K)]))
    inv = float(np.mean([ev[i][1].elapsed_time(ev[i][2]) for i in range(K)]))
    return ms, fwd, inv


def time_graph(torch, plan, beta, g, back, K, W, stream):
    """The step (forward then inverse ALT) captured once in a CUDA graph, then
    W untimed and K timed replays, each bracketed by CUDA events on the
    replaying stream.  Returns (median ms, mean ms over the K-step region)."""
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    with torch.cuda.stream(side):  # warm the capture stream's state once, outside the capture
        plan.forward(beta, out=g)
        plan.inverse(g, out=back)
    stream.wait_stream(side)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        plan.forward(beta, out=g)
        plan.inverse(g, out=back)
    torch.cuda.synchronize()
    for _ in range(W):
        graph.replay()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(K + 1)]
    rs = torch.cuda.current_stream()
    ev[0].record(rs)
    for i in range(K):
        graph.replay()
        ev[i + 1].record(rs)
    torch.cuda.synchronize()
    per = [ev[i].elapsed_time(ev[i + 1]) for i in range(K)]
    del graph
    return float(np.median(per)), ev[0].elapsed_time(ev[K]) / K


def run_e2e(torch, plan, beta_h, g, K, W, barrier, chunk=None):
    """ms per step of host -> device -> forward + inverse ALT -> host for the
    whole batch, pipelined over chunks of `chunk` fields (default 32, one
    field group of the tensor-core kernel) on three streams with two device
    buffers per side, so that one chunk's copy in, the previous chunk's
    transform and the one before's copy out can run at the same time."""
    F = beta_h.shape[0]
    C = min(chunk or 32, F)
    starts = list(range(0, F, C))
    beta_pin = torch.from_numpy(beta_h).pin_memory()
    out_pin = torch.empty(beta_pin.shape, dtype=torch.float64).pin_memory()
    dev_in = [torch.empty((C,) + beta_h.shape[1:], dtype=torch.float64, device="cuda") for _ in range(2)]
    dev_out = [torch.empty_like(dev_in[0]) for _ in range(2)]
    gbuf = g[:C]
    s_in, s_cmp, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    ev = lambda: torch.cuda.Event()
    # per buffer slot: transform done reading dev_in, copy-out done reading dev_out
    cmp_done = [None, None]
    out_done = [None, None]

    def step():
        for c, f0 in enumerate(starts):
            n = min(C, F - f0)
            b = c % 2
            with torch.cuda.stream(s_in):
                if cmp_done[b] is not None:
                    s_in.wait_event(cmp_done[b])
                dev_in[b][:n].copy_(beta_pin[f0:f0 + n], non_blocking=True)
                e_in = ev()
                e_in.record(s_in)
            with torch.cuda.stream(s_cmp):
                s_cmp.wait_event(e_in)
                if out_done[b] is not None:
                    s_cmp.wait_event(out_done[b])
                plan.forward(dev_in[b][:n], out=gbuf[:n])
                plan.inverse(gbuf[:n], out=dev_out[b][:n])
                cmp_done[b] = ev()
                cmp_done[b].record(s_cmp)
            with torch.cuda.stream(s_out):
                s_out.wait_event(cmp_done[b])
                out_pin[f0:f0 + n].copy_(dev_out[b][:n], non_blocking=True)
                out_done[b] = ev()
                out_done[b].record(s_out)

    for _ in range(W):
        step()
    torch.cuda.synchronize()
    barrier()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    main = torch.cuda.current_stream()
    t0.record(main)
    for s_ in (s_in, s_cmp, s_out):
        s_.wait_event(t0)
    for _ in range(K):
        step()
    for s_ in (s_in, s_cmp, s_out):
        e = ev()
        e.record(s_)
        main.wait_event(e)
    t1.record(main)
    torch.cuda.synchronize()
    plan.sync()
    rt = float(np.linalg.norm(out_pin.numpy() - beta_h) / np.linalg.norm(beta_h))
    if not rt < 1e-5:
        raise RuntimeError(f"end-to-end round trip error {rt}")
    return t0.elapsed_time(t1) / K, beta_pin.numel() * 8, len(starts)


def run_ours(args):
    import torch
    import paper_2004_11346_gb300 as sht
    from paper_2004_11346_gb300 import _lib

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev_index = torch.cuda.current_device()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    w = workload(args.workload, args.n0, args.n_leaf)
    N, F = w["N"], w["F"]
    t0 = time.perf_counter()
    # workspace for the whole batch; CUDA events around every apply kernel
    plan = plan_for(sht, w, max_fields=F, flags=_lib.SHT_FLAG_TIMING)
    t_plan = time.perf_counter() - t0
    st = plan.stats()
    beta_h = rank_fields(N, F, w, rank)
    beta = torch.from_numpy(beta_h).cuda()
    g = torch.empty((F, 4 * N - 1, 2 * N, 2), dtype=torch.float64, device="cuda")
    back = torch.empty_like(beta)
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    def max_over_ranks(vals):
        return reduce_max(vals, world, device="cuda")

    for _ in range(args.warmup):
        plan.forward(beta, out=g)
        plan.inverse(g, out=back)
    torch.cuda.synchronize()
    plan.sync()
    rt_err = float((back - beta).norm() / beta.norm())

    K = args.steps
    # mixed: the forward call = the pre-gather kernel, the tensor-core kernel
    # and the output kernel; the inverse call = the pre-gather kernel and the
    # tensor-core kernel, which writes the outputs itself; other precisions one
    # kernel per call
    kernels_per_step = 5 if w["precision"] == "mixed" else 2
    # headline: K replays of the step captured in a CUDA graph, the library's
    # event instrumentation paused; value from the median replay
    plan.set_timing(False)
    barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(dev_index)
    time.sleep(0.3)
    ms, ms_mean = time_graph(torch, plan, beta, g, back, K, max(3, args.warmup), stream)
    clk = clocks.stop()
    launches = K * kernels_per_step
    plan.set_timing(True)
    # separate pass: forward / inverse split and the dominant kernel alone
    # (library CUDA events around each kernel, on the launching stream)
    _, fwd_ms, inv_ms = time_steps(torch, plan, beta, g, back, K, 1, stream)
    plan.kernel_time(reset=True)
    for _ in range(K):
        plan.forward(beta, out=g)
    kf = plan.kernel_time(reset=True)
    main_ms = kf["apply_ms"] / max(1, kf["launches"])
    out_ms = kf["output_ms"] / max(1, kf["launches"])
    for _ in range(K):
        plan.inverse(g, out=back)
    ki = plan.kernel_time(reset=True)
    inv_split = {"apply_ms": ki["apply_ms"] / max(1, ki["launches"]),
                 "output_ms": ki["output_ms"] / max(1, ki["launches"]),
                 "what": "inverse call: pre-gather + tensor-core kernel, whose output warps write the outputs "
                         "(apply; the output interval is empty)"
                 if w["precision"] == "mixed" else "inverse call"}
    barrier()
    plan.sync()
    ms, ms_mean, fwd_ms, inv_ms = max_over_ranks([ms, ms_mean, fwd_ms, inv_ms])
    value = world * F / (ms * 1e-3)

    # end to end through the public API: every step copies the batch in from
    # pinned host memory and reads the result back.  The batch moves in chunks
    # on three streams (copy in, transform, copy out) so that the copies of one
    # chunk overlap the transforms of its neighbours; the transforms themselves
    # stay in order on one stream (calls on one plan must not overlap).
    e2e_ms, io_bytes, e2e_chunks = run_e2e(torch, plan, beta_h, g, K, max(1, args.warmup), barrier,
                                           chunk=args.e2e_chunk)
    e2e_ms = max_over_ranks([e2e_ms])[0]

    flops, entries = program_flops(plan, F)
    roof = roofline(plan, w, F, flops, fwd_ms, main_ms, out_ms)
    line = {
        "metric": METRIC, "value": value, "unit": "fields/s", "n_gpus": world, "steps": K, "warmup": args.warmup,
        "ms_per_step": ms, "ms_per_step_mean": ms_mean,
        "timing": f"median of {K} CUDA-graph replays of the step (event-timed each), instrumentation off",
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "f64", "fp32": "f32", "mixed": "bf16x3 split, f32 accumulate"}[w["precision"]],
        "data": "synthetic", "config": config_of(w, world),
        "forward_ms": fwd_ms, "inverse_ms": inv_ms, "inverse_kernels": inv_split,
        "forward_fields_per_s": world * F / (fwd_ms * 1e-3), "inverse_fields_per_s": world * F / (inv_ms * 1e-3),
        "round_trip_rel_err": rt_err,
        "roofline": roof,
        "e2e": {"value": world * F / (e2e_ms * 1e-3), "unit": "fields/s", "h2d_bytes_per_step": io_bytes,
                "d2h_bytes_per_step": io_bytes, "ms_per_step": e2e_ms, "chunks_per_step": e2e_chunks},
        "gpu_launches": launches,
        "clocks": clk,
        "plan": {"t_factor_s": st["t_factor_s"], "t_create_s": t_plan, "threads": st["threads"],
                 "entries_total": st["entries_total"], "entries_matrix": st["entries_matrix"],
                 "factor_bytes": st["factor_bytes"], "n_ops": st["n_ops"],
                 "blocks": {"idbf": st["n_blocks_idbf"], "lowrank": st["n_blocks_lowrank"],
                            "dense": st["n_blocks_dense"], "dropped": st["n_blocks_dropped"]},
                 "max_rank": st["max_rank"]},
    }
    if rank == 0 and world == 1 and not args.no_compare:
        line["compare"] = compare(torch, sht, _lib, w, plan, beta, g, args, stream)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the oracle's forward outputs of the timed sample double as a parity
        # check of this run's forward ALT of field 0 at those orders
        plan.forward(beta, out=g)
        torch.cuda.synchronize()
        g0 = g[0].cpu().numpy()
        dt, frac, errs = oracle_sample(N, beta_h[0], args.ref_stride, g_check=g0)
        import oracle
        line["cpu_baseline"] = {
            "value": frac / dt, "unit": "fields/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"forward+inverse ALT of every {args.ref_stride}th order |m| of 1 field "
                      f"({frac:.3f} of the transform, {dt:.1f} s), scaled to one field"}
        line["rel_err_vs_oracle"] = {
            "forward_max_per_order": float(max(errs)), "forward_median_per_order": float(np.median(errs)),
            "orders": len(errs), "field": 0,
            "what": "per-order relative l2 error of this run's forward ALT against the oracle's outputs of the "
                    "timed cpu_baseline sample (every sampled order, both signs); the tests check every "
                    "field forward and inverse"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def compare(torch, sht, _lib, w, plan, beta, g, args, stream):
    """The FP64 IDBF path and the dense FP64 transform on the same GPU, one
    field each (round trip), and the headline result's error against the FP64
    IDBF path (itself within 1e-10 of the oracle, see the tests)."""
    N = w["N"]
    out = {}
    K = max(3, args.steps // 2)
    b1 = beta[:1].contiguous()
    g1 = torch.empty((1, 4 * N - 1, 2 * N, 2), dtype=torch.float64, device="cuda")
    r1 = torch.empty_like(b1)
    p64 = sht.Plan(N, 1e-12, precision=_lib.SHT_FP64)
    ms, f, i = time_steps(torch, p64, b1, g1, r1, K, 2, stream)
    out["fp64_idbf"] = {"fields_per_s": 1e3 / ms, "forward_ms": f, "inverse_ms": i, "eps": 1e-12,
                        "entries": p64.stats()["entries_total"], "t_fac_s": p64.stats()["t_factor_s"]}
    ref = None
    if w["precision"] != "fp64":
        F = beta.shape[0]
        ref = torch.empty_like(g)
        p64.forward(beta, out=ref)
        plan.forward(beta, out=g)
        torch.cuda.synchronize()
        d = (g - ref).reshape(F, -1).norm(dim=1) / ref.reshape(F, -1).norm(dim=1)
        out["rel_err_vs_fp64_idbf"] = {"max": float(d.max()), "median": float(d.median()),
                                       "fields": F, "per_field": [float(v) for v in d.tolist()]}
        # like against like: the unfactored O(N^3) transform on the same
        # tensor-core kernels and precision, same fields, same step
        F = beta.shape[0]
        pdm = sht.Plan(N, w["eps"], precision=_lib.SHT_MIXED, flags=_lib.SHT_FLAG_DENSE, max_fields=F)
        back2 = torch.empty_like(beta)
        med, mean = time_graph(torch, pdm, beta, g, back2, K, 2, stream)
        pdm.forward(beta, out=g)
        torch.cuda.synchronize()
        pdm.sync()
        d = (g - ref).reshape(F, -1).norm(dim=1) / ref.reshape(F, -1).norm(dim=1)
        st = pdm.stats()
        out["dense_mixed"] = {"fields_per_s": F / (med * 1e-3), "ms_per_step": med, "ms_per_step_mean": mean,
                              "entries": st["entries_total"], "image_bytes": st["factor_bytes"],
                              "rel_err_vs_fp64_idbf_max": float(d.max()),
                              "what": "SHT_FLAG_DENSE plan, same tensor-core kernels, same 64 fields, "
                                      "forward + inverse, median of CUDA-graph replays"}
        del pdm, back2, ref
        torch.cuda.empty_cache()
    out["sht"] = sht_timings(torch, w, plan, beta, g, K, stream, p64=p64)
    del p64
    pd = sht.Plan(N, 1e-12, precision=_lib.SHT_FP64, flags=_lib.SHT_FLAG_DENSE)
    ms, f, i = time_steps(torch, pd, b1, g1, r1, K, 2, stream)
    out["dense_fp64"] = {"fields_per_s": 1e3 / ms, "forward_ms": f, "inverse_ms": i,
                         "entries": pd.stats()["entries_total"], "t_mat_s": pd.stats()["t_factor_s"]}
    del pd
    # the dense FP64 transform with the recurrence on the fly (nothing stored),
    # on 16 fields: its GEMM tiles take 64 right-hand sides, 4 per field
    F16 = min(16, beta.shape[0])
    b16 = beta[:F16].contiguous()
    g16 = torch.empty((F16, 4 * N - 1, 2 * N, 2), dtype=torch.float64, device="cuda")
    r16 = torch.empty_like(b16)
    pdd = sht.Plan(N, 1e-12, precision=_lib.SHT_FP64, flags=_lib.SHT_FLAG_DIRECT, max_fields=F16)
    ms, f, i = time_steps(torch, pdd, b16, g16, r16, 1, 1, stream)
    out["dense_direct_fp64"] = {"fields_per_s": F16 * 1e3 / ms, "forward_ms": f, "inverse_ms": i, "fields": F16,
                                "round_trip_rel_err": float((r16 - b16).norm() / b16.norm()),
                                "tflops": 2 * 2 * 2 * N ** 3 * 4 * F16 / ms / 1e9,
                                "what": "SHT_FLAG_DIRECT plan: Legendre recurrence on the fly, FP64, nothing stored"}
    del pdd, b16, g16, r16
    torch.cuda.empty_cache()
    # the paper's speedup ratios (its last experiment), FP64 on both sides: the
    # dense transform's time over the IDBF apply's, and building the dense
    # matrices over factoring them
    fp, dn = out["fp64_idbf"], out["dense_fp64"]
    out["paper_ratios"] = {"t_dir_over_t_app": (dn["forward_ms"] + dn["inverse_ms"]) / (fp["forward_ms"] + fp["inverse_ms"]),
                           "t_mat_over_t_fac": dn["t_mat_s"] / fp["t_fac_s"] if fp["t_fac_s"] > 0 else None}
    return out


def sht_timings(torch, w, plan, beta_in, g, K, stream, p64=None):
    """The phi-direction DFT (synthesis + analysis) and the full SHT (ALT + DFT,
    both directions) of the same F fields, and cuFFT of the same batch of
    length-(4N-1) transforms as comparators, precision against precision: the
    plan's FP32 DFT against complex64 cuFFT, the FP64 plan's DFT against
    complex128 cuFFT (cuFFT without the half-sample shift and the transpose:
    a lower bound on a library DFT of this layout)."""
    N, F = w["N"], g.shape[0]
    f = torch.empty((F, 2 * N, 4 * N - 1, 2), dtype=torch.float64, device="cuda")
    g2 = torch.empty_like(g)
    beta = torch.empty_like(beta_in)

    def timed(fn):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(K):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / K

    phi_ms = timed(lambda: (plan.phi_synthesis(g, out=f), plan.phi_analysis(f, out=g2)))
    phi_err = float((g2 - g).norm() / g.norm())
    sht_ms = timed(lambda: (plan.sht_forward(beta_in, out=f), plan.sht_inverse(f, out=beta)))
    plan.sync()
    sht_err = float((beta - beta_in).norm() / beta_in.norm())
    gc = torch.view_as_complex(g)
    fft128_ms = timed(lambda: (torch.fft.ifft(gc, dim=1), torch.fft.fft(gc, dim=1)))
    g64 = gc.to(torch.complex64)
    fft64_ms = timed(lambda: (torch.fft.ifft(g64, dim=1), torch.fft.fft(g64, dim=1)))
    del g64
    # like against like: the library calls' own contract (FP64 g in the order
    # storage sequence -> FP64 theta-major f and back, half-sample shift
    # included) done with torch operations around complex64 cuFFT
    lib_ms, lib_err = torch_phi_same_contract(torch, N, g, f, timed)
    phi_bytes = 2 * 2 * g.numel() * 8  # each direction reads and writes F x (4N-1) x 2N complex FP64
    out = {"phi_round_trip_ms": phi_ms, "phi_round_trip_rel_err": phi_err,
           "phi_GBps": phi_bytes / (phi_ms * 1e-3) / 1e9,
           "phi_hbm_frac": phi_bytes / (phi_ms * 1e-3) / 1e9 / measured_peaks()["hbm"],
           "sht_round_trip_ms": sht_ms, "sht_fields_per_s": F / (sht_ms * 1e-3),
           "sht_round_trip_rel_err": sht_err,
           "phi_arith": "f64" if w["precision"] == "fp64" else "f32",
           "cufft_c64_round_trip_ms": fft64_ms, "cufft_c128_round_trip_ms": fft128_ms,
           "torch_cufft_c64_same_contract_round_trip_ms": lib_ms,
           "torch_cufft_c64_same_contract_vs_ours_rel_diff": lib_err}
    if p64 is not None and w["precision"] != "fp64":
        # the FP64 plan's own phi transform on the same batch, against complex128 cuFFT
        phi64_ms = timed(lambda: (p64.phi_synthesis(g, out=f), p64.phi_analysis(f, out=g2)))
        p64.sync()
        out["phi_fp64_round_trip_ms"] = phi64_ms
        out["phi_fp64_round_trip_rel_err"] = float((g2 - g).norm() / g.norm())
    return out


def torch_phi_same_contract(torch, N, g, f_ours, timed):
    """The phi round trip with the library's layouts and half-sample shift,
    written with torch operations around complex64 cuFFT (reorder the orders
    to DFT positions, shift, transpose, inverse FFT, FP64 out; and back):
    returns (ms per round trip, relative difference of its synthesis from
    ours)."""
    import math
    M, K = 4 * N - 1, 2 * N
    dev = g.device
    ms = torch.arange(-(K - 1), K, device=dev)
    slot = torch.where(ms == 0, torch.zeros_like(ms), torch.where(ms > 0, 2 * ms - 1, -2 * ms))
    pos = torch.remainder(ms, M)
    by_pos = torch.argsort(pos)                 # natural-order index of the order at DFT position j
    slot_at_pos = slot[by_pos]
    ang = math.pi * ms.to(torch.float64) / M
    shift = torch.polar(torch.ones_like(ang), ang).to(torch.complex64)
    shift_at_pos = shift[by_pos]
    pos_at_slot = torch.empty_like(pos)
    pos_at_slot[slot] = pos                     # DFT position of the order in storage slot s
    cshift_at_slot = torch.empty_like(shift)
    cshift_at_slot[slot] = shift.conj() / M
    out = {}

    def syn():
        x = torch.view_as_complex(g).to(torch.complex64).index_select(1, slot_at_pos) * shift_at_pos[None, :, None]
        y = torch.fft.ifft(x.transpose(1, 2).contiguous(), dim=2, norm="forward")
        out["f"] = torch.view_as_real(y.to(torch.complex128))

    def ana():
        y = torch.fft.fft(torch.view_as_complex(out["f"]).to(torch.complex64), dim=2)
        z = y.index_select(2, pos_at_slot) * cshift_at_slot[None, None, :]
        out["g"] = torch.view_as_real(z.transpose(1, 2).contiguous().to(torch.complex128))

    ms_rt = timed(lambda: (syn(), ana()))
    syn()
    err = float((out["f"] - f_ours).norm() / f_ours.norm())
    out.clear()
    torch.cuda.empty_cache()
    return ms_rt, err


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return {"hbm": float(d["hbm_gbs"]), "bf16": float(d["bf16_tflops"]),
                "bf16_sustained": float(d["bf16_tflops_sustained"]), "source": "measured"}
    except (OSError, ValueError, KeyError):
        return {"hbm": 6800.0, "bf16": 1900.0, "bf16_sustained": 1700.0, "source": "fallback"}


def roofline(plan, w, F, flops, fwd_ms, main_ms, out_ms):
    """Roofline of the dominant kernel (the forward block-product kernel, timed
    with the library's CUDA events on the launching stream): algorithmic FLOPs
    and bytes per launch.  For the tensor-core path the kernel's time includes
    its pre-gather (one event pair brackets both), and the forward apply as a
    whole (those plus the output kernel) is reported under "apply"."""
    N = w["N"]
    beta_bytes = F * 4 * N * N * 16          # FP64 complex coefficients
    g_bytes = F * (4 * N - 1) * 2 * N * 16  # FP64 complex values at the nodes
    io_bytes = beta_bytes + g_bytes
    prec = w["precision"]
    t = main_ms * 1e-3
    if prec == "fp64":
        kname, peak, src = "alt_forward_f64_kernel", FP64_PEAK_GFLOPS, \
            "GB300 nominal FP64 1.25 TFLOP/s (FMA-chain probe: 1.197)"
        ops = plan.program(parts=("ops",))["ops"]
        fac = int((ops["ld"].astype(np.int64) * ops["ni"]).sum()) * 8
        tr, tsrc = traffic_for(kname, w["name"], fac + io_bytes)
        return {"kernel": kname, "bound": "alu", "achieved": flops / t / 1e9, "peak": peak, "unit": "GFLOP/s",
                "frac": flops / t / 1e9 / peak, "traffic": tr, "traffic_source": tsrc, "kernel_ms": main_ms,
                "bytes_per_launch": fac + io_bytes, "flops_per_launch": flops, "peak_source": src}
    if prec == "fp32":
        kname, peak = "alt_forward_f32_kernel", FP32_PEAK_GFLOPS
        return {"kernel": kname, "bound": "alu", "achieved": flops / t / 1e9, "peak": peak, "unit": "GFLOP/s",
                "frac": flops / t / 1e9 / peak, "traffic": traffic_for(kname, w["name"])[0], "kernel_ms": main_ms,
                "flops_per_launch": flops,
                "peak_source": "128 FP32 lanes x 2 FLOP x 152 SMs x 2.07 GHz (FMA-chain probe: 73.2)"}
    # tensor-core split-BF16 path: each product costs 6 BF16 MMAs.  The
    # dominant kernel reads the operand images and beta once and writes the
    # accumulated FP32 node values (Y: 4 real right-hand sides x 4 bytes per
    # node, order and field); the output kernel turns those into g.
    pk = measured_peaks()
    ops = plan.program(parts=("ops",))["ops"]
    # algorithmic factor bytes: 6 bytes (three BF16 pieces) per stored entry,
    # with no tile padding or group widening
    img = 6 * int((ops["mo"].astype(np.int64) * ops["ni"].astype(np.int64)).sum())
    y_bytes = F * 2 * N * 2 * N * 16
    algo_bytes = img + beta_bytes + y_bytes
    tens_peak = pk["bf16_sustained"] / 6.0 * 1e3  # GFLOP/s of FP32-quality split products
    t_frac = flops / t / 1e9 / tens_peak
    h_frac = algo_bytes / t / 1e9 / pk["hbm"]
    kname = "alt_tc_kernel"
    tr, tsrc = traffic_for(kname, w["name"], algo_bytes)
    apply_bytes = img + io_bytes
    base = {"kernel": kname, "kernel_ms": main_ms,
            "kernel_ms_covers": "the pre-gather (tc_in_kernel) and alt_tc_kernel, timed together by the library's "
                                "events: the algorithmic work is charged to both",
            "traffic": tr, "traffic_source": tsrc,
            "traffic_over_algorithmic": (tr / algo_bytes) if tr else None, "flops_per_launch": flops,
            "bytes_per_launch": algo_bytes, "factor_image_bytes": img,
            "factor_image_bytes_stored_both_directions": plan.stats()["factor_bytes"],
            "beta_bytes": beta_bytes, "y_bytes": y_bytes,
            "apply": {"kernels": "tc_in_kernel + alt_tc_kernel + tc_out_kernel", "ms": fwd_ms, "output_kernel_ms": out_ms,
                      "bytes": apply_bytes, "GBps": apply_bytes / (fwd_ms * 1e-3) / 1e9,
                      "hbm_frac": apply_bytes / (fwd_ms * 1e-3) / 1e9 / pk["hbm"]}}
    if t_frac >= h_frac:
        return {**base, "bound": "tensor", "achieved": flops / t / 1e12, "peak": tens_peak / 1e3, "unit": "TFLOP/s",
                "frac": t_frac, "peak_source": f"{pk['source']} bf16 sustained {pk['bf16_sustained']} TFLOP/s / 6 "
                                               f"MMAs per split product; HBM frac {h_frac:.3f}"}
    return {**base, "bound": "hbm", "achieved": algo_bytes / t / 1e9, "peak": pk["hbm"], "unit": "GB/s",
            "frac": h_frac, "peak_source": f"{pk['source']} HBM copy {pk['hbm']} GB/s; tensor frac {t_frac:.3f}"}


def traffic_for(kernel, workload_name, algo_bytes=None):
    """DRAM bytes per launch of `kernel` from a committed ncu capture (profiles/traffic.json).

    A capture of the same workload is used as it is; otherwise a capture of a
    smaller case of the same kernel is scaled by the ratio of algorithmic bytes
    (traffic assumed proportional), and the source says so.
    """
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            table = json.load(fh).get(kernel, {})
    except (OSError, ValueError):
        return None, None
    if workload_name in table:
        return table[workload_name], f"ncu capture of {workload_name}"
    ref_name = TRAFFIC_REF.get(workload_name)
    if algo_bytes and ref_name in table and table.get("_algorithmic_" + ref_name):
        return (algo_bytes * table[ref_name] / table["_algorithmic_" + ref_name],
                f"ncu capture of {ref_name}, scaled by algorithmic bytes")
    if algo_bytes:
        for w, v in table.items():
            ref = table.get("_algorithmic_" + w)
            if not w.startswith("_") and ref:
                return algo_bytes * v / ref, f"ncu capture of {w}, scaled by algorithmic bytes"
    return None, None


UNEVEN_PREFIX = "uneven_"


def uneven_sizes(name):
    """'uneven_N128-1024_F256' -> ((128, 256, 512, 1024), 256): powers of two from the first to the last N."""
    body = name[len(UNEVEN_PREFIX):]
    ns, fs = body.split("_F")
    lo, hi = (int(v) for v in ns.lstrip("N").split("-"))
    sizes = []
    n = lo
    while n <= hi:
        sizes.append(n)
        n *= 2
    return tuple(sizes), int(fs)


def run_uneven(args):
    """One step = forward + inverse ALT of an uneven batch (fields of several
    orders N, one plan per N) in one tensor-core launch per direction, through
    alt_forward_batch / alt_inverse_batch.  Compared with the same fields run
    plan by plan (one launch per plan and direction)."""
    import torch
    import paper_2004_11346_gb300 as sht
    from paper_2004_11346_gb300 import _lib

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    sizes, F = uneven_sizes(args.workload)
    eps = 1e-7
    per_field, coeffs = inputs.uneven_batch(F, seed=1 + rank, sizes=sizes)
    Ns = sorted(coeffs)
    t0 = time.perf_counter()
    plans = [sht.Plan(N, eps, precision=_lib.SHT_MIXED, max_fields=coeffs[N].shape[0]) for N in Ns]
    t_plan = time.perf_counter() - t0
    counts = [coeffs[N].shape[0] for N in Ns]
    batch = sht.Batch(plans, counts)
    betas = [torch.from_numpy(coeffs[N]).cuda() for N in Ns]
    gs = [torch.empty((c, 4 * N - 1, 2 * N, 2), dtype=torch.float64, device="cuda") for N, c in zip(Ns, counts)]
    backs = [torch.empty_like(b) for b in betas]
    bptr, gptr, kptr = [b.data_ptr() for b in betas], [g.data_ptr() for g in gs], [k.data_ptr() for k in backs]
    stream = torch.cuda.current_stream()

    def step_batch():
        _lib.alt_forward_batch(batch.handle, bptr, gptr, stream.cuda_stream)
        _lib.alt_inverse_batch(batch.handle, gptr, kptr, stream.cuda_stream)

    def step_plans():
        for p, b, g, k in zip(plans, betas, gs, backs):
            p.forward(b, out=g)
            p.inverse(g, out=k)

    def timed(fn, steps):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        clock = ClockSampler(torch.cuda.current_device())
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        clk = clock.stop()
        ms = e0.elapsed_time(e1) / steps
        return reduce_max([ms], world, device="cuda")[0], clk

    ms_b, clk = timed(step_batch, args.steps)
    batch.sync()
    err = []
    for b, k in zip(betas, backs):
        d = (k - b).reshape(k.shape[0], -1).norm(dim=1) / b.reshape(b.shape[0], -1).norm(dim=1)
        err.append(float(d.max()))
    ms_p, _ = timed(step_plans, max(1, args.steps // 2))
    value = F * world / (ms_b * 1e-3)
    line = {
        "metric": METRIC, "value": value, "unit": "fields/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_b, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16x3 split, f32 accumulate", "data": "synthetic",
        "config": {"workload": args.workload, "sizes": list(Ns), "fields_per_size": counts, "fields_per_rank": F,
                   "global_batch": F * world, "eps": eps, "precision": "mixed",
                   "step": "forward ALT + inverse ALT of the whole batch, one tensor-core launch per direction",
                   "parallelism": f"replicas{world}"},
        "round_trip_rel_err_max_per_size": dict(zip([str(n) for n in Ns], err)),
        "plan_by_plan": {"ms_per_step": ms_p, "fields_per_s": F * world / (ms_p * 1e-3),
                         "launches_per_direction": 2 * len(Ns)},
        "plan_s": t_plan, "clocks": clk, "roofline": None, "cpu_baseline": None,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_only(args):
    """One component on the workload's N and F, for profiling captures and
    component timings (not the benchmark line): "phi", the phi-direction
    synthesis then analysis of F random grids in the plan precision's
    arithmetic; "direct", the forward then inverse ALT of the on-the-fly dense
    FP64 transform.  Prints one JSON line."""
    import torch
    import paper_2004_11346_gb300 as sht
    from paper_2004_11346_gb300 import _lib
    w = workload(args.workload)
    N, F = w["N"], w["F"]
    prec = _lib.SHT_FP64 if args.only == "direct" or w["precision"] == "fp64" else _lib.SHT_MIXED
    plan = sht.Plan(N, w["eps"], precision=prec, flags=_lib.SHT_FLAG_DIRECT, max_fields=F)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(w["seed"])
    if args.only == "phi":
        a = torch.randn((F, 4 * N - 1, 2 * N, 2), dtype=torch.float64, device="cuda", generator=gen)
        b = torch.empty((F, 2 * N, 4 * N - 1, 2), dtype=torch.float64, device="cuda")
        back = torch.empty_like(a)

        def step():
            plan.phi_synthesis(a, out=b)
            plan.phi_analysis(b, out=back)
    else:
        a = torch.from_numpy(rank_fields(N, F, w, 0)).cuda()
        b = torch.empty((F, 4 * N - 1, 2 * N, 2), dtype=torch.float64, device="cuda")
        back = torch.empty_like(a)

        def step():
            plan.forward(a, out=b)
            plan.inverse(b, out=back)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / max(1, args.steps)
    print(json.dumps({"component": args.only, "workload": args.workload, "N": N, "fields": F, "ms_per_step": ms,
                      "fields_per_s": F / (ms * 1e-3), "round_trip_rel_err": float((back - a).norm() / a.norm())}),
          flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--ref-stride", type=int, default=8, help="oracle samples every n-th order")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-compare", action="store_true", help="skip the FP64 IDBF and dense comparators")
    ap.add_argument("--n0", type=int, default=None, help="override the workload's partition stop size n0")
    ap.add_argument("--n-leaf", type=int, default=None, help="override the workload's IDBF leaf size")
    ap.add_argument("--e2e-chunk", type=int, default=None,
                    help="fields per host-copy chunk of the end-to-end loop (default 32)")
    ap.add_argument("--only", choices=["phi", "direct"], default=None,
                    help="time one component on the workload's N and fields instead of the benchmark step")
    args = ap.parse_args()
    if args.only:
        run_only(args)
    elif args.impl == "reference":
        run_reference(args)
    elif args.workload.startswith(UNEVEN_PREFIX):
        run_uneven(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
