"""Benchmark: encrypted 64x64 matrix products per second (the paper's packed
O(h)-rotation HE-MatMult, Alg. 3 with App. B/E) on one GB300, batched.

Workload (one step): 32 independent 64x64 FP64 products, packed two per
ciphertext pair (beta = 2), i.e. 16 ciphertext pairs in one batched call;
CKKS N = 2^14, Q = 1x60 + 7x45 bits, P = 2x60 bits, scale 2^45, matrix
entries uniform in [-1, 1] from fixed seeds.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl hx|reference]

--impl reference times the CPU oracle (oracle/) on the host cores on the
same workload, one ciphertext pair (two products) per step.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import re
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

LOG_N, Q_BITS, P_BITS, LOG2_SCALE = 14, [60] + [45] * 7, [60, 60], 45
H, PAIRS = 64, 16
N_SLOTS = (1 << LOG_N) // 2
BETA = N_SLOTS // (H * H)
PRODUCTS = PAIRS * BETA
METRIC = "encrypted 64x64 matmuls/s (batched HE-MatMult, CKKS N=2^14)"
# The 64-bit modular-multiply ceiling of the GB300 (the ALU roofline of the NTT): 152 SMs x 4
# sub-partitions at the 2070 MHz maximum SM clock, each sub-partition's FMA-heavy pipe finishing
# one lane's 64-bit Shoup product y*w - floor(y*w'/2^64)*q per cycle (a warp-wide product issues
# 10 instructions on that pipe and holds it 32 cycles: ncu pipe counters on the calibration kernel)
GPU_SMS, GPU_SUBPARTITIONS, GPU_MAX_SM_MHZ, SHOUP_PIPE_CYCLES_PER_WARP = 152, 4, 2070, 32
ALU_PEAK_SHOUP = GPU_SMS * GPU_SUBPARTITIONS * GPU_MAX_SM_MHZ * 1e6 * 32 / SHOUP_PIPE_CYCLES_PER_WARP
ALU_PEAK_KIND = ("derived: 152 SMs x 4 sub-partitions x 2070 MHz x 32 lanes / 32 FMA-heavy pipe cycles per "
                 "warp-wide 64-bit Shoup product")
WORKLOAD = ("cfg1: %d independent 64x64 products per step = %d ciphertext pairs x beta=%d packed products; "
            "CKKS N=2^14, Q=1x60+7x45 bit, P=2x60 bit, scale 2^45, entries U[-1,1] seeded" % (PRODUCTS, PAIRS, BETA))


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def sha_of(path):
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def ntt_kernels_sha():
    """Hash of the source of the per-ring NTT phase kernels: ntt.cu without its marked
    several-ring sections (kernels and launcher, which those phase kernels do not use) and without
    its marked host launcher and autotuner (which pick and time the kernels, changing none)."""
    with open(os.path.join(ROOT, "paper_2207_04620_gb300", "csrc", "ntt.cu")) as f:
        src = f.read()
    src = re.sub(r"// ---- several rings in one launch.*?// ---- end of the several-ring kernels\n\n", "", src,
                 flags=re.S)
    src = re.sub(r"// ---- several rings: launcher\n.*?// ---- end of the several-ring launcher\n\n", "", src,
                 flags=re.S)
    src = re.sub(r"// ---- autotuner[^\n]*\n.*?// ---- end of the autotuner\n\n", "", src, flags=re.S)
    src = re.sub(r"// ---- launcher[^\n]*\n.*?// ---- end of the launcher\n\n", "", src, flags=re.S)
    return hashlib.sha256(src.encode()).hexdigest()[:16]


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid=None):
        self.proc = None
        cmd = ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits", "-lms", "200"]
        if uuid:
            cmd[1:1] = ["-i", uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---- CPU oracle (baseline leg and reference arm) -----------------------------------------

def oracle_setup():
    from oracle import ckks as C
    from oracle import hercules as Hc
    from paper_2207_04620_gb300 import workloads

    octx = C.Context(LOG_N, Q_BITS, P_BITS, LOG2_SCALE)
    steps = Hc.matmul_rotation_steps(H, BETA, len(Q_BITS))
    oks = C.keygen(octx, 2, 2024, rot_steps=steps)
    masks = Hc.MaskProvider(octx, H, len(Q_BITS))
    for i in range(len(masks.entries)):
        masks.coeffs(i)
    a = C.encrypt(octx, oks, workloads.pack(workloads.matrices(100, BETA, H), H, BETA), 1)
    b = C.encrypt(octx, oks, workloads.pack(workloads.matrices(200, BETA, H), H, BETA), 2)
    return octx, oks, masks, a, b


def oracle_step(state):
    from oracle import ckks as C
    from oracle import hercules as Hc

    octx, oks, masks, a, b = state
    t0 = time.perf_counter()
    Hc.matmul(C.Evaluator(octx, oks), a, b, H, masks)
    return time.perf_counter() - t0


def cpu_cores():
    return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


def run_reference(args, world, rank):
    if rank != 0:
        return
    state = oracle_setup()
    for _ in range(args.warmup):
        oracle_step(state)
    ts = [oracle_step(state) for _ in range(args.steps)]
    t = sum(ts) / len(ts)
    value = BETA / t
    sample = "one ciphertext pair (%d packed 64x64 products) per step through the oracle's full Alg. 3 schedule" % BETA
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "matmul/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": sample},
            "cpu_baseline": {"value": value, "unit": "matmul/s", "cores": cpu_cores(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "matmul/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---- GPU arm ----------------------------------------------------------------------------

def other_metrics(args):
    """The rest of the headline metric in compact, time-bounded form, each with its own clocks:
    the NTT alone (N=2^14, 1600 limbs, forward and inverse GB/s), the config-2 composite sign
    (64 ciphertexts, 3 timed steps) and a short serving stream (300 requests at 0.8x capacity).
    A record that fails carries its error instead, so the headline line is still printed."""
    out = {}

    def ntt_micro():
        ns = argparse.Namespace(**vars(args))
        ns.log_n, ns.rows, ns.steps, ns.warmup, ns.tiles, ns.reps = 14, 1600, 5, 3, None, 200
        m = run_micro(ns)
        r = {k: (round(v, 4) if isinstance(v, float) else v) for k, v in m.items()
             if k in ("log_n", "rows", "tiles", "fwd_ms", "inv_ms", "fwd_gbs", "inv_gbs", "fwd_frac", "inv_frac",
                      "fwd_alu_frac", "inv_alu_frac", "fwd_calibrated_frac", "inv_calibrated_frac", "peak_gbs",
                      "peak_kind", "clocks")}
        r["what"] = "forward / inverse NTT of 1600 limbs of N=2^14 (210 MB, > L2) in place; " \
                    "CUDA events around 200 transforms per direction, median of 5 steps"
        return r

    def sign_cfg2():
        ns = argparse.Namespace(**vars(args))
        ns.steps, ns.warmup, ns.relu, ns.alpha = 3, 1, False, None
        sg = run_sign(ns)
        r = {k: sg[k] for k in ("value", "unit", "ms_per_step", "steps", "max_err_vs_exact",
                                "max_err_vs_fp64_composite", "clocks", "kernel_shares")}
        r["what"] = sg["metric"] + "; " + sg["config"]["workload"]
        return r

    def serve():
        ns = argparse.Namespace(**vars(args))
        ns.requests, ns.load, ns.lanes, ns.max_batch, ns.full, ns.sweep = 300, 0.8, 4, 16, False, False
        sv = run_serve(ns)
        return {"p50_ms": sv["value"], "p99_ms": sv["p99_ms"], "throughput_req_s": sv["throughput_req_s"],
                "offered_req_s": sv["offered_req_s"], "capacity_req_s": sv["capacity_req_s"],
                "requests": sv["requests"], "clocks": sv["clocks"], "what": "serving stream, " + sv["config"]["workload"]}

    for name, fn in (("ntt_micro", ntt_micro), ("sign_cfg2", sign_cfg2), ("serve", serve)):
        try:
            out[name] = fn()
        except Exception as e:  # noqa: BLE001 -- reported on the line, the headline stands
            out[name] = {"error": "%s: %s" % (type(e).__name__, e)}
            print("bench: %s failed: %s" % (name, e), file=sys.stderr, flush=True)
    return out


def run_hx(args, world, rank, local):
    import torch

    from paper_2207_04620_gb300 import hx, workloads

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if rank == 0:
        import __graft_entry__

        __graft_entry__.build()
    barrier(world)
    stream = torch.cuda.current_stream()
    ctx = hx.hx_context_create(LOG_N, Q_BITS, P_BITS, LOG2_SCALE)
    if args.tiles is None:
        tiles = hx.hx_autotune(ctx, stream=torch.cuda.current_stream())
    else:  # fixed NTT variants for every batch size (signed widths per phase)
        tiles = hx.hx_ntt_tiles(ctx, [int(t) for t in args.tiles.split(",")])
    ntt_tuning = hx.hx_ntt_tuning(ctx)  # variants per batch-size bucket and phase
    limbs = len(Q_BITS)
    steps = hx.hx_matmul_rotation_steps(ctx, H, limbs)
    ks = hx.hx_keygen(ctx, 2, 2024 + rank, steps)
    plan = hx.hx_matmul_plan_create(ctx, H, limbs)
    hx.hx_matmul_plan_bind_keys(ctx, plan, ks)  # Step 2 selection folded into the rotation keys
    premasked_bytes = hx.hx_matmul_plan_bound_bytes(plan)
    mats_a = [workloads.matrices(1000 * rank + 2 * i, BETA, H) for i in range(PAIRS)]
    mats_b = [workloads.matrices(1000 * rank + 2 * i + 1, BETA, H) for i in range(PAIRS)]
    A = [hx.hx_encrypt(ctx, ks, workloads.pack(m, H, BETA), 0, 10 + i) for i, m in enumerate(mats_a)]
    B = [hx.hx_encrypt(ctx, ks, workloads.pack(m, H, BETA), 0, 50 + i) for i, m in enumerate(mats_b)]
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2

    def step():
        outs = hx.hx_matmul_batch(ctx, ks, plan, A, B, H, stream=stream)
        return outs

    def drop(outs):
        for o in outs:
            hx.hx_ct_destroy(o)

    props = torch.cuda.get_device_properties(dev)
    sampler = ClockSampler(getattr(props, "uuid", None) and "GPU-" + str(props.uuid))
    for _ in range(args.warmup):
        drop(step())
    torch.cuda.synchronize()
    # accuracy of one output pair against FP64
    outs = step()
    got = workloads.unpack(hx.hx_decrypt(ctx, ks, outs[0]), H, BETA)
    max_err = float(max(np.abs(g - a @ b).max() for g, a, b in zip(got, mats_a[0], mats_b[0])))
    drop(outs)

    # the batched schedule captured once into a CUDA graph; timed region: its replays,
    # events on the launching stream, L2 flushed between steps
    scale_in = hx.hx_ct_info(A[0])[2]
    ex = hx.hx_matmul_exec_create(ctx, ks, plan, PAIRS, scale_in)
    graph_launches = hx.hx_matmul_exec_launches(ex)
    for _ in range(2):
        drop(hx.hx_matmul_exec_run(ex, A, B, stream=stream))
    c0 = hx.hx_counters(ctx)
    times = []
    for _ in range(args.steps):
        flush.zero_()
        barrier(world)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push("timed")
        e0.record(stream)
        outs = hx.hx_matmul_exec_run(ex, A, B, stream=stream)
        e1.record(stream)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
        drop(outs)
    c1 = hx.hx_counters(ctx)
    clocks = sampler.stop()
    ms = sum(times) / len(times)
    ms_max = max_over_ranks(ms, world)
    value = PRODUCTS * world / (ms_max / 1e3)
    launches = (c1["launches"] - c0["launches"])

    # the same step as one plain batched call (no graph)
    p_times = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        outs = step()
        e1.record(stream)
        torch.cuda.synchronize()
        p_times.append(e0.elapsed_time(e1))
        drop(outs)
    plain_ms = max_over_ranks(sum(p_times) / len(p_times), world)

    # live per-kernel timing (profiling pass over the same step, events on the launching stream)
    hx.hx_profile_enable(ctx, True)
    flush.zero_()
    torch.cuda.synchronize()
    drop(step())
    prof = hx.hx_profile_read(ctx)
    hx.hx_profile_enable(ctx, False)
    total_ms = sum(v[1] for v in prof.values())
    shares = {k: round(v[1] / total_ms, 4) for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])}
    dom = max(prof, key=lambda k: prof[k][1])
    n_launch, dom_ms, dom_bytes = prof[dom]
    achieved = dom_bytes / (dom_ms / 1e3) / 1e9
    peak, peak_kind = peaks()
    traffic = None
    tfile = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tfile):
        with open(tfile) as f:
            tj = json.load(f)
        ent = tj.get(dom)
        if ent and ent.get("kernels_sha") == ntt_kernels_sha():
            # captured on a smaller launch of the same kernel; traffic grows with the residues processed
            traffic = round(ent["dram_bytes_per_alg_byte"] * dom_bytes / n_launch)
    method = ("one profiled step of the same batched schedule with its chains run one after another "
              "on the launching stream (CUDA events around every launch of a class); the timed graph "
              "overlaps the chains, so these are per-kernel speeds, not shares of the graph's time; "
              "traffic: ncu DRAM bytes per algorithmic byte of the NTT phase kernels "
              "(profiles/traffic.json) times this launch's algorithmic bytes")
    hbm = {"achieved": round(achieved, 1), "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
           "peak_kind": peak_kind, "alg_bytes_per_launch": dom_bytes / n_launch}
    if dom == "ntt":
        # bound by its 64-bit integer multiplies, not by HBM: one Shoup product per butterfly,
        # log2(N)/32 butterflies per algorithmic byte (N/2 log2 N butterflies per 16 N bytes)
        shoup_s, mac_s = hx.hx_alu_calibrate(ctx, stream=stream)
        bfly_s = achieved * 1e9 * LOG_N / 32.0
        roofline = {"bound": "alu", "kernel": dom, "achieved": round(bfly_s / 1e9, 1),
                    "peak": round(ALU_PEAK_SHOUP / 1e9, 1), "unit": "G Shoup products/s (one per butterfly)",
                    "frac": round(bfly_s / ALU_PEAK_SHOUP, 4), "traffic": traffic, "peak_kind": ALU_PEAK_KIND,
                    "launches": n_launch, "avg_launch_us": round(dom_ms / n_launch * 1e3, 2),
                    "alg_butterflies_per_launch": dom_bytes / n_launch * LOG_N / 32.0,
                    "hbm": hbm,
                    "calibrated": {"shoup_products_per_s": round(shoup_s / 1e9, 1), "unit": "G/s",
                                   "frac": round(bfly_s / shoup_s, 4), "mac128_per_s": round(mac_s / 1e9, 1),
                                   "what": "measured on this GPU by hx_alu_calibrate (8 independent chains "
                                           "per thread)"},
                    "method": method}
    else:
        roofline = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                    "frac": round(achieved / peak, 4), "traffic": traffic, "peak_kind": peak_kind,
                    "launches": n_launch, "avg_launch_us": round(dom_ms / n_launch * 1e3, 2),
                    "alg_bytes_per_launch": dom_bytes / n_launch, "method": method}
    # every kernel class of the step against the same HBM peak (algorithmic bytes of its
    # launches / their event-timed duration), the key-switching classes among them
    class_roofline = {c: {"launches": v[0], "ms": round(v[1], 3), "gbs": round(v[2] / (v[1] / 1e3) / 1e9, 1),
                          "frac": round(v[2] / (v[1] / 1e3) / 1e9 / peak, 4)}
                      for c, v in sorted(prof.items(), key=lambda kv: -kv[1][1]) if v[1] > 0 and v[2] > 0}

    # end to end through the C ABI with host buffers: every step copies its input
    # ciphertexts from page-locked host memory, replays the graph and copies its
    # products back (hx_matmul_exec_run_host); two executors on two streams let one
    # batch's copies overlap the other's evaluation.  Each step streams ~2 GB of
    # Galois keys, far more than L2, so no flush is needed between steps.
    n = 1 << LOG_N
    host_a = torch.from_numpy(np.stack([hx.hx_ct_export(ctx, x) for x in A]).view(np.int64)).pin_memory()
    host_b = torch.from_numpy(np.stack([hx.hx_ct_export(ctx, x) for x in B]).view(np.int64)).pin_memory()
    ex2 = hx.hx_matmul_exec_create(ctx, ks, plan, PAIRS, scale_in)
    out_limbs, out_scale = hx.hx_matmul_exec_out_info(ex)
    execs = [ex, ex2]
    e2e_streams = [stream, torch.cuda.Stream(device=dev)]
    host_out = [torch.empty((PAIRS, 2, out_limbs, n), dtype=torch.int64).pin_memory() for _ in range(2)]
    h2d = (host_a.numel() + host_b.numel()) * 8
    d2h = host_out[0].numel() * 8

    def e2e_step(it):
        k = it % 2
        hx.hx_matmul_exec_run_host(execs[k], host_a.data_ptr(), host_b.data_ptr(), host_out[k].data_ptr(),
                                   stream=e2e_streams[k])

    for it in range(2):
        e2e_step(it)
    torch.cuda.synchronize()
    # the host copy of a product decrypts to A @ B
    chk = hx.hx_ct_import(ctx, host_out[0][0].numpy().view(np.uint64), out_scale)
    got = workloads.unpack(hx.hx_decrypt(ctx, ks, chk), H, BETA)
    e2e_err = float(max(np.abs(g - a @ b).max() for g, a, b in zip(got, mats_a[0], mats_b[0])))
    hx.hx_ct_destroy(chk)
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for it in range(args.steps):
        e2e_step(it)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks((time.perf_counter() - t0) / args.steps, world)
    hx.hx_matmul_exec_destroy(ex2)
    hx.hx_matmul_exec_destroy(ex)

    # one launch sequence per product pair (no batching) on the same GPU
    per_op_pairs = min(args.per_op_pairs, PAIRS)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(per_op_pairs):
        o = hx.hx_matmul(ctx, ks, A[i], B[i], H, stream=stream)
        torch.cuda.synchronize()
        hx.hx_ct_destroy(o)
    per_op = per_op_pairs * BETA / (time.perf_counter() - t0)

    line = None
    if rank == 0:
        line = {"metric": METRIC, "value": round(value, 2), "unit": "matmul/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": round(ms_max, 3), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
                "config": {"workload": WORKLOAD, "parallelism": "replicas only (one independent batch per GPU)",
                           "l2": "flushed between timed steps (512 MB write outside the events)",
                           "per_step_launch": "one hx_matmul_exec_run C-ABI call: the batched schedule "
                                              "(hx_matmul_batch) captured once into a CUDA graph",
                           "ntt_tiles_autotuned": tiles,
                           "ntt_tuning": ntt_tuning,
                           "step2_premasked_key_bytes": premasked_bytes},
                "e2e": {"value": round(PRODUCTS * world / e2e_s, 2), "unit": "matmul/s",
                        "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                        "what": "hx_matmul_exec_run_host per step: H2D of the 32 input ciphertexts from page-locked "
                                "memory, graph replay, D2H of the 16 product ciphertexts; two executors on two "
                                "streams, host wall clock over all steps",
                        "max_abs_err_vs_fp64": e2e_err},
                "gpu_launches": launches,
                "clocks": clocks,
                "roofline": roofline,
                "kernel_shares": shares, "class_roofline": class_roofline,
                "graph_kernel_nodes": graph_launches,
                "plain_batched": {"value": round(PRODUCTS * world / (plain_ms / 1e3), 2), "unit": "matmul/s",
                                  "ms_per_step": round(plain_ms, 3),
                                  "what": "the same step as one hx_matmul_batch call, no graph"},
                "per_op": {"value": round(per_op, 2), "unit": "matmul/s",
                           "what": "hx_matmul on one ciphertext pair per call, %d pairs, synchronised" % per_op_pairs},
                "accuracy": {"max_abs_err_vs_fp64": max_err, "bound": 2.0 ** -18}}
    hx.hx_matmul_plan_destroy(plan)
    for x in A + B:
        hx.hx_ct_destroy(x)
    hx.hx_keyset_destroy(ks)
    hx.hx_context_destroy(ctx)
    if rank == 0 and world == 1 and not args.no_extras:
        line.update(other_metrics(args))
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            state = oracle_setup()
            t = oracle_step(state)
            line["cpu_baseline"] = {"value": round(BETA / t, 4), "unit": "matmul/s", "cores": cpu_cores(),
                                    "kind": "oracle",
                                    "sample": "one ciphertext pair (%d packed products) through the oracle's Alg. 3, "
                                              "%.1f s" % (BETA, t)}
        except Exception as e:  # noqa: BLE001 -- reported on the line, the headline stands
            line["cpu_baseline"] = {"value": None, "unit": "matmul/s", "kind": "oracle",
                                    "error": "%s: %s" % (type(e).__name__, e)}
            print("bench: cpu_baseline failed: %s" % e, file=sys.stderr, flush=True)
    if line is not None:
        print(json.dumps(line), flush=True)


def g4_iter(x, k):
    """FP64 g_4^(k) with the printed g_4 = (35m^9 - 180m^7 + 378m^5 - 420m^3 + 315m)/128 (Sec. 4.2)."""
    for _ in range(k):
        y = x * x
        x = x * ((((35 * y - 180) * y + 378) * y - 420) * y + 315) / 128.0
    return x


def run_sign(args):
    """Config 2: g_4^(8) (sign, or ReLU with --relu) on 64 ciphertexts of 16384 slots each, CKKS
    N=2^15, Q = 60 + 15x40 bit, P = 3x60 bit, scale 2^40, inputs uniform in [-1,-2^-8] U [2^-8,1];
    the collective refresh (DBootstrap on the device) runs after compositions 3 and 6 and
    is inside the timed region."""
    import torch

    from paper_2207_04620_gb300 import hx, workloads

    import __graft_entry__

    __graft_entry__.build()
    log_n, qb, pb, count, d, k = 15, [60] + [40] * 15, [60] * 3, 64, 4, 8
    # digits of four 40-bit primes: products up to about P (three 60-bit primes), the
    # relinearisation noise stays far below the scale and the sign keeps its accuracy
    alpha = 4 if args.alpha is None else args.alpha
    ctx = hx.hx_context_create(log_n, qb, pb, 40, alpha=alpha)
    hx.hx_autotune(ctx)
    ks = hx.hx_keygen(ctx, 2, 77, [])
    n_slots = (1 << log_n) // 2
    xs = [workloads.sign_inputs(500 + i, n_slots) for i in range(count)]
    cts = [hx.hx_encrypt(ctx, ks, x, 0, 900 + i) for i, x in enumerate(xs)]
    stream = torch.cuda.current_stream()

    def step(seed):
        return hx.hx_sign_approx_batch(ctx, ks, cts, d, k, relu=args.relu, allow_refresh=True, refresh_seed=seed,
                                       stream=stream)

    for w in range(args.warmup):
        for o in step(w):
            hx.hx_ct_destroy(o)
    torch.cuda.synchronize()
    sampler = ClockSampler()
    times = []
    for it in range(args.steps):
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("timed")
        t0 = time.perf_counter()
        outs = step(100 + it)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
        torch.cuda.nvtx.range_pop()
        if it < args.steps - 1:
            for o in outs:
                hx.hx_ct_destroy(o)
    clocks = sampler.stop()
    t = sum(times) / len(times)
    # live per-kernel-class shares of one more step (CUDA events per launch, chains serial)
    hx.hx_profile_enable(ctx, True)
    for o in step(999):
        hx.hx_ct_destroy(o)
    prof = hx.hx_profile_read(ctx)
    hx.hx_profile_enable(ctx, False)
    total_ms = sum(v[1] for v in prof.values())
    shares = {c: round(v[1] / total_ms, 4) for c, v in sorted(prof.items(), key=lambda kv: -kv[1][1])}
    errs_sgn, errs_g = [], []
    for i in range(4):
        got = hx.hx_decrypt(ctx, ks, outs[i])
        g = g4_iter(xs[i], k)
        ref = xs[i] * (1 + g) / 2 if args.relu else g
        exact = np.maximum(xs[i], 0) if args.relu else np.sign(xs[i])
        errs_sgn.append(float(np.abs(got - exact).max()))
        errs_g.append(float(np.abs(got - ref).max()))
    for o in outs:
        hx.hx_ct_destroy(o)
    line = {"metric": "composite %s approximation, ciphertexts/s (g_4^(8), CKKS N=2^15)" % ("ReLU" if args.relu else "sign"),
            "value": round(count / t, 3), "unit": "ct/s", "slots_per_s": round(count * n_slots / t, 1),
            "ms_per_step": round(t * 1e3, 2), "steps": args.steps, "warmup": args.warmup, "n_gpus": 1,
            "higher_is_better": True, "dtype": "u64", "data": "synthetic",
            "config": {"workload": "cfg2: 64 ciphertexts x 16384 slots, |x| in [2^-8, 1], d=4, k=8, two collective "
                                   "refreshes per entry (DBootstrap shares on the device), host wall clock",
                       "primes_per_digit": alpha or 3},
            "max_err_vs_exact": max(errs_sgn), "max_err_vs_fp64_composite": max(errs_g), "clocks": clocks,
            "kernel_shares": shares, "kernel_ms_profiled": round(total_ms, 2)}
    hx.hx_keyset_destroy(ks)
    hx.hx_context_destroy(ctx)
    return line


def run_dense(args):
    """Config 3: one encrypted dense layer 784 -> 128, feedforward and backpropagation (Fig. 5),
    batch of 64 inputs, 64 x 64 blocks (2 x 13 block products, packed 4 per ciphertext: 8
    ciphertext pairs per HE-MatMult batch), ReLU by g_4^(8)(E/4), CKKS N=2^15, Q = 60 + 15x40 bit,
    P = 3x60 bit, scale 2^40; weights N(0, 0.05), inputs U[0,1], upstream gradient N(0, 0.1).
    The collective refreshes inside the composite sign are in the timed region."""
    import torch

    from paper_2207_04620_gb300 import hx, workloads

    import __graft_entry__

    __graft_entry__.build()
    cfg = workloads.CONFIGS["cfg3_dense784x128_n15"]
    h, d, k, div = cfg["h"], cfg["d"], cfg["k"], cfg["input_div"]
    ctx = hx.hx_context_create(cfg["log_n"], cfg["q_bits"], cfg["p_bits"], cfg["log2_scale"], alpha=args.alpha or 0)
    hx.hx_autotune(ctx)
    ks = hx.hx_keygen(ctx, 2, 81, hx.hx_dense_rotation_steps(ctx, h))
    beta = (1 << cfg["log_n"]) // 2 // (h * h)
    W, X, G = workloads.dense_inputs(3, cfg["rows"], cfg["n_in"], cfg["batch"])
    Wp, Xp, Gp = workloads.dense_pack(W, X, G, h, beta)
    n_out, groups = len(Wp), len(Xp)
    Wc = [hx.hx_encrypt(ctx, ks, Wp[i][g], 0, 1000 + 10 * i + g) for i in range(n_out) for g in range(groups)]
    Xc = [hx.hx_encrypt(ctx, ks, Xp[g], 0, 2000 + g) for g in range(groups)]
    Gc = [hx.hx_encrypt(ctx, ks, Gp[i], 0, 3000 + i) for i in range(n_out)]
    stream = torch.cuda.current_stream()

    def step(seed):
        return hx.hx_dense_layer(ctx, ks, Wc, Xc, Gc, h, n_out, groups, d, k, div, refresh_seed=seed, stream=stream)

    def free(res):
        for part in res:
            for c in part:
                hx.hx_ct_destroy(c)

    for w in range(args.warmup):
        free(step(w))
    torch.cuda.synchronize()
    sampler = ClockSampler()
    times = []
    for it in range(args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = step(100 + it)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
        if it < args.steps - 1:
            free(res)
    clocks = sampler.stop()
    t = sum(times) / len(times)
    # live per-kernel-class shares of one more step (CUDA events per launch, chains serial)
    hx.hx_profile_enable(ctx, True)
    free(step(999))
    prof = hx.hx_profile_read(ctx)
    hx.hx_profile_enable(ctx, False)
    total_ms = sum(v[1] for v in prof.values())
    shares = {c: round(v[1] / total_ms, 4) for c, v in sorted(prof.items(), key=lambda kv: -kv[1][1])}
    E, M, dW = res
    Wb = workloads.blocks(W, h)
    Xb = [r[0] for r in workloads.blocks(X, h)]
    Gb = [r[0] for r in workloads.blocks(G, h)]
    err = {"E": 0.0, "relu_vs_fp64_composite": 0.0, "relu_vs_exact": 0.0, "dW_vs_fp64_composite": 0.0}
    for i in range(n_out):
        e_ref = sum(a @ b for a, b in zip(Wb[i], Xb))
        s_ref = g4_iter(e_ref / div, k)
        l_ref = (1 + s_ref) / 2 * Gb[i]
        e = workloads.unpack(hx.hx_decrypt(ctx, ks, E[i]), h, beta)[0]
        m = workloads.unpack(hx.hx_decrypt(ctx, ks, M[i]), h, beta)[0]
        err["E"] = max(err["E"], float(np.abs(e - e_ref).max()))
        err["relu_vs_fp64_composite"] = max(err["relu_vs_fp64_composite"],
                                            float(np.abs(m - e_ref * (1 + s_ref) / 2).max()))
        err["relu_vs_exact"] = max(err["relu_vs_exact"], float(np.abs(m - np.maximum(e_ref, 0)).max()))
        for g in range(groups):
            got = workloads.unpack(hx.hx_decrypt(ctx, ks, dW[i * groups + g]), h, beta)
            for q in range(beta):
                j = beta * g + q
                if j < len(Xb):
                    err["dW_vs_fp64_composite"] = max(err["dW_vs_fp64_composite"],
                                                      float(np.abs(got[q] - l_ref @ Xb[j].T).max()))
    free(res)
    line = {"metric": "encrypted dense layer 784->128 forward+backward, layers/s (batch 64, CKKS N=2^15)",
            "value": round(1.0 / t, 4), "unit": "layer/s", "ms_per_step": round(t * 1e3, 1),
            "steps": args.steps, "warmup": args.warmup, "n_gpus": 1, "higher_is_better": True, "dtype": "u64",
            "data": "synthetic",
            "config": {"workload": "cfg3: W 128x784 (padded 128x832), X 784x64, h=64, beta=4, 8+8 ciphertext pairs "
                                   "per HE-MatMult batch, ReLU g_4^(8)(E/4), collective refreshes timed (host wall clock)"},
            "max_abs_err": err, "clocks": clocks, "kernel_shares": shares, "kernel_ms_profiled": round(total_ms, 2)}
    print(json.dumps(line), flush=True)
    hx.hx_keyset_destroy(ks)
    hx.hx_context_destroy(ctx)


def run_serve(args):
    """Serving stream (config-4 pattern): Poisson arrivals of mixed requests -- encrypted
    matmuls (h in {16, 32, 64}, as the ring allows; 128 with --full) and composite sign (g_4, one
    composition) -- over CKKS rings N in {2^13, 2^14, 2^15} (and 2^16 with --full), chain 60 + 19x40
    bit, P = 3x60 bit, limb counts drawn per request (matmul U{3..20}: 3 runs the depth-2 product;
    sign U{5..20}); rotation keys resident; HBM-budget admission.
    Capacity is measured closed-loop first; the open-loop run offers 0.8x capacity."""
    import torch

    from paper_2207_04620_gb300 import hx, workloads

    import __graft_entry__

    __graft_entry__.build()
    rng = np.random.default_rng(2026)
    log_ns = [13, 14, 15] + ([16] if args.full else [])
    qb, pb = [60] + [40] * 19, [60] * 3
    ctxs, keys = {}, {}
    t_setup = time.perf_counter()
    for ln in log_ns:
        ctx = hx.hx_context_create(ln, qb, pb, 40)
        hx.hx_autotune(ctx)
        s = (1 << ln) // 2
        hs = [h for h in (16, 32, 64, 128) if h * h <= s and (h <= 64 or args.full)]
        steps = sorted({k for h in hs for lv in (3, 8) for k in hx.hx_matmul_rotation_steps(ctx, h, lv)})
        ctxs[ln] = (ctx, hs)
        keys[ln] = hx.hx_keygen(ctx, 2, 4000 + ln, steps)
    n_req = args.requests
    # Request parameters (kind, ring, h, level) come from the seeded generator; the encrypted
    # inputs from small pools, two per (ring, h, level) for products and per (ring, level) for
    # signs, so that 10k requests do not hold 10k input ciphertexts on the device.
    pools = {}

    def pooled(key, make):
        if key not in pools:
            pools[key] = [make(j) for j in range(2)]
        return pools[key][int(rng.integers(0, 2))]

    reqs = []
    for i in range(n_req):
        ln = int(rng.choice(log_ns))
        ctx, hs = ctxs[ln]
        s = (1 << ln) // 2
        if rng.random() < 0.5:
            h = int(rng.choice(hs))
            limbs = int(rng.integers(3, 21))
            beta = s // (h * h)

            def make(j, ctx=ctx, ln=ln, h=h, beta=beta, limbs=limbs):
                sd = 97 * (ln * 1000 + h * 32 + limbs) + j
                return tuple(hx.hx_encrypt(ctx, keys[ln], workloads.pack(workloads.matrices(2 * sd + e, beta, h), h,
                                                                          beta), limbs, 2 * sd + e) for e in (0, 1))
            a, b = pooled(("m", ln, h, limbs), make)
            reqs.append(("matmul", ln, (a, b, h), limbs))
        else:
            limbs = int(rng.integers(5, 21))

            def make(j, ctx=ctx, ln=ln, s=s, limbs=limbs):
                sd = 89 * (ln * 100 + limbs) + j
                return hx.hx_encrypt(ctx, keys[ln], workloads.sign_inputs(sd, s), limbs, sd)
            x = pooled(("s", ln, limbs), make)
            reqs.append(("sign", ln, (x, 4, 1, 7 * i + 1), limbs))
    if args.full:
        # plans (encoded masks per ring, h and level; about 200 GB for every combination) are
        # built on first use, and past a per-ring cap the least recently used are freed: the
        # free memory less 24 GB for the server's batches, shared in proportion to N
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        room = max(0, free0 - (24 << 30))
        weight = sum(1 << ln for ln in log_ns)
        for ln in log_ns:
            hx.hx_context_set_plan_cache(ctxs[ln][0], max(1, room * (1 << ln) // weight))
    else:
        # build every plan once (library masks) before timing
        seen = set()
        for kind, ln, a, limbs in reqs:
            if kind == "matmul" and (ln, a[2], limbs) not in seen:
                seen.add((ln, a[2], limbs))
                hx.hx_ct_destroy(hx.hx_matmul(ctxs[ln][0], keys[ln], a[0], a[1], a[2]))
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t_setup
    # the server counts registered keys against its budget: give it the free memory (less what
    # the capped plan caches may still take, and a margin) plus the keys already resident
    probe = hx.hx_server_create(1 << 62, 1, 1)
    for ln in log_ns:
        hx.hx_server_register_keys(probe, keys[ln])
    key_bytes = hx.hx_server_stats(probe)["key_bytes"]
    hx.hx_server_destroy(probe)
    free, total = torch.cuda.mem_get_info()
    plan_room = 0
    if args.full:
        for ln in log_ns:
            info = hx.hx_context_plan_cache_info(ctxs[ln][0])
            plan_room += max(0, info["cap"] - info["bytes"])
    budget = int(max(0, free - plan_room) * 0.9) + key_bytes
    sv = hx.hx_server_create(budget, args.lanes, args.max_batch)
    for ln in log_ns:
        hx.hx_server_register_keys(sv, keys[ln])

    def submit(r):
        kind, ln, a, _ = r
        ctx = ctxs[ln][0]
        if kind == "matmul":
            return hx.hx_server_submit_matmul(sv, ctx, keys[ln], a[0], a[1], a[2])
        return hx.hx_server_submit_sign(sv, ctx, keys[ln], a[0], a[1], a[2], False, a[3])

    def drain(pending_ids, lat):
        for rid, res, st, l in hx.hx_server_poll(sv, wait=False):
            if st != 0:
                raise RuntimeError("request %d failed with status %d" % (rid, st))
            lat[rid] = l
            hx.hx_ct_destroy(res)
            pending_ids.discard(rid)

    # closed loop: the first 20% at once -> capacity
    n_cap = max(20, n_req // 5)
    lat_cap, pend = {}, set()
    t0 = time.perf_counter()
    for r in reqs[:n_cap]:
        pend.add(submit(r))
    while pend:
        for rid, res, st, l in hx.hx_server_poll(sv, wait=True):
            lat_cap[rid] = l
            hx.hx_ct_destroy(res)
            pend.discard(rid)
    capacity = n_cap / (time.perf_counter() - t0)
    # open loop: Poisson arrivals at a fixed fraction of the capacity
    def open_loop(load, batch):
        rate = load * capacity
        gaps = rng.exponential(1.0 / rate, len(batch))
        lat, pend = {}, set()
        t0 = time.perf_counter()
        t_next = t0
        for r, g in zip(batch, gaps):
            t_next += g
            while True:
                now = time.perf_counter()
                if now >= t_next:
                    break
                drain(pend, lat)
                time.sleep(min(0.0005, t_next - now))
            pend.add(submit(r))
        while pend:
            for rid, res, st, l in hx.hx_server_poll(sv, wait=True):
                if st != 0:
                    raise RuntimeError("request %d failed with status %d" % (rid, st))
                lat[rid] = l
                hx.hx_ct_destroy(res)
                pend.discard(rid)
        return lat, rate, time.perf_counter() - t0

    sampler = ClockSampler()
    lat, rate, elapsed = open_loop(args.load, reqs[n_cap:])
    clocks = sampler.stop()
    stats = hx.hx_server_stats(sv)
    # the same request stream at other offered loads (below, near and above capacity)
    sweep = []
    for load in ((0.5, 0.9, 1.1) if getattr(args, "sweep", True) else ()):
        lt, rt, el = open_loop(load, reqs[n_cap:])
        Ls = np.array(sorted(lt.values()))
        sweep.append({"load": load, "offered_req_s": round(rt, 2), "throughput_req_s": round(len(Ls) / el, 2),
                      "p50_ms": round(float(np.percentile(Ls, 50)), 3),
                      "p99_ms": round(float(np.percentile(Ls, 99)), 3)})
    hx.hx_server_destroy(sv)
    L = np.array(sorted(lat.values()))
    line = {"metric": "serving p50/p99 ms (continuous batching, mixed encrypted matmul + sign)",
            "value": round(float(np.percentile(L, 50)), 3), "p99_ms": round(float(np.percentile(L, 99)), 3),
            "unit": "ms", "higher_is_better": False, "throughput_req_s": round(len(L) / elapsed, 2),
            "offered_req_s": round(rate, 2), "capacity_req_s": round(capacity, 2), "requests": len(L),
            "n_gpus": 1, "dtype": "u64", "data": "synthetic",
            "config": {"workload": "Poisson arrivals at %.1fx closed-loop capacity; 50%% matmul h in %s "
                                   "(feasible per ring), 50%% sign g_4 (k=1); N in %s; Q=60+19x40, P=3x60 bit; "
                                   "matmul limbs U{3..20}, sign limbs U{5..20}"
                                   % (args.load, sorted({h for ln in log_ns for h in ctxs[ln][1]}),
                                      [2 ** l for l in log_ns]),
                       "inputs": "two seeded ciphertexts (pairs) per (ring, h, level) and per (ring, level) for "
                                 "signs, drawn per request",
                       "plans": ("built on first use, least recently used freed past a per-ring cap (free memory "
                                 "less 24 GB, in proportion to N)" if args.full else "all built before timing"),
                       "lanes": args.lanes, "max_batch": args.max_batch, "hbm_budget_bytes": budget,
                       "setup_s": round(setup_s, 1)},
            "server": stats, "clocks": clocks, "load_sweep": sweep,
            "plan_cache": {str(2 ** ln): hx.hx_context_plan_cache_info(ctxs[ln][0]) for ln in log_ns}}
    for entries in pools.values():
        for e in entries:
            for h in (e if isinstance(e, tuple) else (e,)):
                hx.hx_ct_destroy(h)
    for ln in log_ns:
        hx.hx_keyset_destroy(keys[ln])
        hx.hx_context_destroy(ctxs[ln][0])
    return line


def run_micro(args):
    """NTT alone: forward then inverse transform of `rows` limbs of one ring
    degree, in place, timed with CUDA events.  Algorithmic traffic: one read
    and one write of every residue per transform (16 B per coefficient)."""
    import torch

    from paper_2207_04620_gb300 import hx, workloads

    import __graft_entry__

    __graft_entry__.build()
    log_n = args.log_n
    ctx = hx.hx_context_create(log_n, Q_BITS, P_BITS, LOG2_SCALE)
    tiles = hx.hx_autotune(ctx) if args.tiles is None else hx.hx_ntt_tiles(ctx, [int(t) for t in args.tiles.split(",")])
    primes = hx.hx_context_primes(ctx)
    n = 1 << log_n
    rows = args.rows
    per = len(primes)
    polys = max(1, rows // per)
    x = torch.from_numpy(workloads.residues(7, primes, polys, n).view(np.int64)).cuda()
    stream = torch.cuda.current_stream()
    idx = list(range(per))
    for _ in range(args.warmup):
        hx.hx_ntt(ctx, x.data_ptr(), polys, idx, False, stream)
        hx.hx_ntt(ctx, x.data_ptr(), polys, idx, True, stream)
    torch.cuda.synchronize()
    fw, iv = [], []
    # each timed step repeats each direction `reps` times between its events (inputs larger
    # than L2), long enough for the clock sampler to see the GPU under load
    reps = max(1, int(getattr(args, "reps", 1)))
    sampler = ClockSampler()
    for _ in range(args.steps):
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record(stream)
        for _ in range(reps):
            hx.hx_ntt(ctx, x.data_ptr(), polys, idx, False, stream)
        e[1].record(stream)
        for _ in range(reps):
            hx.hx_ntt(ctx, x.data_ptr(), polys, idx, True, stream)
        e[2].record(stream)
        torch.cuda.synchronize()
        fw.append(e[0].elapsed_time(e[1]) / reps)
        iv.append(e[1].elapsed_time(e[2]) / reps)
    clocks = sampler.stop()
    byt = 16.0 * polys * per * n
    peak, kind = peaks()
    shoup_s, _ = hx.hx_alu_calibrate(ctx, stream=stream)
    res = {"micro": "ntt", "log_n": log_n, "rows": polys * per, "bytes_per_transform": byt, "tiles": tiles,
           "fwd_ms": statistics.median(fw), "inv_ms": statistics.median(iv),
           "fwd_gbs": byt / statistics.median(fw) / 1e6, "inv_gbs": byt / statistics.median(iv) / 1e6,
           "peak_gbs": peak, "peak_kind": kind, "clocks": clocks}
    res["fwd_frac"] = res["fwd_gbs"] / peak
    res["inv_frac"] = res["inv_gbs"] / peak
    # the ALU roofline: butterflies/s (one Shoup product each) against the derived ceiling, and
    # against the Shoup products/s the calibration kernel reaches
    res["shoup_products_per_s"] = shoup_s
    res["alu_peak_shoup_per_s"] = ALU_PEAK_SHOUP
    res["fwd_alu_frac"] = res["fwd_gbs"] * 1e9 * log_n / 32.0 / ALU_PEAK_SHOUP
    res["inv_alu_frac"] = res["inv_gbs"] * 1e9 * log_n / 32.0 / ALU_PEAK_SHOUP
    res["fwd_calibrated_frac"] = res["fwd_gbs"] * 1e9 * log_n / 32.0 / shoup_s
    res["inv_calibrated_frac"] = res["inv_gbs"] * 1e9 * log_n / 32.0 / shoup_s
    hx.hx_context_destroy(ctx)
    return res


def run_rmatmul(args):
    """Rectangular products (App. D, Alg. "41") at the config-1 ring: 16 ciphertext pairs x beta=2,
    each a (t x 64) . (64 x 64) product with A packed as 64/t vertical copies; CKKS N=2^14,
    Q = 60 + 7x45 bit, P = 2x60 bit; L2 flushed between steps.  The square product of the same
    batch is timed beside it."""
    import torch

    from paper_2207_04620_gb300 import hx, workloads

    import __graft_entry__

    __graft_entry__.build()
    t, pairs = args.t, PAIRS
    ctx = hx.hx_context_create(LOG_N, Q_BITS, P_BITS, LOG2_SCALE)
    hx.hx_autotune(ctx)
    limbs = len(Q_BITS)
    ks = hx.hx_keygen(ctx, 2, 31, sorted(set(hx.hx_rmatmul_rotation_steps(ctx, H, t, limbs))
                                         | set(hx.hx_matmul_rotation_steps(ctx, H, limbs))))
    plan = hx.hx_matmul_plan_create(ctx, H, limbs)
    rng = np.random.default_rng(5)
    As = [[rng.uniform(-1, 1, (t, H)) for _ in range(BETA)] for _ in range(pairs)]
    Bs = [workloads.matrices(300 + i, BETA, H) for i in range(pairs)]
    At = [hx.hx_encrypt(ctx, ks, workloads.pack([np.vstack([a] * (H // t)) for a in As[i]], H, BETA), 0, 10 + i)
          for i in range(pairs)]
    Bc = [hx.hx_encrypt(ctx, ks, workloads.pack(Bs[i], H, BETA), 0, 50 + i) for i in range(pairs)]
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")

    def timed(fn):
        for _ in range(args.warmup):
            for o in fn():
                hx.hx_ct_destroy(o)
        ts, outs = [], None
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            outs = fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
            if len(ts) < args.steps:
                for o in outs:
                    hx.hx_ct_destroy(o)
        return sum(ts) / len(ts), outs

    rect_ms, outs = timed(lambda: hx.hx_rmatmul_batch(ctx, ks, plan, At, Bc, H, t, stream=stream))
    got = workloads.unpack(hx.hx_decrypt(ctx, ks, outs[0]), H, BETA)
    err = float(max(np.abs(g - np.vstack([a @ b] * (H // t))).max() for g, a, b in zip(got, As[0], Bs[0])))
    for o in outs:
        hx.hx_ct_destroy(o)
    sq_ms, outs = timed(lambda: hx.hx_matmul_batch(ctx, ks, plan, At, Bc, H, stream=stream))
    for o in outs:
        hx.hx_ct_destroy(o)
    n = pairs * BETA
    line = {"metric": "encrypted (%dx64).(64x64) rectangular products/s (HE-RMatMult, CKKS N=2^14)" % t,
            "value": round(n / (rect_ms / 1e3), 2), "unit": "product/s", "ms_per_step": round(rect_ms, 3),
            "steps": args.steps, "warmup": args.warmup, "n_gpus": 1, "higher_is_better": True, "dtype": "u64",
            "data": "synthetic",
            "config": {"workload": "32 rectangular products per step (16 ciphertext pairs x beta=2), t=%d, h=64" % t,
                       "l2": "flushed between steps"},
            "square_same_batch": {"value": round(n / (sq_ms / 1e3), 2), "unit": "matmul/s", "ms_per_step": round(sq_ms, 3)},
            "max_abs_err_vs_fp64": err}
    print(json.dumps(line), flush=True)
    hx.hx_keyset_destroy(ks)
    hx.hx_context_destroy(ctx)


def run_micro_encrypt(args):
    """Client side (Fig. 1 items 3 and 5): encode + encrypt 64 slot vectors of 16384 values at the
    config-2 ring (N=2^15, 16 limbs) as one device batch (hx_encrypt_batch, slots from host memory,
    handles out), beside the host encoder + per-ciphertext encryption (hx_encrypt) of the same
    inputs; the two give identical ciphertexts."""
    import torch

    from paper_2207_04620_gb300 import hx

    import __graft_entry__

    __graft_entry__.build()
    log_n, qb, pb, count = 15, [60] + [40] * 15, [60] * 3, 64
    ctx = hx.hx_context_create(log_n, qb, pb, 40)
    ks = hx.hx_keygen(ctx, 2, 3, [])
    z = np.random.default_rng(2).uniform(-1, 1, (count, (1 << log_n) // 2))
    seeds = list(range(1000, 1000 + count))
    for _ in range(args.warmup):
        for o in hx.hx_encrypt_batch(ctx, ks, z, seeds):
            hx.hx_ct_destroy(o)
    torch.cuda.synchronize()
    ts = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        outs = hx.hx_encrypt_batch(ctx, ks, z, seeds)
        torch.cuda.synchronize()
        ts.append(time.perf_counter() - t0)
        for o in outs[1:]:
            hx.hx_ct_destroy(o)
        first = outs[0]
        if len(ts) < args.steps:
            hx.hx_ct_destroy(first)
    t_dev = statistics.median(ts)
    host_n = 8
    t0 = time.perf_counter()
    ref = [hx.hx_encrypt(ctx, ks, z[i], 0, seeds[i]) for i in range(host_n)]
    t_host = (time.perf_counter() - t0) / host_n
    same = bool(np.array_equal(hx.hx_ct_export(ctx, first), hx.hx_ct_export(ctx, ref[0])))
    for o in ref + [first]:
        hx.hx_ct_destroy(o)
    res = {"micro": "encrypt", "log_n": log_n, "limbs": len(qb), "count": count,
           "device_batch_ct_per_s": round(count / t_dev, 1), "device_batch_ms": round(t_dev * 1e3, 2),
           "host_path_ct_per_s": round(1.0 / t_host, 1), "speedup": round(t_host * count / t_dev, 1),
           "identical_to_host_path": same,
           "note": "host wall clock; the device batch includes the H2D of the slots and the handle copies"}
    print(json.dumps(res), flush=True)
    hx.hx_keyset_destroy(ks)
    hx.hx_context_destroy(ctx)


def run_micro_ntt_multi(args):
    """Rings of uneven degree and limb count through one launch per phase (hx_ntt_multi) against one
    hx_ntt call per ring, forward transforms in place, CUDA events on the stream: a large mix
    (N = 2^13 with 12 limbs x 8 polynomials, 2^14 8 x 16, 2^15 16 x 4, 2^16 20 x 2) and 48 small
    rings (N 2^12..2^14, 1..4 limbs, one polynomial each, the shape of a serving mix)."""
    import torch

    from paper_2207_04620_gb300 import hx, workloads

    import __graft_entry__

    __graft_entry__.build()
    stream = torch.cuda.current_stream()
    ctx_of = {}

    def make_jobs(specs):
        jobs, bufs, byt = [], [], 0.0
        for ln, limbs, polys in specs:
            if ln not in ctx_of:
                c = hx.hx_context_create(ln, [60] + [40] * 19, [60] * 2, 40)
                hx.hx_autotune(c)
                ctx_of[ln] = c
            ctx = ctx_of[ln]
            primes = hx.hx_context_primes(ctx)[:limbs]
            x = torch.from_numpy(workloads.residues(ln + len(jobs), primes, polys, 1 << ln).view(np.int64)).cuda()
            bufs.append(x)
            jobs.append((ctx, x.data_ptr(), polys, list(range(limbs))))
            byt += 16.0 * polys * limbs * (1 << ln)
        return jobs, bufs, byt

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        ts = []
        for _ in range(args.steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    peak, kind = peaks()
    cases = {"large": [(13, 12, 8), (14, 8, 16), (15, 16, 4), (16, 20, 2)],
             "many_small": [(12 + (i % 3), 1 + (i % 4), 1) for i in range(48)]}
    out = {"micro": "ntt_multi", "peak_gbs": peak, "peak_kind": kind,
           "note": "fused: one persistent launch per phase for all rings (128-thread tiles, next tile "
                   "prefetched); per-ring: one hx_ntt call (two launches, autotuned persistent kernels) per ring"}
    for name, specs in cases.items():
        jobs, bufs, byt = make_jobs(specs)

        def separate():
            for ctx, ptr, polys, pr in jobs:
                hx.hx_ntt(ctx, ptr, polys, pr, False, stream)

        def fused():
            hx.hx_ntt_multi(jobs, False, stream)

        ms_sep, ms_fus = timed(separate), timed(fused)
        out[name] = {"rings": len(specs), "bytes": byt, "fused_ms": round(ms_fus, 4), "per_ring_ms": round(ms_sep, 4),
                     "fused_gbs": round(byt / ms_fus / 1e6, 1), "per_ring_gbs": round(byt / ms_sep / 1e6, 1),
                     "launches": {"fused": 2, "per_ring": 2 * len(specs)}}
    print(json.dumps(out), flush=True)
    for c in ctx_of.values():
        hx.hx_context_destroy(c)


def run_matmul_jobs(args):
    """Products over several rings, levels and sizes in one hx_matmul_jobs call against the same
    groups as one call each, one after another on the stream (same cached plans and keys).  Groups:
    N = 2^12 (Q = 60 + 4x45 bit) h = 16, N = 2^13 (60 + 5x45) h = 32, N = 2^14 (60 + 7x45, config 1's
    ring) h = 64 and h = 32, N = 2^14 at 6 limbs h = 64; 8 ciphertext pairs each, P = 2x60 bit,
    scale 2^45, entries U[-1, 1] seeded; CUDA events on the stream, L2 flushed between steps."""
    import torch

    from paper_2207_04620_gb300 import hx, workloads

    import __graft_entry__

    __graft_entry__.build()
    stream = torch.cuda.current_stream()
    rings = {12: [60] + [45] * 4, 13: [60] + [45] * 5, 14: [60] + [45] * 7}
    groups = [(12, 16, 5), (13, 32, 6), (14, 64, 8), (14, 32, 8), (14, 64, 6)]  # (log N, h, limbs)
    pairs = 8
    ctxs, kss = {}, {}
    for ln, qb in rings.items():
        ctx = hx.hx_context_create(ln, qb, [60, 60], 45)
        hx.hx_autotune(ctx, stream=stream)
        steps = sorted({s for g in groups if g[0] == ln for s in hx.hx_matmul_rotation_steps(ctx, g[1], g[2])})
        ctxs[ln], kss[ln] = ctx, hx.hx_keygen(ctx, 2, 70 + ln, steps)
    jobs_of, products = [], 0
    for gi, (ln, h, limbs) in enumerate(groups):
        beta = (1 << ln) // 2 // (h * h)
        js = []
        for i in range(pairs):
            a = workloads.pack(workloads.matrices(1000 * gi + 2 * i, beta, h), h, beta)
            b = workloads.pack(workloads.matrices(1000 * gi + 2 * i + 1, beta, h), h, beta)
            A = hx.hx_encrypt(ctxs[ln], kss[ln], a, limbs, 10 + i)
            B = hx.hx_encrypt(ctxs[ln], kss[ln], b, limbs, 50 + i)
            js.append((ctxs[ln], kss[ln], A, B, h))
        jobs_of.append(js)
        products += pairs * beta
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")

    def one_call():
        return hx.hx_matmul_jobs([j for js in jobs_of for j in js], stream=stream)

    def per_group():
        return [o for js in jobs_of for o in hx.hx_matmul_jobs(js, stream=stream)]

    def timed(fn):
        for _ in range(max(args.warmup, 1)):
            for o in fn():
                hx.hx_ct_destroy(o)
        ts = []
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            outs = fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
            for o in outs:
                hx.hx_ct_destroy(o)
        return statistics.median(ts)

    sampler = ClockSampler()
    ms_one = timed(one_call)
    ms_seq = timed(per_group)
    clocks = sampler.stop()
    out = {"workload": "matmul_jobs", "unit": "products/s", "products_per_step": products,
           "groups": [{"log_n": ln, "h": h, "limbs": limbs, "pairs": pairs,
                       "products": pairs * ((1 << ln) // 2 // (h * h))} for ln, h, limbs in groups],
           "one_call": {"ms": round(ms_one, 3), "value": round(products / (ms_one / 1e3), 1)},
           "one_call_per_group": {"ms": round(ms_seq, 3), "value": round(products / (ms_seq / 1e3), 1)},
           "speedup": round(ms_seq / ms_one, 3), "clocks": clocks,
           "what": "hx_matmul_jobs over every group (groups side by side on per-context stream pools) "
                   "against one hx_matmul_jobs call per group, one after another"}
    print(json.dumps(out), flush=True)
    for js in jobs_of:
        for j in js:
            hx.hx_ct_destroy(j[2])
            hx.hx_ct_destroy(j[3])
    for ln in rings:
        hx.hx_keyset_destroy(kss[ln])
        hx.hx_context_destroy(ctxs[ln])


def run_micro_rotate_jobs(args):
    """Rotations of ciphertexts of several rings in one hx_rotate_jobs call (each key-switching
    stage one launch over all of them) against one hx_rotate call per ciphertext, CUDA events on
    the stream: 48 small jobs (N = 2^12 .. 2^14, 2 .. 5 limbs, the shape of a serving mix) and
    16 jobs of the config-1 ring (N = 2^14, 8 limbs).  Chains of 60 + 7x45 bit, P = 2x60 bit."""
    import torch

    from paper_2207_04620_gb300 import hx

    import __graft_entry__

    __graft_entry__.build()
    stream = torch.cuda.current_stream()
    steps_set = [1, 3, -2, 5]
    ctxs, kss = {}, {}
    for ln in (12, 13, 14):
        ctxs[ln] = hx.hx_context_create(ln, [60] + [45] * 7, [60, 60], 45)
        hx.hx_autotune(ctxs[ln], stream=stream)
        kss[ln] = hx.hx_keygen(ctxs[ln], 2, 90 + ln, steps_set)
    rng = np.random.default_rng(5)

    def make(specs):
        jobs = []
        for i, (ln, limbs, k) in enumerate(specs):
            z = rng.uniform(-1, 1, (1 << ln) // 2)
            jobs.append((ctxs[ln], kss[ln], hx.hx_encrypt(ctxs[ln], kss[ln], z, limbs, 700 + i), k))
        return jobs

    def timed(fn):
        for _ in range(max(args.warmup, 1)):
            for o in fn():
                hx.hx_ct_destroy(o)
        ts = []
        for _ in range(args.steps):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            outs = fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
            for o in outs:
                hx.hx_ct_destroy(o)
        return statistics.median(ts)

    cases = {"many_small": [(12 + i % 3, 2 + i % 4, steps_set[i % 4]) for i in range(48)],
             "config1_ring": [(14, 8, steps_set[i % 4]) for i in range(16)]}
    out = {"micro": "rotate_jobs", "what": "one hx_rotate_jobs call (13 launches for all jobs) against one hx_rotate "
                                          "call (13 launches) per ciphertext, median over the timed steps"}
    for name, specs in cases.items():
        jobs = make(specs)
        ms_jobs = timed(lambda: hx.hx_rotate_jobs(jobs, stream=stream))
        ms_each = timed(lambda: [hx.hx_rotate(c, k_, h, st, stream=stream) for c, k_, h, st in jobs])
        out[name] = {"jobs": len(specs), "one_call_ms": round(ms_jobs, 4), "per_ciphertext_ms": round(ms_each, 4),
                     "speedup": round(ms_each / ms_jobs, 2)}
        for j in jobs:
            hx.hx_ct_destroy(j[2])
    print(json.dumps(out), flush=True)
    for ln in ctxs:
        hx.hx_keyset_destroy(kss[ln])
        hx.hx_context_destroy(ctxs[ln])


def run_micro_aggregate(args):
    """Alg. 6 Aggregation alone: the model update w - eta/(B N) * sum_i g_i for the 8
    gradient ciphertexts of one 784->128 layer (h=64, beta=4 packing) from 16 parties,
    CKKS N=2^15, 16 limbs.  The streaming sum reads every party's ciphertext once
    (algorithmic traffic: (parties + 1) ciphertexts of 2 x 16 x 2^15 words per model
    ciphertext); the rescale and the final addition follow it."""
    import torch

    from paper_2207_04620_gb300 import hx

    import __graft_entry__

    __graft_entry__.build()
    log_n, qb, pb = 15, [60] + [40] * 15, [60] * 3
    parties, count = args.parties, 8
    ctx = hx.hx_context_create(log_n, qb, pb, 40)
    ks = hx.hx_keygen(ctx, 2, 5, [])
    n_slots = (1 << log_n) // 2
    rng = np.random.default_rng(11)
    w = [rng.normal(0, 0.05, n_slots) for _ in range(count)]
    wc = [hx.hx_encrypt(ctx, ks, w[m], 0, 10 + m) for m in range(count)]
    g0 = [rng.normal(0, 0.01, n_slots) for _ in range(count)]
    gc = []
    for i in range(parties):
        for m in range(count):
            gc.append(hx.hx_encrypt(ctx, ks, g0[m] * (1 + 0.01 * i), 0, 1000 + 100 * i + m))
    c = 0.1 / (4 * parties)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        for o in hx.hx_aggregate(ctx, gc, parties, wc, c, stream=stream):
            hx.hx_ct_destroy(o)
    torch.cuda.synchronize()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    times = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        outs = hx.hx_aggregate(ctx, gc, parties, wc, c, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
        for o in outs[1:]:
            hx.hx_ct_destroy(o)
        last = outs[0]
        if len(times) < args.steps:
            hx.hx_ct_destroy(last)
    want = w[0] - c * sum(g0[0] * (1 + 0.01 * i) for i in range(parties))
    err = float(np.abs(hx.hx_decrypt(ctx, ks, last) - want).max())
    hx.hx_ct_destroy(last)
    # the streaming kernel alone, from the library's per-class CUDA events
    hx.hx_profile_enable(ctx, True)
    flush.zero_()
    torch.cuda.synchronize()
    for o in hx.hx_aggregate(ctx, gc, parties, wc, c, stream=stream):
        hx.hx_ct_destroy(o)
    prof = hx.hx_profile_read(ctx)
    hx.hx_profile_enable(ctx, False)
    _, agg_ms, agg_bytes = prof["aggregate"]
    peak, kind = peaks()
    gbs = agg_bytes / (agg_ms / 1e3) / 1e9
    res = {"micro": "aggregate", "parties": parties, "ciphertexts": count, "log_n": log_n, "limbs": len(qb),
           "call_ms": statistics.median(times), "kernel_ms": agg_ms, "kernel_bytes": agg_bytes,
           "kernel_gbs": round(gbs, 1), "peak_gbs": peak, "peak_kind": kind, "frac": round(gbs / peak, 4),
           "max_abs_err_vs_fp64": err,
           "note": "call = sum + constant (one streaming kernel), rescale, addition, handle copies"}
    print(json.dumps(res), flush=True)
    hx.hx_keyset_destroy(ks)
    hx.hx_context_destroy(ctx)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--micro", choices=["ntt", "aggregate", "encrypt", "ntt-multi", "rotate-jobs"], default=None)
    ap.add_argument("--parties", type=int, default=16)
    ap.add_argument("--workload", choices=["matmul", "sign", "dense", "serve", "rmatmul", "jobs"], default="matmul")
    ap.add_argument("--t", type=int, default=16, help="rows of A in the rectangular product")
    ap.add_argument("--requests", type=int, default=1000)
    ap.add_argument("--load", type=float, default=0.8)
    ap.add_argument("--lanes", type=int, default=4)
    ap.add_argument("--max-batch", type=int, default=16)
    ap.add_argument("--full", action="store_true", help="serving: add N=2^16 and h=128")
    ap.add_argument("--relu", action="store_true")
    ap.add_argument("--alpha", type=int, default=None,
                    help="sign/dense: primes per key-switching digit (0: K; default 4 for sign, K for dense)")
    ap.add_argument("--log-n", type=int, default=14)
    ap.add_argument("--rows", type=int, default=1600)
    ap.add_argument("--reps", type=int, default=1, help="NTT micro-benchmark: transforms per timed step")
    ap.add_argument("--tiles", default=None, help="NTT tile widths per phase, e.g. 16,16,16,16 (default: autotune)")
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="hx", choices=["hx", "reference"])
    ap.add_argument("--per-op-pairs", type=int, default=4)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="default line without the NTT, sign and serving sub-records")
    args = ap.parse_args()
    if args.micro == "aggregate":
        return run_micro_aggregate(args)
    if args.micro == "encrypt":
        return run_micro_encrypt(args)
    if args.micro == "ntt-multi":
        return run_micro_ntt_multi(args)
    if args.micro == "rotate-jobs":
        return run_micro_rotate_jobs(args)
    if args.micro:
        return print(json.dumps(run_micro(args)), flush=True)
    if args.workload == "sign":
        return print(json.dumps(run_sign(args)), flush=True)
    if args.workload == "serve":
        return print(json.dumps(run_serve(args)), flush=True)
    if args.workload == "dense":
        return run_dense(args)
    if args.workload == "rmatmul":
        return run_rmatmul(args)
    if args.workload == "jobs":
        return run_matmul_jobs(args)
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_hx(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
