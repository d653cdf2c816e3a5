#!/usr/bin/env python
"""Throughput of the population simulator: variant-steps/s at 4096 uneven
robots on one B300 (per GPU; weak scaling over GPUs).

Workload: 4096 seeded tree-grammar robots (2..20 hinged bricks, seed 3 + rank),
dt = 0.002 s, the first 15000 steps of their run: the default --steps 3 bench
steps of 5000 simulation steps each (one sim_step_n call = one CUDA-graph
replay of one persistent 5000-step launch).  W warm-up bench steps run first,
then the state is reset to the workload's start, so the timed region is steps
0..K*chunk of the run.

Printed JSON (rank 0):
  value    device time of the timed sim_step_n calls (CUDA events on the
           simulator's stream), inputs resident in HBM, L2 flushed (256 MiB
           write) between timed bench steps;
  e2e      the same metric through the C ABI with pinned host buffers:
           host->device state upload, the steps, device->host state read per
           bench step;
  roofline step kernel vs the FP32 ALU peak measured on the same GPU by the
           library's FFMA-loop kernel (scaled to the SM clock of the timed
           steps); algorithmic flops per variant-step counted by the FP64
           oracle on a sample of the same workload (contact-dependent phases
           scaled to the GPU's own contact count);
  surrogate  the learned part at the screening sizes: training time per
           epoch over 50000 pairs, predict + top-k of 65536 offspring;
  cpu_baseline  the FP64 oracle on the host cores, on a sample (every 16th
           robot, 2000 steps).
--impl reference times that oracle alone (bounded sample per bench step).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "variant-steps/s at 4096 uneven robots (1 B300)"
UNIT = "variant-steps/s"
SM_COUNT_NOMINAL = 148
FP32_LANES_PER_SM = 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3, help="timed bench steps")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--variants", type=int, default=4096)
    ap.add_argument("--chunk", type=int, default=5000, help="simulation steps per bench step")
    ap.add_argument("--seed", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def dist_init(world, local):
    if world <= 1:
        return None
    import torch
    import torch.distributed as dist
    os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
    backend = "nccl" if torch.cuda.is_available() else "gloo"
    if backend == "nccl":
        torch.cuda.set_device(local)
    dist.init_process_group(backend=backend)
    return dist


def reduce_max(dist, x, device):
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(dist, x, device):
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def barrier(dist):
    if dist is not None:
        dist.barrier()


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons (200 ms)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.gpu)], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("step_kernel.cuh", "step_common.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2502_11129_b300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic():
    """Per-launch DRAM bytes of the step kernel from the committed ncu summary,
    if it was captured from the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "step_kernel_traffic.json")
    try:
        d = json.load(open(path))
    except (OSError, ValueError):
        return None
    if d.get("source_hash") != kernel_source_hash():
        return None
    return d.get("dram_bytes_per_launch_full_workload")


def oracle_sample(pop, steps, threads):
    """FP64 oracle on the host cores: returns (variant-steps/s, flop stats)."""
    from oracle import oracle as O
    from paper_2502_11129_b300 import population as P
    s0 = P.cpg_initial(pop)
    models = O.models_from_population(pop)
    t0 = time.perf_counter()
    q, v, s, st, stats = O.run_population(pop, pop.q0, pop.v0, s0, steps, threads=threads, models=models)
    dt = time.perf_counter() - t0
    d = O.stats_dict(stats)
    vs = pop.n * steps
    return vs / dt, d, dt


def surrogate_record(device):
    """The learned half of the headline metric at the screening sizes (a
    128 -> 256 -> 256 -> 1 BF16 MLP, every dense layer on tcgen05): training
    time per epoch over 50000 (genotype, displacement) pairs, predicting and
    ranking 65536 offspring (top 4096), each call with its host copies."""
    from paper_2502_11129_b300 import surrogate as SG
    t = SG.timing(n_train=50000, n_screen=65536, k=4096, epochs=3, batch=1024, seed=0)
    return {"train_pairs": 50000, "train_s_per_epoch": t["train_s_per_epoch"],
            "train_s_3_epochs_incl_upload": t["train_s"],
            "train_tflops_incl_host": t["train_tflops_incl_host"],
            "screen_n": 65536, "screen_topk": 4096, "predict_s": t["predict_s"], "topk_s": t["topk_s"],
            "screen_per_s": 65536 / (t["predict_s"] + t["topk_s"]),
            "predict_tflops_incl_host": t["predict_tflops_incl_host"],
            "note": "wall time of each C-ABI call, host<->device copies included (per epoch: the slope "
                    "between a 1- and a 3-epoch call, one CUDA-graph replay each); encode of 2048 robots "
                    f"{t['encode_2048_s'] * 1e3:.2f} ms"}


def run_ours(args, world, rank, local, dist):
    import torch
    from paper_2502_11129_b300 import population as P
    from paper_2502_11129_b300 import sim as S

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    # one non-default stream shared by the simulator, the L2 flush and the
    # timing events (the legacy default stream cannot host graph capture)
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    pop = P.grammar(args.variants, seed=args.seed + 1000 * rank)
    s0 = P.cpg_initial(pop)
    Q0, V0, S0 = S.state_rows(pop, pop.q0, pop.v0, s0)
    sm = S.Sim(device=local, stream=stream.cuda_stream)
    sm.set_population(pop)
    sm.set_state(Q0, V0, S0)
    for _ in range(args.warmup):
        sm.step(args.chunk)
    # launch shapes probed from a settled, contact-rich state (the state is
    # kept), then one more untimed bench step captures the chosen shape's graph
    sm.autotune(min(500, args.chunk))
    sm.step(args.chunk)
    torch.cuda.synchronize(dev)
    sm.set_state(Q0, V0, S0)
    c_before = sm.counters()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = Clocks(local)
    torch.cuda.synchronize(dev)
    barrier(dist)
    clocks.start()
    for k in range(args.steps):
        flush.fill_(float(k))
        ev[k][0].record(stream)
        sm.step(args.chunk)
        ev[k][1].record(stream)
    torch.cuda.synchronize(dev)
    barrier(dist)
    clk = clocks.stop()
    ms = [a.elapsed_time(b) for a, b in ev]
    total_s = sum(ms) / 1e3
    total_s = reduce_max(dist, total_s, dev)
    c_after = sm.counters()
    vsteps = c_after["variant_steps"] - c_before["variant_steps"]
    contacts_per_vs = (c_after["contacts"] - c_before["contacts"]) / max(vsteps, 1)
    frozen = int(np.count_nonzero(sm.read_state()[3] & 5))
    # executed variant-steps over all ranks (a variant frozen by a non-finite
    # state stops advancing)
    value = reduce_sum(dist, vsteps, dev) / total_s
    shape = sm.launch_shape()
    spl = min(shape["steps_per_launch"], args.chunk)
    launches_per_chunk = -(-args.chunk // spl)
    launch_s = total_s / (args.steps * launches_per_chunk)

    # end to end through the C ABI with pinned host buffers
    e2e = None
    if not args.no_e2e:
        pin = lambda a: torch.from_numpy(a).pin_memory()
        hq, hv, hs = pin(Q0), pin(V0), pin(S0)
        oq, ov, os_ = pin(np.zeros_like(Q0)), pin(np.zeros_like(V0)), pin(np.zeros_like(S0))
        ost = torch.zeros(args.variants, dtype=torch.int32).pin_memory()
        torch.cuda.synchronize(dev)
        barrier(dist)
        t0 = time.perf_counter()
        for k in range(args.steps):
            sm.set_state_ptr(0, args.variants, hq.data_ptr(), hv.data_ptr(), hs.data_ptr())
            sm.step(args.chunk)
            sm.read_state_ptr(0, args.variants, oq.data_ptr(), ov.data_ptr(), os_.data_ptr(), ost.data_ptr())
            hq, oq = oq, hq
            hv, ov = ov, hv
            hs, os_ = os_, hs
        e2e_s = reduce_max(dist, time.perf_counter() - t0, dev)
        h2d = Q0.nbytes + V0.nbytes + S0.nbytes
        d2h = h2d + 4 * args.variants
        e2e = {"value": args.variants * args.chunk * args.steps * world / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": total_s * 1e3 / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": f"{args.variants} tree-grammar robots (2-20 hinges, seed {args.seed}+1000*rank), "
                                  f"dt 0.002 s, steps 0..{args.steps * args.chunk} as {args.steps} x "
                                  f"{args.chunk}-step graph replays",
                      "variants_per_gpu": args.variants, "sim_steps_per_bench_step": args.chunk,
                      "steps_per_launch": spl, "warps_per_block": shape["warps_per_block"],
                      "warps_per_sm": shape["warps_per_sm"],
                      "l2": "flushed between timed steps (256 MiB write)",
                      "contacts_per_variant_step": contacts_per_vs, "frozen_variants": frozen,
                      "parallelism": f"dp{world} (independent robots per GPU)"},
           # per launch: the slowest-first order (one cost_sort up to 8192 robots, else
           # cost_histogram + cost_scatter) and the step_kernel
           "gpu_launches": args.steps * launches_per_chunk * (2 if args.variants <= 8192 else 3),
           "e2e": e2e, "clocks": clk}

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from paper_2502_11129_b300 import population as P2
        sample = pop.subset(np.arange(0, pop.n, 16))
        threads = len(os.sched_getaffinity(0))
        rate, d, dt = oracle_sample(sample, 2000, threads)
        out["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
                               "sample": f"every 16th robot ({sample.n}) x 2000 steps from step 0, FP64, "
                                         f"{threads} pthreads, {dt:.1f} s"}
        vs_o = d["steps"]
        fl_contact = (d["flops_jac"] + d["flops_pgs"]) / vs_o
        fl_rest = (d["flops_total"] / vs_o) - fl_contact
        c_o = d["contacts"] / vs_o
        fl_per_vs = fl_rest + fl_contact * (contacts_per_vs / c_o if c_o > 0 else 1.0)
        props = torch.cuda.get_device_properties(dev)
        sms = props.multi_processor_count
        max_mhz = (clk or {}).get("sm_max_mhz") or 2032.0
        nominal = sms * FP32_LANES_PER_SM * 2 * max_mhz * 1e6 / 1e12
        units_per_launch = args.variants * spl
        achieved = fl_per_vs * units_per_launch / launch_s / 1e12
        # measured FP32 peak: the library's FFMA-loop kernel, clocks sampled
        # while it runs, scaled to the SM clock sampled during the timed steps
        fclk = Clocks(local)
        fclk.start()
        pk = S.fp32_peak(local, 25)
        fc = fclk.stop() or {}
        bench_mhz = (clk or {}).get("sm_mhz")
        ffma_mhz = fc.get("sm_mhz")
        scale = bench_mhz / ffma_mhz if bench_mhz and ffma_mhz else 1.0
        peak = pk["tflops"] * scale
        out["roofline"] = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                           "frac": achieved / peak, "traffic": ncu_traffic(),
                           "flops_per_unit": fl_per_vs, "unit_name": "variant-step",
                           "units_per_launch": units_per_launch, "launch_ms": launch_s * 1e3,
                           "peak_basis": "measured",
                           "peak_measurement": {
                               "kernel": "FFMA loop (sim_fp32_peak: 8 independent chains a thread, 64 warps per SM)",
                               "tflops": pk["tflops"], "ms": pk["ms"], "sm_mhz": ffma_mhz,
                               "reasons": fc.get("reasons"), "scaled_to_bench_sm_mhz": bench_mhz,
                               "flops_per_sm_cycle": (pk["tflops"] * 1e12 / (sms * ffma_mhz * 1e6)
                                                      if ffma_mhz else None)},
                           "peak_nominal": nominal,
                           "nominal_basis": f"{sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x {max_mhz:.0f} MHz",
                           "oracle_contacts_per_variant_step": c_o}
        out["surrogate"] = surrogate_record(local)
    sm.close()
    return out


def run_reference(args, world, rank):
    """The FP64 oracle alone, each bench step a bounded sample: every 16th
    robot x 200 continuing simulation steps."""
    if rank != 0:
        return None
    from oracle import oracle as O
    from paper_2502_11129_b300 import population as P
    pop = P.grammar(args.variants, seed=args.seed)
    sample = pop.subset(np.arange(0, pop.n, 16))
    models = O.models_from_population(sample)
    threads = len(os.sched_getaffinity(0))
    q, v, s = sample.q0.copy(), sample.v0.copy(), P.cpg_initial(sample)
    per = 200
    for _ in range(args.warmup):
        q, v, s, st, _ = O.run_population(sample, q, v, s, per, threads=threads, models=models)
    q, v, s = sample.q0.copy(), sample.v0.copy(), P.cpg_initial(sample)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        q, v, s, st, _ = O.run_population(sample, q, v, s, per, threads=threads, models=models)
    dt = time.perf_counter() - t0
    value = sample.n * per * args.steps / dt
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"{args.variants} tree-grammar robots (seed {args.seed}); bench step = "
                                   f"every 16th robot x {per} continuing steps on the FP64 oracle",
                       "variants_sampled": sample.n},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"{sample.n} robots x {per} steps per bench step, {threads} pthreads"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}


def main():
    args = parse()
    world, rank, local = dist_env()
    if args.impl == "reference":
        out = run_reference(args, world, rank)
        if out is not None:
            print(json.dumps(out), flush=True)
        return
    dist = dist_init(world, local)
    out = run_ours(args, world, rank, local, dist)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
