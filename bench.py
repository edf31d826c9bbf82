#!/usr/bin/env python3
"""Benchmark: Lawler-network pins per second to the exact minimum cut.

Workload (one step): on the 2,000,000-vertex / 3,000,000-net ring hypergraph
(2 + Zipf(2.5) pins per net, capped at 5,000, window 4,096; net weights
1..10; halves bipartition; region = vertices within 200,000 positions of the
two cut points), build the flow network of the region, compute the maximum
flow by push-relabel, and extract the minimal source-side cut S_r.
value = Lawler-network pins (p_N, s/t pins included) / step time, summed over
ranks (independent replicas; the single max flow does not shard).

The line also carries "kway", the second half of the metric (k-way refine
time at equal connectivity - 1):
  - "batched": rounds of Algorithm 1 on the 8,000,000-vertex / 12,000,000-net
    ring (2 + Zipf(2.5) pins capped at 10,000, k = 64 contiguous arcs, 5 % of
    the vertices moved to a neighbouring block), all FlowCutter problems of a
    round in one batched launch (with several ranks the round's block pairs
    are split across them);
  - "compare": from one start partition of the same generator at a smaller
    size, the plain round (one FlowCutter problem after another), the batched
    round (identical partitions), the batched round pruned by the learned
    scheduler with the committed weights (train_scheduler.py), and batched
    rounds under the paper's active block scheduling, to convergence or a
    round limit: seconds, pairs refined and final (lambda - 1) per arm;
  - every round's (lambda - 1) recomputed on the host from the returned
    partition ("certificate").

cpu_baseline: the CPU oracle (Dinic on the explicit Lawler graph) on a 1/10
sample of the workload, plus the sequential FIFO push-relabel (SeqPR) on the
full workload, one host core each.  --impl reference times the oracle on the
sample.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

WORKLOAD = "ring_n2M_zipf"
METRIC = "Lawler-network pins/s to exact min cut (1 GB300)"
UNIT = "pins/s"
L2_BYTES = 129 * 1024 * 1024
# Oracle sample: the same generator at 1/10 scale (about 10-30 s of CPU work).
SAMPLE = dict(n=200_000, m=300_000, radius=20_000)

# algorithmic bytes per counted item of the engine (the roofline model)
B_HYPER = 28   # incidence (8) + w(e) (4) + f_in (4) + f_out (4) + two labels (8)
B_NET = 12     # pin (4) + pin flow (4) + label (4)
B_NODE = 24    # list entry (4) + label (4) + excess (8) + delta (8)
B_PUSH = 16    # flow write (4) + excess-delta atomic (8) + stamp (4)


def env_rank():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, device):
        self.device = device
        self.samples = []
        self.proc = None

    def start(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 7:
                self.samples.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4)
                          if s[3 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.samples)}


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


ENGINE_SOURCES = ("engine.cu", "engine.cuh", "common.cuh", "kernels.cuh")


def engine_code_sha256(read):
    """sha256 of the engine sources with comments and blank lines removed, so
    that an edit of comments alone keeps the hash (the sources hold no string
    literal with a comment marker)."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in ENGINE_SOURCES:
        text = re.sub(r"/\*.*?\*/|//[^\n]*", "", read(f), flags=re.S)
        lines = [ln.rstrip() for ln in text.splitlines() if ln.strip()]
        h.update(("\n".join(lines) + "\n").encode())
    return h.hexdigest()


def engine_traffic_ratio():
    """DRAM bytes per modelled byte of the engine kernel from the committed ncu
    summary, if the engine code is unchanged since that capture."""
    import re
    path = os.path.join(ROOT, "profiles", "engine_kernel_ring_n1M.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    m1 = re.search(r"traffic_per_modelled_byte = ([0-9.]+)", text)
    m2 = re.search(r"engine_source_sha256 = ([0-9a-f]+)", text)
    if not (m1 and m2):
        return None
    def read(f):
        with open(os.path.join(ROOT, "paper_2201_01556_gb300", "csrc", f)) as fh:
            return fh.read()
    return float(m1.group(1)) if engine_code_sha256(read) == m2.group(1) else None


def oracle_step(inst):
    import oracle
    H = inst["H"]
    t0 = time.perf_counter()
    net = oracle.build_network(H, inst["part"], inst["region"])
    mc = oracle.max_flow_min_cut(net)
    dt = time.perf_counter() - t0
    return net.p, dt, mc.flow


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    inst = synth.instance(WORKLOAD, args.seed, **SAMPLE)
    for _ in range(args.warmup if args.warmup < 1 else 1):
        oracle_step(inst)
    times, pins = [], 0
    for _ in range(args.steps):
        p, dt, _ = oracle_step(inst)
        times.append(dt)
        pins = p
    v = pins / statistics.mean(times)
    sample = (f"ring n={SAMPLE['n']}, m={SAMPLE['m']}, radius={SAMPLE['radius']} "
              f"({pins} Lawler-network pins), same generator as the workload")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * statistics.mean(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "seed": args.seed,
                       "sample": sample},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample, "nproc": host_cpu()[0],
                             "cpu_model": host_cpu()[1]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def km1_host(H, part):
    """(lambda - 1) recomputed on the host from a partition (Section 2): one
    64-bit block mask per net, its population count minus one, times w(e)."""
    bits = np.left_shift(np.uint64(1), part[H.pins].astype(np.uint64))
    off = H.net_off.astype(np.int64)
    masks = np.zeros(H.m, np.uint64)
    full = off[1:] > off[:-1]          # empty nets keep mask 0
    if full.any():
        masks[full] = np.bitwise_or.reduceat(bits, off[:-1][full])
    lam = np.unpackbits(masks.view(np.uint8).reshape(-1, 8), axis=1).sum(1).astype(np.int64)
    return int((np.maximum(lam - 1, 0) * H.net_w.astype(np.int64)).sum())


def kway_batched(hfp, ctx, args, world):
    """Batched k-way rounds on the large ring, each round's (lambda - 1)
    checked against a host recount of the returned partition.  With several
    ranks the rounds split their block pairs across the ranks (one all-gather
    of move sets per round) and every rank runs this."""
    import torch
    from paper_2201_01556_gb300 import sharded
    n = args.kway_n
    inst = synth.instance("ring_n8M_zipf_k64", args.seed, n=n, m=n * 3 // 2)
    H, part = inst["H"], inst["part"]
    hg = hfp.HGraph(ctx, H.net_off, H.pins, H.net_w, H.node_w, H.n)
    pd = torch.from_numpy(part.copy()).cuda()
    conn = [hfp.connectivity(hg, pd, 64)]
    cert = [km1_host(H, part) == conn[0]]
    G, tune = args.kway_group, None
    if G <= 0:
        # CTAs per FlowCutter problem: hfp_autotune_round times the first
        # round's batched launch per candidate (untimed here; outcomes do not
        # depend on the group size)
        cands = (4, 8, 16)
        G, tms = hfp.autotune_round(hg, pd, 64, cands)
        tune = {"candidates": list(cands), "launch_ms": [round(float(x), 1) for x in tms]}
    secs, pairs, fc_ms, parts = [], [], [], []
    for _ in range(args.kway_rounds):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if world > 1:
            st, _ = sharded.refine_round_sharded(hg, pd, 64, group_ctas=G)
        else:
            st, _, ms = hfp.refine_round_batched(hg, pd, 64, group_ctas=G)
            fc_ms.append(round(ms, 1))
        torch.cuda.synchronize()
        secs.append(round(time.perf_counter() - t0, 3))
        conn.append(int(st.connectivity_after))
        cert.append(km1_host(H, pd.cpu().numpy()) == int(st.connectivity_after)
                    and int(st.connectivity_before) - int(st.gain) == int(st.connectivity_after))
        pairs.append(int(st.pairs))
        parts.append({f: round(getattr(st, "ms_" + f), 1)
                      for f in ("pairs", "prepare", "flow", "finish", "apply")})
    hg.close()
    out = {"workload": f"ring n={n} m={n * 3 // 2} k=64 (2+Zipf(2.5) <= 10000, 5% moved)",
           "pins_H": int(H.p), "group_ctas": G, "group_autotune": tune,
           "pairs_split_over_ranks": world,
           "seconds_per_round": secs, "connectivity_minus_1": conn, "pairs_per_round": pairs,
           "round_parts_ms": parts, "certificate": all(cert)}
    if fc_ms:
        out["flowcutter_launch_ms"] = fc_ms
    return out


def kway_compare(hfp, ctx, args):
    """Plain vs batched vs batched + learned rounds from one start partition
    (seed 1001, held out from the scheduler's training seeds)."""
    import torch
    from paper_2201_01556_gb300 import eval_scheduler, scheduler, train_scheduler
    n, k = args.compare_n, 64
    inst = synth.instance("ring_n8M_zipf_k64", 1001, n=n, m=n * 3 // 2)
    H, part = inst["H"], inst["part"]
    loaded = train_scheduler.load_params()
    mlp = torch.from_numpy(loaded[0]).cuda() if loaded is not None else None
    r = eval_scheduler.compare(hfp, scheduler, ctx, H, part, k, args.compare_rounds, mlp,
                               plain=True) if mlp is not None else None
    out = {"workload": f"ring n={n} m={n * 3 // 2} k={k} seed 1001 (held out)",
           "rounds_max": args.compare_rounds}
    if r is None:
        out["unavailable"] = "no committed scheduler weights"
        return out
    for a, v in r.items():
        out[a] = {"seconds": round(v["seconds"], 3), "pairs": v["pairs"],
                  "rounds": len(v["connectivity"]),
                  "connectivity_minus_1": v["connectivity"][-1]}
    out["plain_identical_to_batched"] = r["plain"]["identical_to_batched"]
    b = out["batched"]["connectivity_minus_1"]
    out["learned_vs_unpruned"] = out["learned"]["connectivity_minus_1"] / b - 1.0 if b else None
    out["within_0.5pct"] = out["learned_vs_unpruned"] is not None and \
        out["learned_vs_unpruned"] <= 0.005
    out["speedup_batched_over_plain"] = out["plain"]["seconds"] / out["batched"]["seconds"]
    out["speedup_learned_over_plain"] = out["plain"]["seconds"] / out["learned"]["seconds"]
    if "active" in out and b:
        out["active_vs_unpruned"] = out["active"]["connectivity_minus_1"] / b - 1.0
        out["speedup_active_over_plain"] = out["plain"]["seconds"] / out["active"]["seconds"]
    out["scheduler_training"] = loaded[1]
    return out


def host_cpu():
    """Host core count and CPU model (for the CPU baselines)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if model is None:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    import platform
    return os.cpu_count(), model or platform.machine()


def cpu_baselines(args, full_inst, gpu_value):
    """The oracle on the 1/10 sample and SeqPR on the full workload."""
    import oracle
    nproc, model = host_cpu()
    sinst = synth.instance(WORKLOAD, args.seed, **SAMPLE)
    p, dt, _ = oracle_step(sinst)
    golden = None
    try:
        with open(os.path.join(ROOT, "tests", "golden", f"{WORKLOAD}_seed1_maxflow.json")) as f:
            golden = json.load(f).get("oracle_seconds")
    except (OSError, ValueError):
        pass
    out = {"value": p / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"1/10-size sample: ring n={SAMPLE['n']}, m={SAMPLE['m']}, radius="
                     f"{SAMPLE['radius']} ({p} Lawler-network pins), one run, {dt:.1f} s; "
                     f"Dinic is super-linear here, so the sample flatters the oracle",
           "nproc": nproc, "cpu_model": model,
           "oracle_full_size_seconds": golden,
           "oracle_full_size_note": "the oracle on the full workload when its golden file was "
                                    "written (tests/golden), one core"}
    if not args.no_seqpr:
        H = full_inst["H"]
        t0 = time.perf_counter()
        net = oracle.build_network(H, full_inst["part"], full_inst["region"])
        r = oracle.seqpr(net)
        ds = time.perf_counter() - t0
        out["seqpr"] = {"value": net.p / ds, "unit": UNIT, "seconds": round(ds, 2), "cores": 1,
                        "kind": "sequential FIFO push-relabel with global relabeling (SeqPR)",
                        "sample": "the full workload", "flow": r.flow,
                        "gpu_over_seqpr": gpu_value / (net.p / ds)}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    # smaller rings of the same generator, for profiling captures
    ap.add_argument("--n", type=int, default=None)
    ap.add_argument("--m", type=int, default=None)
    ap.add_argument("--radius", type=int, default=None)
    ap.add_argument("--kway-rounds", type=int, default=2,
                    help="k-way refinement rounds to time (0: none)")
    ap.add_argument("--kway-n", type=int, default=8_000_000)
    ap.add_argument("--kway-group", type=int, default=0,
                    help="CTAs per FlowCutter problem; 0: hfp_autotune_round picks from 4, 8, 16")
    ap.add_argument("--compare-n", type=int, default=200_000,
                    help="ring size of the plain / batched / learned comparison (0: skip)")
    ap.add_argument("--compare-rounds", type=int, default=3)
    ap.add_argument("--no-seqpr", action="store_true", help="skip the full-size SeqPR timing")
    args = ap.parse_args()
    rank, world, local = env_rank()
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2201_01556_gb300 import hfp
    hfp.load()

    inst = synth.instance(WORKLOAD, args.seed, n=args.n, m=args.m, radius=args.radius)
    H, part, region = inst["H"], inst["part"], inst["region"]
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).cuda()
    d_off, d_pins, d_netw, d_nodew = dev(H.net_off), dev(H.pins), dev(H.net_w), dev(H.node_w)
    d_region, d_side = dev(region), dev(part)
    stream = torch.cuda.current_stream()
    ctx = hfp.ctx_create(local, stream.cuda_stream)
    out_region = torch.empty(len(region), dtype=torch.uint8, device="cuda")
    flush = torch.empty(2 * L2_BYTES, dtype=torch.uint8, device="cuda")

    def step(keep_stats=None):
        net = hfp.build_flow_network(ctx, d_off, d_pins, d_netw, d_nodew, d_region, d_side, H.n)
        flow = hfp.max_flow(net)
        ws = hfp.min_cut_source_side_device(net, out_region)
        if keep_stats is not None:
            keep_stats.append((net.info.p_pins, hfp.net_stats(net), flow, ws))
        net.close()
        return flow

    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = Clocks(local)
    clocks.start()
    launches0 = hfp.kernel_launches()
    stats = []
    ms = []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step(stats)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    launches = hfp.kernel_launches() - launches0
    clk = clocks.stop()
    total_ms = sum(ms)
    if dist:
        t = torch.tensor([total_ms], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
        dist.barrier()
    p_pins = stats[0][0]
    value = world * p_pins * args.steps / (total_ms / 1e3)

    # end to end through the public API with host buffers
    e2e_ms = []
    h2d = (H.net_off.nbytes + H.pins.nbytes + H.net_w.nbytes + H.node_w.nbytes + region.nbytes
           + part.nbytes)
    d2h = len(region) + 8
    for _ in range(0 if args.no_e2e else max(1, min(args.steps, 3))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        net = hfp.build_flow_network(ctx, H.net_off, H.pins, H.net_w, H.node_w, region, part, H.n)
        hfp.max_flow(net)
        _, reg, _, _ = hfp.min_cut_source_side(net, lawler=False, cut_cap=0)
        torch.cuda.synchronize()
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
        net.close()
    e2e_value = world * p_pins / (statistics.mean(e2e_ms) / 1e3) if e2e_ms else None
    kway = {}
    if args.kway_rounds > 0:
        kway["batched"] = kway_batched(hfp, ctx, args, world)
    if args.compare_n > 0 and world == 1:
        kway["compare"] = kway_compare(hfp, ctx, args)

    if rank != 0:
        return 0
    # roofline of the dominant kernel (the persistent flow engine)
    eng_ns = sum(s[1]["engine_ns"] for s in stats)
    eng_launches = sum(s[1]["engine_launches"] for s in stats)
    model = sum(s[1]["items_hyper"] * B_HYPER + s[1]["items_net"] * B_NET
                + s[1]["node_visits"] * B_NODE + s[1]["pushes"] * B_PUSH for s in stats)
    peak, peak_kind = load_peaks()
    achieved = (model / eng_launches) / (eng_ns / eng_launches / 1e9) / 1e9 if eng_ns else None
    ratio = engine_traffic_ratio()
    traffic = ratio * model / eng_launches if (ratio is not None and eng_launches) else None
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": (achieved / peak) if achieved else None, "traffic": traffic,
            "traffic_note": "DRAM bytes per launch, scaled from the ncu capture in "
                            "profiles/engine_kernel_ring_n1M.md by modelled bytes"
                            if traffic is not None else "kernel changed since the ncu capture",
            "kernel": "engine_kernel", "peak_kind": peak_kind,
            "engine_ms_per_step": eng_ns / 1e6 / args.steps,
            "engine_launches_per_step": eng_launches / args.steps}
    st = stats[0][1]
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": WORKLOAD if args.n is None else f"{WORKLOAD} scaled to n={H.n}",
                       "seed": args.seed, "n": H.n,
                       "m": H.m, "pins_H": H.p, "region": len(region), "lawler_pins": p_pins,
                       "flow": stats[0][2], "source_weight": stats[0][3],
                       "l2": "flushed between timed steps (2x L2 buffer write)",
                       "parallelism": f"replicas{world}"},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": int(launches),
            "clocks": clk, "roofline": roof,
            "engine": {"rounds": st["rounds"], "global_relabels": st["global_relabels"],
                       "gr_levels": st["gr_levels"], "pushes": st["pushes"],
                       "gr_queue_entries": st["gr_queue_entries"],
                       "gr_queue_overflows": st["gr_queue_overflows"]}}
    if kway:
        line["kway"] = kway
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baselines(args, inst, value)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
