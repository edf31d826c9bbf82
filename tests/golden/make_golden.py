"""Writes the full-size expected values in tests/golden/ from the CPU oracle.

Only oracle/ (and the seeded generators in synth/) are called: no value here
comes from the CUDA path.  Each run takes tens of minutes on one core.

    python tests/golden/make_golden.py maxflow     # 2M-vertex ring, seed 1
    python tests/golden/make_golden.py flowcutter  # 500k-vertex ring, seed 1
"""
import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import synth  # noqa: E402


def digest(mask: np.ndarray) -> str:
    """sha256 of a 0/1 vector packed to bits (little bit order)."""
    return hashlib.sha256(np.packbits(np.asarray(mask, dtype=np.uint8), bitorder="little")
                          .tobytes()).hexdigest()


def maxflow(seed: int = 1):
    inst = synth.instance("ring_n2M_zipf", seed)
    t0 = time.time()
    net = oracle.build_network(inst["H"], inst["part"], inst["region"])
    mc = oracle.max_flow_min_cut(net)
    out = {
        "citation": "Maximum flow and minimal cut sides on the Lawler expansion (Section 2, "
                    "'Flows' and 'Flows on Hypergraphs'; Section 6 construction), computed by "
                    "the CPU oracle (Dinic) on the 2,000,000-vertex ring workload.",
        "workload": "ring_n2M_zipf", "seed": seed,
        "n_nodes": net.n_nodes, "m_nets": net.m_nets, "p_pins": net.p,
        "flow": mc.flow,
        "source_side_count": int(mc.source_side.sum()),
        "source_side_sha256": digest(mc.source_side),
        "sink_side_count": int(mc.sink_side.sum()),
        "sink_side_sha256": digest(mc.sink_side),
        "oracle_seconds": round(time.time() - t0, 1),
    }
    with open(os.path.join(HERE, f"ring_n2M_zipf_seed{seed}_maxflow.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(out)


def flowcutter(seed: int = 1):
    inst = synth.instance("ring_n500k_zipf_fc", seed)
    H, part, region = inst["H"], inst["part"], inst["region"]
    t0 = time.time()
    net = oracle.build_network(H, part, region)
    L = oracle.max_block_weight(int(net.node_w.sum()), 2, 3)
    dist = oracle.dist_from_cut(H, part, region)
    orig, d, gid = oracle.node_arrays(net, part, region, dist)
    r = oracle.flowcutter(net, L, orig, d, gid, seed=seed)
    out = {
        "citation": "FlowCutter, Algorithm 2 (Section 7) with the piercing rules of Section 7 "
                    "'Piercing' as read in the oracle, on the 500,000-vertex ring workload "
                    "(vertex weights 1..4, eps = 0.03), computed by the CPU oracle.",
        "workload": "ring_n500k_zipf_fc", "seed": seed, "fc_seed": seed,
        "max_block_weight": L, "status": r.status, "flow": r.flow,
        "iterations": r.iterations, "result_side": r.result_side,
        "source_weight": r.source_weight,
        "pierce_side": r.pierce_side.tolist(), "pierce_node": r.pierce_node.tolist(),
        "final_side_sha256": digest(r.final_side[2:]),
        "final_side_count": int(r.final_side[2:].sum()),
        "oracle_seconds": round(time.time() - t0, 1),
    }
    with open(os.path.join(HERE, f"ring_n500k_zipf_fc_seed{seed}_flowcutter.json"), "w") as f:
        json.dump(out, f, indent=1)
    print({k: v for k, v in out.items() if k not in ("pierce_side", "pierce_node")})


if __name__ == "__main__":
    what = sys.argv[1] if len(sys.argv) > 1 else "maxflow"
    {"maxflow": maxflow, "flowcutter": flowcutter}[what]()
