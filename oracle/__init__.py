"""CPU oracle for the flow-based refinement hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  It shares no
code with the CUDA library (``paper_2201_01556_gb300``) and never imports it.

The C routines in ``oracle.c`` are plain textbook code on the explicit Lawler
expansion (Section 2); this module only marshals numpy arrays.  Every function
cites the paper passage it follows.  Parity status of each part:
  - network construction, max flow, S_r / T_r: pinned (brute force, scipy's
    maximum_flow, Edmonds-Karp vs Dinic, hand-built fixtures, invariants);
  - FlowCutter: pinned by invariants and brute force on small cases only; the
    paper prints no worked example, so the piercing sequence itself follows
    the stated readings (parity of the sequence is by construction).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lib = None

OK, ERR_INVALID, ERR_OOM, ITER_LIMIT, NO_BALANCED_CUT, ABORTED_WORSE = 0, -1, -2, -4, -5, -6
DIST_FAR = (1 << 20) - 1


def build(force: bool = False) -> str:
    """Compile oracle.c (plain gcc, portable flags)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


class _FcResult(ctypes.Structure):
    _fields_ = [("flow", ctypes.c_int64), ("iterations", ctypes.c_int32),
                ("n_pierced", ctypes.c_int32), ("result_side", ctypes.c_int32),
                ("status", ctypes.c_int32), ("source_weight", ctypes.c_int64),
                ("bulk_steps", ctypes.c_int32), ("mb_steps", ctypes.c_int32)]


class _FcOptions(ctypes.Structure):
    _fields_ = [("bulk_beta_pct", ctypes.c_int32), ("bulk_warmup", ctypes.c_int32),
                ("mb_reps", ctypes.c_int32), ("pad", ctypes.c_int32)]


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P, i32, i64, u32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
        lib.or_build_network.restype = i64
        lib.or_build_network.argtypes = [i32, i32, P, P, P, P, P, P, i32, P, P, P, P, P, P]
        lib.or_dist_from_cut.restype = i32
        lib.or_dist_from_cut.argtypes = [i32, i32, P, P, P, P, i32, P]
        lib.or_dedup_nets.restype = i32
        lib.or_dedup_nets.argtypes = [i32, P, P, P, P, P, P, P, P, P]
        lib.or_seqpr.restype = i64
        lib.or_seqpr.argtypes = [i32, i32, P, P, P, P, P, P]
        lib.or_lawler_create.restype = P
        lib.or_lawler_create.argtypes = [i32, i32, P, P, P, P]
        lib.or_lawler_free.restype = None
        lib.or_lawler_free.argtypes = [P]
        lib.or_lawler_nodes.restype = i32
        lib.or_lawler_nodes.argtypes = [P]
        lib.or_lawler_arcs.restype = i64
        lib.or_lawler_arcs.argtypes = [P]
        lib.or_augment.restype = i64
        lib.or_augment.argtypes = [P, P, P, i32]
        lib.or_reset_flow.restype = None
        lib.or_reset_flow.argtypes = [P]
        lib.or_flow_value.restype = i64
        lib.or_flow_value.argtypes = [P, P]
        lib.or_reach_from.restype = None
        lib.or_reach_from.argtypes = [P, P, P]
        lib.or_reach_to.restype = None
        lib.or_reach_to.argtypes = [P, P, P]
        lib.or_export_arcs.restype = None
        lib.or_export_arcs.argtypes = [P, P, P, P, P]
        lib.or_bruteforce.restype = i32
        lib.or_bruteforce.argtypes = [i32, i32, P, P, P, P, i64, P, P, P, P, P]
        lib.or_flowcutter_ex.restype = i32
        lib.or_flowcutter_ex.argtypes = [P, i64, P, P, P, u32, i64, i32, i32, P, P, P, P, i32,
                                         P]
        lib.or_flowcutter.restype = i32
        lib.or_flowcutter.argtypes = [P, i64, P, P, P, u32, i64, i32, i32, P, P, P, i32,
                                      ctypes.POINTER(_FcResult)]
        _lib = lib
    return _lib


def _p(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


@dataclass
class FlowNetwork:
    """Flow hypergraph of a region (Section 6): hypernode 0 = s, 1 = t,
    2 + i = region[i]; nets in ascending id of H; pins of a net are its region
    pins in H's order, then s, then t."""
    n_nodes: int
    m_nets: int
    net_off: np.ndarray    # uint32[m_nets+1]
    pins: np.ndarray       # int32[p]
    net_w: np.ndarray      # int32[m_nets]
    net_gid: np.ndarray    # int32[m_nets]: id of the net in H
    node_w: np.ndarray     # int64[n_nodes]

    @property
    def p(self) -> int:
        return int(self.net_off[-1])

    @property
    def lawler_nodes(self) -> int:
        return self.n_nodes + 2 * self.m_nets


def build_network(H, side, region) -> FlowNetwork:
    """Section 6, "Construction Algorithms", first algorithm (net scan)."""
    lib = _load()
    side = _c(side, np.int32)
    region = _c(region, np.int32)
    nr = len(region)
    out_m = np.zeros(1, dtype=np.int32)
    cap_p = H.p + 2 * H.m + 1
    nnet_off = np.zeros(H.m + 1, dtype=np.uint32)
    npins = np.zeros(cap_p, dtype=np.int32)
    nnet_w = np.zeros(max(H.m, 1), dtype=np.int32)
    nnet_gid = np.zeros(max(H.m, 1), dtype=np.int32)
    nnode_w = np.zeros(nr + 2, dtype=np.int64)
    p = lib.or_build_network(H.n, H.m, _p(_c(H.net_off, np.uint32)), _p(_c(H.pins, np.int32)),
                             _p(_c(H.net_w, np.int32)), _p(_c(H.node_w, np.int32)), _p(side),
                             _p(region), nr, _p(out_m), _p(nnet_off), _p(npins), _p(nnet_w),
                             _p(nnet_gid), _p(nnode_w))
    if p < 0:
        raise ValueError(f"or_build_network failed: {p}")
    mm = int(out_m[0])
    return FlowNetwork(nr + 2, mm, nnet_off[: mm + 1].copy(), npins[:p].copy(),
                       nnet_w[:mm].copy(), nnet_gid[:mm].copy(), nnode_w)


def dedup_network(net: FlowNetwork) -> FlowNetwork:
    """Identical net removal (Section 6, "Identical Net Removal"), read as in
    oracle.c: the flow hypergraph with every net merged into the smallest-id
    net with the same pin set (found through (fingerprint, size) groups)."""
    lib = _load()
    m = net.m_nets
    off = np.zeros(m + 1, np.uint32)
    pins = np.zeros(max(net.p, 1), np.int32)
    w = np.zeros(max(m, 1), np.int32)
    gid = np.zeros(max(m, 1), np.int32)
    rep = np.zeros(max(m, 1), np.int32)
    mm = lib.or_dedup_nets(m, _p(_c(net.net_off, np.uint32)), _p(_c(net.pins, np.int32)),
                           _p(_c(net.net_w, np.int32)), _p(_c(net.net_gid, np.int32)), _p(off),
                           _p(pins), _p(w), _p(gid), _p(rep))
    if mm < 0:
        raise MemoryError("or_dedup_nets failed")
    return FlowNetwork(net.n_nodes, int(mm), off[: mm + 1].copy(), pins[: off[mm]].copy(),
                       w[:mm].copy(), gid[:mm].copy(), net.node_w.copy())


def dist_from_cut(H, side, region) -> np.ndarray:
    """Hop distance from the original cut inside the region (reading of
    Section 6 "Region Growing" / Section 7 "Piercing"); per region position."""
    lib = _load()
    region = _c(region, np.int32)
    dist = np.zeros(max(len(region), 1), dtype=np.int32)
    rc = lib.or_dist_from_cut(H.n, H.m, _p(_c(H.net_off, np.uint32)), _p(_c(H.pins, np.int32)),
                              _p(_c(side, np.int32)), _p(region), len(region), _p(dist))
    if rc != 0:
        raise ValueError(f"or_dist_from_cut failed: {rc}")
    return dist[: len(region)]


class Lawler:
    """Explicit Lawler expansion of a flow hypergraph (Section 2) with a flow
    on its arcs.  Node ids: hypernode h, in-node n_nodes + e, out-node
    n_nodes + m_nets + e."""

    def __init__(self, net: FlowNetwork):
        lib = _load()
        self.net = net
        self._keep = (_c(net.net_off, np.uint32), _c(net.pins, np.int32),
                      _c(net.net_w, np.int32), _c(net.node_w, np.int64))
        self.h = lib.or_lawler_create(net.n_nodes, net.m_nets, *[_p(a) for a in self._keep])
        if not self.h:
            raise MemoryError("or_lawler_create failed")
        self.N = lib.or_lawler_nodes(self.h)
        self.A = lib.or_lawler_arcs(self.h)

    def __del__(self):
        if getattr(self, "h", None):
            _load().or_lawler_free(self.h)
            self.h = None

    def mask(self, nodes) -> np.ndarray:
        m = np.zeros(self.N, dtype=np.uint8)
        m[np.asarray(list(nodes), dtype=np.int64)] = 1
        return m

    def augment(self, S: np.ndarray, T: np.ndarray, algo: str = "dinic") -> int:
        """Augment the current flow to a maximum S-T flow; returns flow added."""
        r = _load().or_augment(self.h, _p(_c(S, np.uint8)), _p(_c(T, np.uint8)),
                               1 if algo == "ek" else 0)
        if r < 0:
            raise MemoryError("augment failed")
        return int(r)

    def reset(self):
        _load().or_reset_flow(self.h)

    def flow_value(self, S: np.ndarray) -> int:
        return int(_load().or_flow_value(self.h, _p(_c(S, np.uint8))))

    def reach_from(self, seed: np.ndarray) -> np.ndarray:
        """Nodes reachable from `seed` by residual arcs (source-side cut)."""
        out = np.zeros(self.N, dtype=np.uint8)
        _load().or_reach_from(self.h, _p(_c(seed, np.uint8)), _p(out))
        return out

    def reach_to(self, seed: np.ndarray) -> np.ndarray:
        """Nodes with a residual path into `seed` (sink-side cut)."""
        out = np.zeros(self.N, dtype=np.uint8)
        _load().or_reach_to(self.h, _p(_c(seed, np.uint8)), _p(out))
        return out

    def arcs(self):
        A = self.A
        tail = np.zeros(A, np.int32); head = np.zeros(A, np.int32)
        cap = np.zeros(A, np.int64); flow = np.zeros(A, np.int64)
        _load().or_export_arcs(self.h, _p(tail), _p(head), _p(cap), _p(flow))
        return tail, head, cap, flow


@dataclass
class MinCut:
    flow: int
    source_side: np.ndarray   # uint8[N]: S_r, the minimal source side
    sink_side: np.ndarray     # uint8[N]: T_r, the minimal sink side
    lawler: Lawler


def max_flow_min_cut(net: FlowNetwork, algo: str = "dinic") -> MinCut:
    """Maximum s-t flow on the Lawler expansion and both minimal cut sides:
    S_r by forward residual BFS from s, T_r by reverse BFS into t (Section 2,
    last paragraph of "Flows")."""
    G = Lawler(net)
    S = G.mask([0])
    T = G.mask([1])
    G.augment(S, T, algo)
    return MinCut(G.flow_value(S), G.reach_from(S), G.reach_to(T), G)


@dataclass
class SeqPRResult:
    flow: int
    source_side: np.ndarray   # uint8[N]: S_r
    sink_side: np.ndarray     # uint8[N]: T_r
    pushes: int
    relabels: int
    global_relabels: int


def seqpr(net: FlowNetwork) -> SeqPRResult:
    """Sequential FIFO push-relabel on the flow hypergraph with global
    relabeling, to a maximum preflow (the paper's SeqPR baseline, Appendix
    "Flow Algorithms"; Section 2, "Push-Relabel Algorithm"), with both
    minimal cut sides."""
    lib = _load()
    N = net.lawler_nodes
    src = np.zeros(max(N, 1), np.uint8)
    snk = np.zeros(max(N, 1), np.uint8)
    st = np.zeros(4, np.int64)
    f = lib.or_seqpr(net.n_nodes, net.m_nets, _p(_c(net.net_off, np.uint32)),
                     _p(_c(net.pins, np.int32)), _p(_c(net.net_w, np.int32)), _p(src), _p(snk),
                     _p(st))
    if f < 0:
        raise MemoryError(f"or_seqpr failed: {f}")
    return SeqPRResult(int(f), src[:N], snk[:N], int(st[0]), int(st[1]), int(st[2]))


def cut_weight(net: FlowNetwork, in_source_h: np.ndarray) -> int:
    """Hypergraph cut of a bipartition of the flow hypergraph's hypernodes:
    sum of w(e) over nets with pins on both sides (Section 2)."""
    side = np.asarray(in_source_h, dtype=bool)
    total = 0
    for e in range(net.m_nets):
        ps = net.pins[net.net_off[e]:net.net_off[e + 1]]
        s = side[ps]
        if s.any() and not s.all():
            total += int(net.net_w[e])
    return total


def bruteforce(net: FlowNetwork, max_w: int = -1):
    """Enumerate every bipartition of the region (<= 24 vertices): minimum cut,
    intersection / union of the minimising source sets (as region bitmasks),
    number of minimisers, and the minimum cut among bipartitions with both
    sides <= max_w (-1 if none)."""
    lib = _load()
    mc = np.zeros(1, np.int64); am = np.zeros(1, np.uint32); om = np.zeros(1, np.uint32)
    nm = np.zeros(1, np.int64); mb = np.zeros(1, np.int64)
    rc = lib.or_bruteforce(net.n_nodes, net.m_nets, _p(_c(net.net_off, np.uint32)),
                           _p(_c(net.pins, np.int32)), _p(_c(net.net_w, np.int32)),
                           _p(_c(net.node_w, np.int64)), int(max_w), _p(mc), _p(am), _p(om),
                           _p(nm), _p(mb))
    if rc != 0:
        raise ValueError("bruteforce: too many region vertices")
    return dict(min_cut=int(mc[0]), and_mask=int(am[0]), or_mask=int(om[0]),
                n_min=int(nm[0]), min_balanced=int(mb[0]))


def max_block_weight(total_w: int, k: int, eps_pct: int) -> int:
    """Balance bound L = (1 + eps) * ceil(c(V) / k) (Section 2), in exact
    integers: floor((100 + eps_pct) * ceil(W / k) / 100)."""
    return ((100 + eps_pct) * (-(-total_w // k))) // 100


@dataclass
class FlowCutterResult:
    status: int
    flow: int
    iterations: int
    final_side: np.ndarray     # uint8[n_nodes]
    pierce_side: np.ndarray    # int32[n_pierced]
    pierce_node: np.ndarray    # int32[n_pierced] (flow-hypergraph node ids)
    result_side: int
    source_weight: int
    bulk_steps: int = 0        # iterations that pierced several nodes
    mb_steps: int = 0          # path-free piercings after the first balanced cut


def flowcutter(net: FlowNetwork, max_w: int, orig_side: np.ndarray, dist: np.ndarray,
               gid: np.ndarray, seed: int = 0, flow_bound: int = -1, max_iter: int = 1 << 30,
               recompute: bool = False, bulk_beta_pct: int = 0, bulk_warmup: int = 3,
               mb_reps: int = 0) -> FlowCutterResult:
    """FlowCutter core, Algorithm 2 (Section 7), with the piercing rules of
    Section 7 "Piercing" as read in oracle.c.  Per hypernode arrays:
    orig_side (0/1), dist (distance from the original cut), gid (id in H).
    bulk_beta_pct > 0 turns on bulk piercing (Section 7, "Bulk Piercing";
    beta in percent, `bulk_warmup` single piercings per side first);
    mb_reps > 0 continues to the most balanced cut (Section 7, "Most
    Balanced Cut") with that many repetitions.  The readings are in
    oracle.c."""
    lib = _load()
    G = Lawler(net)
    nh = net.n_nodes
    final = np.zeros(nh, np.uint8)
    cap = (nh + 1) * (1 + max(int(mb_reps), 0))
    ps = np.zeros(cap, np.int32); pn = np.zeros(cap, np.int32)
    res = _FcResult()
    opt = _FcOptions(int(bulk_beta_pct), int(bulk_warmup), int(mb_reps), 0)
    lib.or_flowcutter_ex(G.h, int(max_w), _p(_c(orig_side, np.int32)), _p(_c(dist, np.int32)),
                         _p(_c(gid, np.int32)), ctypes.c_uint32(seed & 0xFFFFFFFF),
                         int(flow_bound), int(min(max_iter, 2**31 - 1)), 1 if recompute else 0,
                         ctypes.byref(opt), _p(final), _p(ps), _p(pn), cap, ctypes.byref(res))
    k = min(res.n_pierced, cap)
    return FlowCutterResult(res.status, res.flow, res.iterations, final, ps[:k].copy(),
                            pn[:k].copy(), res.result_side, res.source_weight, res.bulk_steps,
                            res.mb_steps)


def node_arrays(net: FlowNetwork, side, region, dist_region):
    """Per-hypernode orig_side, dist and gid arrays for flowcutter():
    s is side 0, t side 1; region vertices take side[v] and their distance."""
    region = np.asarray(region, dtype=np.int64)
    orig = np.zeros(net.n_nodes, np.int32)
    orig[1] = 1
    orig[2:] = np.asarray(side)[region]
    dist = np.zeros(net.n_nodes, np.int32)
    dist[2:] = dist_region
    gid = np.full(net.n_nodes, -1, np.int32)
    gid[2:] = region
    return orig, dist, gid


# ---------------------------------------------------------------------------
# k-way refinement (Section 4, Algorithm 1; Section 5; Section 6)

def _kway_sig():
    lib = _load()
    P, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    if not hasattr(lib, "_kway_ready"):
        lib.or_connectivity.restype = i64
        lib.or_connectivity.argtypes = [i32, P, P, P, P, i32]
        lib.or_quotient.restype = None
        lib.or_quotient.argtypes = [i32, P, P, P, P, i32, P, P]
        lib.or_grow_region.restype = i32
        lib.or_grow_region.argtypes = [i32, i32, P, P, P, P, i32, i32, i32, i32, P, P, P]
        lib.or_apply_moves.restype = i64
        lib.or_apply_moves.argtypes = [i32, i32, P, P, P, P, P, i32, i64, P, i32, P, P]
        lib._kway_ready = True
    return lib


def _hp(H):
    return (_c(H.net_off, np.uint32), _c(H.pins, np.int32), _c(H.net_w, np.int32),
            _c(H.node_w, np.int32))


def connectivity(H, part, k: int) -> int:
    """(lambda - 1)(Pi) = sum_e (lambda(e) - 1) w(e) (Section 2)."""
    off, pins, nw, _ = _hp(H)
    return int(_kway_sig().or_connectivity(H.m, _p(off), _p(pins), _p(nw),
                                           _p(_c(part, np.int32)), k))


def quotient(H, part, k: int):
    """Quotient graph (Section 5): per block pair i < j, number and weight of
    nets with pins in both.  Returns (nets[k, k], weight[k, k])."""
    off, pins, nw, _ = _hp(H)
    a = np.zeros((k, k), np.int64)
    b = np.zeros((k, k), np.int64)
    _kway_sig().or_quotient(H.m, _p(off), _p(pins), _p(nw), _p(_c(part, np.int32)), k, _p(a),
                            _p(b))
    return a, b


def grow_region(H, part, bi: int, bj: int, alpha_eps_pct: int = 48, delta: int = 2):
    """Region of the pair (bi, bj) and the distances of its vertices
    (Section 6, "Region Growing"; see oracle.c for the readings)."""
    off, pins, nw, cw = _hp(H)
    region = np.zeros(max(H.n, 1), np.int32)
    dist = np.zeros(max(H.n, 1), np.int32)
    nr = np.zeros(1, np.int32)
    _kway_sig().or_grow_region(H.n, H.m, _p(off), _p(pins), _p(cw), _p(_c(part, np.int32)),
                               bi, bj, alpha_eps_pct, delta, _p(region), _p(dist), _p(nr))
    k = int(nr[0])
    return region[:k].copy(), dist[:k].copy()


def apply_moves(H, part: np.ndarray, k: int, max_w: int, moves: np.ndarray):
    """Section 5, "Apply Moves": returns (gain, applied, n_valid); part is
    updated in place.  moves: int32[n, 3] rows (vertex, from, to)."""
    off, pins, nw, cw = _hp(H)
    assert part.dtype == np.int32 and part.flags.c_contiguous
    mv = _c(moves, np.int32).reshape(-1)
    applied = np.zeros(1, np.int32)
    nv = np.zeros(1, np.int32)
    g = _kway_sig().or_apply_moves(H.n, H.m, _p(off), _p(pins), _p(nw), _p(cw), _p(part), k,
                                   int(max_w), _p(mv) if len(mv) else None, len(mv) // 3,
                                   _p(applied), _p(nv))
    return int(g), int(applied[0]), int(nv[0])


@dataclass
class PairResult:
    bi: int
    bj: int
    status: int
    moves: np.ndarray        # int32[n, 3]: (vertex, from, to)
    delta_exp: int
    flow: int
    original_cut: int
    region_size: int
    pins: int


def refine_block_pair(H, part, k: int, bi: int, bj: int, eps_pct: int = 3,
                      alpha_eps_pct: int = 48, delta: int = 2, seed: int = 0) -> PairResult:
    """One block pair of Algorithm 1: region (Section 6), flow network,
    FlowCutter with the k-way balance bound and the original pair cut as flow
    bound (Section 7; Section 8.3 "Flow Value"), moves and the expected gain
    Delta_exp = original cut on the network's nets - final flow."""
    part = np.asarray(part, np.int32)
    side = np.where(part == bi, 0, np.where(part == bj, 1, -1)).astype(np.int32)
    region, dist = grow_region(H, part, bi, bj, alpha_eps_pct, delta)
    net = build_network(H, side, region)
    L = max_block_weight(int(np.asarray(H.node_w, np.int64).sum()), k, eps_pct)
    in_src = np.zeros(net.n_nodes, bool)
    in_src[0] = True
    in_src[2:] = side[region] == 0
    cut0 = cut_weight(net, in_src)
    orig, d, gid = node_arrays(net, side, region, dist)
    r = flowcutter(net, L, orig, d, gid, seed=seed, flow_bound=cut0)
    empty = np.zeros((0, 3), np.int32)
    if r.status != OK:
        return PairResult(bi, bj, r.status, empty, 0, r.flow, cut0, len(region), net.p)
    fin = r.final_side[2:]
    ch = np.nonzero(fin != side[region])[0]
    frm = np.where(side[region[ch]] == 0, bi, bj)
    to = np.where(fin[ch] == 0, bi, bj)
    moves = np.stack([region[ch], frm, to], axis=1).astype(np.int32) if len(ch) else empty
    return PairResult(bi, bj, OK, moves, cut0 - r.flow, r.flow, cut0, len(region), net.p)


def refine_round(H, part, k: int, eps_pct: int = 3, alpha_eps_pct: int = 48, delta: int = 2,
                 seed: int = 0, pairs=None):
    """One synchronous round of Algorithm 1: every pair of adjacent blocks is
    refined against the same partition; the move sets with Delta_exp >= 0 are
    applied in descending Delta_exp (ties: ascending (i, j)) with the
    conflict rules of Section 5.  pairs: optional list of (i, j) to refine
    (default: every quotient-graph edge).  Returns (new part, total gain,
    results, gains)."""
    part = np.array(part, dtype=np.int32)
    if pairs is None:
        qn, _ = quotient(H, part, k)
        pairs = [(i, j) for i in range(k) for j in range(i + 1, k) if qn[i, j] > 0]
    res = [refine_block_pair(H, part, k, i, j, eps_pct, alpha_eps_pct, delta, seed)
           for i, j in pairs]
    total, gains = apply_round(H, part, k, res, eps_pct)
    return part, total, res, gains


def apply_round(H, part: np.ndarray, k: int, res, eps_pct: int = 3):
    """The apply step of a round (Section 5, "Apply Moves"): the move sets
    of the results with status OK, Delta_exp >= 0 and moves, in descending
    Delta_exp (ties: ascending (i, j)), each through apply_moves.  part
    (int32) is updated in place.  Returns (total gain, {(i, j): (gain,
    applied, valid moves)})."""
    L = max_block_weight(int(np.asarray(H.node_w, np.int64).sum()), k, eps_pct)
    order = sorted((r for r in res if r.status == OK and r.delta_exp >= 0 and len(r.moves)),
                   key=lambda r: (-r.delta_exp, r.bi, r.bj))
    gains = {}
    total = 0
    for r in order:
        g, applied, nv = apply_moves(H, part, k, L, r.moves)
        gains[(r.bi, r.bj)] = (g, applied, nv)
        total += g
    return total, gains
