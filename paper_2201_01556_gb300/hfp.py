"""Python binding of libhfp (include/hfp.h): argument marshalling only.

Every function here maps one-to-one onto a C entry point of the same name
(``build_flow_network`` -> ``hfp_build_flow_network`` ...).  Inputs are numpy
arrays (host memory) or CUDA torch tensors (device memory); outputs are
numpy arrays unless a device output is requested.  There is no fallback: if
libhfp.so cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import _build

OK = 0
ERR_INVALID, ERR_OOM, ERR_CUDA, ERR_ITER_LIMIT = -1, -2, -3, -4
NO_BALANCED_CUT, ABORTED_WORSE, ERR_BUFFER_TOO_SMALL, ERR_STATE = -5, -6, -7, -8
MEM_HOST, MEM_DEVICE = 0, 1

_lib = None


class HfpError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"hfp status {status}: {msg}")
        self.status = status


class _Hypergraph(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("m", ctypes.c_int32), ("net_off", ctypes.c_void_p),
                ("pins", ctypes.c_void_p), ("net_w", ctypes.c_void_p), ("node_w", ctypes.c_void_p)]


class _NetInfo(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int32), ("m_nets", ctypes.c_int32),
                ("p_pins", ctypes.c_int64), ("lawler_nodes", ctypes.c_int32),
                ("pad", ctypes.c_int32), ("total_weight", ctypes.c_int64)]


class _Stats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint64) for k in
                ("rounds", "global_relabels", "gr_levels", "items_hyper", "items_net",
                 "node_visits", "pushes", "engine_launches", "engine_ns", "gr_queue_entries",
                 "gr_queue_overflows")]


class Tuning(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint32) for k in ("gr_work_x100", "stall_rounds", "stall_nodes",
                                               "tail_enter", "tail_exit", "max_rounds",
                                               "bfs_enter", "bfs_exit", "pierce_relabel",
                                               "stall_rounds_pierce", "batch_cluster",
                                               "batch_big_ctas", "batch_big_groups",
                                               "async_gr", "gr_warps", "fused_rounds",
                                               "identical_nets", "batch_fused_rounds",
                                               "batch_async_gr", "parpr_block",
                                               "construction", "batch_gr_work_x100",
                                               "batch_stall_rounds_pierce", "wait_timeout_ms",
                                               "prep_streams")]


class RefineParams(ctypes.Structure):
    _fields_ = [("eps_pct", ctypes.c_int32), ("alpha_eps_pct", ctypes.c_int32),
                ("delta", ctypes.c_int32), ("seed", ctypes.c_uint32)]


class PairResult(ctypes.Structure):
    _fields_ = [("bi", ctypes.c_int32), ("bj", ctypes.c_int32), ("status", ctypes.c_int32),
                ("region_size", ctypes.c_int32), ("pins", ctypes.c_int64),
                ("original_cut", ctypes.c_int64), ("flow", ctypes.c_int64),
                ("delta_exp", ctypes.c_int64), ("n_moves", ctypes.c_int32),
                ("iterations", ctypes.c_int32), ("applied", ctypes.c_int32),
                ("valid_moves", ctypes.c_int32), ("gain", ctypes.c_int64),
                ("device_us", ctypes.c_int32), ("group_ctas", ctypes.c_int32)]


class RoundStats(ctypes.Structure):
    _fields_ = [("connectivity_before", ctypes.c_int64), ("connectivity_after", ctypes.c_int64),
                ("gain", ctypes.c_int64), ("moves_applied", ctypes.c_int64),
                ("pairs", ctypes.c_int32), ("pairs_improved", ctypes.c_int32),
                ("pairs_applied", ctypes.c_int32), ("pairs_skipped", ctypes.c_int32),
                ("ms_pairs", ctypes.c_float), ("ms_prepare", ctypes.c_float),
                ("ms_flow", ctypes.c_float), ("ms_finish", ctypes.c_float),
                ("ms_apply", ctypes.c_float), ("pad", ctypes.c_int32)]


class AdamParams(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_float), ("eps", ctypes.c_float), ("beta1", ctypes.c_double),
                ("beta2", ctypes.c_double)]


class _NetworkView(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int32), ("m_nets", ctypes.c_int32),
                ("p_pins", ctypes.c_int64), ("net_off", ctypes.c_void_p),
                ("pins", ctypes.c_void_p), ("net_w", ctypes.c_void_p),
                ("node_off", ctypes.c_void_p), ("inc_slot", ctypes.c_void_p),
                ("node_w", ctypes.c_void_p)]


class FcParams(ctypes.Structure):
    _fields_ = [("max_block_weight", ctypes.c_int64), ("flow_bound", ctypes.c_int64),
                ("seed", ctypes.c_uint32), ("max_iterations", ctypes.c_int32),
                ("bulk_beta_pct", ctypes.c_int32), ("bulk_warmup", ctypes.c_int32),
                ("mb_reps", ctypes.c_int32), ("pad", ctypes.c_int32)]


class _FcResult(ctypes.Structure):
    _fields_ = [("flow", ctypes.c_int64), ("source_weight", ctypes.c_int64),
                ("iterations", ctypes.c_int32), ("n_pierced", ctypes.c_int32),
                ("result_side", ctypes.c_int32), ("device_us", ctypes.c_int32),
                ("bulk_steps", ctypes.c_int32), ("mb_steps", ctypes.c_int32)]


class _FcTask(ctypes.Structure):
    _fields_ = [("net", ctypes.c_void_p), ("params", FcParams), ("final_side", ctypes.c_void_p),
                ("pierce_side", ctypes.c_void_p), ("pierce_node", ctypes.c_void_p),
                ("pierce_cap", ctypes.c_int32), ("status", ctypes.c_int32),
                ("result", _FcResult)]


def library_path() -> str:
    return _build.LIB


def load():
    """Load libhfp.so (building it first when sources are newer)."""
    global _lib
    if _lib is not None:
        return _lib
    if not _build.up_to_date():
        _build.build()
    if not os.path.exists(_build.LIB):
        raise ImportError("libhfp.so is missing: the CUDA library was not built")
    lib = ctypes.CDLL(_build.LIB)
    P, i32, i64, u32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
    sig = {
        "hfp_ctx_create": (i32, [P, i32, P]),
        "hfp_ctx_destroy": (None, [P]),
        "hfp_last_error": (ctypes.c_char_p, []),
        "hfp_kernel_launches": (ctypes.c_uint64, []),
        "hfp_build_flow_network": (i32, [P, ctypes.POINTER(_Hypergraph), i32, P, i32, P, P, P]),
        "hfp_net_destroy": (None, [P]),
        "hfp_net_get_info": (i32, [P, ctypes.POINTER(_NetInfo)]),
        "hfp_net_export": (i32, [P, i32, P, P, P, P, P, P, P, P]),
        "hfp_net_export_flow": (i32, [P, i32, P, P, P, P, P, P]),
        "hfp_net_get_stats": (i32, [P, ctypes.POINTER(_Stats)]),
        "hfp_max_flow": (i32, [P, P]),
        "hfp_min_cut_source_side": (i32, [P, i32, P, P, P, i32, P, P]),
        "hfp_min_cut_sink_side": (i32, [P, i32, P, P, P]),
        "hfp_pierce_and_augment": (i32, [P, i32, P, i32, ctypes.POINTER(FcParams), P, P]),
        "hfp_flowcutter": (i32, [P, ctypes.POINTER(FcParams), P, P, P, i32,
                                 ctypes.POINTER(_FcResult)]),
        "hfp_max_flow_noalloc": (i32, [i32, P, ctypes.POINTER(_NetworkView), P, P, P]),
        "hfp_net_enable_trace": (i32, [P, i32]),
        "hfp_hgraph_create": (i32, [P, ctypes.POINTER(_Hypergraph), i32, P]),
        "hfp_hgraph_destroy": (None, [P]),
        "hfp_connectivity": (i32, [P, P, i32, P]),
        "hfp_refine_block_pair": (i32, [P, P, i32, i32, i32, ctypes.POINTER(RefineParams), P,
                                        i32, ctypes.POINTER(PairResult)]),
        "hfp_refine_round": (i32, [P, P, i32, ctypes.POINTER(RefineParams), P, ctypes.c_float,
                                   ctypes.POINTER(RoundStats), P, i32, P]),
        "hfp_ctx_get_tuning": (i32, [P, ctypes.POINTER(Tuning)]),
        "hfp_ctx_set_tuning": (i32, [P, ctypes.POINTER(Tuning)]),
        "hfp_net_get_trace": (i32, [P, P, P, P, i32, P]),
        "hfp_pair_features": (i32, [P, P, i32, i32, P, P, P, i32, P]),
        "hfp_flowcutter_batch": (i32, [P, P, i32, i32]),
        "hfp_ctx_batch_profile": (i32, [P, P, P, P, P, i32, i32]),
        "hfp_ctx_wait_selftest": (i32, [P, i32, ctypes.POINTER(ctypes.c_float)]),
        "hfp_ctx_last_batch_layout": (i32, [P, P, P, P]),
        "hfp_refine_round_batched": (i32, [P, P, i32, ctypes.POINTER(RefineParams), P,
                                           ctypes.c_float, i32, ctypes.POINTER(RoundStats), P,
                                           i32, P, P]),
        "hfp_autotune_round": (i32, [P, P, i32, ctypes.POINTER(RefineParams), P, i32, P, P]),
        "hfp_autotune_round_engine": (i32, [P, P, i32, ctypes.POINTER(RefineParams), i32, P, i32,
                                            P, ctypes.POINTER(Tuning)]),
        "hfp_mlp_forward": (i32, [P, P, P, i32, P]),
        "hfp_mlp_grad": (i32, [P, P, P, P, i32, P, P]),
        "hfp_mlp_train": (i32, [P, P, P, P, P, P, P, i32, i32, ctypes.POINTER(AdamParams), P,
                                i32]),
        "hfp_pair_scores": (i32, [P, P, i32, i32, P, P, P]),
        "hfp_round_pairs": (i32, [P, P, i32, P, ctypes.c_float, P, P, i32, P, P]),
        "hfp_refine_pairs_batched": (i32, [P, P, i32, ctypes.POINTER(RefineParams), P, i32, i32,
                                           P, P, ctypes.c_int64, P, P]),
        "hfp_apply_moves": (i32, [P, P, i32, ctypes.POINTER(RefineParams), P, P, P, i32,
                                  ctypes.POINTER(RoundStats)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(status: int, allow=()):
    if status != OK and status not in allow:
        raise HfpError(status, load().hfp_last_error().decode(errors="replace"))
    return status


def _is_dev(a) -> bool:
    return hasattr(a, "is_cuda") and a.is_cuda


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    return ctypes.c_void_p(a.ctypes.data)


def _host(a, dtype):
    return None if a is None else np.ascontiguousarray(a, dtype=dtype)


class Context:
    """hfp_ctx: a device and the stream every call of this context uses."""

    def __init__(self, device: int = 0, stream: int | None = None):
        lib = load()
        h = ctypes.c_void_p()
        _check(lib.hfp_ctx_create(ctypes.byref(h), device, ctypes.c_void_p(stream or 0)))
        self.h = h
        self.device = device

    def close(self):
        if getattr(self, "h", None):
            load().hfp_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ctx_create(device: int = 0, stream: int | None = None) -> Context:
    return Context(device, stream)


def ctx_get_tuning(ctx: Context) -> dict:
    """hfp_ctx_get_tuning."""
    t = Tuning()
    _check(load().hfp_ctx_get_tuning(ctx.h, ctypes.byref(t)))
    return {k: int(getattr(t, k)) for k, _ in Tuning._fields_}


def ctx_set_tuning(ctx: Context, **kw):
    """hfp_ctx_set_tuning: change the given knobs, keep the others."""
    cur = ctx_get_tuning(ctx)
    cur.update(kw)
    t = Tuning(**cur)
    _check(load().hfp_ctx_set_tuning(ctx.h, ctypes.byref(t)))


@dataclass
class NetInfo:
    n_nodes: int
    m_nets: int
    p_pins: int
    lawler_nodes: int
    total_weight: int


class Net:
    """hfp_net: a flow network resident on the device with its flow state."""

    def __init__(self, ctx: Context, handle, n_region: int):
        self.ctx = ctx
        self.h = handle
        self.n_region = n_region
        inf = _NetInfo()
        _check(load().hfp_net_get_info(self.h, ctypes.byref(inf)))
        self.info = NetInfo(inf.n_nodes, inf.m_nets, inf.p_pins, inf.lawler_nodes, inf.total_weight)

    def close(self):
        if getattr(self, "h", None):
            load().hfp_net_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def build_flow_network(ctx: Context, net_off, pins, net_w, node_w, region, side, n: int,
                       dist_from_cut=None) -> Net:
    """hfp_build_flow_network.  All arrays numpy (host) or all CUDA tensors."""
    dev = _is_dev(pins) or _is_dev(net_off)
    if dev:
        arrs = dict(net_off=net_off, pins=pins, net_w=net_w, node_w=node_w, region=region,
                    side=side, dist=dist_from_cut)
    else:
        arrs = dict(net_off=_host(net_off, np.uint32), pins=_host(pins, np.int32),
                    net_w=_host(net_w, np.int32), node_w=_host(node_w, np.int32),
                    region=_host(region, np.int32), side=_host(side, np.int32),
                    dist=_host(dist_from_cut, np.int32))
    m = len(arrs["net_off"]) - 1
    H = _Hypergraph(n, m, _ptr(arrs["net_off"]), _ptr(arrs["pins"]), _ptr(arrs["net_w"]),
                    _ptr(arrs["node_w"]))
    h = ctypes.c_void_p()
    nr = len(arrs["region"])
    _check(load().hfp_build_flow_network(ctx.h, ctypes.byref(H), MEM_DEVICE if dev else MEM_HOST,
                                         _ptr(arrs["region"]), nr, _ptr(arrs["side"]),
                                         _ptr(arrs["dist"]), ctypes.byref(h)))
    return Net(ctx, h, nr)


def net_export(net: Net) -> dict:
    """hfp_net_export to host numpy arrays."""
    i = net.info
    out = dict(net_off=np.zeros(i.m_nets + 1, np.uint32), pins=np.zeros(i.p_pins, np.int32),
               net_w=np.zeros(i.m_nets, np.int32), net_gid=np.zeros(i.m_nets, np.int32),
               node_w=np.zeros(i.n_nodes, np.int32), node_off=np.zeros(i.n_nodes + 1, np.uint32),
               inc_slot=np.zeros(i.p_pins, np.int32), dist=np.zeros(i.n_nodes, np.int32))
    _check(load().hfp_net_export(net.h, MEM_HOST, *[_ptr(out[k]) for k in
                                                    ("net_off", "pins", "net_w", "net_gid",
                                                     "node_w", "node_off", "inc_slot", "dist")]))
    return out


def net_export_flow(net: Net) -> dict:
    """hfp_net_export_flow to host numpy arrays: per-arc flows, excess,
    pending deltas and terminal flags."""
    i = net.info
    out = dict(f_in=np.zeros(i.p_pins, np.int32), f_out=np.zeros(i.p_pins, np.int32),
               f_b=np.zeros(i.m_nets, np.int32), excess=np.zeros(i.lawler_nodes, np.int64),
               delta=np.zeros(i.lawler_nodes, np.int64), flags=np.zeros(i.lawler_nodes, np.uint8))
    _check(load().hfp_net_export_flow(net.h, MEM_HOST, *[_ptr(out[k]) for k in
                                                         ("f_in", "f_out", "f_b", "excess",
                                                          "delta", "flags")]))
    return out


def net_export_device(net: Net) -> dict:
    """hfp_net_export into CUDA int32 tensors (the layout hfp_max_flow_noalloc
    reads)."""
    import torch
    i = net.info
    z = lambda k: torch.zeros(max(k, 1), dtype=torch.int32, device=f"cuda:{net.ctx.device}")
    out = dict(net_off=z(i.m_nets + 1), pins=z(i.p_pins), net_w=z(i.m_nets),
               node_w=z(i.n_nodes), node_off=z(i.n_nodes + 1), inc_slot=z(i.p_pins))
    _check(load().hfp_net_export(net.h, MEM_DEVICE, _ptr(out["net_off"]), _ptr(out["pins"]),
                                 _ptr(out["net_w"]), None, _ptr(out["node_w"]),
                                 _ptr(out["node_off"]), _ptr(out["inc_slot"]), None))
    return out


def max_flow_noalloc(device: int, stream: int, view: dict, n_nodes: int, m_nets: int,
                     p_pins: int, in_source_lawler=None):
    """hfp_max_flow_noalloc: max flow and S_r without any allocation in the
    call.  view holds CUDA tensors in hfp_net_export's layout.  Returns
    (flow value, c(S_r))."""
    v = _NetworkView(n_nodes, m_nets, p_pins, _ptr(view["net_off"]), _ptr(view["pins"]),
                     _ptr(view["net_w"]), _ptr(view["node_off"]), _ptr(view["inc_slot"]),
                     _ptr(view["node_w"]))
    flow = ctypes.c_int64()
    w = ctypes.c_int64()
    _check(load().hfp_max_flow_noalloc(device, ctypes.c_void_p(stream or 0), ctypes.byref(v),
                                       ctypes.byref(flow), _ptr(in_source_lawler),
                                       ctypes.byref(w)))
    return int(flow.value), int(w.value)


STATE_NAMES = ("done", "push", "relabel", "gr_init", "gr_level", "sr_init", "sr_level",
               "dist_init", "dist_level", "other")


# engine states 0 .. 20 (the numbering of the batched-launch profile)
ENGINE_STATES = ("done", "push", "relabel", "gr_init", "gr_level", "sr_init", "sr_level",
                 "dist_init", "dist_level", "one_cta", "fc_saturate", "fc_select", "unused12",
                 "fc_mark_s", "fc_mark_t", "sr_add", "gr_add", "gr_seed", "gr_run", "round",
                 "flush")


def ctx_batch_profile(ctx: Context, reset: bool = True) -> dict:
    """hfp_ctx_batch_profile -> {state: (device ns, phases, light input
    nodes, heavy input nodes)} of the batched launches since the last reset,
    summed over their networks (states with no phase are left out)."""
    ns, cnt, li, hi = (np.zeros(24, np.uint64) for _ in range(4))
    _check(load().hfp_ctx_batch_profile(ctx.h, _ptr(ns), _ptr(cnt), _ptr(li), _ptr(hi), 24,
                                        1 if reset else 0))
    out = {}
    for i in range(24):
        if cnt[i]:
            name = ENGINE_STATES[i] if i < len(ENGINE_STATES) else f"state{i}"
            out[name] = (int(ns[i]), int(cnt[i]), int(li[i]), int(hi[i]))
    return out


def ctx_last_batch_layout(ctx: Context) -> dict:
    """hfp_ctx_last_batch_layout -> {groups, group_ctas, cluster} of the
    context's last batched FlowCutter launch."""
    g, c, cl = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(load().hfp_ctx_last_batch_layout(ctx.h, ctypes.byref(g), ctypes.byref(c),
                                            ctypes.byref(cl)))
    return {"groups": g.value, "group_ctas": c.value, "cluster": cl.value}


def ctx_wait_selftest(ctx: Context, barrier: int) -> tuple[int, float]:
    """hfp_ctx_wait_selftest -> (status, device ms of the launch): a barrier
    wait (0 grid, 1 group in global memory, 2 cluster) that only the
    context's wait_timeout_ms ends; ERR_ITER_LIMIT is the designed outcome.
    Other errors raise HfpError."""
    ms = ctypes.c_float()
    st = load().hfp_ctx_wait_selftest(ctx.h, barrier, ctypes.byref(ms))
    if st not in (OK, ERR_ITER_LIMIT):
        _check(st)
    return st, float(ms.value)


def net_enable_trace(net: Net, phases: int):
    """hfp_net_enable_trace: record the next `phases` engine phases."""
    _check(load().hfp_net_enable_trace(net.h, phases))


def net_trace(net: Net, cap: int = 0) -> dict:
    """hfp_net_get_trace -> per-state device time and counts, and the
    per-phase trace (state, CTA-alone flag, input and output list sizes,
    flow value, device time)."""
    ns = np.zeros(10, np.uint64)
    cnt = np.zeros(10, np.uint64)
    buf = np.zeros(max(4 * cap, 4), np.uint64)
    n = ctypes.c_int32()
    _check(load().hfp_net_get_trace(net.h, _ptr(ns), _ptr(cnt), _ptr(buf), cap, ctypes.byref(n)))
    k = min(n.value, cap)
    tr = buf[: 4 * k].reshape(-1, 4)
    w0 = tr[:, 0]
    m29 = np.uint64((1 << 29) - 1)
    return dict(state_ns={STATE_NAMES[i]: int(ns[i]) for i in range(10)},
                state_cnt={STATE_NAMES[i]: int(cnt[i]) for i in range(10)},
                phases=int(n.value),
                state=((w0 >> np.uint64(58)) & np.uint64(31)).astype(np.int64),
                solo=((w0 >> np.uint64(63)) & np.uint64(1)).astype(np.int64),
                light_in=((w0 >> np.uint64(29)) & m29).astype(np.int64),
                heavy_in=(w0 & m29).astype(np.int64),
                light_out=(tr[:, 1] >> np.uint64(32)).astype(np.int64),
                heavy_out=(tr[:, 1] & np.uint64(0xFFFFFFFF)).astype(np.int64),
                flow=tr[:, 2].astype(np.int64), ns=tr[:, 3].astype(np.int64))


class HGraph:
    """hfp_hgraph: a hypergraph resident on the device for k-way refinement."""

    def __init__(self, ctx: Context, net_off, pins, net_w, node_w, n: int):
        arrs = dict(net_off=_host(net_off, np.uint32), pins=_host(pins, np.int32),
                    net_w=_host(net_w, np.int32), node_w=_host(node_w, np.int32))
        H = _Hypergraph(n, len(arrs["net_off"]) - 1, _ptr(arrs["net_off"]), _ptr(arrs["pins"]),
                        _ptr(arrs["net_w"]), _ptr(arrs["node_w"]))
        h = ctypes.c_void_p()
        _check(load().hfp_hgraph_create(ctx.h, ctypes.byref(H), MEM_HOST, ctypes.byref(h)))
        self.ctx, self.h, self.n = ctx, h, n

    def close(self):
        if getattr(self, "h", None):
            load().hfp_hgraph_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def refine_params(eps_pct=3, alpha_eps_pct=48, delta=2, seed=0) -> RefineParams:
    return RefineParams(eps_pct, alpha_eps_pct, delta, seed & 0xFFFFFFFF)


def connectivity(hg: HGraph, part_dev, k: int) -> int:
    """hfp_connectivity (part: CUDA int32 tensor)."""
    v = ctypes.c_int64()
    _check(load().hfp_connectivity(hg.h, _ptr(part_dev), k, ctypes.byref(v)))
    return int(v.value)


def refine_block_pair(hg: HGraph, part_dev, k: int, bi: int, bj: int,
                      params: RefineParams | None = None):
    """hfp_refine_block_pair -> (PairResult, moves int32[n, 3])."""
    params = params or refine_params()
    res = PairResult()
    cap = hg.n
    moves = np.zeros(3 * max(cap, 1), np.int32)
    _check(load().hfp_refine_block_pair(hg.h, _ptr(part_dev), k, bi, bj, ctypes.byref(params),
                                        _ptr(moves), cap, ctypes.byref(res)))
    return res, moves[: 3 * res.n_moves].reshape(-1, 3).copy()


def refine_round(hg: HGraph, part_dev, k: int, params: RefineParams | None = None,
                 pair_scores=None, min_score: float = 0.0):
    """hfp_refine_round (part updated in place) -> (RoundStats, [PairResult])."""
    params = params or refine_params()
    stats = RoundStats()
    cap = k * k
    arr = (PairResult * cap)()
    n = ctypes.c_int32()
    sc = None if pair_scores is None else np.ascontiguousarray(pair_scores, np.float32)
    _check(load().hfp_refine_round(hg.h, _ptr(part_dev), k, ctypes.byref(params), _ptr(sc),
                                   ctypes.c_float(min_score), ctypes.byref(stats), arr, cap,
                                   ctypes.byref(n)))
    return stats, [arr[i] for i in range(n.value)]


MLP_FEATURES, MLP_HIDDEN, MLP_PARAMS = 16, 64, 5313


def flowcutter_batch(ctx: Context, nets, params, group_ctas: int = 0,
                     pierce_cap: int | None = None):
    """hfp_flowcutter_batch: FlowCutter on every network in one launch ->
    [FlowCutterResult] (params: one FcParams per network)."""
    n = len(nets)
    tasks = (_FcTask * max(n, 1))()
    keep = []
    for i, (net, prm) in enumerate(zip(nets, params)):
        cap = net.info.n_nodes if pierce_cap is None else pierce_cap
        fs = np.zeros(max(net.n_region, 1), np.uint8)
        ps = np.zeros(max(cap, 1), np.int32)
        pn = np.zeros(max(cap, 1), np.int32)
        keep.append((fs, ps, pn))
        tasks[i].net = net.h
        tasks[i].params = prm
        tasks[i].final_side = fs.ctypes.data
        tasks[i].pierce_side = ps.ctypes.data
        tasks[i].pierce_node = pn.ctypes.data
        tasks[i].pierce_cap = cap
    _check(load().hfp_flowcutter_batch(ctx.h, tasks, n, group_ctas))
    out = []
    for i, net in enumerate(nets):
        t = tasks[i]
        fs, ps, pn = keep[i]
        k = min(t.result.n_pierced, t.pierce_cap)
        out.append(FlowCutterResult(t.status, t.result.flow, t.result.source_weight,
                                    t.result.iterations, t.result.result_side,
                                    fs[: net.n_region], ps[:k].copy(), pn[:k].copy()))
    return out


def refine_round_batched(hg: HGraph, part_dev, k: int, params: RefineParams | None = None,
                         pair_scores=None, min_score: float = 0.0, group_ctas: int = 0):
    """hfp_refine_round_batched -> (RoundStats, [PairResult], FlowCutter launch ms)."""
    params = params or refine_params()
    stats = RoundStats()
    cap = k * k
    arr = (PairResult * cap)()
    n = ctypes.c_int32()
    ms = ctypes.c_float()
    sc = None if pair_scores is None else np.ascontiguousarray(pair_scores, np.float32)
    _check(load().hfp_refine_round_batched(hg.h, _ptr(part_dev), k, ctypes.byref(params), _ptr(sc),
                                           ctypes.c_float(min_score), group_ctas,
                                           ctypes.byref(stats), arr, cap, ctypes.byref(n),
                                           ctypes.byref(ms)))
    return stats, [arr[i] for i in range(n.value)], float(ms.value)


def round_pairs(hg: HGraph, part_dev, k: int, pair_scores=None, min_score: float = 0.0):
    """hfp_round_pairs -> (pairs int32[P, 2], nets in both blocks int64[P],
    connectivity)."""
    cap = k * (k - 1) // 2
    pairs = np.zeros((max(cap, 1), 2), np.int32)
    nets = np.zeros(max(cap, 1), np.int64)
    n = ctypes.c_int32()
    conn = ctypes.c_int64()
    sc = None if pair_scores is None else np.ascontiguousarray(pair_scores, np.float32)
    _check(load().hfp_round_pairs(hg.h, _ptr(part_dev), k, _ptr(sc), ctypes.c_float(min_score),
                                  _ptr(pairs), _ptr(nets), cap, ctypes.byref(n),
                                  ctypes.byref(conn)))
    return pairs[:n.value].copy(), nets[:n.value].copy(), int(conn.value)


def refine_pairs_batched(hg: HGraph, part_dev, k: int, pairs, params: RefineParams | None = None,
                         group_ctas: int = 0):
    """hfp_refine_pairs_batched -> ([PairResult], moves int32[M, 3], offsets
    int64[n + 1], FlowCutter launch ms); part is not changed."""
    params = params or refine_params()
    pr = np.ascontiguousarray(np.asarray(pairs, np.int32).reshape(-1, 2))
    n = len(pr)
    res = (PairResult * max(n, 1))()
    off = np.zeros(n + 1, np.int64)
    ms = ctypes.c_float()
    # moves are region vertices whose block changes: the vertex count covers
    # them unless vertices move in several pairs' regions at once; if not,
    # the call reports the exact need and runs again
    cap = max(int(hg.n), 1)
    for _ in range(2):
        moves = np.empty((max(cap, 1), 3), np.int32)
        st = _check(load().hfp_refine_pairs_batched(hg.h, _ptr(part_dev), k, ctypes.byref(params),
                                                    _ptr(pr), n, group_ctas, res, _ptr(moves),
                                                    cap, _ptr(off), ctypes.byref(ms)),
                    allow=(ERR_BUFFER_TOO_SMALL,))
        if st == OK:
            return [res[i] for i in range(n)], moves[:off[n]].copy(), off, float(ms.value)
        cap = int(off[n])
    raise HfpError(ERR_BUFFER_TOO_SMALL, "moves did not fit")


def apply_moves(hg: HGraph, part_dev, k: int, results, moves, offsets,
                params: RefineParams | None = None):
    """hfp_apply_moves (part updated in place) -> (RoundStats, [PairResult]
    with applied / valid_moves / gain)."""
    params = params or refine_params()
    n = len(results)
    arr = (PairResult * max(n, 1))(*results)
    mv = np.ascontiguousarray(np.asarray(moves, np.int32).reshape(-1, 3))
    off = np.ascontiguousarray(offsets, np.int64)
    stats = RoundStats()
    _check(load().hfp_apply_moves(hg.h, _ptr(part_dev), k, ctypes.byref(params), arr, _ptr(mv),
                                  _ptr(off), n, ctypes.byref(stats)))
    return stats, [arr[i] for i in range(n)]


def autotune_round(hg: HGraph, part_dev, k: int, candidates, params: RefineParams | None = None):
    """hfp_autotune_round -> (best group size, ms per candidate)."""
    params = params or refine_params()
    c = np.ascontiguousarray(candidates, np.int32)
    ms = np.zeros(len(c), np.float32)
    best = ctypes.c_int32()
    _check(load().hfp_autotune_round(hg.h, _ptr(part_dev), k, ctypes.byref(params), _ptr(c), len(c),
                                     _ptr(ms), ctypes.byref(best)))
    return int(best.value), ms


def autotune_round_engine(hg: HGraph, part_dev, k: int, params: RefineParams | None = None,
                          group_ctas: int = 0):
    """hfp_autotune_round_engine -> (chosen tuning dict, launch ms per try)."""
    params = params or refine_params()
    ms = np.zeros(32, np.float32)
    n = ctypes.c_int32()
    t = Tuning()
    _check(load().hfp_autotune_round_engine(hg.h, _ptr(part_dev), k, ctypes.byref(params),
                                            group_ctas, _ptr(ms), len(ms), ctypes.byref(n),
                                            ctypes.byref(t)))
    return {f: int(getattr(t, f)) for f, _ in Tuning._fields_}, ms[: n.value]


def pair_features(hg: HGraph, part_dev, k: int, eps_pct: int = 3, prev_gain=None):
    """hfp_pair_features -> (pairs CUDA int32[P, 2], features CUDA float32[P, 16])."""
    import torch
    cap = k * (k - 1) // 2
    dev = part_dev.device
    feat = torch.zeros((max(cap, 1), MLP_FEATURES), dtype=torch.float32, device=dev)
    pairs = torch.zeros((max(cap, 1), 2), dtype=torch.int32, device=dev)
    pg = None if prev_gain is None else np.ascontiguousarray(prev_gain, np.int64)
    n = ctypes.c_int32()
    _check(load().hfp_pair_features(hg.h, _ptr(part_dev), k, eps_pct, _ptr(pg), _ptr(feat),
                                    _ptr(pairs), cap, ctypes.byref(n)))
    return pairs[: n.value], feat[: n.value]


def mlp_forward(ctx: Context, params_dev, x_dev):
    """hfp_mlp_forward -> scores (CUDA float32[rows])."""
    import torch
    rows = int(x_dev.shape[0])
    out = torch.zeros(max(rows, 1), dtype=torch.float32, device=x_dev.device)
    _check(load().hfp_mlp_forward(ctx.h, _ptr(params_dev), _ptr(x_dev), rows, _ptr(out)))
    return out[:rows]


def mlp_grad(ctx: Context, params_dev, x_dev, y_dev):
    """hfp_mlp_grad -> (mean loss, gradient CUDA float32[MLP_PARAMS])."""
    import torch
    g = torch.zeros(MLP_PARAMS, dtype=torch.float32, device=x_dev.device)
    loss = ctypes.c_float()
    _check(load().hfp_mlp_grad(ctx.h, _ptr(params_dev), _ptr(x_dev), _ptr(y_dev),
                               int(x_dev.shape[0]), _ptr(g), ctypes.byref(loss)))
    return float(loss.value), g


class MlpState:
    """Parameters, Adam moments and step counter of the scheduler, on the
    device (float32 CUDA tensors; the counter an int32 tensor)."""

    def __init__(self, params_dev):
        import torch
        self.params = params_dev.contiguous()
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.step = torch.zeros(1, dtype=torch.int32, device=self.params.device)


def mlp_train(ctx: Context, state: MlpState, x_dev, y_dev, steps: int, lr: float = 1e-3,
              beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
    """hfp_mlp_train: `steps` Adam steps in place -> losses CUDA float32[steps]."""
    import torch
    losses = torch.zeros(max(steps, 1), dtype=torch.float32, device=x_dev.device)
    opt = AdamParams(lr, eps, beta1, beta2)
    _check(load().hfp_mlp_train(ctx.h, _ptr(state.params), _ptr(state.m), _ptr(state.v),
                                _ptr(state.step), _ptr(x_dev), _ptr(y_dev), int(x_dev.shape[0]),
                                steps, ctypes.byref(opt), _ptr(losses), steps))
    return losses[:steps]


def pair_scores(hg: HGraph, part_dev, k: int, params_dev, eps_pct: int = 3, prev_gain=None):
    """hfp_pair_scores -> host float32[k, k] (-1 where blocks share no net)."""
    out = np.zeros((k, k), np.float32)
    pg = None if prev_gain is None else np.ascontiguousarray(prev_gain, np.int64)
    _check(load().hfp_pair_scores(hg.h, _ptr(part_dev), k, eps_pct, _ptr(pg), _ptr(params_dev),
                                  _ptr(out)))
    return out


def net_stats(net: Net) -> dict:
    s = _Stats()
    _check(load().hfp_net_get_stats(net.h, ctypes.byref(s)))
    return {k: int(getattr(s, k)) for k, _ in _Stats._fields_}


def kernel_launches() -> int:
    """hfp_kernel_launches: kernels this library launched in the process."""
    return int(load().hfp_kernel_launches())


def max_flow(net: Net) -> int:
    """hfp_max_flow: augment to a maximum preflow; returns the flow value."""
    v = ctypes.c_int64()
    _check(load().hfp_max_flow(net.h, ctypes.byref(v)))
    return int(v.value)


def min_cut_source_side(net: Net, lawler: bool = True, cut_cap: int | None = None):
    """hfp_min_cut_source_side -> (in_source_lawler | None, in_source_region,
    cut_net_ids, source_weight)."""
    i = net.info
    law = np.zeros(i.lawler_nodes, np.uint8) if lawler else None
    reg = np.zeros(max(net.n_region, 1), np.uint8)
    cap = i.m_nets if cut_cap is None else cut_cap
    cuts = np.zeros(cap, np.int32) if cap > 0 else None
    ncut = ctypes.c_int32()
    w = ctypes.c_int64()
    _check(load().hfp_min_cut_source_side(net.h, MEM_HOST, _ptr(law), _ptr(reg), _ptr(cuts), cap,
                                          ctypes.byref(ncut), ctypes.byref(w)))
    cut_ids = cuts[: ncut.value] if cuts is not None else np.zeros(0, np.int32)
    return law, reg[: net.n_region], cut_ids, int(w.value)


def min_cut_source_side_device(net: Net, in_source_region, in_source_lawler=None) -> int:
    """hfp_min_cut_source_side with device outputs (CUDA uint8 tensors);
    returns c(S_r)."""
    w = ctypes.c_int64()
    _check(load().hfp_min_cut_source_side(net.h, MEM_DEVICE, _ptr(in_source_lawler),
                                          _ptr(in_source_region), None, 0, None, ctypes.byref(w)))
    return int(w.value)


def min_cut_sink_side(net: Net, lawler: bool = True):
    """hfp_min_cut_sink_side -> (in_sink_lawler | None, in_sink_region, sink_weight)."""
    i = net.info
    law = np.zeros(i.lawler_nodes, np.uint8) if lawler else None
    reg = np.zeros(max(net.n_region, 1), np.uint8)
    w = ctypes.c_int64()
    _check(load().hfp_min_cut_sink_side(net.h, MEM_HOST, _ptr(law), _ptr(reg), ctypes.byref(w)))
    return law, reg[: net.n_region], int(w.value)


def fc_params(max_block_weight: int, flow_bound: int = -1, seed: int = 0,
              max_iterations: int = 0, bulk_beta_pct: int = 0, bulk_warmup: int = 3,
              mb_reps: int = 0) -> FcParams:
    return FcParams(int(max_block_weight), int(flow_bound), int(seed) & 0xFFFFFFFF,
                    int(max_iterations), int(bulk_beta_pct), int(bulk_warmup), int(mb_reps), 0)


def pierce_and_augment(net: Net, side: int, nodes=None, params: FcParams | None = None):
    """hfp_pierce_and_augment -> (pierced node, new flow value)."""
    arr = None if nodes is None else _host(nodes, np.int32)
    pierced = ctypes.c_int32(-1)
    v = ctypes.c_int64()
    _check(load().hfp_pierce_and_augment(net.h, side, _ptr(arr), 0 if arr is None else len(arr),
                                         ctypes.byref(params) if params is not None else None,
                                         ctypes.byref(pierced), ctypes.byref(v)))
    return int(pierced.value), int(v.value)


@dataclass
class FlowCutterResult:
    status: int
    flow: int
    source_weight: int
    iterations: int
    result_side: int
    final_side: np.ndarray
    pierce_side: np.ndarray
    pierce_node: np.ndarray
    bulk_steps: int = 0
    mb_steps: int = 0


def flowcutter(net: Net, params: FcParams, pierce_cap: int | None = None) -> FlowCutterResult:
    """hfp_flowcutter.  Statuses NO_BALANCED_CUT / ABORTED_WORSE are returned
    in the result rather than raised."""
    cap = (net.info.n_nodes + 1) * (1 + max(params.mb_reps, 0)) if pierce_cap is None \
        else pierce_cap
    fs = np.zeros(max(net.n_region, 1), np.uint8)
    ps = np.zeros(max(cap, 1), np.int32)
    pn = np.zeros(max(cap, 1), np.int32)
    r = _FcResult()
    st = _check(load().hfp_flowcutter(net.h, ctypes.byref(params), _ptr(fs), _ptr(ps), _ptr(pn),
                                      cap, ctypes.byref(r)),
                allow=(NO_BALANCED_CUT, ABORTED_WORSE))
    k = min(r.n_pierced, cap)
    return FlowCutterResult(st, r.flow, r.source_weight, r.iterations, r.result_side,
                            fs[: net.n_region], ps[:k].copy(), pn[:k].copy(), r.bulk_steps,
                            r.mb_steps)
