"""Seeded synthetic inputs shared by the CPU oracle and the CUDA path.

The generators draw ring hypergraphs shaped like the paper's workloads
(Section 8, "Instances": unit vertex weights or small integer weights,
heavy-tailed net sizes, multi-million pins).  They hold none of the flow
method's arithmetic: the region of a flow problem and the block assignment
are inputs, defined here by their positions on the ring.

The C source ``gen.c`` is compiled on first use (or by ``build()``) into
``synth/_build/libsynth.so``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libsynth.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile gen.c into a shared library (plain gcc, no -march flags)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
                               "-std=c11", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        lib.synth_net_sizes.restype = ctypes.c_int64
        lib.synth_net_sizes.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                        ctypes.c_uint64, P]
        lib.synth_ring_pins.restype = ctypes.c_int64
        lib.synth_ring_pins.argtypes = [ctypes.c_int32, ctypes.c_int32, P, ctypes.c_int32,
                                        ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                        ctypes.c_int32, ctypes.c_uint64, P, P, P, P]
        lib.synth_kway_partition.restype = ctypes.c_int32
        lib.synth_kway_partition.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                             ctypes.c_uint64, P]
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


@dataclass
class Hypergraph:
    """Net -> pins CSR of a hypergraph H = (V, E, c, w) (Section 2)."""
    n: int
    m: int
    net_off: np.ndarray   # uint32[m+1]
    pins: np.ndarray      # int32[net_off[m]]
    net_w: np.ndarray     # int32[m]
    node_w: np.ndarray    # int32[n]

    @property
    def p(self) -> int:
        return int(self.net_off[-1])


GEOMETRIC, ZIPF = 0, 1


def ring_hypergraph(n: int, m: int, dist: int, cap: int, window: int,
                    w_range=(1, 1), c_range=(1, 1), seed: int = 1) -> Hypergraph:
    """Ring hypergraph: each net's pins are drawn without replacement from a
    window around a uniform centre; sizes are 2+Geometric(1/2) or 2+Zipf(2.5)."""
    lib = _load()
    sizes = np.empty(m, dtype=np.int32)
    total = lib.synth_net_sizes(m, dist, cap, seed, _ptr(sizes))
    if total < 0:
        raise ValueError("bad size-distribution arguments")
    if total > 0xFFFFFFFF:
        raise ValueError("too many pins for uint32 offsets")
    net_off = np.empty(m + 1, dtype=np.uint32)
    pins = np.empty(int(total), dtype=np.int32)
    net_w = np.empty(m, dtype=np.int32)
    node_w = np.empty(n, dtype=np.int32)
    got = lib.synth_ring_pins(n, m, _ptr(sizes), window, int(w_range[0]), int(w_range[1]),
                              int(c_range[0]), int(c_range[1]), seed,
                              _ptr(net_off), _ptr(pins), _ptr(net_w), _ptr(node_w))
    if got < 0:
        raise ValueError("bad ring arguments")
    return Hypergraph(n, m, net_off, pins[: int(got)].copy() if got != total else pins, net_w, node_w)


def halves(n: int) -> np.ndarray:
    """Bipartition of the ring into [0, n/2) -> block 0 and [n/2, n) -> block 1."""
    part = np.zeros(n, dtype=np.int32)
    part[n // 2:] = 1
    return part


def region_near_cuts(n: int, radius: int) -> np.ndarray:
    """Vertices within `radius` positions of either cut point of the halves
    bipartition (cut points 0 and n/2): v is in the region iff
    (v - c) mod n < radius or (c - 1 - v) mod n < radius.  Ascending ids."""
    v = np.arange(n, dtype=np.int64)
    keep = np.zeros(n, dtype=bool)
    for c in (0, n // 2):
        keep |= ((v - c) % n) < radius
        keep |= ((c - 1 - v) % n) < radius
    return np.nonzero(keep)[0].astype(np.int32)


def kway_partition(n: int, k: int, frac_ppm: int, seed: int) -> np.ndarray:
    """k contiguous arcs, then frac_ppm parts-per-million of vertices moved to
    an adjacent block."""
    part = np.empty(n, dtype=np.int32)
    if _load().synth_kway_partition(n, k, frac_ppm, seed, _ptr(part)) < 0:
        raise ValueError("bad partition arguments")
    return part


# The workloads, by name.  Sizes are the full ones; instance() may shrink n,
# m, radius, window and cap for quick cases of the same shape.
WORKLOADS = {
    "ring_n4096_geom": dict(name="ring_n4096_geom", n=4096, m=6144, dist=GEOMETRIC, cap=16, window=64,
            w_range=(1, 4), c_range=(1, 1), radius=48, k=2),
    "ring_n2M_zipf": dict(name="ring_n2M_zipf", n=2_000_000, m=3_000_000, dist=ZIPF, cap=5000, window=4096,
            w_range=(1, 10), c_range=(1, 1), radius=200_000, k=2),
    "ring_n500k_zipf_fc": dict(name="ring_n500k_zipf_fc", n=500_000, m=750_000, dist=ZIPF, cap=5000, window=4096,
            w_range=(1, 10), c_range=(1, 4), radius=50_000, k=2, eps_pct=3),
    "ring_n8M_zipf_k64": dict(name="ring_n8M_zipf_k64", n=8_000_000, m=12_000_000, dist=ZIPF, cap=10000,
            window=4096, w_range=(1, 10), c_range=(1, 1), k=64, frac_ppm=50_000),
}


def instance(workload: str, seed: int, n: int | None = None, m: int | None = None,
             radius: int | None = None, window: int | None = None, cap: int | None = None):
    """Hypergraph plus partition (and, for bipartitions, the flow region) of a
    workload; n, m, radius, window and cap may be overridden for smaller cases."""
    c = dict(WORKLOADS[workload])
    if n is not None:
        c["n"] = n
    if m is not None:
        c["m"] = m
    if radius is not None:
        c["radius"] = radius
    if window is not None:
        c["window"] = window
    if cap is not None:
        c["cap"] = cap
    H = ring_hypergraph(c["n"], c["m"], c["dist"], c["cap"], c["window"], c["w_range"],
                        c["c_range"], seed)
    out = dict(workload=c, H=H, seed=seed)
    if c["k"] == 2:
        out["part"] = halves(c["n"])
        out["region"] = region_near_cuts(c["n"], c["radius"])
    else:
        out["part"] = kway_partition(c["n"], c["k"], c["frac_ppm"], seed)
    return out
