"""CPU oracle of the learned block-pair scheduler.

TEST INFRASTRUCTURE ONLY (same rule as the rest of ``oracle/``): only
``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
may import it; it never imports the CUDA package.

The paper has no learned component.  Its round refines every edge of the
quotient graph (Section 5, "Quotient Graph Construction" and "Parallel
Scheduling").  The scheduler scores each edge with a small multilayer
perceptron so that pairs unlikely to improve (lambda - 1) can be skipped.
Everything here is a plain definition:
  - pair_features: 16 numbers per quotient-graph edge from counts over the
    nets joining the two blocks, the block weights and the previous round;
  - bf16: round-to-nearest-even of float32 to bfloat16 (8 exponent bits,
    7 fraction bits), written from the bit-level definition;
  - forward / backward: 16 -> 64 -> 64 -> 1 with ReLU and a sigmoid output,
    bf16-rounded weights and matmul inputs, float32 arithmetic, the
    binary cross-entropy loss on the logit and its exact gradient
    (straight-through for the rounding);
  - adam_step: Adam (Kingma and Ba, 2015, Algorithm 1) with bias
    correction.
Parity status: pinned (finite differences in float64, hand examples, the
bf16 rounding of torch, the quotient graph of ``oracle.quotient``).
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _c, _hp, _load, _p

N_FEATURES = 16
HIDDEN = 64
# flat parameter layout: W1[64,16], b1[64], W2[64,64], b2[64], w3[64], b3[1]
SHAPES = (("W1", (HIDDEN, N_FEATURES)), ("b1", (HIDDEN,)), ("W2", (HIDDEN, HIDDEN)),
          ("b2", (HIDDEN,)), ("w3", (HIDDEN,)), ("b3", (1,)))
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unflatten(flat: np.ndarray) -> dict:
    out, o = {}, 0
    for name, shape in SHAPES:
        size = int(np.prod(shape))
        out[name] = flat[o:o + size].reshape(shape)
        o += size
    return out


def flatten(p: dict) -> np.ndarray:
    return np.concatenate([np.asarray(p[name]).reshape(-1) for name, _ in SHAPES])


# ---------------------------------------------------------------------------
# bfloat16

def bf16(x: np.ndarray) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even), returned
    as float32.  bfloat16 keeps the upper 16 bits of the float32 pattern; the
    dropped 16 bits decide the rounding: above half -> up, below -> down,
    exactly half -> towards an even kept pattern.  NaN stays NaN."""
    a = np.ascontiguousarray(x, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    keep = u >> 16
    low = u & 0xFFFF
    up = (low > 0x8000) | ((low == 0x8000) & ((keep & 1) == 1))
    r = ((keep + up.astype(np.uint64)) << 16).astype(np.uint32)
    out = r.view(np.float32).copy()
    nan = np.isnan(a)
    out[nan] = a[nan]
    return out.reshape(np.shape(x))


# ---------------------------------------------------------------------------
# features

def pair_stats(H, part, k: int) -> np.ndarray:
    """int64[k, k, 8] counts over the nets joining blocks i < j (oracle.c
    or_pair_stats)."""
    lib = _load()
    if not hasattr(lib, "_mlp_ready"):
        lib.or_pair_stats.restype = None
        lib.or_pair_stats.argtypes = [ctypes.c_int32] + [ctypes.c_void_p] * 4 + \
            [ctypes.c_int32, ctypes.c_void_p]
        lib._mlp_ready = True
    off, pins, nw, _ = _hp(H)
    s = np.zeros((k, k, 8), np.int64)
    lib.or_pair_stats(H.m, _p(off), _p(pins), _p(nw), _p(_c(part, np.int32)), k, _p(s))
    return s


def pair_features(H, part, k: int, max_w: int, prev_gain=None):
    """Features of every quotient-graph edge (i < j with a joining net), in
    row-major pair order.  prev_gain: int64[k, k] gain the pair achieved in
    the previous round, -1 where it was not refined (None: no previous
    round).  Returns (pairs int32[P, 2], features float32[P, 16]).

      0 log1p(nets)          1 log1p(weight)         2 log1p(pins)
      3 log1p(largest net)   4 log1p(nets2)          5 log1p(weight2)
      6 weight2 / weight     7 log1p(pins2)          8 c(Vi) / L
      9 c(Vj) / L           10 (c(Vi) + c(Vj)) / (2L) 11 log1p(pins / nets)
     12 log1p(max(prev, 0)) 13 1 if prev >= 0 else 0 14 log2(k) / 6
     15 weight * P / (sum of weight over all P pairs)
    where "nets2" are the joining nets whose blocks are exactly {i, j}."""
    f32 = np.float32
    st = pair_stats(H, part, k)
    bw = np.bincount(np.asarray(part, np.int64), weights=np.asarray(H.node_w, np.float64),
                     minlength=k).astype(np.int64)
    pairs = [(i, j) for i in range(k) for j in range(i + 1, k) if st[i, j, 0] > 0]
    P = len(pairs)
    X = np.zeros((P, N_FEATURES), f32)
    if P == 0:
        return np.zeros((0, 2), np.int32), X
    tot = f32(sum(int(st[i, j, 1]) for i, j in pairs))
    L = f32(max_w)
    for r, (i, j) in enumerate(pairs):
        s = st[i, j]
        prev = -1 if prev_gain is None else int(prev_gain[i, j])
        X[r, 0] = np.log1p(f32(s[0]))
        X[r, 1] = np.log1p(f32(s[1]))
        X[r, 2] = np.log1p(f32(s[2]))
        X[r, 3] = np.log1p(f32(s[3]))
        X[r, 4] = np.log1p(f32(s[4]))
        X[r, 5] = np.log1p(f32(s[5]))
        X[r, 6] = f32(s[5]) / f32(s[1])
        X[r, 7] = np.log1p(f32(s[6]))
        X[r, 8] = f32(bw[i]) / L
        X[r, 9] = f32(bw[j]) / L
        X[r, 10] = f32(bw[i] + bw[j]) / (f32(2) * L)
        X[r, 11] = np.log1p(f32(s[2]) / f32(s[0]))
        X[r, 12] = np.log1p(f32(max(prev, 0)))
        X[r, 13] = f32(1 if prev >= 0 else 0)
        X[r, 14] = f32(np.log2(f32(k))) / f32(6)
        X[r, 15] = f32(s[1]) * f32(P) / tot
    return np.array(pairs, np.int32), X


# ---------------------------------------------------------------------------
# the network

def forward(flat, X, quant: bool = True, dtype=np.float32):
    """Scores and the intermediates backward needs.  With quant, weights and
    the inputs of the two matrix products are rounded to bfloat16; the
    products accumulate in dtype (float32 by default), biases, ReLU, the
    last layer (a 64-term dot product with bf16 weights) and the sigmoid stay
    in dtype."""
    q = (lambda a: bf16(a).astype(dtype)) if quant else (lambda a: np.asarray(a, dtype))
    p = unflatten(np.asarray(flat, dtype))
    W1, W2, w3 = (q(p[n]) for n in ("W1", "W2", "w3"))
    b1, b2, b3 = (p[n].astype(dtype) for n in ("b1", "b2", "b3"))
    x = q(X)
    a1 = x @ W1.T + b1
    h1 = np.maximum(a1, 0)
    h1q = q(h1)
    a2 = h1q @ W2.T + b2
    h2 = np.maximum(a2, 0)
    z = h2 @ w3 + b3[0]
    ez = np.exp(-np.abs(z))                      # sigmoid without overflow
    s = np.where(z >= 0, 1 / (1 + ez), ez / (1 + ez))
    return s, dict(x=x, a1=a1, h1q=h1q, a2=a2, h2=h2, z=z, W1=W1, W2=W2, w3=w3)


def bce_loss(z, y):
    """Mean binary cross-entropy of the logits z against 0/1 labels y, in the
    overflow-free form max(z, 0) - z*y + log(1 + exp(-|z|))."""
    return float(np.mean(np.maximum(z, 0) - z * y + np.log1p(np.exp(-np.abs(z)))))


def backward(flat, X, y, quant: bool = True, dtype=np.float32):
    """(loss, gradient of the mean BCE loss w.r.t. the flat parameters).
    The rounding to bfloat16 passes gradients straight through."""
    s, c = forward(flat, X, quant, dtype)
    y = np.asarray(y, dtype)
    B = len(y)
    dz = (s - y) / dtype(B)
    g = {}
    g["w3"] = c["h2"].T @ dz
    g["b3"] = np.array([dz.sum()], dtype)
    da2 = np.outer(dz, c["w3"]) * (c["a2"] > 0)
    g["W2"] = da2.T @ c["h1q"]
    g["b2"] = da2.sum(axis=0)
    da1 = (da2 @ c["W2"]) * (c["a1"] > 0)
    g["W1"] = da1.T @ c["x"]
    g["b1"] = da1.sum(axis=0)
    return bce_loss(c["z"], y), flatten(g).astype(dtype)


def adam_step(flat, grad, m, v, t: int, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba, 2015): returns new (params, m, v);
    t is the 1-based step number."""
    f = np.float32
    g = np.asarray(grad, f)
    m = f(beta1) * m + f(1 - beta1) * g
    v = f(beta2) * v + f(1 - beta2) * g * g
    mh = m / f(1 - beta1 ** t)
    vh = v / f(1 - beta2 ** t)
    return (flat - f(lr) * mh / (np.sqrt(vh) + f(eps))).astype(f), m, v
