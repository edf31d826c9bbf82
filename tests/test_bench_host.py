"""Host-side pieces of bench.py, checked on the CPU: the (lambda - 1) recount
that certifies every benchmarked k-way round, against the oracle's
connectivity (Section 2) and a plain loop; and the engine-source hash that
decides whether the committed ncu traffic figure still applies to the
engine the bench runs."""
import importlib.util
import os
import re

import numpy as np
import pytest

import oracle
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _loop_km1(H, part):
    tot = 0
    for e in range(H.m):
        blocks = {int(part[v]) for v in H.pins[H.net_off[e]:H.net_off[e + 1]]}
        tot += max(len(blocks) - 1, 0) * int(H.net_w[e])
    return tot


@pytest.mark.parametrize("seed,n,m,k", [(1, 3000, 4500, 64), (2, 5000, 2000, 7), (3, 800, 1200, 2)])
def test_km1_host_matches_oracle(bench, seed, n, m, k):
    inst = synth.instance("ring_n8M_zipf_k64", seed, n=n, m=m)
    H = inst["H"]
    part = inst["part"] if k == 64 else synth.kway_partition(n, k, 200, seed)
    got = bench.km1_host(H, part)
    assert got == oracle.connectivity(H, part, k) == _loop_km1(H, part)
    assert got > 0


def test_km1_host_empty_and_single_pin_nets(bench):
    # nets: empty (first), {0,1}, single pin, empty, {2,3,4}, empty (last)
    off = np.array([0, 0, 2, 3, 3, 6, 6], np.uint32)
    pins = np.array([0, 1, 2, 2, 3, 4], np.int32)
    w = np.array([5, 3, 7, 2, 4, 9], np.int32)
    H = synth.Hypergraph(5, 6, off, pins, w, np.ones(5, np.int32))
    part = np.array([0, 1, 1, 63, 0], np.int32)
    # {0,1}: 2 blocks -> 3; {2}: 0; {2,3,4}: blocks {1,63,0} -> 2 * 4
    assert bench.km1_host(H, part) == 3 + 8 == _loop_km1(H, part)


def test_engine_hash_ignores_comments_only(bench):
    csrc = os.path.join(ROOT, "paper_2201_01556_gb300", "csrc")
    files = {f: open(os.path.join(csrc, f)).read() for f in bench.ENGINE_SOURCES}
    base = bench.engine_code_sha256(lambda f: files[f])
    commented = dict(files)
    commented["engine.cu"] = "// a new comment\n\n/* block\n comment */\n" + files["engine.cu"]
    assert bench.engine_code_sha256(lambda f: commented[f]) == base
    changed = dict(files)
    changed["common.cuh"] = files["common.cuh"] + "\nconstexpr int kNewConstant = 1;\n"
    assert bench.engine_code_sha256(lambda f: changed[f]) != base


def test_traffic_ratio_follows_the_committed_capture(bench):
    text = open(os.path.join(ROOT, "profiles", "engine_kernel_ring_n1M.md")).read()
    ratio = float(re.search(r"traffic_per_modelled_byte = ([0-9.]+)", text).group(1))
    sha = re.search(r"engine_source_sha256 = ([0-9a-f]+)", text).group(1)
    csrc = os.path.join(ROOT, "paper_2201_01556_gb300", "csrc")
    cur = bench.engine_code_sha256(lambda f: open(os.path.join(csrc, f)).read())
    got = bench.engine_traffic_ratio()
    assert got == (ratio if cur == sha else None)
    assert 0.0 < ratio < 10.0
