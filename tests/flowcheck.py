"""Feasibility check of a (pre)flow in the flow-hypergraph representation.

Per-arc flows of a maximum flow are not unique, so the CUDA path's flows are
checked for what every maximum preflow satisfies (Section 2, "Flows";
Section 8.3, "Restricting Capacities"), not compared with the oracle's:
  - capacities: 0 <= f(u, e_in) <= w(e) (the cap), 0 <= f(e_in, e_out) <= w(e),
    f(e_out, u) >= 0;
  - conservation: every non-terminal Lawler node has inflow - outflow equal to
    its stored excess, and that excess is >= 0 (a preflow);
  - value: the net inflow of the sink set equals the reported flow value, and
    the net outflow of the source set equals it plus the excess left inside.
Test infrastructure: reads exported arrays only.
"""
import numpy as np


def net_inflow(n_nodes, net_off, pins, f_in, f_out, f_b):
    """Inflow - outflow of every Lawler node (hypernode h -> h, in-node of net
    e -> n_nodes + e, out-node -> n_nodes + m + e)."""
    m = len(net_off) - 1
    net_off = np.asarray(net_off, np.int64)
    f_in = np.asarray(f_in, np.int64)
    f_out = np.asarray(f_out, np.int64)
    f_b = np.asarray(f_b, np.int64)
    inflow = np.zeros(n_nodes + 2 * m, np.int64)
    # hypernode u: receives f(e_out, u), sends f(u, e_in)
    np.add.at(inflow, np.asarray(pins, np.int64), f_out - f_in)
    net_of_slot = np.repeat(np.arange(m), np.diff(net_off))
    sum_in = np.bincount(net_of_slot, weights=f_in, minlength=m).astype(np.int64)
    sum_out = np.bincount(net_of_slot, weights=f_out, minlength=m).astype(np.int64)
    inflow[n_nodes:n_nodes + m] += sum_in - f_b
    inflow[n_nodes + m:] += f_b - sum_out
    return inflow


def check_preflow(n_nodes, net_off, pins, net_w, fl, flow_value):
    """fl: dict of hfp_net_export_flow arrays (f_in, f_out, f_b, excess,
    delta, flags).  Raises AssertionError on the first violated property."""
    m = len(net_off) - 1
    net_w = np.asarray(net_w, np.int64)
    w_slot = np.repeat(net_w, np.diff(np.asarray(net_off, np.int64)))
    f_in, f_out, f_b = fl["f_in"], fl["f_out"], fl["f_b"]
    assert (f_b >= 0).all() and (f_b <= net_w).all(), "bridge flow outside [0, w(e)]"
    assert (f_in >= 0).all() and (f_in <= w_slot).all(), "(u, e_in) flow outside [0, w(e)]"
    assert (f_out >= 0).all(), "negative (e_out, u) flow"
    assert (fl["delta"] == 0).all(), "unapplied pushes after the flow returned"
    inflow = net_inflow(n_nodes, net_off, pins, f_in, f_out, f_b)
    flags = fl["flags"]
    src = (flags & 1) != 0
    snk = (flags & 2) != 0
    inner = ~(src | snk)
    assert not (src & snk).any(), "a node in both S and T"
    ex = fl["excess"]
    assert (inflow[inner] == ex[inner]).all(), "conservation: inflow - outflow != excess"
    assert (ex[inner] >= 0).all(), "negative excess (not a preflow)"
    assert int(inflow[snk].sum()) == flow_value, "net inflow of T != flow value"
    assert int(-inflow[src].sum()) == flow_value + int(ex[inner].sum()), \
        "net outflow of S != flow value + excess left inside"
    assert m == len(f_b)
