"""The preflow checker used on the CUDA path's flows rejects what it must
(CPU only): a hand-built feasible flow passes; planted capacity, conservation
and value errors fail."""
import numpy as np
import pytest

from tests.flowcheck import check_preflow, net_inflow

# flow hypergraph: s = 0, t = 1, a = 2; nets e0 = {a, s} w 5, e1 = {a, t} w 3.
# Lawler ids: hypernodes 0..2, in-nodes 3, 4, out-nodes 5, 6.
NET_OFF = np.array([0, 2, 4], np.uint32)
PINS = np.array([2, 0, 2, 1], np.int32)
NET_W = np.array([5, 3], np.int32)


def _flow():
    # s -> e0_in -> e0_out -> a (3 units), a -> e1_in -> e1_out -> t (3 units)
    return dict(f_in=np.array([0, 3, 3, 0], np.int32),
                f_out=np.array([3, 0, 0, 3], np.int32),
                f_b=np.array([3, 3], np.int32),
                excess=np.zeros(7, np.int64), delta=np.zeros(7, np.int64),
                flags=np.array([1, 2, 0, 0, 0, 0, 0], np.uint8))


def test_feasible_flow_passes():
    fl = _flow()
    assert net_inflow(3, NET_OFF, PINS, fl["f_in"], fl["f_out"], fl["f_b"]).tolist() == \
        [-3, 3, 0, 0, 0, 0, 0]
    check_preflow(3, NET_OFF, PINS, NET_W, fl, 3)


def test_preflow_with_excess_passes():
    fl = _flow()
    fl["f_in"][1] = 5      # s pushes 5 into e0_in, only 3 leave
    fl["excess"][3] = 2
    check_preflow(3, NET_OFF, PINS, NET_W, fl, 3)


@pytest.mark.parametrize("plant", ["over_cap_in", "over_cap_bridge", "negative_out",
                                   "not_conserved", "negative_excess", "wrong_value",
                                   "pending_delta"])
def test_planted_errors_fail(plant):
    fl = _flow()
    value = 3
    if plant == "over_cap_in":
        fl["f_in"][2] = 4; fl["f_b"][1] = 4; fl["f_out"][3] = 4; fl["f_out"][0] = 4
        fl["f_in"][1] = 4; fl["f_b"][0] = 4; value = 4   # 4 > w(e1) = 3 on (a, e1_in)
    elif plant == "over_cap_bridge":
        fl["f_b"][1] = 4; fl["excess"][4] = -1
    elif plant == "negative_out":
        fl["f_out"][0] = -1
    elif plant == "not_conserved":
        fl["f_out"][0] = 2
    elif plant == "negative_excess":
        fl["f_b"][0] = 2; fl["excess"][3] = 1; fl["excess"][5] = -1; fl["f_out"][0] = 3
    elif plant == "wrong_value":
        value = 2
    elif plant == "pending_delta":
        fl["delta"][2] = 1
    with pytest.raises(AssertionError):
        check_preflow(3, NET_OFF, PINS, NET_W, fl, value)
