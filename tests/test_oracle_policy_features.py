"""Pins of the learned policy's features (the network inputs at the decision
hop) against hand-worked values in tests/golden/policy_features.txt.

Cases A-D give list states entry by entry and check the oracle's feature
function on them: at least k passing, fewer than k, none, and a fully
expanded list with a clamped estimate.  The last two lines run the oracle's
search with a FORCED policy on the hand-worked 5-point graph and check the
features it records after one and after two hops, which ties the feature
function to the search state it is computed from (Algorithm 1 after h0
iterations)."""
import os
import struct

import numpy as np
import pytest

from oracle import jag_oracle as O
from paper_2602_10258_gb300 import datagen as D

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "policy_features.txt")


def _num(tok):
    """A fixture number: 0x... is an fp32 (or uint32) bit pattern, else a decimal."""
    if tok.startswith("0x"):
        return struct.unpack("<f", struct.pack("<I", int(tok, 16)))[0]
    return float(tok)


def _read():
    cases, searches, cur = [], [], None
    for line in open(GOLD):
        line = line.split("#")[0].strip()
        if not line:
            continue
        t = line.split()
        if t[0] == "case":
            cur = {"name": t[1], "k": int(t[3]), "est": int(t[5]), "kind": int(t[7]), "entries": []}
            cases.append(cur)
        elif t[0] == "entry":
            k1 = int(t[1], 16) if t[1].startswith("0x") else int(t[1])
            cur["entries"].append((k1, float(t[2]), int(t[3])))
        elif t[0] == "features" and cur is not None and "features" not in cur:
            cur["features"] = np.array([_num(v) for v in t[1:]], np.float32)
        elif t[0] == "search":
            searches.append((int(t[2]), np.array([_num(v) for v in t[4:]], np.float32)))
    return cases, searches


CASES, SEARCHES = _read()


def test_fixture_is_complete():
    assert [c["name"] for c in CASES] == ["A", "B", "C", "D"]
    assert all(len(c["features"]) == O.NFEAT for c in CASES)
    assert [h for h, _ in SEARCHES] == [1, 2]


@pytest.mark.parametrize("case", CASES, ids=[c["name"] for c in CASES])
def test_features_of_hand_worked_lists(case):
    e = case["entries"]
    f = O.policy_features([v[0] for v in e], [v[1] for v in e], [v[2] for v in e], case["k"], case["est"],
                          case["kind"])
    # bit-exact: every expected value is the fp32 the definition rounds to
    assert f.view(np.uint32).tolist() == case["features"].view(np.uint32).tolist(), (f, case["features"])


def _five_point_index():
    x = np.array([[0], [2], [3], [7], [9]], np.float32)
    graph = np.array([[2, 1], [2, 0], [1, 3], [2, 4], [3, -1]], np.int32)
    return O.Index(x, attr_i32=np.arange(5, dtype=np.int32), dist_a=O.K_LABEL, R=2, graph=graph, entry=2)


@pytest.mark.parametrize("h0,want", SEARCHES, ids=["h0=%d" % h for h, _ in SEARCHES])
def test_features_of_the_search_state(h0, want):
    ix = _five_point_index()
    f = D.filters_range_i32([0], [1])
    pol = O.Policy(O.POL_FORCED, h0=h0, forced=np.zeros((1, 2), np.int32), nq=1, want_features=True)
    ids, dist, _ = O.query_policy(ix, np.array([[6.0]], np.float32), f, np.zeros(8, np.uint8), 2, 2, pol)
    assert pol.features[0].view(np.uint32).tolist() == want.view(np.uint32).tolist(), (pol.features[0], want)
    # the decision keeps the beam and sets no stop, so the answer is the plain one
    assert list(ids[0]) == [1, 0] and list(dist[0]) == [16.0, 36.0]
