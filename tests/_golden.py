"""Readers for the text fixtures under tests/golden/."""
import os

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_build_golden():
    """Rows, entry, query and answer of the hand-worked 5-point build."""
    rows, entry, query, answer = {}, None, None, None
    for line in open(os.path.join(GOLD, "build_1d_5pts.txt")):
        line = line.split("#")[0].strip()
        if not line:
            continue
        tok = line.split()
        if tok[0] == "entry":
            entry = int(tok[1])
        elif tok[0] == "row":
            rows[int(tok[1])] = [int(t) for t in tok[2:]]
        elif tok[0] == "query":
            query = [float(t) for t in tok[1:]]
        elif tok[0] == "answer":
            answer = [float(t) for t in tok[1:]]
    return rows, entry, query, answer
