"""Pins of the oracle's low-precision storage (BF16, FP8-E4M3 with a per-row
scale) and of the FP32 re-rank, against the number formats' definitions,
exact rational arithmetic and special cases.  CPU only."""
from fractions import Fraction

import numpy as np
import pytest

from oracle import jag_oracle as O
from paper_2602_10258_gb300 import datagen as D


def _bf16_value(h):
    return float(np.array([int(h) << 16], np.uint32).view(np.float32)[0])


def test_bf16_is_nearest_ties_to_even():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(3000).astype(np.float32) * np.float32(10) ** rng.uniform(-4, 4, 3000).astype(np.float32),
                        np.array([1.0, -2.5, 3.0e-5, 65504.0], np.float32)])
    # exact halfway points between neighbouring bf16 values
    base = rng.integers(0x3000, 0x4F00, 500).astype(np.uint32)
    half = ((base << 16) | 0x8000).view(np.float32)
    x = np.concatenate([x, half, -half])
    enc = O.bf16_encode(x)
    for xi, hi in zip(x, enc):
        b = int(np.array([xi], np.float32).view(np.uint32)[0])
        t = b >> 16
        cands = [t, t + 1]
        ex = Fraction(float(xi))
        dist = [abs(Fraction(_bf16_value(c)) - ex) for c in cands]
        if dist[0] < dist[1]:
            want = cands[0]
        elif dist[1] < dist[0]:
            want = cands[1]
        else:
            want = cands[0] if cands[0] % 2 == 0 else cands[1]
        assert int(hi) == want, (xi, hi, want)


def test_fp8_published_values():
    # OCP 8-bit floating point, E4M3: bias 7, max 448, min normal 2^-6,
    # min subnormal 2^-9, 1.0 = 0 0111 000
    v = O.fp8_decode(np.array([0x38, 0x7E, 0x08, 0x01, 0x07, 0x00, 0xB8, 0xFE], np.uint8))
    assert list(v) == [1.0, 448.0, 2.0 ** -6, 2.0 ** -9, 7 * 2.0 ** -9, 0.0, -1.0, -448.0]
    pos = O.fp8_decode(np.arange(127, dtype=np.uint8))
    assert (np.diff(pos) > 0).all()                       # increasing with the code
    assert len(set(pos.tolist())) == 127


def test_fp8_round_trip_midpoints_and_saturation():
    codes = np.array([c for c in range(256) if c not in (127, 255)], np.uint8)
    vals = O.fp8_decode(codes)
    back = O.fp8_encode(vals)
    assert (back[codes != 0x80] == codes[codes != 0x80]).all()
    assert O.fp8_encode(np.float32(-0.0))[0] == 0x80
    pos = O.fp8_decode(np.arange(127, dtype=np.uint8)).astype(np.float64)
    for c in range(126):
        mid = (pos[c] + pos[c + 1]) / 2                  # exact in fp32 (few bits)
        m32 = np.float32(mid)
        assert float(m32) == mid
        even = c if c % 2 == 0 else c + 1
        assert O.fp8_encode(m32)[0] == even
        assert O.fp8_encode(np.nextafter(m32, np.float32(np.inf)))[0] == c + 1
        assert O.fp8_encode(np.nextafter(m32, np.float32(-np.inf)))[0] == c
    for big in (448.0001, 464.0, 1e9):
        assert O.fp8_encode(np.float32(big))[0] == 0x7E
        assert O.fp8_encode(np.float32(-big))[0] == 0xFE


def test_fp8_quantize_scale_and_error():
    rng = np.random.default_rng(3)
    x = (rng.standard_normal((200, 37)) * 3).astype(np.float32)
    x[5] = 0.0
    q, s = O.quantize(x, O.FMT_FP8)
    assert q.shape == (200, 48)                            # 37 bytes padded to 16-byte chunks
    assert (q[:, 37:] == 0).all()
    assert s[5] == 1.0 and (q[5, :37] == 0).all()
    for i in range(200):
        if i == 5:
            continue
        mx = np.abs(x[i]).max()
        assert s[i] == np.float32(mx / np.float32(448.0))
        j = int(np.argmax(np.abs(x[i])))
        assert q[i, j] & 0x7F == 0x7E                      # the largest element lands on +-448
        deq = (s[i] * O.fp8_decode(q[i, :37])).astype(np.float64)
        err = np.abs(deq - x[i])
        # half a unit in the last place: 2^-4 relative above 2^-6, s * 2^-10 absolute below
        bound = np.maximum(np.abs(x[i]) * 2.0 ** -4, s[i] * 2.0 ** -10) * (1 + 1e-6)
        assert (err <= bound).all()


def test_bf16_quantize_layout():
    x = np.arange(-50, 50, dtype=np.float32).reshape(10, 10)
    q, s = O.quantize(x, O.FMT_BF16)
    assert q.shape == (10, 32) and (s == 1).all()
    h = q[:, :20].copy().view(np.uint16)
    assert (np.array([_bf16_value(v) for v in h.ravel()]).reshape(10, 10) == x).all()


@pytest.mark.parametrize("fmt", [O.FMT_BF16, O.FMT_FP8])
def test_quantized_distance_exact_on_small_integers(fmt):
    """Integers in [-16, 16] are exact in BF16 and, with scale 1 (a row whose
    largest magnitude is 448), in E4M3: every partial sum is exact, so the
    distance is the exact sum whatever the chunking."""
    rng = np.random.default_rng(4)
    for d in (1, 7, 16, 33, 100, 128, 300):
        x = rng.integers(-16, 17, (20, d)).astype(np.float32)
        if fmt == O.FMT_FP8:
            x[:, 0] = 448.0
        q = rng.integers(-16, 17, (20, d)).astype(np.float32)
        rows, s = O.quantize(x, fmt)
        got = O.dist_canon_q_rows(q, rows, s, fmt)
        exact = ((q.astype(np.int64) - x.astype(np.int64)) ** 2).sum(1)
        assert (got == exact).all()


@pytest.mark.parametrize("fmt", [O.FMT_BF16, O.FMT_FP8])
def test_quantized_distance_error_bound(fmt):
    """Against the exact distance to the dequantized row (rational
    arithmetic): within the summation bound gamma_(d+2)."""
    rng = np.random.default_rng(5)
    d = 100
    x = rng.standard_normal((10, d)).astype(np.float32)
    q = rng.standard_normal((10, d)).astype(np.float32)
    rows, s = O.quantize(x, fmt)
    got = O.dist_canon_q_rows(q, rows, s, fmt)
    u = 2.0 ** -24
    gamma = (d + 2) * u / (1 - (d + 2) * u)
    for i in range(10):
        if fmt == O.FMT_BF16:
            deq = [Fraction(_bf16_value(h)) for h in rows[i, :2 * d].copy().view(np.uint16)]
        else:
            deq = [Fraction(float(np.float32(s[i] * v))) for v in O.fp8_decode(rows[i, :d])]
        exact = sum((Fraction(float(a)) - b) ** 2 for a, b in zip(q[i], deq))
        assert abs(Fraction(float(got[i])) - exact) <= Fraction(gamma) * exact


@pytest.fixture(scope="module")
def built_small():
    w = D.make_range_i32(n=1500, d=24, nq=40, seed=13, width=200)
    ix = O.Index.from_workload(w, R=16)
    O.build(ix, lb=32)
    return w, ix


@pytest.mark.parametrize("fmt", [O.FMT_BF16, O.FMT_FP8])
def test_quantized_search_literal_equals_direct(built_small, fmt):
    w, ix = built_small
    qx = O.Index.from_workload(w, R=16, graph=ix.graph, entry=ix.entry, storage=fmt)
    for ls in (10, 20, 64):
        a, da, _ = O.query(qx, w.q, w.filters, w.aux, 10, ls)
        b, db, _ = O.query(qx, w.q, w.filters, w.aux, 10, ls, literal=True)
        assert (a == b).all() and (da == db).all()


@pytest.mark.parametrize("fmt", [O.FMT_BF16, O.FMT_FP8])
def test_quantized_search_reranks_in_fp32(built_small, fmt):
    """Answers carry exact fp32 distances, sorted; with a full beam the top 4k
    by the stored-format distance contain the exact top k."""
    w, ix = built_small
    qx = O.Index.from_workload(w, R=16, graph=ix.graph, entry=ix.entry, storage=fmt)
    ids, dist, _ = O.query(qx, w.q, w.filters, w.aux, 10, ix.n)
    bi, bd, _, _ = O.brute_force(ix, w.q, w.filters, w.aux, 10)
    assert (ids == bi).all() and (dist == bd).all()
    ids, dist, _ = O.query(qx, w.q, w.filters, w.aux, 10, 32)
    for i in range(len(ids)):
        m = ids[i] >= 0
        ref = O.dist_canon_rows(np.repeat(w.q[i:i + 1], m.sum(), 0), w.x[ids[i][m]])
        assert (ref == dist[i][m]).all()
        assert (np.diff(dist[i][m]) >= 0).all()
