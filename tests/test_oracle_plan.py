"""Pins of the oracle's pencil plan (paper Sec. II-B; Table 1)."""
import math
import os

import numpy as np
import pytest

from oracle.plan import Plan, split, message_bytes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_message_sizes.txt")


def _table1():
    rows = []
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            n, *mb = line.split()
            rows.append((int(n), [float(x) for x in mb]))
    return rows


def _matches(mib, printed):
    # printed to two decimals; exact ties are printed either way in the table
    # (53.125 -> 53.13 for rate 8 at N=4, 1.625 -> 1.62 for float32 at N=100)
    return abs(mib - printed) <= 0.005 + 1e-12


@pytest.mark.parametrize("N,mb", _table1())
def test_table1_message_sizes(N, mb):
    p = int(round(math.sqrt(N)))
    plan = Plan(2560, 1280, 137, p, p, transposition=0, dims=3, mode="table1")
    m = plan.messages[0]
    got = [message_bytes(m, r, 3) / 2 ** 20 for r in (0, -16, 16, 8)]
    assert all(_matches(g, x) for g, x in zip(got, mb)), (got, mb)
    # every message of the Table-1 plan has the same size
    for r in (0, -16, 16, 8):
        assert len({message_bytes(x, r, 3) for x in plan.messages}) == 1


def test_table1_1281_latitudes_does_not_fit():
    # the reading above: 1281 latitudes fails rows N=9 and N=49
    bad = []
    for N, mb in _table1():
        p = int(round(math.sqrt(N)))
        m = Plan(2560, 1281, 137, p, p, 0, 3, "table1").messages[0]
        got = [message_bytes(m, r, 3) / 2 ** 20 for r in (0, -16, 16, 8)]
        if not all(_matches(g, x) for g, x in zip(got, mb)):
            bad.append(N)
    assert bad == [9, 49]


def test_balanced_split():
    for e in range(1, 60):
        for p in range(1, 9):
            parts = split(e, p)
            assert sum(L for _, L in parts) == e
            assert max(L for _, L in parts) - min(L for _, L in parts) <= 1
            assert all(parts[i][0] + parts[i][1] == parts[i + 1][0] for i in range(p - 1))


@pytest.mark.parametrize("t", [0, 1])
@pytest.mark.parametrize("pr,pc", [(1, 1), (2, 3), (3, 2), (4, 4)])
def test_messages_cover_field_once(t, pr, pc):
    n = (13, 11, 9)
    plan = Plan(*n, pr, pc, transposition=t)
    cnt = np.zeros((n[2], n[1], n[0]), dtype=np.int64)
    for m in plan.messages:
        cnt[m.z0:m.z0 + m.nz, m.y0:m.y0 + m.ny, m.x0:m.x0 + m.nx] += 1
        if t == 0:   # all-to-all by rows: same grid row
            assert m.src // pc == m.dst // pc
        else:        # by columns: same grid column
            assert m.src % pc == m.dst % pc
    assert np.all(cnt == 1)
    per = pc if t == 0 else pr
    assert len(plan.messages) == pr * pc * per


def test_pencils_after_transposition():
    # z->lambda: each destination receives all longitudes of its (lat, lev)
    # part; lambda->theta: all latitudes of its (lon, lev) part.
    n = (16, 12, 10)
    for t in (0, 1):
        plan = Plan(*n, 2, 3, transposition=t)
        by_dst = {}
        for m in plan.messages:
            by_dst.setdefault(m.dst, []).append(m)
        for d, ms in by_dst.items():
            if t == 0:
                assert sum(m.nx for m in ms) == n[0]
                assert len({(m.y0, m.ny, m.z0, m.nz) for m in ms}) == 1
            else:
                assert sum(m.ny for m in ms) == n[1]
                assert len({(m.x0, m.nx, m.z0, m.nz) for m in ms}) == 1


@pytest.mark.parametrize("rate", [0, -16, 8, 16])
def test_layout_offsets(rate):
    plan = Plan(37, 23, 17, 3, 2, transposition=0)
    so, ro, total = plan.layout(rate)
    for offs in (so, ro):
        spans = sorted((offs[(m.src, m.dst)], message_bytes(m, rate)) for m in plan.messages)
        for (a, la), (b, _) in zip(spans, spans[1:]):
            assert a % 256 == 0 and a + la <= b
        assert spans[-1][0] + spans[-1][1] <= total
    # send order = by source rank then destination; receive = by destination then source
    srt = sorted(plan.messages, key=lambda m: so[(m.src, m.dst)])
    assert [(m.src, m.dst) for m in srt] == sorted((m.src, m.dst) for m in plan.messages)
    rrt = sorted(plan.messages, key=lambda m: ro[(m.src, m.dst)])
    assert [(m.dst, m.src) for m in rrt] == sorted((m.dst, m.src) for m in plan.messages)
