"""The communication-time model of the row transposition (Sec. III-E, Sec. V-B;
Table 1 message sizes): closed forms, limits and the pipelining bound.  Host
only: the message sizes come from the library's plan, no kernel runs."""
import math

import pytest

from paper_2609_24294_gb300 import netmodel as nm


@pytest.fixture(scope="module")
def sizes():
    from paper_2609_24294_gb300 import build
    build.build()
    return nm.message_sizes()


def test_machine_matches_the_paper():
    t = nm.Dragonfly()
    # 27 groups x 16 chassis x 4 routers x 1 node; the paper's total of 6480 nodes
    # does not follow from these counts (only the first two groups hold N <= 121)
    assert t.nodes == 1728
    assert t.link_bytes_s == 25e9                       # 200 Gb/s
    assert t.hop_s == 1e-6


def test_hops_symmetric_and_ordered_by_distance():
    t = nm.Dragonfly()
    assert t.hops(5, 5) == 0
    assert t.hops(0, 1) == 3                            # same chassis
    assert t.hops(0, 4) == 5                            # next chassis, same group
    assert t.hops(0, 64) == 7                           # next group
    for a, b in ((0, 1), (3, 60), (10, 700), (1727, 0)):
        assert t.hops(a, b) == t.hops(b, a)
    with pytest.raises(ValueError):
        t.hops(0, 1728)
    t2 = nm.Dragonfly(nodes_per_router=2)
    assert t2.hops(0, 1) == 2


def test_table1_sizes_from_the_plan(sizes):
    # Table 1 in MB (MiB): float32, float16, rate-16, rate-8; the two printed ties
    # (53.125, 1.625 ...) are accepted either way.
    table1 = {4: (212.50, 106.25, 106.25, 53.13), 9: (62.38, 31.19, 33.54, 16.77),
              16: (26.56, 13.28, 14.06, 7.03), 25: (13.50, 6.75, 7.00, 3.50),
              36: (7.62, 3.81, 4.23, 2.12), 49: (4.81, 2.41, 2.58, 1.29),
              64: (3.32, 1.66, 1.95, 0.98), 81: (2.31, 1.15, 1.25, 0.62),
              100: (1.62, 0.81, 1.00, 0.50), 121: (1.23, 0.62, 0.62, 0.31)}
    for N, row in table1.items():
        for s, mb in zip(nm.STRATEGIES, row):
            assert abs(sizes[N][s] / 2 ** 20 - mb) <= 0.0051, (N, s)


def test_alltoall_is_rounds_of_latency_plus_link_time():
    t = nm.Dragonfly()
    m = 1 << 20
    # 4 ranks on one chassis: 3 rounds of (3 hops x 1 us + m / 25 GB/s)
    assert nm.alltoall_time([0, 1, 2, 3], m, t) == pytest.approx(3 * (3e-6 + m / 25e9), rel=1e-12)
    # without latency the exchange is (p - 1) m / beta, for any placement
    t0 = nm.Dragonfly(hop_s=0.0)
    for N in nm.TABLE1_N:
        p = nm.grid_side(N)
        assert nm.exchange_time(N, m, t0) == pytest.approx((p - 1) * m / 25e9, rel=1e-12)
    # pieces only add latency
    assert nm.alltoall_time([0, 1, 2, 3], m, t, pieces=4) == pytest.approx(3 * (4 * 3e-6 + m / 25e9), rel=1e-12)
    assert nm.alltoall_time([7], m, t) == 0.0
    with pytest.raises(ValueError):
        nm.grid_side(8)


def test_rows_that_cross_a_group_are_the_slowest():
    t = nm.Dragonfly()
    # N = 121: rows of 11 consecutive nodes; row 5 spans nodes 55..65 (groups 0 and 1)
    slow = nm.alltoall_time(nm.row_nodes(121, 5), 1 << 20, t)
    fast = nm.alltoall_time(nm.row_nodes(121, 0), 1 << 20, t)
    assert slow > fast
    assert nm.exchange_time(121, 1 << 20, t) == pytest.approx(max(
        nm.alltoall_time(nm.row_nodes(121, r), 1 << 20, t) for r in range(11)))


def test_pipeline_bounds():
    for tp, tc, tu in ((1.0, 2.0, 0.5), (3.0, 0.2, 3.0), (0.0, 1.0, 0.0)):
        ser = nm.serial_total(tp, tc, tu)
        assert nm.pipelined_total(tp, tc, tu, 1) == pytest.approx(ser)
        prev = ser
        for k in (2, 4, 8, 64, 4096):
            t = nm.pipelined_total(tp, tc, tu, k)
            assert max(tp, tc, tu) - 1e-12 <= t <= prev + 1e-12      # never below the slowest stage
            prev = t
        assert nm.pipelined_total(tp, tc, tu, 10 ** 7) == pytest.approx(max(tp, tc, tu), rel=1e-5)


def test_flowshop_equal_pieces_is_the_closed_form():
    # k equal pieces through three stages: the first piece passes every stage, the
    # rest follow one slowest-stage time apart
    for tp, tc, tu in ((1.0, 2.0, 0.5), (3.0, 0.2, 3.0), (0.4, 0.4, 0.4)):
        for k in (1, 2, 5, 8):
            pieces = [(tp / k, tc / k, tu / k)] * k
            assert nm.flowshop(pieces) == pytest.approx(nm.pipelined_total(tp, tc, tu, k), rel=1e-12)


def test_flowshop_by_hand():
    # pieces (pack, exchange, unpack): (1,3,1), (2,1,2), (1,1,1)
    # stage ends: piece 0: 1, 4, 5; piece 1: 3, 5, 7; piece 2: 4, 6, 8
    assert nm.flowshop([(1, 3, 1), (2, 1, 2), (1, 1, 1)]) == pytest.approx(8.0)
    assert nm.flowshop([(2.0, 0.0, 0.0)]) == 2.0 and nm.flowshop([]) == 0.0


def test_model_with_measured_pieces(sizes):
    per = {N: {s: (40e-6, 40e-6) for s in nm.STRATEGIES} for N in nm.TABLE1_N}
    # pieces as fast as an equal split: the same result as the formula; pieces that
    # cost more than their share (launch overheads) make pipelining worth less
    even = {N: {s: {k: [(40e-6 / k, 40e-6 / k)] * k for k in (1, 2, 4)} for s in nm.STRATEGIES}
            for N in nm.TABLE1_N}
    slow = {N: {s: {k: [(40e-6 / k + 10e-6, 40e-6 / k + 10e-6)] * k for k in (1, 2, 4)} for s in nm.STRATEGIES}
            for N in nm.TABLE1_N}
    a = nm.model(nm.TABLE1_N, sizes, per, pieces=(1, 2, 4))
    b = nm.model(nm.TABLE1_N, sizes, per, per_rank_pieces=even)
    c = nm.model(nm.TABLE1_N, sizes, per, per_rank_pieces=slow)
    for N in nm.TABLE1_N:
        for s in nm.STRATEGIES:
            assert b[N][s]["pipelined_s"] == pytest.approx(a[N][s]["pipelined_s"], rel=1e-12)
            assert c[N][s]["pipelined_s"] >= b[N][s]["pipelined_s"] - 1e-15
            assert c[N][s]["pipelined_s"] <= c[N][s]["serial_s"] + 1e-15


def test_speedups_reduce_to_size_ratios_without_overheads(sizes):
    zero = {N: {s: (0.0, 0.0) for s in nm.STRATEGIES} for N in nm.TABLE1_N}
    res = nm.model(nm.TABLE1_N, sizes, zero, nm.Dragonfly(hop_s=0.0), pieces=(1,))
    for N in nm.TABLE1_N:
        for s in nm.STRATEGIES:
            want = sizes[N]["float32"] / sizes[N][s]
            assert res[N][s]["speedup_serial"] == pytest.approx(want, rel=1e-12)
        assert res[N]["float16"]["speedup_serial"] == pytest.approx(2.0, rel=1e-12)
    # at N = 121 the model's ceiling for rate 8 is the size ratio, 4x (Table 1: 1.23 / 0.31)
    assert res[121]["zfp8"]["speedup_serial"] == pytest.approx(4.0, rel=1e-2)


def test_codec_time_is_added_in_series_and_pipelining_helps(sizes):
    per = {N: {"float32": (0.0, 0.0), "float16": (0.0, 0.0), "zfp16": (50e-6, 50e-6), "zfp8": (40e-6, 40e-6)}
           for N in nm.TABLE1_N}
    res = nm.model(nm.TABLE1_N, sizes, per)
    for N in nm.TABLE1_N:
        r = res[N]["zfp8"]
        assert r["serial_s"] == pytest.approx(r["pack_s"] + r["comm_s"] + r["unpack_s"])
        assert r["pipelined_s"] <= r["serial_s"]
        assert res[N]["zfp8"]["speedup_serial"] < sizes[N]["float32"] / sizes[N]["zfp8"]
    # with codec time on the ZFP side only, rate 16 trails float16 at every N
    # (its messages are as large or larger, Table 1)
    assert all(res[N]["float16"]["speedup_serial"] > res[N]["zfp16"]["speedup_serial"] for N in nm.TABLE1_N)
    assert math.isfinite(res[121]["zfp8"]["speedup_pipelined"])


def test_sht_step_sums_and_dilutes_the_speedup():
    from paper_2609_24294_gb300 import netmodel as nm
    Ns = (16, 64)
    tr = {N: {"float32": (1e-4, 4e-3, 1e-4), "float16": (1e-4, 2e-3, 1e-4),
              "zfp16": (2e-4, 2e-3, 2e-4), "zfp8": (2e-4, 1e-3, 2e-4)} for N in Ns}
    zero = {N: 0.0 for N in Ns}
    r0 = nm.sht_step(Ns, tr, zero, zero)
    for N in Ns:
        for s in nm.STRATEGIES:
            assert abs(r0[N][s]["step_s"] - 2 * sum(tr[N][s])) < 1e-15
            # no local compute: the step's speedup is the transposition's
            assert abs(r0[N][s]["speedup_step"] - r0[N][s]["speedup_transposition"]) < 1e-12
    prev = None
    for c in (1e-4, 1e-3, 1e-2):
        r = nm.sht_step(Ns, tr, {N: c for N in Ns}, {N: 2 * c for N in Ns})
        sp = r[64]["zfp8"]["speedup_step"]
        assert abs(r[64]["zfp8"]["step_s"] - (2 * sum(tr[64]["zfp8"]) + 3 * c)) < 1e-15
        assert 1.0 < sp < r[64]["zfp8"]["speedup_transposition"]        # diluted, still faster
        if prev is not None:
            assert sp < prev                                             # more compute, less speedup
        prev = sp
        assert r[64]["float32"]["speedup_step"] == 1.0


def test_per_rank_work_of_the_t1279_grid():
    from paper_2609_24294_gb300 import netmodel as nm
    assert nm.fft_values_per_rank(1) == 2560 * 1280 * 137
    assert nm.fft_values_per_rank(64) * 64 == 2560 * 1280 * 137
    # T1279 on 1280 latitudes: (T+1)(T+2)/2 coefficients, 640 multiply-adds each per part and level
    assert nm.legendre_flops_per_rank(1) == 4 * 137 * 640 * 1280 * 1281 / 2
    assert abs(nm.legendre_flops_per_rank(121) * 121 - nm.legendre_flops_per_rank(1)) < 1e-3
