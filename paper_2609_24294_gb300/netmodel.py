"""Time model of one compressed pencil transposition: pack side, all-to-all, unpack side.

The paper (Sec. III-E, Sec. V-B) simulates the row all-to-all with SimGrid on a
Dragonfly of 27 groups (4 links between groups), 16 chassis per group (3 links
between chassis), 4 routers per chassis (1 link between routers) and one node
per router, with 200 Gb/s links and 1 us of latency per hop, for N = 4 ... 121
nodes and the per-pair message sizes of Table 1.  The codec times are added in
series, on the sender before the collective and on the receiver after it; the
paper notes that per-block pipelining of compression with the exchange would
bring the total below that serial figure.

This module is a closed-form stand-in for that simulation (SimGrid is not used):

* ranks sit on consecutive nodes; a p x p rank grid (N = p^2) exchanges within
  each row of p ranks (rank = row * p + col), all rows at once;
* the all-to-all is a pairwise exchange of p - 1 rounds; in round s rank i sends
  its message to row peer (i + s) mod p and receives one; a round costs the
  latency of the longest route in it plus the message's time on one link
  (injection-bound: one NIC per node, no link contention modelled, so the
  communication time is a lower bound of what a contended network gives);
* a route's latency is its link count times the per-hop latency, with link
  counts taken as 2 between nodes on one router, 3 within a chassis (one
  router-router hop), 5 within a group (a chassis link plus an intra-chassis
  hop at either end) and 7 between groups (a global link in place of the
  chassis link, plus a chassis link); at these message sizes the latency terms
  are small beside the link time;
* pipelining cuts every message into K pieces that flow through pack-side
  codec, exchange and unpack-side codec as a three-stage pipeline; every piece
  pays the route latency again.

Times are seconds, sizes bytes.  ``per_rank`` times come from measurements of
the pack-side and unpack-side kernels on one rank's pencil (see
``bench.py``); nothing here runs on the GPU.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

# Table 1 node counts and the 2560 x 1280 x 137 grid its message sizes fit.
TABLE1_N = (4, 9, 16, 25, 36, 49, 64, 81, 100, 121)
TABLE1_GRID = (2560, 1280, 137)                   # lon, lat, lev
STRATEGIES = ("float32", "float16", "zfp16", "zfp8")
RATE_OF = {"float32": 0, "float16": -16, "zfp16": 16, "zfp8": 8}

# The paper's own end-to-end speedups over float32 at N = 121 (Table 2), A100
# codec timings plus the SimGrid Dragonfly; quoted beside the model as context.
PAPER_SPEEDUP_N121 = {"float16": 2.05, "zfp16": 1.95, "zfp8": 3.97}


@dataclass(frozen=True)
class Dragonfly:
    """The simulated machine of Sec. III-E (defaults are the paper's)."""
    groups: int = 27
    chassis_per_group: int = 16
    routers_per_chassis: int = 4
    nodes_per_router: int = 1
    link_gbit_s: float = 200.0
    hop_s: float = 1e-6

    @property
    def nodes(self) -> int:
        return self.groups * self.chassis_per_group * self.routers_per_chassis * self.nodes_per_router

    @property
    def link_bytes_s(self) -> float:
        return self.link_gbit_s * 1e9 / 8.0

    def _coords(self, node: int):
        router, _ = divmod(node, self.nodes_per_router)
        chassis, _ = divmod(router, self.routers_per_chassis)
        group, _ = divmod(chassis, self.chassis_per_group)
        return group, chassis, router

    def hops(self, a: int, b: int) -> int:
        """Links on a minimal route between nodes a and b (0 for a == b)."""
        if not (0 <= a < self.nodes and 0 <= b < self.nodes):
            raise ValueError("node outside the machine")
        if a == b:
            return 0
        ga, ca, ra = self._coords(a)
        gb, cb, rb = self._coords(b)
        if ra == rb:
            return 2                  # node -> router -> node
        if ca == cb:
            return 3                  # + one router-router hop
        if ga == gb:
            return 5                  # + chassis link, one intra-chassis hop at each end
        return 7                      # a global link and a chassis link


def row_nodes(N: int, row: int):
    """Nodes of row `row` of the sqrt(N) x sqrt(N) rank grid (rank r on node r)."""
    p = grid_side(N)
    return [row * p + c for c in range(p)]


def grid_side(N: int) -> int:
    p = int(round(math.sqrt(N)))
    if p * p != N or p < 1:
        raise ValueError("N must be a perfect square (a p x p rank grid)")
    return p


def alltoall_time(nodes, m_bytes: float, topo: Dragonfly = Dragonfly(), pieces: int = 1) -> float:
    """Pairwise-exchange all-to-all of one message of m_bytes per ordered pair
    among `nodes`, each message sent as `pieces` back-to-back pieces."""
    p = len(nodes)
    if p <= 1 or m_bytes <= 0:
        return 0.0
    t = 0.0
    for s in range(1, p):
        lat = max(topo.hops(nodes[i], nodes[(i + s) % p]) for i in range(p)) * topo.hop_s
        t += pieces * lat + m_bytes / topo.link_bytes_s
    return t


def exchange_time(N: int, m_bytes: float, topo: Dragonfly = Dragonfly(), pieces: int = 1) -> float:
    """The row transposition: every row's all-to-all at once; the slowest row."""
    p = grid_side(N)
    return max(alltoall_time(row_nodes(N, r), m_bytes, topo, pieces) for r in range(p))


def serial_total(t_pack: float, t_comm: float, t_unpack: float) -> float:
    """The paper's serial model: pack side, then the collective, then unpack side."""
    return t_pack + t_comm + t_unpack


def pipelined_total(t_pack: float, t_comm_k: float, t_unpack: float, k: int) -> float:
    """Three-stage pipeline over k equal pieces: the first piece passes every
    stage, the other k - 1 follow one slowest-stage time apart.  t_comm_k is the
    exchange time with every message in k pieces (it includes k latencies)."""
    if k < 1:
        raise ValueError("k >= 1")
    stages = (t_pack / k, t_comm_k / k, t_unpack / k)
    return sum(stages) + (k - 1) * max(stages)


def flowshop(stage_times) -> float:
    """Makespan of pieces flowing in order through three stages (pack-side codec,
    exchange, unpack-side codec), each stage serving one piece at a time:
    stage_times[i] = (pack s, exchange s, unpack s) of piece i.  A piece enters a
    stage when the stage has finished the previous piece and the piece has left
    the previous stage."""
    done = [0.0, 0.0, 0.0]
    for t in stage_times:
        prev = 0.0
        for s in range(3):
            done[s] = max(done[s], prev) + t[s]
            prev = done[s]
    return done[2]


def message_sizes(N_list=TABLE1_N, grid=TABLE1_GRID, split=None):
    """Per-pair message bytes of the row transposition for each strategy, from
    the library's plan (the Table 1 split by default: every extent divided by p
    and rounded down, level padding to a multiple of 4 for ZFP)."""
    from . import zfpx as z
    split = z.SPLIT_TABLE1 if split is None else split
    out = {}
    for N in N_list:
        p = grid_side(N)
        plan = z.Plan(grid, p, p, 0, 3, split)
        try:
            ranks, _ = plan.messages()[0]
            out[N] = {s: plan.message_bytes(RATE_OF[s], ranks[0], ranks[1]) for s in STRATEGIES}
        finally:
            plan.close()
    return out


def model(N_list, sizes, per_rank, topo: Dragonfly = Dragonfly(), pieces=(1, 2, 4, 8, 16, 32),
          per_rank_pieces=None):
    """Time breakdown and speedups per node count.

    sizes[N][strategy]: per-pair message bytes.  per_rank[N][strategy] =
    (pack-side seconds, unpack-side seconds) for one rank's pencil.  Returns,
    per N and strategy: the three serial terms, the serial total, the best
    pipelined total and its piece count, and the speedups over float32 of both.

    per_rank_pieces[N][strategy][k], when given, is the measured list of k
    (pack s, unpack s) of the rank's pencil cut into k pieces; the pipelined
    total is then the flow shop of those measured pieces (each piece's exchange
    time the k-piece exchange over k), over the k it holds, in place of the
    equal-piece formula.
    """
    res = {}
    for N in N_list:
        row = {}
        for s in STRATEGIES:
            tp, tu = per_rank[N][s]
            tc = exchange_time(N, sizes[N][s], topo)
            ser = serial_total(tp, tc, tu)
            best_k, best = 1, ser
            measured = (per_rank_pieces or {}).get(N, {}).get(s)
            for k in (sorted(measured) if measured else pieces):
                tck = exchange_time(N, sizes[N][s], topo, k)
                if measured:
                    t = flowshop([(a, tck / k, b) for a, b in measured[k]])
                else:
                    t = pipelined_total(tp, tck, tu, k)
                if t < best:
                    best_k, best = k, t
            row[s] = {"message_bytes": sizes[N][s], "pack_s": tp, "comm_s": tc, "unpack_s": tu,
                      "serial_s": ser, "pipelined_s": best, "pieces": best_k}
        for s in STRATEGIES:
            row[s]["speedup_serial"] = row["float32"]["serial_s"] / row[s]["serial_s"]
            row[s]["speedup_pipelined"] = row["float32"]["pipelined_s"] / row[s]["pipelined_s"]
        res[N] = row
    return res


# The forward spectral transform of the Table 1 grid: 2560 longitudes, 1280
# Gaussian latitudes, 137 levels, linear truncation T = 1279.
SHT_GRID = (2560, 1280, 137)
SHT_T = 1279


def fft_values_per_rank(N: int, grid=SHT_GRID) -> float:
    """Grid-point values of one rank's lambda-pencil (the longitude FFT's input)."""
    nlon, nlat, nlev = grid
    return nlon * nlat * nlev / N


def legendre_flops_per_rank(N: int, grid=SHT_GRID, T: int = SHT_T) -> float:
    """Folded float32 flops of one rank's share of the Legendre transform: every
    coefficient takes nlat/2 multiply-adds for each of its real and imaginary
    parts and each level; shared evenly over the N ranks."""
    _, nlat, nlev = grid
    return 2.0 * 2 * nlev * (nlat // 2) * (T + 1) * (T + 2) / 2 / N


def sht_step(N_list, transposition, fft_s, legendre_s):
    """One forward spectral-transform step per node count, in series (Sec. II-B's
    order): the row transposition, the longitude FFT, the column transposition,
    the Legendre transform.

    transposition[N][strategy] = (pack-side s, exchange s, unpack-side s) of the
    row transposition; the column transposition is taken to cost the same (in a
    p x p grid its messages carry the same number of values, now wavenumbers).
    fft_s[N], legendre_s[N]: one rank's compute, the same for every strategy.
    Returns per N and strategy the four terms, the step time and the speedup of
    the step over float32, beside the speedup of the transposition alone."""
    res = {}
    for N in N_list:
        row = {}
        for s in STRATEGIES:
            tp, tc, tu = transposition[N][s]
            t1 = tp + tc + tu
            step = t1 + fft_s[N] + t1 + legendre_s[N]
            row[s] = {"transposition_s": t1, "fft_s": fft_s[N], "legendre_s": legendre_s[N], "step_s": step}
        for s in STRATEGIES:
            row[s]["speedup_step"] = row["float32"]["step_s"] / row[s]["step_s"]
            row[s]["speedup_transposition"] = row["float32"]["transposition_s"] / row[s]["transposition_s"]
        res[N] = row
    return res
