"""Pencil decomposition and message layout (test infrastructure; oracle side).

Restates Sec. II-B of the paper: a 3-D field (N_lambda x N_theta x N_z, held
[lev][lat][lon], lon fastest) is split over a p_r x p_c rank grid; each
transposition is an all-to-all inside one row (z->lambda) or one column
(lambda->theta) of the grid (Sec. II-B: all-to-all by rows, then by columns).

Rank (row, col) has id row * p_c + col.

* z -> lambda (transposition 0): source (row j, col i) holds lon part i (of
  p_c) x lat part j (of p_r) x all levels; destination (row j, col k) holds all
  lon x lat part j x level part k (of p_c).  Message (j,i) -> (j,k) is the box
  lon_i x lat_j x lev_k.
* lambda -> theta (transposition 1): source (row j, col k) holds all lon x lat
  part j x lev part k; destination (row l, col k) holds lon part l (of p_r) x
  all lat x lev part k.  Message (j,k) -> (l,k) is the box lon_l x lat_j x lev_k.

Split rule: "balanced" gives the first (extent mod parts) parts one extra
element; "table1" gives every part floor(extent / parts) and drops the rest,
which is the rule the paper's Table 1 follows (pinned exactly by
tests/test_oracle_plan.py against all 40 entries of Table 1).

Message sizes (bytes): float32 4 per value; float16 2 per value; ZFP rate r
with 3-D blocks: ceil(nx/4) ceil(ny/4) ceil(nz/4) * 8r (every extent padded up
to a multiple of 4, Table 1); 1-D blocks: ceil(nx/4) * ny * nz * r/2.

Buffer layout: the send buffer holds, for source rank 0..P-1 in turn, its
messages in peer order (k for transposition 0, l for transposition 1); the
receive buffer holds, for destination rank 0..P-1, its messages in source
peer order.  Every message starts at a multiple of 256 bytes.
"""
from dataclasses import dataclass
from typing import List, Tuple

ALIGN = 256


def split(extent: int, parts: int, mode: str = "balanced") -> List[Tuple[int, int]]:
    """(start, length) of each part."""
    if mode == "table1":
        L = extent // parts
        return [(i * L, L) for i in range(parts)]
    base, rem = divmod(extent, parts)
    out, s = [], 0
    for i in range(parts):
        L = base + (1 if i < rem else 0)
        out.append((s, L))
        s += L
    return out


@dataclass
class Message:
    src: int
    dst: int
    src_peer: int      # index of src inside the communicator
    dst_peer: int      # index of dst inside the communicator
    x0: int
    nx: int
    y0: int
    ny: int
    z0: int
    nz: int

    @property
    def nvals(self):
        return self.nx * self.ny * self.nz


def _ceil4(v):
    return (v + 3) // 4


def message_bytes(m: Message, rate: int, dims: int = 3) -> int:
    """rate 0 = float32, -16 = float16, r > 0 = ZFP rate r."""
    if rate == 0:
        return 4 * m.nvals
    if rate == -16:
        return 2 * m.nvals
    if dims == 3:
        return _ceil4(m.nx) * _ceil4(m.ny) * _ceil4(m.nz) * 8 * rate
    if dims == 2:
        return _ceil4(m.nx) * _ceil4(m.ny) * m.nz * 2 * rate
    return (_ceil4(m.nx) * m.ny * m.nz * 4 * rate + 7) // 8


def _align(v):
    return (v + ALIGN - 1) // ALIGN * ALIGN


class Plan:
    def __init__(self, nlon, nlat, nlev, pr, pc, transposition=0, dims=3, mode="balanced"):
        self.n = (nlon, nlat, nlev)
        self.pr, self.pc = pr, pc
        self.P = pr * pc
        self.transposition = transposition
        self.dims = dims
        msgs = []
        if transposition == 0:
            lon = split(nlon, pc, mode)
            lat = split(nlat, pr, mode)
            lev = split(nlev, pc, mode)
            for j in range(pr):
                for i in range(pc):
                    for k in range(pc):
                        msgs.append(Message(j * pc + i, j * pc + k, i, k,
                                            lon[i][0], lon[i][1], lat[j][0], lat[j][1],
                                            lev[k][0], lev[k][1]))
        elif transposition == 1:
            lon = split(nlon, pr, mode)
            lat = split(nlat, pr, mode)
            lev = split(nlev, pc, mode)
            for k in range(pc):
                for j in range(pr):
                    for l in range(pr):
                        msgs.append(Message(j * pc + k, l * pc + k, j, l,
                                            lon[l][0], lon[l][1], lat[j][0], lat[j][1],
                                            lev[k][0], lev[k][1]))
        else:
            raise ValueError("transposition must be 0 or 1")
        # send order: by source rank, then destination peer
        self.messages = sorted(msgs, key=lambda m: (m.src, m.dst_peer))

    def layout(self, rate):
        """Returns (send_off, recv_off, total) with offsets keyed by (src, dst)."""
        send_off, off = {}, 0
        for m in self.messages:
            send_off[(m.src, m.dst)] = off
            off = _align(off + message_bytes(m, rate, self.dims))
        total = off
        recv_off, off = {}, 0
        for m in sorted(self.messages, key=lambda m: (m.dst, m.src_peer)):
            recv_off[(m.src, m.dst)] = off
            off = _align(off + message_bytes(m, rate, self.dims))
        assert off == total
        return send_off, recv_off, total
