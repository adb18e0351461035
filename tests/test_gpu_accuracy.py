"""GPU parity of the accuracy mode (variable-rate 3-D blocks to an absolute
tolerance, Sec. II-C's named future mode) through the C ABI against the CPU
oracle: per-block bit counts, total bits and payload bytes bit-exact, decoded
values bit-exact; small ragged and strided arrays and the 1280 x 640 x 137
field."""
import numpy as np
import pytest
import torch

import fieldgen
from oracle import codec as oc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def z():
    from paper_2609_24294_gb300 import build, zfpx
    build.build()
    zfpx.lib()
    return zfpx


def _run(z, src, tol):
    """GPU encode + decode; returns (lengths, payload bytes, total bits, decoded)."""
    n = tuple(reversed(src.shape))
    nblk = ((n[0] + 3) // 4) * ((n[1] + 3) // 4) * ((n[2] + 3) // 4)
    lengths = torch.zeros(nblk, dtype=torch.int16, device="cuda")
    payload = torch.zeros(z.zfpx_accuracy_max_payload_bytes(n), dtype=torch.uint8, device="cuda")
    total = torch.zeros(1, dtype=torch.int64, device="cuda")
    work = torch.zeros(z.zfpx_accuracy_workspace_bytes(n), dtype=torch.uint8, device="cuda")
    z.zfpx_encode_accuracy(src, tol, lengths, payload, total, work)
    torch.cuda.synchronize()
    bits = int(total.item())
    used = 8 * ((bits + 63) // 64)
    dec = torch.full(src.shape, float("nan"), device="cuda")
    z.zfpx_decode_accuracy(lengths, payload[:max(used, 8)], dec, work)
    torch.cuda.synchronize()
    return lengths.cpu().numpy().view(np.uint16), payload.cpu().numpy(), bits, dec.cpu().numpy()


def _check(z, x, src, tol):
    L, P, bits, dec = _run(z, src, tol)
    rL, rP, rbits = oc.encode_accuracy(np.ascontiguousarray(x), tol)
    assert bits == rbits
    np.testing.assert_array_equal(L, rL)
    nb = (bits + 7) // 8
    assert P[:nb].tobytes() == rP[:nb].tobytes()
    assert not P[8 * ((bits + 63) // 64):].any()
    rdec = np.empty_like(np.ascontiguousarray(x))
    oc.decode_accuracy(rL, rP, rdec)
    assert dec.view(np.uint32).tobytes() == rdec.view(np.uint32).tobytes()
    return L, bits


@pytest.mark.parametrize("rel", [1e-1, 1e-3, 1e-5])
@pytest.mark.parametrize("shape", [(1, 1, 1), (4, 4, 4), (7, 5, 3), (9, 13, 22), (17, 26, 37)])
def test_small_arrays(z, shape, rel):
    rng = np.random.default_rng(sum(shape))
    g = np.cumsum(np.cumsum(rng.standard_normal(shape), axis=2), axis=1)
    x = (250.0 + g).astype(np.float32)
    tol = rel * float(np.abs(x).max())
    _check(z, x, torch.from_numpy(x).cuda(), tol)


def test_special_values_and_views(z):
    rng = np.random.default_rng(7)
    big = (rng.standard_normal((12, 20, 40)) * 10.0 ** rng.integers(-30, 30, (12, 20, 40))).astype(np.float32)
    big[0:4, 0:4, 0:4] = 0.0
    big[0:4, 4:8, 0:4] = 3.25
    big[4:8, 0:4, 0:4] = np.float32(5e-40)
    big[5, 5, 5] = np.inf
    big[9, 9, 9] = np.nan
    x = big[1:11, 2:19, 3:37]                                       # unaligned view
    src = torch.from_numpy(big).cuda()[1:11, 2:19, 3:37]
    for tol in (1e-3, 1.0, 1e6):
        _check(z, x, src, tol)


def test_repeated_calls_share_the_workspace(z):
    x = (250.0 + np.cumsum(np.random.default_rng(3).standard_normal((8, 16, 40)), axis=2)).astype(np.float32)
    src = torch.from_numpy(x).cuda()
    a = _run(z, src, 0.01)
    b = _run(z, src, 0.01)
    np.testing.assert_array_equal(a[0], b[0])
    assert a[2] == b[2] and a[1].tobytes() == b[1].tobytes()


def test_t639_field_full_size(z):
    x = fieldgen.t639_field()
    L, bits = _check(z, x, torch.from_numpy(x).cuda(), 1e-3)
    assert 0 < bits < 16 * x.size                                    # variable, below the rate-16 cut


# ---------------------------------------------------------------- plans: the all-to-all-v
@pytest.mark.parametrize("t", [0, 1])
@pytest.mark.parametrize("shape,pr,pc", [((17, 23, 37), 3, 2), ((20, 16, 48), 1, 4), ((3, 8, 8), 2, 4)])
def test_plan_accuracy_matches_oracle(z, shape, pr, pc, t):
    from oracle import plan as opl
    rng = np.random.default_rng(sum(shape) + t)
    nz, ny, nx = shape
    x = (250.0 + np.cumsum(np.cumsum(rng.standard_normal(shape), axis=2), axis=1)).astype(np.float32)
    tol = 1e-3 * float(np.abs(x).max())
    xd = torch.from_numpy(x).cuda()
    dst_store = torch.full((nz, ny, nx + 6), float("nan"), device="cuda")
    dst = dst_store[:, :, :nx]
    plan = z.Plan.for_fields(xd, pr, pc, t, 3, dst=dst)
    acc = z.AccuracyTransposition(plan)
    acc.compress(xd, tol)
    acc.exchange()
    acc.decompress(dst)
    torch.cuda.synchronize()
    oplan = opl.Plan(nx, ny, nz, pr, pc, t, 3)
    msgs = oplan.messages
    exp = []
    for m in msgs:
        box = np.ascontiguousarray(x[m.z0:m.z0 + m.nz, m.y0:m.y0 + m.ny, m.x0:m.x0 + m.nx])
        if box.size == 0:
            exp.append((np.zeros(0, np.uint16), np.zeros(0, np.uint8), 0))
        else:
            exp.append(oc.encode_accuracy(box, tol))
    words = acc.words.cpu().numpy()[:len(msgs)]
    np.testing.assert_array_equal(words, [(b + 63) // 64 for _, _, b in exp])
    G = acc.G
    len_send = acc.len_send.cpu().numpy().view(np.uint16)[:G]
    np.testing.assert_array_equal(len_send, np.concatenate([L for L, _, _ in exp]) if G else len_send)
    pay_send = acc.pay_send.cpu().numpy()
    o = 0
    for (L, P, b), w in zip(exp, words):
        nb = (b + 7) // 8
        assert pay_send[8 * o:8 * o + nb].tobytes() == P[:nb].tobytes()
        o += int(w)
    # receive order: by destination rank, then source peer
    rorder = sorted(range(len(msgs)), key=lambda i: (msgs[i].dst, msgs[i].src_peer))
    len_recv = acc.len_recv.cpu().numpy().view(np.uint16)[:G]
    if G:
        np.testing.assert_array_equal(len_recv, np.concatenate([exp[i][0] for i in rorder]))
    pay_recv = acc.pay_recv.cpu().numpy()
    o = 0
    for i in rorder:
        L, P, b = exp[i]
        nb = (b + 7) // 8
        assert pay_recv[8 * o:8 * o + nb].tobytes() == P[:nb].tobytes()
        o += int(words[i])
    rdst = np.full_like(x, np.nan)
    for m, (L, P, b) in zip(msgs, exp):
        if m.nx * m.ny * m.nz == 0:
            continue
        box = np.empty((m.nz, m.ny, m.nx), np.float32)
        oc.decode_accuracy(L, P, box)
        rdst[m.z0:m.z0 + m.nz, m.y0:m.y0 + m.ny, m.x0:m.x0 + m.nx] = box
    assert dst.cpu().numpy().view(np.uint32).tobytes() == rdst.view(np.uint32).tobytes()
    assert torch.isnan(dst_store[:, :, nx:]).all()


# ---------------------------------------------------------------- precision mode
@pytest.mark.parametrize("p", [4, 12, 20, 32])
def test_precision_arrays_and_plan(z, p):
    from oracle import plan as opl
    rng = np.random.default_rng(50 + p)
    shape = (9, 13, 22)
    x = (np.cumsum(np.cumsum(rng.standard_normal(shape), axis=2), axis=1) * 10.0 ** rng.uniform(-3, 3)).astype(np.float32)
    src = torch.from_numpy(x).cuda()
    n = tuple(reversed(shape))
    nblk = 3 * 4 * 6
    lengths = torch.zeros(nblk, dtype=torch.int16, device="cuda")
    payload = torch.zeros(z.zfpx_accuracy_max_payload_bytes(n), dtype=torch.uint8, device="cuda")
    total = torch.zeros(1, dtype=torch.int64, device="cuda")
    work = torch.zeros(z.zfpx_accuracy_workspace_bytes(n), dtype=torch.uint8, device="cuda")
    z.zfpx_encode_precision(src, p, lengths, payload, total, work)
    dec = torch.full_like(src, float("nan"))
    z.zfpx_decode_accuracy(lengths, payload, dec, work)
    torch.cuda.synchronize()
    rL, rP, rbits = oc.encode_precision(x, p)
    assert int(total.item()) == rbits
    np.testing.assert_array_equal(lengths.cpu().numpy().view(np.uint16), rL)
    assert payload.cpu().numpy()[:(rbits + 7) // 8].tobytes() == rP.tobytes()
    rdec = np.empty_like(x)
    oc.decode_accuracy(rL, rP, rdec)
    assert dec.cpu().numpy().view(np.uint32).tobytes() == rdec.view(np.uint32).tobytes()
    # on a plan, through the all-to-all-v
    plan = z.Plan.for_fields(src, 2, 3, 0, 3)
    acc = z.AccuracyTransposition(plan)
    acc.compress_precision(src, p)
    acc.exchange()
    out = torch.full_like(src, float("nan"))
    acc.decompress(out)
    torch.cuda.synchronize()
    rout = np.full_like(x, np.nan)
    for m in opl.Plan(n[0], n[1], n[2], 2, 3, 0, 3).messages:
        if m.nx * m.ny * m.nz == 0:
            continue
        box = np.ascontiguousarray(x[m.z0:m.z0 + m.nz, m.y0:m.y0 + m.ny, m.x0:m.x0 + m.nx])
        L, P, b = oc.encode_precision(box, p)
        o = np.empty_like(box)
        oc.decode_accuracy(L, P, o)
        rout[m.z0:m.z0 + m.nz, m.y0:m.y0 + m.ny, m.x0:m.x0 + m.nx] = o
    assert out.cpu().numpy().view(np.uint32).tobytes() == rout.view(np.uint32).tobytes()
