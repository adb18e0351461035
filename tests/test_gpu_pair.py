"""The transposition pair (Sec. II-B: z -> lambda by rows, then lambda ->
theta by columns) through the CUDA-graph entry point, against the oracle
running the same two transpositions one after the other."""
import numpy as np
import pytest
import torch

from oracle import packs as op
from oracle import plan as opl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def z():
    from paper_2609_24294_gb300 import build, zfpx
    build.build()
    zfpx.lib()
    return zfpx


def _field(shape, seed):
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    x = np.linspace(0, 2 * np.pi, nx)[None, None, :]
    y = np.linspace(0, np.pi, ny)[None, :, None]
    zz = np.linspace(0, 1, nz)[:, None, None]
    f = 250 + 20 * (np.sin(2 * x + zz) * np.cos(3 * y) + 0.02 * rng.standard_normal(shape))
    return f.astype(np.float32)


@pytest.mark.parametrize("fold", [False, True])
@pytest.mark.parametrize("shape,pr,pc,dims", [((20, 40, 48), 2, 2, 3), ((17, 26, 37), 3, 2, 3),
                                              ((9, 30, 44), 2, 3, 2)])
@pytest.mark.parametrize("rate", [8, 16])
def test_pair_graph_matches_oracle(z, shape, pr, pc, dims, rate, fold):
    x = _field(shape, 1)
    nz, ny, nx = shape
    src = torch.from_numpy(x).cuda()
    mid = torch.full_like(src, float("nan"))
    dst = torch.full_like(src, float("nan"))
    p1 = z.Plan.for_fields(src, pr, pc, 0, dims, dst=mid)
    p2 = z.Plan.for_fields(mid, pr, pc, 1, dims, dst=dst)
    nbuf = max(p1.buffer_bytes(rate), p2.buffer_bytes(rate))
    send = torch.zeros(nbuf, dtype=torch.uint8, device="cuda")
    recv = torch.zeros(nbuf, dtype=torch.uint8, device="cuda")
    g = z.PairGraph(p1, p2, rate, src, mid, dst, send, recv, fold_permute=fold)
    assert g.num_kernels() == (4 if fold else 6)
    before = z.zfpx_launch_count()
    g.launch()
    torch.cuda.synchronize()
    assert z.zfpx_launch_count() - before == g.num_kernels()
    # oracle: the two transpositions in turn
    o1 = opl.Plan(nx, ny, nz, pr, pc, 0, dims)
    o2 = opl.Plan(nx, ny, nz, pr, pc, 1, dims)
    ymid = np.full_like(x, np.nan)
    op.unpack(o1, rate, op.permute(o1, rate, op.pack(o1, rate, x)), ymid)
    zout = np.full_like(x, np.nan)
    op.unpack(o2, rate, op.permute(o2, rate, op.pack(o2, rate, ymid)), zout)
    assert np.array_equal(mid.cpu().numpy().view(np.uint32), ymid.view(np.uint32))
    assert np.array_equal(dst.cpu().numpy().view(np.uint32), zout.view(np.uint32))
    # replaying is deterministic
    dst.fill_(0)
    g.launch()
    torch.cuda.synchronize()
    assert np.array_equal(dst.cpu().numpy().view(np.uint32), zout.view(np.uint32))
    g.close()
