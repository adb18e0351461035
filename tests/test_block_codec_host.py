"""The library's block coders built for the host CPU against the oracle, block
by block and bit for bit (paper Sec. II-C; the readings of the oracle).

`tests/block_codec_host.cpp` compiles the __host__ __device__ functions of
`csrc/zfpx_block.cuh` with a C++ compiler: the 3-D block decoder that the
GPU's decode kernels run (windowed plane parse, transposes, inverse
transform, dequantisation), the scalar two-pass 3-D encoder (the statement
the GPU's warp-uniform encoder follows), and the 2-D and 1-D encoders and
decoders (the 1-D ones with four blocks in lockstep, checked against one
block at a time).
Streams must equal the oracle's byte for byte and decoded floats its bit
patterns, on graded spectra, random blocks over many scales, special values
(zero, signed zero, subnormals, the largest floats, inf and NaN) and, for the
decoders, arbitrary byte streams.  No GPU: a regression in the coding logic
shows here before any GPU run.  (The warp-uniform 3-D encoder the GPU runs,
`csrc/zfpx_enc3.cuh`, is device code; its parity is in the GPU tests.)"""
import shutil
import subprocess
from pathlib import Path

import numpy as np
import pytest

from fieldgen.workloads import graded_blocks
from oracle import codec as oc

ROOT = Path(__file__).resolve().parents[1]
SRC = ROOT / "tests" / "block_codec_host.cpp"
CSRC = ROOT / "paper_2609_24294_gb300" / "csrc"


@pytest.fixture(scope="module")
def host(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = tmp_path_factory.mktemp("block_codec_host") / "block_codec_host"
    subprocess.run([cxx, "-std=c++17", "-O2", "-Wno-unknown-pragmas", "-I", str(CSRC), str(SRC), "-o", str(exe)],
                   check=True)
    return exe


def run(host, mode, rate, data):
    r = subprocess.run([str(host), mode, str(rate)], input=bytes(data), capture_output=True)
    assert r.returncode == 0, (mode, rate, r.returncode)
    return r.stdout


def blocks(dims, n, seed):
    """n blocks of 4^dims float32 values: graded spectra (3-D), normal values
    scaled over many decades, constants, sparse blocks and special values."""
    S = 4 ** dims
    r = np.random.default_rng(seed)
    out = []
    if dims == 3:
        g = graded_blocks(n // 4, seed)                                  # [4][4][4 nb]
        out.append(g.reshape(4, 4, n // 4, 4).transpose(2, 0, 1, 3).reshape(-1, 64))
    m = n - sum(len(o) for o in out)
    k = m // 4
    scale = 10.0 ** r.uniform(-30, 30, (k, 1))
    out.append((r.standard_normal((k, S)) * scale).astype(np.float32))
    out.append(np.repeat(r.standard_normal((k, 1)) * 10.0 ** r.uniform(-8, 8, (k, 1)), S, axis=1).astype(np.float32))
    sparse = np.zeros((k, S), np.float32)
    idx = r.integers(0, S, (k, 2))
    sparse[np.arange(k), idx[:, 0]] = r.standard_normal(k)
    sparse[np.arange(k), idx[:, 1]] = -r.standard_normal(k) * 1e-3
    out.append(sparse)
    fi = np.finfo(np.float32)
    special = [0.0, -0.0, fi.smallest_subnormal, -fi.smallest_subnormal, 2.0 ** -127, 2.0 ** -126, fi.tiny,
               fi.max, -fi.max, np.inf, -np.inf, np.nan, 1.0, -1.0, 250.0, 0.5]
    spec = r.choice(np.array(special, np.float32), (m - 3 * k, S))
    spec[::3] = np.where(r.random(spec[::3].shape) < 0.9, 0.0, spec[::3])
    out.append(spec.astype(np.float32))
    return np.concatenate(out).astype(np.float32)


def oracle_encode(dims, rate, x):
    return np.concatenate([oc.encode_block(dims, rate, b) for b in x])


def oracle_decode(dims, rate, streams):
    B = oc.block_bytes(dims, rate)
    s = np.frombuffer(streams, np.uint8).reshape(-1, B)
    return np.stack([oc.decode_block(dims, rate, b) for b in s])


def random_streams(dims, rate, n, seed):
    r = np.random.default_rng(seed)
    s = r.integers(0, 256, (n, oc.block_bytes(dims, rate)), dtype=np.uint8)
    s[::4, 0] |= 1                                  # a share of headers that say "not a zero block"
    s[1::4, 1:] &= r.integers(0, 256, s[1::4, 1:].shape, dtype=np.uint8)   # sparser planes
    return s.reshape(-1).tobytes()


def bits(a):
    return np.ascontiguousarray(a, np.float32).view(np.uint32)


@pytest.mark.parametrize("rate", [8, 16])
def test_3d_coders_equal_the_oracle(host, rate):
    x = blocks(3, 1200, seed=rate)
    want_s = oracle_encode(3, rate, x)
    assert run(host, "enc3", rate, x.tobytes()) == want_s.tobytes()
    streams = want_s.tobytes() + random_streams(3, rate, 400, seed=100 + rate)
    got = np.frombuffer(run(host, "dec3", rate, streams), np.float32).reshape(-1, 64)
    want = oracle_decode(3, rate, streams)
    assert got.shape == want.shape
    assert np.array_equal(bits(got), bits(want))


@pytest.mark.parametrize("rate", [8, 16])
@pytest.mark.parametrize("dims", [2, 1])
def test_2d_and_1d_coders_equal_the_oracle(host, dims, rate):
    x = blocks(dims, 2400, seed=10 * dims + rate)
    enc = {2: "enc2", 1: "enc1"}[dims]
    dec = {2: "dec2", 1: "dec1"}[dims]
    got_s = np.frombuffer(run(host, enc, rate, x.tobytes()), np.uint8)
    want_s = oracle_encode(dims, rate, x)
    assert got_s.tobytes() == want_s.tobytes()
    streams = want_s.tobytes() + random_streams(dims, rate, 800, seed=200 + 10 * dims + rate)
    got = np.frombuffer(run(host, dec, rate, streams), np.float32).reshape(-1, 4 ** dims)
    want = oracle_decode(dims, rate, streams)
    assert np.array_equal(bits(got), bits(want))


def test_host_program_rejects_bad_input(host):
    for mode, rate, data in [("dec3", 8, b"\0" * 63), ("enc2", 16, b"\0" * 60), ("dec1", 8, b"\0" * 5),
                             ("enc3", 8, b"\0" * 255), ("enc4", 8, b""), ("dec3", 12, b"")]:
        r = subprocess.run([str(host), mode, str(rate)], input=data, capture_output=True)
        assert r.returncode == 2, (mode, rate)
