"""The constants of the plan kernels' block-index division (block_divisor in
csrc/zfpx_internal.h: Granlund and Montgomery's division by an invariant
integer as a multiply-high, an add and shifts), built for the host and
checked against integer division: every divisor up to 4096 with quotients
over the whole 32-bit range, block counts as plans produce them (up to
2^29 blocks along x, 2^31 - 8 rows), powers of two and their neighbours,
and the dividends next to every multiple boundary.  No GPU."""
import os
import shutil
import subprocess
from pathlib import Path

import numpy as np
import pytest

ROOT = Path(__file__).resolve().parents[1]
SRC = ROOT / "tests" / "divisor_host.cpp"
CSRC = ROOT / "paper_2609_24294_gb300" / "csrc"


def _cuda_include():
    for base in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if base and (Path(base) / "include" / "cuda_runtime.h").exists():
            return str(Path(base) / "include")
    nvcc = shutil.which("nvcc")
    if nvcc:
        inc = Path(nvcc).resolve().parents[1] / "include"
        if (inc / "cuda_runtime.h").exists():
            return str(inc)
    return None


@pytest.fixture(scope="module")
def host(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    inc = _cuda_include()
    if cxx is None or inc is None:
        pytest.skip("no C++ compiler or CUDA headers")
    exe = tmp_path_factory.mktemp("divisor_host") / "divisor_host"
    subprocess.run([cxx, "-std=c++17", "-O2", "-I", str(CSRC), "-I", inc, str(SRC), "-o", str(exe)], check=True)
    return exe


def quotients(host, d, n):
    pairs = np.stack([np.asarray(d, np.uint32), np.asarray(n, np.uint32)], axis=1)
    r = subprocess.run([str(host)], input=pairs.tobytes(), capture_output=True)
    assert r.returncode == 0
    return np.frombuffer(r.stdout, np.uint32)


def check(host, d, n):
    d = np.asarray(d, np.uint64)
    n = np.asarray(n, np.uint64)
    got = quotients(host, d, n)
    assert np.array_equal(got, (n // d).astype(np.uint32))


def test_small_divisors_whole_range(host):
    r = np.random.default_rng(3)
    d = np.repeat(np.arange(1, 4097, dtype=np.uint64), 64)
    n = r.integers(0, 1 << 32, d.size, dtype=np.uint64)
    n[::64] = 0
    n[1::64] = (1 << 32) - 1
    n[2::64] = d[2::64] - 1
    n[3::64] = d[3::64]
    check(host, d, n)


def test_plan_sized_divisors_and_boundaries(host):
    r = np.random.default_rng(4)
    ds = [2 ** k + e for k in range(1, 31) for e in (-1, 0, 1)] + [(1 << 29), (1 << 31) - 8, 40, 80, 320, 1284]
    ds += list(r.integers(1, 1 << 31, 200))
    d_all, n_all = [], []
    for d in ds:
        d = int(d)
        ks = r.integers(1, max(2, ((1 << 31) - 1) // d), 20)
        near = np.concatenate([ks * d - 1, ks * d, ks * d + 1]) if d > 1 else ks
        near = near[(near >= 0) & (near < (1 << 32))]
        d_all += [d] * len(near)
        n_all += list(near)
    check(host, d_all, n_all)
