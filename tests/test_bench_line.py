"""The benchmark's last stdout line: one JSON object, short enough for a reader that
keeps only the tail of the output, holding the headline keys; the full record goes
to a side file."""
import json
import os

import bench


def _fake_line():
    kern = {n: {"ms": 0.4123456, "algorithmic_bytes": 711_111_111, "GBps": 1479.123456,
                "f32_GBps": 1100.5, "frac_of_measured_hbm": 0.2181234}
            for n in ("compress_r8", "permute_r8", "decompress_r8",
                      "compress_r16", "permute_r16", "decompress_r16")}
    return {
        "metric": bench.METRIC, "value": 983.123456789, "unit": "GB/s", "n_gpus": 1, "steps": 20,
        "warmup": 3, "ms_per_step": 1.8341234, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": bench.WORKLOAD, "l2": "inputs larger than L2", "ranks": "8x8",
                   "rates": [8, 16], "parallelism": "independent field per GPU"},
        "roofline": {"bound": "hbm", "kernel": "compress_r16", "achieved": 1479.1234, "peak": 6685.8,
                     "peak_kind": "measured", "unit": "GB/s", "frac": 0.2212345, "traffic": 674_500_000,
                     "source_sha": "0123456789abcdef",
                     "limiter": {"unit": "alu pipe (integer)", "alu_pct_of_peak": 63.9,
                                 "issue_slots_pct": 62.3, "dram_pct_of_peak": 17.8,
                                 "source": "ncu --set full, profiles/codec_kernels_1280x640x137.md"}},
        "cpu_baseline": {"value": 0.9012345, "unit": "GB/s", "cores": 16, "kind": "oracle",
                         "sample": "512 of 512 messages of this plan, each through r8 and r16 "
                                   "compress+decompress (1.8 s on 16 threads)",
                         "single_thread": {"value": 0.06, "unit": "GB/s", "sample": "40 messages in 3.0 s"}},
        "e2e": {"value": 354.1234, "unit": "GB/s", "h2d_bytes_per_step": 449_000_000,
                "d2h_bytes_per_step": 898_000_000},
        "gpu_launches": 120,
        "clocks": {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 30},
        "kernels": kern,
    }


def test_headline_is_short_and_parses(tmp_path, capsys):
    line = _fake_line()
    detail = dict(line, extras={"big": ["x" * 100] * 400}, error={}, comparators={})
    path = str(tmp_path / "detail.json")
    bench.emit(line, detail, path)
    out = capsys.readouterr().out.strip().splitlines()
    last = out[-1]
    assert len(last.encode()) <= bench.HEADLINE_MAX_BYTES
    d = json.loads(last)
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e", "clocks",
              "gpu_launches"):
        assert k in d, k
    assert d["value"] > 0 and d["roofline"]["frac"] > 0
    assert set(d["kernels"]) == set(line["kernels"])
    assert "extras" not in d and d["detail_file"] == path
    full = json.load(open(path))
    assert len(full["extras"]["big"]) == 400
    assert os.path.getsize(path) > len(last)


def test_headline_drops_detail_before_exceeding_limit():
    line = _fake_line()
    line["config"]["workload"] = "w" * 3000
    s = bench.headline(line, "d.json")
    d = json.loads(s)
    assert "kernels" not in d and d["value"] > 0
