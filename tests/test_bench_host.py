"""Host-side logic of bench.py that needs no GPU: the clock sampler (against a fake
nvidia-smi) and the rule that DRAM traffic is reported only from a profile taken on the
current kernel source."""
import hashlib
import os
import stat
import sys
import time

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _fake_smi(tmp_path, line):
    d = tmp_path / "bin"
    d.mkdir()
    p = d / "nvidia-smi"
    p.write_text("#!/bin/sh\nwhile true; do echo \"%s\"; sleep 0.02; done\n" % line)
    p.chmod(p.stat().st_mode | stat.S_IEXEC)
    return str(d) + os.pathsep + os.environ.get("PATH", "")   # the fake first; `sleep` still found


def test_clock_sampler_reads_clocks_and_reasons(tmp_path, monkeypatch):
    line = "0, 2070, 2070, 950.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active"
    monkeypatch.setenv("PATH", _fake_smi(tmp_path, line))
    with bench.ClockSampler(0, period_ms=20) as c:
        time.sleep(0.05)              # a warm-up: its samples are not summarised
        c.mark()
        time.sleep(0.1)
    s = c.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]
    assert s["samples"] >= 2
    assert len(c.lines) > s["samples"]


def test_clock_sampler_short_region_still_sampled(tmp_path, monkeypatch):
    line = "0, 1980, 2070, 1200.0, 0x0, Active, Not Active, Not Active, Not Active"
    monkeypatch.setenv("PATH", _fake_smi(tmp_path, line))
    with bench.ClockSampler(0, period_ms=20) as c:
        pass                          # a region far shorter than the sampling period
    s = c.summary()
    assert s["samples"] >= 1 and s["sm_mhz"] == 1980.0
    assert s["reasons"] == ["hw_slowdown"]


def test_clock_sampler_without_nvidia_smi(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))
    with bench.ClockSampler(0) as c:
        pass
    assert c.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}


def test_committed_profile_matches_committed_kernel():
    # the headline kernel's ncu summary was taken on the source in the tree
    t = bench.profiled_traffic("mix_sparse_tmem.cu", "mix_sparse_batched_1024x480000_k16.md")
    assert t == pytest.approx(2.0290e9)


def test_traffic_withheld_when_kernel_changed(tmp_path, monkeypatch):
    (tmp_path / "profiles").mkdir()
    csrc = tmp_path / "paper_1502_03162_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "k.cu").write_text("// kernel v1\n")
    sha = hashlib.sha256(b"// kernel v1\n").hexdigest()
    (tmp_path / "profiles" / "k.md").write_text(
        f"kernel_source_sha256: {sha}\ndram_bytes_per_launch_full_size: 1.5e+09\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profiled_traffic("k.cu", "k.md") == pytest.approx(1.5e9)
    (csrc / "k.cu").write_text("// kernel v2\n")
    assert bench.profiled_traffic("k.cu", "k.md") is None
    assert bench.profiled_traffic("k.cu", "missing.md") is None


def test_profile_summaries_run_committed_files_only():
    import re
    prof = os.path.join(ROOT, "profiles")
    names = [f for f in os.listdir(prof) if f.endswith((".md", ".txt"))]
    assert names
    for f in names:
        text = open(os.path.join(prof, f)).read()
        scripts = re.findall(r"python3?\s+(?:-m\s+)?(\S+\.py)", text)
        assert scripts, f"{f}: no command"
        for s in scripts:
            assert os.path.isfile(os.path.join(ROOT, s)), f"{f}: {s} is not in the repository"
            assert not s.startswith("_work"), f"{f}: {s} is a working file"
        assert "--clock-control none" in text or "ncu" not in text, f"{f}: ncu without clock control"


def test_sliced_oracle_sums_slices_to_the_whole_mix():
    """The all-core CPU baseline (and the full-size parity test) split the sources into one
    slice per spawned worker and sum the slices' mixes in FP64: by linearity (Eq. 2 summed
    over sources) that is the oracle's mix of all sources, up to the order of the FP64 sums."""
    import oracle
    from oracle.pool import SlicedRenderer
    from paper_1502_03162_gb300 import synth
    rng = np.random.default_rng(4)
    S, L = 7, 3001
    cfg = synth.batched_config(S=S, L=L, seed=4, n_dirs=20)
    idx, w, nnz = oracle.topk(cfg["G"], 16)
    tm = SlicedRenderer(cfg["y"], cfg["dirs"], idx, w, nnz, 200, cfg["res"], cores=3)
    try:
        for mode, fn in (("sparse", oracle.render_sparse), ("dense", oracle.render_dense),
                         ("fft", oracle.render_fft)):
            dt, out = tm.run(S, L, mode)
            ref = fn(cfg["y"], cfg["dirs"], idx, w, nnz, 200, cfg["res"], length=L)
            assert dt > 0 and out.shape == ref.shape
            np.testing.assert_allclose(out, ref, rtol=0, atol=1e-12 * np.abs(ref).max())
        dt, out = tm.run(4, L, "sparse", workers=1)
        ref = oracle.render_sparse(cfg["y"][:4], cfg["dirs"][:4], idx, w, nnz, 200, cfg["res"])
        np.testing.assert_allclose(out, ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    finally:
        tm.close()
    del rng


def test_fft_flop_count_of_the_built_design():
    """Per source-ear sample: a 4096-point complex FFT (5 P log2 P flops) per source pair and
    frame shared by 2 sources x 2 ears, 8 flops per bin and ear, inverse FFTs shared by all
    sources; hop 4096 - 232 for a 231-tap HRIR."""
    import bench
    B = 4096 - 232
    want = 5 * 4096 * 12 / (4 * B) + 8 * 2049 / B + 5 * 4096 * 12 / (1024 * B)
    assert abs(bench.fft_flops_per_unit(1024) - want) < 1e-12
    assert 20.0 < bench.fft_flops_per_unit(1024) < 20.4
