"""The balanced work partition of the mixing kernels and the reduction (struct Partition),
checked on the CPU: tests/partition_check.cu compiles the library's own header and replays
how each CTA walks its units and flushes its runs into partial slots (no GPU is used).
Properties: every CTA gets U/P units to within one, every unit has exactly one owner, every
(tile, source) lands in exactly one slot of its tile, the slots of a tile follow source
order (the reduction's fixed summation order), and no run exceeds gs sources.  The second
test replays the moving-source kernel's shared-memory layout the same way."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_partition_invariants(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "partition_check")
    subprocess.run([nvcc, "-std=c++17", "-O1", "-gencode", "arch=compute_103a,code=sm_103a",
                    "-I", os.path.join(ROOT, "paper_1502_03162_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "partition_check.cu"), "-o", exe],
                   check=True, capture_output=True, text=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.startswith("ok"), r.stdout + r.stderr


def test_moving_kernel_shared_memory_layout(tmp_path):
    """The tensor-memory moving-source kernel's shared-memory layout, replayed on the CPU by
    tests/moving_layout_check.cu (which includes the kernel's source): aligned windows, table
    blocks, barriers, tap programs and accumulators for every stage count that fits, no
    overlap, within 227 KB, and at least 5 stages for every accepted tap count."""
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "moving_layout_check")
    subprocess.run([nvcc, "-std=c++17", "-O1", "--expt-relaxed-constexpr",
                    "-gencode", "arch=compute_103a,code=sm_103a",
                    "-I", os.path.join(ROOT, "paper_1502_03162_gb300", "csrc"),
                    "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "moving_layout_check.cu"), "-o", exe],
                   check=True, capture_output=True, text=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.startswith("ok"), r.stdout + r.stderr
