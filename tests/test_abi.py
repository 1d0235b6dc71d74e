"""The C-ABI library loads and exports every symbol include/hrir.h declares (no GPU needed;
no compute call is made)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hrir.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hrir_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1502_03162_gb300 import build, hrir
    build.build()
    return hrir.load_library()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("hrir_load_filters", "hrir_render_batch", "hrir_create", "hrir_sync"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1502_03162_gb300 import hrir
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} not exported by libhrir.so"
        assert name in hrir.SIGNATURES, f"{name} has no Python binding"


def test_version_and_cpu_only_create_fails_cleanly(lib):
    from paper_1502_03162_gb300 import hrir
    assert hrir.hrir_version() >= 1
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(hrir.HRIRError) as ei:
        hrir.hrir_create(0)
    assert ei.value.status == hrir.HRIR_ECUDA


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_1502_03162_gb300 import hrir
    import importlib
    mod = importlib.reload(hrir)
    saved = mod._lib
    try:
        mod._lib = None
        with pytest.raises(RuntimeError):
            mod.load_library(str(tmp_path / "missing.so"))
    finally:
        mod._lib = saved


def test_every_declared_function_is_documented():
    # each declaration in the header sits below a comment block that documents it (the
    # block may document a group of related calls declared together)
    lines = open(HEADER).read().splitlines()
    decl = re.compile(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(hrir_[a-z0-9_]+)\s*\(")
    for i, ln in enumerate(lines):
        m = decl.match(ln)
        if not m:
            continue
        j = i - 1
        # skip continuation lines, neighbouring declarations and a typedef the block also
        # documents (the kernel-family enum of the timing calls)
        while j >= 0 and not lines[j].rstrip().endswith("*/") and (
                decl.match(lines[j]) or lines[j].startswith((" ", "\t", "typedef", "}"))
                or (lines[j].strip() == "" and j > 0 and lines[j - 1].startswith("}"))):
            j -= 1
        assert j >= 0 and lines[j].rstrip().endswith("*/"), f"{m.group(1)} has no doc comment"
