"""The C-ABI library builds for sm_103a, loads, and exports every entry point
include/dnnmg.h declares (no GPU needed: no compute calls)."""
import os
import re

import pytest

from paper_2307_14837_gb300 import build, capi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "dnnmg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dnnmg_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return capi.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_binding_names_match_header():
    assert sorted(capi.exported_symbols()) == _declared()


def test_status_strings(lib):
    assert capi.load().dnnmg_strerror(0) == b"ok"
    assert capi.load().dnnmg_strerror(-1) == b"invalid argument"
    assert capi.load().dnnmg_strerror(-99) == b"unknown status"


def test_create_rejects_bad_arguments_without_a_gpu(lib):
    # argument validation happens before any CUDA call
    mesh = dict(xyz=[[0.0, 0, 0]], cells=[[0, 0, 0, 0, 0, 0, 0, 0]], vertex_bc=[0])
    with pytest.raises(capi.DnnmgError) as e:
        capi.dnnmg_create(mesh, 0.01, 0.01, 1.0, capi.FP64)
    assert e.value.status == -1
    with pytest.raises(capi.DnnmgError):
        capi.dnnmg_create(mesh, 0.01, -1.0, 1.0, capi.FP64)     # dt <= 0



def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    # no CPU fallback: without the built library the binding raises
    monkeypatch.setattr(capi, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        capi.load(str(tmp_path / "libdnnmg.so"))


def test_product_package_does_not_import_the_oracle():
    # the oracle is test infrastructure: no module of the package imports it
    pkg = os.path.join(ROOT, "paper_2307_14837_gb300")
    for name in os.listdir(pkg):
        if name.endswith(".py"):
            src = open(os.path.join(pkg, name)).read()
            assert not re.search(r"^\s*(from|import)\s+oracle\b", src, flags=re.M), name


def test_build_targets_sm103a_only():
    assert build.ARCH_FLAGS == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_noalloc_limit_matches_header():
    src = open(os.path.join(ROOT, "include", "dnnmg.h")).read()
    m = re.search(r"#define\s+DNNMG_NOALLOC_MAX_PATCHES\s+(\d+)", src)
    assert m and int(m.group(1)) == capi.NOALLOC_MAX_PATCHES


def test_training_data_calls_reject_bad_arguments_without_a_gpu(lib):
    # argument checks come before any CUDA call: EINVAL (-1) on the CPU
    L = capi.load()
    fake = 4096                                   # never dereferenced on these paths
    FP32, BF16 = capi.FP32, capi.BF16
    assert L.dnnmg_column_stats(None, FP32, 10, 4, 4, fake, fake, None) == -1
    assert L.dnnmg_column_stats(fake, FP32, 1, 4, 4, fake, fake, None) == -1     # rows < 2
    assert L.dnnmg_column_stats(fake, FP32, 10, 8, 4, fake, fake, None) == -1    # ld < cols
    assert L.dnnmg_column_stats(fake, 7, 10, 4, 4, fake, fake, None) == -1       # unknown dtype
    assert L.dnnmg_standardize(fake, BF16, 10, 0, 4, fake, fake, fake, None) == -1
    assert L.dnnmg_standardize(fake, BF16, 0, 4, 4, fake, fake, fake, None) == 0  # nothing to do
    assert L.dnnmg_gather_rows(fake, 10, 0, fake, 5, fake, None) == -1           # row_bytes
    assert L.dnnmg_gather_rows(fake, 10, 16, fake, 0, fake, None) == 0
    assert L.dnnmg_add_noise(None, BF16, 10, 0, 4, 8, 0.1, 1, None) == -1
    assert L.dnnmg_add_noise(fake, BF16, 10, 4, 2, 8, 0.1, 1, None) == -1        # c1 < c0
    assert L.dnnmg_add_noise(fake, BF16, 10, 0, 9, 8, 0.1, 1, None) == -1        # c1 > ld
    assert L.dnnmg_add_noise(fake, BF16, 10, 0, 4, 8, -0.1, 1, None) == -1       # sigma < 0
    assert L.dnnmg_add_noise(fake, BF16, 10, 0, 4, 8, 0.0, 1, None) == 0         # no noise: no launch
    assert L.dnnmg_patch_targets(None, fake, fake, fake, 81) == -1
