"""Host-side checks of the C ABI library (no GPU needed): it builds for sm_103a, loads,
exports every entry point include/phmm.h declares, and fails cleanly without a device."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2606_25738_gb300 import build
    build.build()
    from paper_2606_25738_gb300 import phmm
    return phmm


def _declared():
    src = open(os.path.join(ROOT, "include", "phmm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(phmm_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_entry_points():
    names = _declared()
    for n in ("phmm_create", "phmm_submit_batch", "phmm_poll", "phmm_destroy"):
        assert n in names


def test_exports_every_declared_symbol(lib):
    names = _declared()
    so = lib.library()
    for n in names:
        assert hasattr(so, n), n
    assert sorted(lib.SYMBOLS) == names


def test_abi_version_and_strerror(lib):
    src = open(os.path.join(ROOT, "include", "phmm.h")).read()
    ver = int(re.search(r"#define PHMM_ABI_VERSION (\d+)", src).group(1))
    so = lib.library()
    assert so.phmm_abi_version() == ver
    for code in (0, 1, -1, -2, -3, -4, -5, -6, -7):
        assert so.phmm_strerror(code)
    assert so.phmm_strerror(12345) == b"unknown status"


def test_missing_library_fails_loudly(lib, monkeypatch):
    monkeypatch.setattr(lib, "LIB_PATH", "/nonexistent/libphmm.so")
    with pytest.raises(RuntimeError):
        lib._load()


def test_create_rejects_bad_config(lib):
    import ctypes
    so = lib.library()
    h = ctypes.c_void_p()
    cfg = lib.Config(0, 7, 0, 0, 0, None, 0, 0)  # bad precision
    assert so.phmm_create(ctypes.byref(cfg), ctypes.byref(h)) == lib.PHMM_EINVAL
    cfg = lib.Config(0, 0, 0, 0, 0, None, 13, 0)  # bad columns per lane
    assert so.phmm_create(ctypes.byref(cfg), ctypes.byref(h)) == lib.PHMM_EINVAL
    cfg = lib.Config(0, 0, 0, 0, 0, None, 12, 2)  # 12 is a packed width only
    assert so.phmm_create(ctypes.byref(cfg), ctypes.byref(h)) == lib.PHMM_EINVAL
    cfg = lib.Config(0, 0, 0, 0, 0, None, 0, 7)  # bad variant
    assert so.phmm_create(ctypes.byref(cfg), ctypes.byref(h)) == lib.PHMM_EINVAL
    cfg = lib.Config(0, 0, 0, 0, 0, None, 0, 0, -1e-3)  # negative FP32 tolerance
    assert so.phmm_create(ctypes.byref(cfg), ctypes.byref(h)) == lib.PHMM_EINVAL
    cfg = lib.Config(0, 0, 0, 0, 0, None, 0, 0, float("nan"))
    assert so.phmm_create(ctypes.byref(cfg), ctypes.byref(h)) == lib.PHMM_EINVAL
    cfg = lib.Config(0, 0, 0, 0, lib.F_LONG_LEAN | lib.F_LONG_PIPE24, None, 0, 0)  # two forced kernels
    assert so.phmm_create(ctypes.byref(cfg), ctypes.byref(h)) == lib.PHMM_EINVAL
    cfg = lib.Config(0, 0, 0, 0, lib.F_LONG_SERIAL | lib.F_LONG_PIPE32, None, 0, 0)
    assert so.phmm_create(ctypes.byref(cfg), ctypes.byref(h)) == lib.PHMM_EINVAL
    cfg = lib.Config(0, 0, 0, 0, lib.F_LONG_WAVE | lib.F_LONG_WAVE16, None, 0, 0)
    assert so.phmm_create(ctypes.byref(cfg), ctypes.byref(h)) == lib.PHMM_EINVAL
    assert so.phmm_create(None, ctypes.byref(h)) == lib.PHMM_EINVAL


def test_create_without_gpu_reports_cuda_error(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(lib.PhmmError) as e:
        lib.Context()
    assert e.value.status == lib.PHMM_ECUDA


def test_null_arguments(lib):
    so = lib.library()
    import ctypes
    t = ctypes.c_uint64()
    assert so.phmm_submit_batch(None, None, ctypes.byref(t)) == lib.PHMM_EINVAL
    assert so.phmm_poll(None, 1, 0) == lib.PHMM_EINVAL
    so.phmm_destroy(None)


def test_ctypes_structs_match_header(lib, tmp_path):
    """The binding's ctypes structs have the C header's sizes and field offsets (gcc)."""
    import ctypes
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    assert lib.ABI_VERSION == lib.library().phmm_abi_version()
    pairs = [("phmm_config", lib.Config), ("phmm_batch", lib.Batch), ("phmm_stats", lib.Stats),
             ("phmm_server_config", lib.ServerConfig), ("phmm_server_stats", lib.ServerStats)]
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "phmm.h"', "int main(void) {"]
    for cname, cls in pairs:
        lines.append('printf("%%zu\\n", sizeof(%s));' % cname)
        for f, _ in cls._fields_:
            lines.append('printf("%%zu\\n", offsetof(%s, %s));' % (cname, f))
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True,
                                          check=True).stdout.split()]
    want = []
    for _, cls in pairs:
        want.append(ctypes.sizeof(cls))
        want += [getattr(cls, f).offset for f, _ in cls._fields_]
    assert got == want


def test_cpu_library_exports_its_header():
    """libphmm_cpu.so (the row-wise CPU comparator) exports what include/phmm_cpu.h declares,
    and the GPU library does not contain it (no CPU path behind the GPU ABI)."""
    import ctypes
    from paper_2606_25738_gb300 import build
    build.build()
    path = build.build_cpu()
    src = open(os.path.join(ROOT, "include", "phmm_cpu.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = sorted(set(re.findall(r"\b(phmm_[a-z_0-9]+)\s*\(", src)))
    assert names == ["phmm_cpu_forward"]
    so = ctypes.CDLL(path)
    for n in names:
        assert hasattr(so, n), n
    gpu = ctypes.CDLL(build.LIB)
    assert not hasattr(gpu, "phmm_cpu_forward")
