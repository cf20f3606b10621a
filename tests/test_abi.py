"""Host-side checks of the C ABI: the library builds and loads, it exports every entry point
that include/qoc.h declares, the ctypes structures match the C layouts, and it fails loudly
(an error status, no fallback) where no GPU is present.  No kernel is launched here."""
import os
import re
import subprocess
import tempfile

import pytest

import paper_1612_04929_gb300 as qoc
from paper_1612_04929_gb300 import build as qbuild
from paper_1612_04929_gb300 import qoc as qmod

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "qoc.h")


@pytest.fixture(scope="module")
def lib():
    qbuild.build()
    return qoc.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(qoc_[a-z_]+)\s*\(", text)))


def test_header_declarations_match_binding():
    assert declared_functions() == sorted(qmod.ABI_SYMBOLS)


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", qbuild.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (qoc_\w+)", out))
    for name in declared_functions():
        assert name in exported, name
        getattr(lib, name)


def test_status_strings(lib):
    for code, name in qmod.STATUS_NAMES.items():
        assert qoc.qoc_status_string(code) == name


def test_default_options(lib):
    o = qoc.qoc_default_options()
    assert o.precision == 0 and o.tol == 0.0 and o.ckpt_stride == 0 and o.n_override == -1
    assert o.p_override == 0 and o.profile == 0 and o.stream is None and o.plain_fp32_exp == 0


def test_struct_layouts_match_c(lib):
    """Compile a tiny C program against include/qoc.h and compare sizes and offsets."""
    src = r"""
#include <stdio.h>
#include <stddef.h>
#include "qoc.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu\n", sizeof(qoc_options), offsetof(qoc_options, stream),
         offsetof(qoc_options, profile), offsetof(qoc_options, plain_fp32_exp), sizeof(qoc_info),
         offsetof(qoc_info, device_bytes));
  printf("%zu %zu %zu\n", sizeof(qoc_profile), offsetof(qoc_profile, launches), offsetof(qoc_profile, total_ms));
  return 0;
}
"""
    import ctypes as ct
    with tempfile.TemporaryDirectory() as t:
        c = os.path.join(t, "l.c")
        open(c, "w").write(src)
        exe = os.path.join(t, "l")
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        lines = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    a = [int(x) for x in lines[0].split()]
    b = [int(x) for x in lines[1].split()]
    assert a == [ct.sizeof(qmod.qoc_options), qmod.qoc_options.stream.offset, qmod.qoc_options.profile.offset,
                 qmod.qoc_options.plain_fp32_exp.offset, ct.sizeof(qmod.qoc_info), qmod.qoc_info.device_bytes.offset]
    assert b == [ct.sizeof(qmod.qoc_profile), qmod.qoc_profile.launches.offset, qmod.qoc_profile.total_ms.offset]


def _has_gpu():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.mark.skipif(_has_gpu(), reason="checks the no-GPU failure mode")
def test_create_fails_loudly_without_gpu(lib):
    with pytest.raises(qoc.QocError) as e:
        qoc.Context("fp32")
    assert e.value.status == 7


def test_missing_library_raises(tmp_path, monkeypatch):
    monkeypatch.setattr(qmod, "_lib", None)
    with pytest.raises(qoc.QocError):
        qmod.load(str(tmp_path / "absent.so"))


def test_null_context_is_rejected(lib):
    assert lib.qoc_set_system(None, 2, 0, None, None, 1.0, 1) == 1
    assert lib.qoc_evaluate_device(None, None, None, None) == 1
    lib.qoc_destroy(None)


@pytest.mark.parametrize("field,value", [("precision", 4), ("precision", -1), ("tol", -1.0), ("theta_max", -0.5),
                                         ("ckpt_stride", -2), ("wave_slices", -1), ("sweep", 3), ("gradient", 2),
                                         ("adjoint", 2), ("fault_inject", 2)])
def test_invalid_options_are_rejected_before_the_device(lib, field, value):
    """qoc_create validates every option on the host before it touches a device: an out-of-range
    value is QOC_ERR_ARG (1) on any machine, and no context is returned."""
    import ctypes as ct
    opt = qmod.qoc_options()
    lib.qoc_default_options(ct.byref(opt))
    setattr(opt, field, value)
    out = ct.c_void_p(1)
    assert lib.qoc_create(ct.byref(out), ct.byref(opt)) == 1
    assert not out.value
