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
  printf("%zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(qoc_options), offsetof(qoc_options, stream),
         offsetof(qoc_options, profile), offsetof(qoc_options, plain_fp32_exp), sizeof(qoc_info),
         offsetof(qoc_info, device_bytes), offsetof(qoc_options, taylor_scheme), offsetof(qoc_info, taylor_scheme));
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
                 qmod.qoc_options.plain_fp32_exp.offset, ct.sizeof(qmod.qoc_info), qmod.qoc_info.device_bytes.offset,
                 qmod.qoc_options.taylor_scheme.offset, qmod.qoc_info.taylor_scheme.offset]
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


def test_reversal_needs_the_fp64_form(lib):
    """Reversal regenerates states through the stored propagators: the FP32 forms refuse it on
    the host (QOC_ERR_UNSUPPORTED) before touching a device."""
    import ctypes as ct
    opt = qmod.qoc_options()
    lib.qoc_default_options(ct.byref(opt))
    opt.precision, opt.reversal = 1, 1
    out = ct.c_void_p(1)
    assert lib.qoc_create(ct.byref(out), ct.byref(opt)) == 9
    assert not out.value


@pytest.mark.parametrize("field,value", [("precision", 4), ("precision", -1), ("tol", -1.0), ("theta_max", -0.5),
                                         ("ckpt_stride", -2), ("wave_slices", -1), ("sweep", 3), ("gradient", 2),
                                         ("adjoint", 2), ("fault_inject", 2), ("reversal", 2),
                                         ("propagation", 2), ("propagation", -1), ("exponential", 2),
                                         ("taylor_scheme", 2), ("taylor_scheme", -1), ("autotune", 2),
                                         ("autotune", -1)])
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


# ------------------------------------------------------------------ allocation-free entry point
ARENA_BYTES = 32 << 20
PARAM_BLOCK_BYTES = 1072     # the device parameter block at the start of the array


def static_arena_bytes(d, M, N, S):
    """The fixed array's use by qoc_evaluate_static, as include/qoc.h states it: every piece
    starts on a 256-byte boundary; U_j and U_j^dag take 2 ceil16(d^2) complex128 numbers per
    slice, the d x S blocks are padded to Spad columns (panels of min(S, 8) columns)."""
    cb = min(S, 8)
    spad = -(-S // cb) * cb
    blk = d * spad
    d2 = -(-d * d // 16) * 16
    pieces = [PARAM_BLOCK_BYTES, 8 * (M + 2), 16 * blk, 16 * blk, 16 * N * 2 * d2, 16 * (N + 1) * blk,
              16 * N * blk, 16 * N * blk, 16 * blk, 16 * N, 8 * N, 16, 8 * (M * N + 1), 8 * spad, 4 * d]
    used = 0
    for p in pieces:
        used = -(-used // 256) * 256 + p
    return used


def static_n_max(d, M, S):
    lo, hi = 1, 1 << 22
    while lo < hi:
        mid = (lo + hi + 1) // 2
        if static_arena_bytes(d, M, mid, S) <= ARENA_BYTES:
            lo = mid
        else:
            hi = mid - 1
    return lo


STATIC_SHAPES = [(48, 2, 1), (48, 3, 8), (44, 2, 41), (8, 3, 3), (1, 0, 1), (30, 64, 30)]


def _static_status(lib, d, M, N, S):
    import ctypes as ct
    alpha = (ct.c_double * 5)(1, 0, 0, 0, 0)
    fake = ct.c_void_p(16)   # never dereferenced: these calls return before any device work
    return lib.qoc_evaluate_static(d, M, N, S, ct.c_double(0.1), fake, fake, fake, fake, fake, None, alpha,
                                   fake, fake, None)


@pytest.mark.parametrize("shape", STATIC_SHAPES, ids=lambda s: "d%dM%dS%d" % s)
def test_static_arena_rejects_one_slice_past_the_stated_bound(lib, shape):
    """The size check comes before any CUDA call: one slice beyond the bound that the header
    states is QOC_ERR_SHAPE on any machine (the GPU test runs the largest admitted N)."""
    d, M, S = shape
    n = static_n_max(d, M, S)
    assert _static_status(lib, d, M, n + 1, S) == 2
    assert _static_status(lib, d, M, 10 * n, S) == 2


@pytest.mark.skipif(_has_gpu(), reason="the admitted size would run kernels on a GPU")
@pytest.mark.parametrize("shape", STATIC_SHAPES, ids=lambda s: "d%dM%dS%d" % s)
def test_static_arena_admits_the_stated_bound_without_gpu(lib, shape):
    """Up to the stated bound the size check passes, and without a GPU the call then fails
    loudly at its first CUDA call (QOC_ERR_CUDA), with no fallback."""
    d, M, S = shape
    assert _static_status(lib, d, M, static_n_max(d, M, S), S) == 7
