"""The C-ABI library builds, loads without a GPU and exports what the header declares.

No compute call is made here: these run on machines without a GPU.
"""

import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gravdenoise.h")


@pytest.fixture(scope="module")
def native():
    from paper_2512_10386_gb300 import build as nb
    nb.build()
    from paper_2512_10386_gb300 import _native
    return _native


def _declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|size_t|const char \*)\s*(denoise_\w+)\s*\(", text, re.M)))


def test_header_declares_the_binding_names(native):
    assert _declared() == sorted(native.EXPORTED)


def test_library_exports_every_declared_symbol(native):
    L = native.lib()
    for name in _declared():
        assert hasattr(L, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", native.LIB_PATH], capture_output=True, text=True).stdout
    for name in _declared():
        assert re.search(rf"\bT {name}$", out, re.M), name


def test_strerror_is_callable_without_gpu(native):
    assert native.strerror(0) == "ok"
    assert "NaN" in native.strerror(native.DENOISE_E_NONFINITE)
    assert native.strerror(12345) == "unknown status"


def test_ctypes_structs_match_c_layout(native, tmp_path):
    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "gravdenoise.h"\n'
                   'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu\\n", sizeof(denoise_params), sizeof(denoise_stats),'
                   ' sizeof(denoise_debug), offsetof(denoise_params, temperature), offsetof(denoise_stats, stage_ms),'
                   ' sizeof(denoise_tuning), offsetof(denoise_tuning, leaf_threads));'
                   'return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    want = [ctypes.sizeof(native.denoise_params), ctypes.sizeof(native.denoise_stats),
            ctypes.sizeof(native.denoise_debug), native.denoise_params.temperature.offset,
            native.denoise_stats.stage_ms.offset, ctypes.sizeof(native.denoise_tuning),
            native.denoise_tuning.leaf_threads.offset]
    assert got == want


def test_create_without_gpu_fails_cleanly(native):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    st = native.lib().denoise_create(ctypes.byref(h), 0, 1000, 1)
    assert st == native.DENOISE_E_CUDA and not h.value


def test_package_has_no_cpu_fallback(native):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2512_10386_gb300 import Denoiser
    with pytest.raises(RuntimeError):
        Denoiser(max_points=10)


def test_noalloc_scratch_size_matches_the_header(native):
    """The no-allocation entry point's static scratch covers the leaf kernel's
    spill stride (the query returns 0 otherwise) and has the documented size."""
    import re
    hdr = open(os.path.join(ROOT, "include", "gravdenoise.h")).read()
    documented = {int(v.replace(",", "")) for v in re.findall(r"\(([0-9,]+) bytes per GPU", hdr)}
    documented |= {int(v.replace(",", "")) for v in re.findall(r"scratch array \(([0-9,]+)\)", hdr)}
    got = native.denoise_noalloc_scratch_bytes()
    assert got > 0
    assert documented == {got}
