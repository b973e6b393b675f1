"""The C-ABI library builds for sm_103a, loads, and exports every entry point that
include/ov.h declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

from paper_1604_08057_gb300 import binding, build

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "ov.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ov_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("ov_apply_H", "ov_tsl_sign", "ov_tsl_sign_vjp", "ov_context_create", "ov_strerror"):
        assert n in names


def test_library_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    for n in declared_functions():
        assert hasattr(lib, n), n
    assert set(declared_functions()) <= set(binding.EXPORTS)


def test_binding_fails_loudly_without_library(tmp_path):
    import pytest
    saved = binding._lib
    binding._lib = None
    try:
        with pytest.raises(RuntimeError):
            binding.load(str(tmp_path / "missing.so"))
    finally:
        binding._lib = saved


def test_strerror_without_gpu():
    lib = binding.load(build.build())
    assert lib.ov_strerror(-3).decode().startswith("Lanczos breakdown")
    assert lib.ov_strerror(0).decode() == "success"


def test_ctypes_structs_match_the_c_layout(tmp_path):
    """Sizes and field offsets of the ABI structs as gcc lays them out from ov.h
    equal those of the binding's ctypes mirrors."""
    import shutil
    import subprocess
    import pytest
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    structs = {"ov_options": binding.Options, "ov_tsl_info": binding.Info,
               "ov_tune_report": binding.TuneReport, "ov_problem": binding.Problem}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "ov.h"', "int main(void) {"]
    for cname, cls in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(line.split()[:2]): int(line.split()[2]) for line in out if line.strip()}
    for cname, cls in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert got[(cname, fname)] == getattr(cls, fname).offset, (cname, fname)


def test_nested_option_and_stage_reject_bad_arguments_without_gpu():
    """options.nested outside 0..OV_NESTED_MAX and ov_tridiag_sign_nested's size and
    pointer checks are decided on the host, before any CUDA call."""
    import numpy as np
    lib = binding.load(build.build())
    h = ctypes.c_void_p()
    for bad in (-1, 1025):
        opt = binding.Options(0, 1, 2, 0)
        opt.nested = bad
        assert lib.ov_context_create(ctypes.byref(h), ctypes.byref(opt), None) == -1
    k = 8
    a = np.ones(k, dtype=np.complex128)
    d = np.zeros(k)
    y = np.zeros(k, dtype=np.complex128)
    it = ctypes.c_int32(0)

    def call(ctx, kk, m, beta0=1.0, yp=y.ctypes.data):
        return lib.ov_tridiag_sign_nested(ctx, kk, a.ctypes.data, a.ctypes.data, d.ctypes.data, m, beta0, yp,
                                          ctypes.byref(it))
    assert call(None, k, 4) == -1                       # no context
    fake = ctypes.c_void_p(1)                           # never dereferenced: the sizes fail first
    assert call(fake, 1, 4) == -1                       # k < 2
    assert call(fake, 4097, 4) == -1                    # k > 4096
    assert call(fake, k, -1) == -1                      # m < 0
    assert call(fake, k, 1025) == -1                    # m > OV_NESTED_MAX
    assert call(fake, k, 4, float("nan")) == -1         # non-finite beta0
    assert call(fake, k, 4, 1.0, None) == -1            # no output
