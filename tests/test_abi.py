"""The C-ABI library loads and exports every entry point of include/bsf.h.

CPU only: no compute call is made; host-only entry points (defaults,
buffer sizes, status strings, argument validation) are exercised.
"""
import os
import re

import numpy as np

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "bsf.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(bsf_[a-z_0-9]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_1003_2022_gb300 import build
    build.build()
    from paper_1003_2022_gb300 import _lib
    return _lib


def test_every_declared_symbol_is_exported(lib):
    so = lib.load()
    names = _declared()
    assert len(names) >= 10
    for n in names:
        assert hasattr(so, n), n
    assert sorted(lib.EXPORTS) == names


def test_host_only_calls(lib):
    o = lib.default_opts()
    assert o.precision == lib.BSF_PREC_EXACT and abs(o.eps - 1e-3) < 1e-9 and o.halo == 0
    assert lib.bsf_buffer_bytes(lib.BSF_U8, 10, 20, 4, 3, lib.BSF_PREC_EXACT) == 16 * 26 * 8
    assert lib.bsf_buffer_bytes(lib.BSF_F32, 10, 20, 4, 3, lib.BSF_PREC_EXACT) == 16 * 26 * 16
    assert lib.bsf_buffer_bytes(lib.BSF_F32, 10, 20, 4, 3, lib.BSF_PREC_FP64) == 16 * 26 * 8
    with pytest.raises(lib.BsfError) as e:
        lib.bsf_buffer_bytes(lib.BSF_U8, 10, 20, 6, 3, lib.BSF_PREC_EXACT)
    assert e.value.code == lib.BSF_EUNSUPPORTED
    with pytest.raises(lib.BsfError):
        lib.bsf_buffer_bytes(lib.BSF_U8, 0, 20, 4, 3, lib.BSF_PREC_EXACT)
    for code in range(0, 11):
        assert lib.status_string(code) not in ("", "unknown status")
    # null context and null pointers are rejected before any CUDA call
    assert lib.bsf_filter(None, 0, 0, 1, 1, 8, 8, 4, 0, 0, None, 0, 0) == lib.BSF_EINVAL
    assert lib.bsf_scales_from_cov(None, 0, 2, 10, 4, None, 0, 0, 0) == lib.BSF_EINVAL
    assert lib.bsf_filter_host(None, 0, 0, 1, 1, 8, 8, 4, 0, 0, None, 0) == lib.BSF_EINVAL
    assert lib.bsf_host_sync(None) == lib.BSF_EINVAL


def test_python_binding_refuses_to_run_without_library(tmp_path, lib):
    import importlib
    mod = importlib.import_module("paper_1003_2022_gb300._lib")
    saved = mod._lib
    try:
        mod._lib = None
        with pytest.raises(RuntimeError):
            mod.load(str(tmp_path / "missing.so"))
    finally:
        mod._lib = saved


def test_halo_bounds_rejected_before_any_device_call(lib):
    """A halo beyond the library's bound, or an image whose buffer exceeds the
    fixed scratch of the allocation-free entry point, is an argument error
    returned on the host: nothing is planned or launched (a huge halo once
    overflowed the padded size and divided by zero in the scan planner)."""
    o = lib.default_opts()
    o.halo = 2 ** 31 - 1
    dummy = 16  # non-null pointers that are never dereferenced
    assert lib.bsf_filter_noalloc(dummy, lib.BSF_U8, 2, 2, 4, dummy, lib.BSF_PARAM_SCALES, o, dummy, 0) \
        == lib.BSF_EINVAL
    o.halo = 1 << 20
    assert lib.bsf_filter_noalloc(dummy, lib.BSF_U8, 1 << 20, 1 << 20, 4, dummy, lib.BSF_PARAM_SCALES, o, dummy,
                                  0) == lib.BSF_ENOSCRATCH
    o.halo = 4
    assert lib.bsf_filter_noalloc(dummy, lib.BSF_F32, 4096, 4096, 4, dummy, lib.BSF_PARAM_SCALES, o, dummy, 0) \
        == lib.BSF_ENOSCRATCH
    with pytest.raises(lib.BsfError) as e:
        lib.bsf_buffer_bytes(lib.BSF_U8, 10, 20, 4, (1 << 20) + 1, lib.BSF_PREC_EXACT)
    assert e.value.code == lib.BSF_EINVAL
    assert lib.bsf_buffer_bytes(lib.BSF_U8, 1 << 20, 1 << 20, 4, 1 << 20, lib.BSF_PREC_EXACT) \
        == (3 << 20) * (3 << 20) * 8


def test_query_workspace_host_only(lib):
    """bsf_query_workspace needs no context and no device: the N=4 figure is the
    pre-integrated buffers of one launch plus the scan carries; N=6 a bound."""
    o = lib.default_opts()
    o.max_scale = 32.0
    n4 = lib.bsf_query_workspace(None, lib.BSF_U8, 1, 1, 2048, 2048, 4, lib.BSF_PARAM_SRT, o)
    P = int(np.ceil(0.5 * 8.364 * 32)) + 4
    Lp = 2048 + 2 * P
    buf = Lp * Lp * 8
    carries = 10 * (-(-Lp // 8)) * Lp * 8  # ten carry rows per band, bands of at least 8 rows
    assert buf <= n4 <= buf + carries
    n4f = lib.bsf_query_workspace(None, lib.BSF_F32, 1, 1, 2048, 2048, 4, lib.BSF_PARAM_SRT, o)
    assert n4f > 1.9 * buf  # 16-byte elements
    o.iterations = 2
    assert lib.bsf_query_workspace(None, lib.BSF_U8, 1, 1, 2048, 2048, 4, lib.BSF_PARAM_SRT, o) == n4 + 2048 * 2048 * 4
    o.iterations = 1
    o.max_scale = 48.0
    n6 = lib.bsf_query_workspace(None, lib.BSF_F32, 4, 3, 4096, 4096, 6, lib.BSF_PARAM_SRT, o)
    assert n6 >= 4 * 6 * 4096 * 4096 * 8
    o.max_scale = 0.0
    with pytest.raises(lib.BsfError) as e:
        lib.bsf_query_workspace(None, lib.BSF_U8, 1, 1, 64, 64, 4, lib.BSF_PARAM_SRT, o)
    assert e.value.code == lib.BSF_EINVAL
    o.halo = 20
    assert lib.bsf_query_workspace(None, lib.BSF_U8, 1, 1, 64, 64, 4, lib.BSF_PARAM_SRT, o) >= 104 * 104 * 8
    with pytest.raises(lib.BsfError) as e:
        lib.bsf_query_workspace(None, lib.BSF_U8, 1, 1, 64, 64, 5, lib.BSF_PARAM_SRT, o)
    assert e.value.code == lib.BSF_EUNSUPPORTED


def test_opts_layout_matches_the_header(lib, tmp_path):
    """The ctypes bsf_opts has the C struct's size and field offsets (compiled
    from include/bsf.h with the host compiler), and the defaults of the
    optional modes are off."""
    import ctypes
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("needs a C compiler")
    fields = [f[0] for f in lib.bsf_opts._fields_]
    src = tmp_path / "layout.c"
    body = "\n".join(f'    printf("{n} %zu\\n", offsetof(bsf_opts, {n}));' for n in fields)
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "bsf.h"\nint main(void) {\n'
                   '    printf("sizeof %zu\\n", sizeof(bsf_opts));\n' + body + "\n    return 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True,
                   capture_output=True)
    out = dict(line.split() for line in subprocess.run([str(exe)], check=True, capture_output=True,
                                                       text=True).stdout.split("\n") if line)
    assert int(out["sizeof"]) == ctypes.sizeof(lib.bsf_opts)
    for n in fields:
        assert int(out[n]) == getattr(lib.bsf_opts, n).offset, n
    o = lib.default_opts()
    assert o.map_lut == 0 and o.staging == lib.BSF_STAGING_L1 and o.boundary == lib.BSF_BOUNDARY_ZERO
