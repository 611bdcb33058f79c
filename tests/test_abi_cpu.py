"""C ABI checks that need no GPU: the library builds and loads, exports every function that
include/rfsr.h declares, its enums match the binding, and the product path never reaches the
oracle or a CPU fallback."""
import ctypes
import os
import re

import pytest

from paper_2203_09200_gb300 import build as pbuild
from paper_2203_09200_gb300 import rfsr

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rfsr.h")


@pytest.fixture(scope="module")
def lib():
    pbuild.build()
    return rfsr.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rfsr_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_serving_interface():
    names = declared_functions()
    for n in ("rfsr_create_stream", "rfsr_push_frame", "rfsr_get_frame", "rfsr_destroy"):
        assert n in names


def test_every_declared_function_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
        assert n in rfsr.SYMBOLS, f"binding lacks {n}"


def test_enums_match_binding():
    text = open(HEADER).read()

    def val(name):
        return int(re.search(rf"\b{name}\s*=\s*(-?\d+)", text).group(1))
    assert val("RFSR_EMASK") == rfsr.RFSR_EMASK
    assert val("RFSR_ETIMEDOUT") == rfsr.RFSR_ETIMEDOUT
    for k, v in rfsr.CC_MODES.items():
        assert val("RFSR_CC_" + k.upper()) == v
    assert val("RFSR_DEC_ACCEPT") == rfsr.DEC_ACCEPT
    assert val("RFSR_DBG_RMV") == rfsr.DBG_RMV


def test_struct_layouts_match_header(lib):
    # the default-config calls write through our ctypes structs: a size mismatch would show as
    # garbage in the trailing fields
    c = rfsr.rfsr_stream_config()
    lib.rfsr_stream_config_default(ctypes.byref(c))
    assert (c.height, c.width, c.num_refs, c.template_size, c.search_radius) == (720, 1280, 3, 9, 8)
    assert c.fsr_iterations == 100 and abs(c.fsr_rho - 0.7) < 1e-7 and c.keep_f32 == 0
    e = rfsr.rfsr_engine_config()
    lib.rfsr_engine_config_default(ctypes.byref(e))
    assert e.max_inflight == 4 and e.batched == 0 and e.autotune == 1


def test_struct_sizes_match_a_c_compiler(tmp_path):
    """sizeof / offsetof of every public struct as a C compiler sees the header, against ctypes."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"rfsr_engine_config": rfsr.rfsr_engine_config,
               "rfsr_stream_config": rfsr.rfsr_stream_config,
               "rfsr_stream_info": rfsr.rfsr_stream_info,
               "rfsr_batch_shape": rfsr.rfsr_batch_shape,
               "rfsr_tuning": rfsr.rfsr_tuning,
               "rfsr_state_header": rfsr.rfsr_state_header,
               "rfsr_engine_info": rfsr.rfsr_engine_info}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "rfsr.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for fname, _ in cls._fields_:
            lines.append(f'printf("{name}.{fname} %zu\\n", offsetof({name}, {fname}));')
    lines += ["return 0; }"]
    src = tmp_path / "sizes.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "sizes"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = dict(l.rsplit(" ", 1) for l in subprocess.run([str(exe)], check=True, capture_output=True,
                                                       text=True).stdout.splitlines())
    for name, cls in structs.items():
        assert int(out[name]) == ctypes.sizeof(cls), name
        for fname, _ in cls._fields_:
            assert int(out[f"{name}.{fname}"]) == getattr(cls, fname).offset, f"{name}.{fname}"


def test_errors_without_gpu_are_loud(lib):
    if os.environ.get("CUDA_VISIBLE_DEVICES", None) is None:
        try:
            import torch
            if torch.cuda.is_available():
                pytest.skip("a GPU is present")
        except ImportError:
            pass
    with pytest.raises(rfsr.RfsrError) as ei:
        rfsr.Engine()
    assert ei.value.code in (rfsr.RFSR_EDEVICE, rfsr.RFSR_EINVAL)
    assert lib.rfsr_kernel_launches() == 0


def test_null_arguments_are_einval(lib):
    assert lib.rfsr_engine_create(None, None) == rfsr.RFSR_EINVAL
    assert lib.rfsr_push_frame(None, None, None) == rfsr.RFSR_EINVAL
    assert lib.rfsr_get_frame(None, None, None, 0) == rfsr.RFSR_EINVAL
    assert lib.rfsr_destroy(None) == rfsr.RFSR_EINVAL
    assert b"NULL" in lib.rfsr_last_error()


def test_product_path_has_no_oracle_or_fallback():
    pkg = os.path.join(ROOT, "paper_2203_09200_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cpp", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f
                assert "orc_" not in src, f
    # the oracle does not import the product path either
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".py", ".c")):
            src = open(os.path.join(ROOT, "oracle", f)).read()
            assert not re.search(r"(import|from)\s+paper_2203_09200_gb300", src), f
            assert not re.search(r"#include\s+\"(rfsr\.h|rfsr_internal\.h)\"", src), f


def test_missing_library_fails_loudly(tmp_path):
    with pytest.raises(RuntimeError):
        rfsr.load.__wrapped__(str(tmp_path / "nope.so")) if hasattr(rfsr.load, "__wrapped__") \
            else _load_fresh(str(tmp_path / "nope.so"))


def _load_fresh(path):
    saved = rfsr._lib
    rfsr._lib = None
    try:
        return rfsr.load(path)
    finally:
        rfsr._lib = saved
