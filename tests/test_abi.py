"""The C ABI library builds, loads and exports every symbol dc.h declares
(CPU only: no compute calls)."""

import ctypes
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def declared_functions():
    names = []
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^DC_API\s+[\w\s\*]*?\b(\w+)\s*\(", text, flags=re.M)
    return names


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("no nvcc to build the library")
    from paper_2508_04951_gb300 import build
    path = build.build()
    return path


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("doppler_resample", "iono_correct", "correct_batch", "correct_bank",
                     "resample_exact_batch", "dc_create", "dc_destroy", "dc_check"):
        assert required in names


def c_layout(exprs):
    """Evaluate sizeof / offsetof expressions over include/dc.h with the host C
    compiler."""
    import tempfile
    hdr = os.path.join(ROOT, "include")
    body = "".join(f'  printf("%zu\\n", (size_t)({e}));\n' for e in exprs)
    src = f"#include <stdio.h>\n#include <stddef.h>\n#include \"dc.h\"\nint main(void) {{\n{body}  return 0;\n}}\n"
    with tempfile.TemporaryDirectory() as d:
        c, exe = os.path.join(d, "t.c"), os.path.join(d, "t")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-I", hdr, c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    return [int(v) for v in out.split()]


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    declared = set(declared_functions())
    assert declared <= exported, declared - exported
    # nothing else leaks out of the C ABI
    assert exported <= declared, exported - declared
    handle = ctypes.CDLL(lib)
    for name in declared:
        assert getattr(handle, name) is not None


def test_binding_names_match_header(lib):
    import paper_2508_04951_gb300 as dcg
    assert set(dcg.exported_symbols()) <= set(declared_functions())
    dcg.load()
    o = dcg.dc_opts_default()
    assert (o.taps, o.kaiser_beta, o.mode, o.n_out, o.carrier_shift, o.freq_ref) == (32, 8.0, 0, 0, 0, 0.0)
    assert dcg.ITEM_DTYPE.itemsize == 64
    # the binding's struct layouts are the header's, as a C compiler lays them out
    sizes = c_layout(["sizeof(dc_opts)", "sizeof(dc_item)", "offsetof(dc_opts, freq_ref)",
                      "offsetof(dc_opts, carrier_shift)"])
    assert sizes == [ctypes.sizeof(dcg.DcOpts), dcg.ITEM_DTYPE.itemsize, dcg.DcOpts.freq_ref.offset,
                     dcg.DcOpts.carrier_shift.offset]


def test_status_strings(lib):
    import paper_2508_04951_gb300 as dcg
    L = dcg.load()
    assert L.dc_status_str(0) == b"DC_OK"
    assert L.dc_status_str(5) == b"DC_ETIMEOUT"


def test_create_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_2508_04951_gb300 as dcg
    with pytest.raises(dcg.DcError):
        dcg.Context(0)
