"""The C-ABI library builds for sm_103a, loads, and exports every entry point
include/rad.h, rad_mlp.h and rad_pic.h declare (no compute calls: this runs
without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols(header="rad.h"):
    txt = open(os.path.join(ROOT, "include", header)).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(rad_[a-z_0-9]+)\s*\(", txt)))


def test_header_declares_the_binding_names():
    from paper_1003_1140_gb300 import rad
    assert sorted(rad.EXPORTED) == declared_symbols()


def test_library_builds_loads_and_exports_everything():
    from paper_1003_1140_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    for header in ("rad.h", "rad_mlp.h", "rad_pic.h"):
        for name in declared_symbols(header):
            assert hasattr(lib, name), name


def test_mlp_header_declares_the_binding_names():
    from paper_1003_1140_gb300 import mlp
    assert sorted(mlp.EXPORTED) == declared_symbols("rad_mlp.h")


def test_pic_header_declares_the_binding_names():
    from paper_1003_1140_gb300 import pic
    assert sorted(pic.EXPORTED) == declared_symbols("rad_pic.h")


def test_null_context_calls_fail_cleanly():
    from paper_1003_1140_gb300 import build
    lib = ctypes.CDLL(build.build())
    lib.rad_last_error.restype = ctypes.c_char_p
    lib.rad_last_error.argtypes = [ctypes.c_void_p]
    lib.rad_spectrum_size.restype = ctypes.c_int64
    lib.rad_spectrum_size.argtypes = [ctypes.c_void_p]
    lib.rad_finalize.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    lib.rad_reset.argtypes = [ctypes.c_void_p]
    lib.rad_destroy.argtypes = [ctypes.c_void_p]
    assert lib.rad_last_error(None) == b"null context"
    assert lib.rad_spectrum_size(None) == -1
    assert lib.rad_finalize(None, None) == -1
    assert lib.rad_reset(None) == -1
    lib.rad_destroy(None)


def test_rad_init_rejects_null_out_pointer():
    from paper_1003_1140_gb300 import build
    lib = ctypes.CDLL(build.build())
    lib.rad_init.restype = ctypes.c_int
    assert lib.rad_init(None, None, 0, None, None, 0, ctypes.c_double(0.0), None, 0, None, 0,
                        0, 0, ctypes.c_double(0.0), None) == -1


def test_fault_hook_tokens_are_checked_before_any_device_call(monkeypatch):
    """RAD_FAULT is parsed at rad_init before the device is touched: an unknown
    token or a malformed step number is RAD_EINVAL on any machine."""
    import numpy as np
    from paper_1003_1140_gb300 import rad as R
    args = (np.array([[0.0, 1.0, 0.0]]), [np.linspace(1.0, 2.0, 4)], 0.1, [(8, -1.0)],
            [(0, 4, 1, 0)])
    for bad in ("explode", "stall,step:", "step:-2", "step:3x", "alloc, graph"):
        monkeypatch.setenv("RAD_FAULT", bad)
        with pytest.raises(R.RadError) as ei:
            R.Radiation(*args)
        assert ei.value.code == -1, bad
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        # accepted tokens get past the parse and stop at the device query
        monkeypatch.setenv("RAD_FAULT", "alloc,graph,stall,step:3,")
        with pytest.raises(R.RadError) as ei:
            R.Radiation(*args)
        assert ei.value.code == -3


def test_trajectory_pusher_builds():
    pytest.importorskip("torch")
    from trajgen import gpu
    assert os.path.exists(gpu.build())


def test_headers_are_plain_c_and_every_symbol_links(tmp_path):
    """A C program (C99, -pedantic -Werror) that includes all three headers and takes
    the address of every declared function links against the library; running it
    calls only entry points that reject their arguments before touching a device."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no gcc")
    from paper_1003_1140_gb300 import build
    lib = build.build()
    names = sorted(set(declared_symbols("rad.h") + declared_symbols("rad_mlp.h")
                       + declared_symbols("rad_pic.h")))
    src = tmp_path / "abi.c"
    src.write_text(
        "#include <stddef.h>\n#include <stdio.h>\n"
        '#include "rad.h"\n#include "rad_mlp.h"\n#include "rad_pic.h"\n'
        "typedef void (*fn)(void);\n"
        "static const fn every[] = {\n" + ",\n".join(f"    (fn){n}" for n in names) + "\n};\n"
        "int main(void) {\n"
        "    rad_options o = {0};\n"
        "    int bad = 0;\n"
        "    (void)o;\n"
        "    bad |= rad_init(NULL, NULL, 0, NULL, NULL, 0, 0.0, NULL, 0, NULL, 0, 0, 0, 0.0,\n"
        "                    NULL) != RAD_EINVAL;\n"
        "    bad |= rad_pic_init(NULL, 0, 0.0, 0.0, NULL, 0, NULL, NULL, NULL) != RAD_PIC_EINVAL;\n"
        "    bad |= rad_mlp_init(NULL, NULL, 0, 0, NULL) != RAD_MLP_EINVAL;\n"
        "    bad |= rad_spectrum_size(NULL) != -1;\n"
        "    printf(\"%d symbols\\n\", (int)(sizeof every / sizeof every[0]));\n"
        "    return bad;\n"
        "}\n")
    exe = tmp_path / "abi"
    libdir = os.path.dirname(lib)
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                        "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe),
                        "-L", libdir, "-l:" + os.path.basename(lib), "-Wl,-rpath," + libdir],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.strip() == f"{len(names)} symbols"
