"""The C-ABI library loads on the CPU and exports every entry point that
include/kf.h declares; the Python binding carries the same names.  No compute
call is made (no GPU here)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "kf.h")


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(kf_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1912_07133_gb300 import build as B
    B.build()
    from paper_1912_07133_gb300 import kf
    return kf.load()


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ("kf_create", "kf_destroy", "kf_last_error", "kf_design", "kf_filter_bank",
                 "kf_detect_blobs", "kf_bank_opts_default", "kf_kernel_times"):
        assert name in syms


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name
    from paper_1912_07133_gb300 import build as B
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (kf_\w+)", out))
    assert set(declared_symbols()) <= exported


def test_binding_names_match_header():
    from paper_1912_07133_gb300 import kf
    assert sorted(kf.ENTRY_POINTS) == declared_symbols()
    for name in kf.ENTRY_POINTS:
        assert callable(getattr(kf, name))


def test_struct_layouts_match_header(lib):
    """ctypes mirrors of the ABI structs have the C sizes (no GPU needed)."""
    import ctypes
    from paper_1912_07133_gb300 import kf
    assert ctypes.sizeof(kf.kf_frame) == 32
    assert ctypes.sizeof(kf.kf_blob) == 32
    assert ctypes.sizeof(kf.kf_blob_shape) == 16
    assert ctypes.sizeof(kf.kf_bank_opts) == 4 * 4 + 8 + 8 + 8 + 32
    assert ctypes.sizeof(kf.kf_kernel_time) == 40
    o = kf.kf_bank_opts_default()
    assert o.threshold == 0.05 and o.fir_kmax == 96 and o.storage == kf.KF_DTYPE_F32


def test_no_device_is_a_loud_error(lib):
    """Without a GPU the binding refuses instead of computing anything."""
    import torch
    from paper_1912_07133_gb300 import kf
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(kf.KfError):
        kf.kf_create(0)


def test_field_offsets_match_the_c_compiler(tmp_path):
    """Every field of the ctypes mirrors sits at the offset gcc gives it in
    include/kf.h."""
    import ctypes
    from paper_1912_07133_gb300 import kf
    structs = {"kf_frame": kf.kf_frame, "kf_bank_opts": kf.kf_bank_opts, "kf_blob": kf.kf_blob,
               "kf_blob_shape": kf.kf_blob_shape,
               "kf_kernel_time": kf.kf_kernel_time, "kf_coeffs": kf.kf_coeffs}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "kf.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'  printf("{name} sizeof %zu\\n", sizeof({name}));')
        for fname, _ in cls._fields_:
            lines.append(f'  printf("{name} {fname} %zu\\n", offsetof({name}, {fname}));')
    lines.append("  return 0; }")
    src = tmp_path / "probe.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for name, cls in structs.items():
        assert got[(name, "sizeof")] == ctypes.sizeof(cls), name
        for fname, _ in cls._fields_:
            assert got[(name, fname)] == getattr(cls, fname).offset, (name, fname)


def test_quartic_entry_points_reject_bad_arguments_without_a_device(lib):
    """The D = 5 calls check their arguments before any CUDA call: a NULL
    context or NULL pointers give KF_EINVAL with a message."""
    from paper_1912_07133_gb300 import kf
    assert lib.kf_quartic_bank(None, None, None, 1, kf.KF_IIR_REPEATED_POLE, 4, None, 0) == kf.KF_EINVAL
    assert b"ctx" in lib.kf_last_error(None)
    assert lib.kf_quartic_steer(None, None, 10, 1, 0.5, None) == kf.KF_EINVAL
    assert kf.KF_QUARTIC_CHANNELS == 15 and len(kf.QUARTIC_CHANNELS) == 15
    assert kf.QUARTIC_CHANNELS[:3] == ((0, 0), (1, 0), (0, 1))
