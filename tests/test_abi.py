"""CPU checks of the C-ABI boundary: the library builds for sm_103a, loads, and exports every
entry point include/painn.h declares; argument validation that needs no GPU; the parameter
blob layout the header documents."""
import os
import re
import struct
import subprocess

import numpy as np
import pytest

import synthetic as syn

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "painn.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ctd_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import paper_2506_04055_gb300 as eng
    eng.build()
    return eng.load()


def test_every_declared_symbol_is_exported(lib):
    from paper_2506_04055_gb300 import _lib
    declared = _declared()
    assert declared == sorted(_lib.EXPORTS)
    so = os.path.join(ROOT, "paper_2506_04055_gb300", "libctd_painn.so")
    syms = subprocess.run(["nm", "-D", "--defined-only", so], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (ctd_[a-z_0-9]+)\b", syms))
    for name in declared:
        assert name in exported, name
        getattr(lib, name)


def test_library_targets_sm103a(lib):
    """Every translation unit is compiled for compute_103a/sm_103a only, and the assembler's own
    report of each build names sm_103a for every kernel it compiled."""
    from paper_2506_04055_gb300 import buildlib
    assert buildlib.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    for src in buildlib.SOURCES:
        log = open(os.path.join(buildlib.BUILD, src + ".ptxas.txt")).read()
        targets = set(re.findall(r"for '(sm_[0-9a-z]+)'", log))
        assert targets <= {"sm_103a"}, (src, targets)
        if "__global__" in open(os.path.join(buildlib.SRC, src)).read():
            assert targets == {"sm_103a"}, src


def test_invalid_model_description_rejected(lib):
    from paper_2506_04055_gb300 import _lib
    for desc in (_lib.ctd_model_desc(48, 20, 3, 2, 5.0, 0), _lib.ctd_model_desc(64, 40, 3, 2, 5.0, 0),
                 _lib.ctd_model_desc(64, 20, 3, 2, -1.0, 0), _lib.ctd_model_desc(64, 20, 3, 2, 5.0, 7)):
        with pytest.raises(_lib.CtdError) as ei:
            _lib.ctd_create(desc)
        assert ei.value.code == _lib.CTD_ERR_INVALID_ARG


def test_no_device_is_an_error_not_a_fallback(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2506_04055_gb300 import _lib
    with pytest.raises(_lib.CtdError) as ei:
        _lib.ctd_create(_lib.ctd_model_desc(64, 20, 3, 2, 5.0, 0))
    assert ei.value.code == _lib.CTD_ERR_CUDA


def test_param_blob_layout():
    F, K, T, S = 64, 20, 3, 2
    blob = syn.params_blob(F, K, T, S, rc=5.0, e_scale=2.0, seed=0)
    assert blob[:8] == b"CTDPAINN"
    ver, f, k, t, s, _ = struct.unpack("<iiiiii", blob[8:32])
    rc, eps, esc, nval = struct.unpack("<dddq", blob[32:64])
    assert (ver, f, k, t, s, rc, esc) == (1, F, K, T, S, 5.0, 2.0)
    per = F * F + F + 3 * F * F + 3 * F + 3 * F * K + 3 * F + 2 * F * F + 2 * F * F + F + 3 * F * F + 3 * F
    assert nval == S * F + T * per + (F // 2) * F + F // 2 + F // 2 + 1 == (len(blob) - 64) // 8
    vals = np.frombuffer(blob[64:], np.float64)
    P = syn.unpack_params(vals.copy(), F, K, T, S)
    bound = np.sqrt(6.0 / (F + F))
    assert np.abs(P["W1_0"]).max() <= bound and np.abs(P["W1_0"]).max() > 0.9 * bound
    assert np.all(P["b1_0"] == 0)


def test_local_param_blob_layout():
    """The strictly local model's blob: the header the library checks and the value count of
    the documented order (A0, c0, P0; per layer Q, M, m and, before the last, Gs, Gv; R1, d1,
    R2, d2)."""
    F, K, L, S, C = 64, 20, 3, 2, 16
    blob = syn.local_params_blob(F, K, L, S, C, rc=5.0, e_scale=0.5, seed=0)
    assert blob[:8] == b"CTDLOCAL"
    ver, f, k, layers, s, c = struct.unpack("<iiiiii", blob[8:32])
    rc, _, esc, nval = struct.unpack("<dddq", blob[32:64])
    assert (ver, f, k, layers, s, c, rc, esc) == (1, F, K, L, S, C, 5.0, 0.5)
    C2, Fh = 2 * C, F // 2
    count = (K + 2 * S) * F + F + F * C2 + L * (F * C2 + (F + C2) * F + F) + (L - 1) * 2 * C2 * C
    count += F * Fh + Fh + Fh + 1
    assert nval == count == (len(blob) - 64) // 8
    names = [n for n, _ in syn.local_param_shapes(F, K, L, S, C)]
    assert names[:3] == ["A0", "c0", "P0"] and names[-4:] == ["R1", "d1", "R2", "d2"]
    assert "Gs3" not in names and "Gs2" in names


def test_struct_layouts_match_the_header():
    """ctypes mirrors of ctd_model_desc, ctd_stats and ctd_domain_info have the C compiler's sizes and offsets
    (a program built from include/painn.h with gcc prints them)."""
    import ctypes

    from paper_2506_04055_gb300 import _lib
    out_dir = os.path.join(ROOT, "_build")
    os.makedirs(out_dir, exist_ok=True)
    src = os.path.join(out_dir, "layout.c")
    exe = os.path.join(out_dir, "layout")
    fields = {"ctd_model_desc": [f for f, _ in _lib.ctd_model_desc._fields_],
              "ctd_stats": [f for f, _ in _lib.ctd_stats._fields_],
              "ctd_domain_info": [f for f, _ in _lib.ctd_domain_info._fields_]}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "painn.h"', "int main(void) {"]
    for st, names in fields.items():
        lines.append(f'  printf("{st} size %zu\\n", sizeof({st}));')
        for f in names:
            lines.append(f'  printf("{st} {f} %zu\\n", offsetof({st}, {f}));')
    lines += ["  return 0;", "}"]
    with open(src, "w") as fh:
        fh.write("\n".join(lines) + "\n")
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True)
    got = {}
    for line in subprocess.run([exe], capture_output=True, text=True, check=True).stdout.splitlines():
        st, key, val = line.split()
        got[(st, key)] = int(val)
    for st in fields:
        cls = getattr(_lib, st)
        assert got[(st, "size")] == ctypes.sizeof(cls), st
        for f in fields[st]:
            assert got[(st, f)] == getattr(cls, f).offset, (st, f)
