"""The oracle and the CUDA path share no code.

Checked on the sources: the library (Python binding and CUDA/C++ sources)
never imports or includes the oracle, the oracle never references the library
or its headers, and the input generators (the one module both sides use)
import neither.
"""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1407_1465_gb300")
ORACLE = os.path.join(ROOT, "oracle")


def _files(top, exts):
    for dirpath, _, names in os.walk(top):
        if "_build" in dirpath or "__pycache__" in dirpath:
            continue
        for n in names:
            if n.endswith(exts):
                yield os.path.join(dirpath, n)


def _text(path):
    with open(path, encoding="utf-8", errors="replace") as f:
        return f.read()


def test_library_does_not_use_the_oracle():
    for path in _files(PKG, (".py", ".cu", ".cuh", ".h", ".cpp")):
        text = _text(path)
        assert not re.search(r"^\s*(import|from)\s+oracle\b", text, re.M), path
        assert "rsa_oracle" not in text, path


def test_oracle_does_not_use_the_library():
    for path in _files(ORACLE, (".py", ".c", ".h")):
        text = _text(path)
        assert not re.search(r"^\s*(import|from)\s+paper_1407_1465_gb300\b", text, re.M), path
        assert not re.search(r'#include\s+[<"]rsa_gb300\.h', text) and "librsagpu" not in text, path
        assert not re.search(r'#include\s+"(mont|kernels|crt_tc|keyrec|tc)\.', text), path


def test_input_generators_import_neither_side():
    text = _text(os.path.join(ROOT, "workloads.py"))
    assert not re.search(r"^\s*(import|from)\s+(oracle|paper_1407_1465_gb300)\b", text, re.M)
