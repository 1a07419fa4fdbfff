"""A plain C program builds against include/trstmi.h, links the library and,
on a machine without a GPU, gets TRSTMI_ECUDA from trstmi_create (the
library has no CPU fallback).  CPU only."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_c_program_links_and_fails_loudly_without_a_gpu(tmp_path):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2207_06374_gb300 import trstmi as T
    T.lib()   # builds the library if needed
    libdir = os.path.dirname(T.LIB_PATH)
    exe = tmp_path / "search_example"
    subprocess.check_call(["gcc", "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                           os.path.join(ROOT, "tests", "c", "search_example.c"), "-o", str(exe),
                           "-L", libdir, "-ltrstmi", f"-Wl,-rpath,{libdir}"])
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 3, (r.returncode, r.stdout, r.stderr)
    assert "CUDA" in r.stdout
