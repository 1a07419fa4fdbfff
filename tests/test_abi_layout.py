"""The Python binding's structures have the layout of the C header's (CPU only):
a small C program compiled against include/trstmi.h prints the size of every
public structure and the offset of every field, and the ctypes / numpy
mirrors must agree field by field."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

T = pytest.importorskip("paper_2207_06374_gb300.trstmi")

# C structure -> its mirror in the binding (ctypes.Structure or numpy dtype)
MIRRORS = {
    "trstmi_options": T.Options,
    "trstmi_trace_row": T.TraceRow,
    "trstmi_step_info": T.StepInfo,
    "trstmi_multistart_result": T.MultistartResult,
    "trstmi_server_opts": T.ServerOpts,
    "trstmi_request": T.Request,
    "trstmi_result": T.Result,
    "trstmi_server_stats_t": T.ServerStats,
    "trstmi_certificates": T.Certificates,
    "trstmi_tr_options": T.TrOptions,
    "trstmi_tr_row": T.TR_ROW_DTYPE,
    "trstmi_peaks": T.Peaks,
}


def _fields(mirror):
    if isinstance(mirror, np.dtype):
        return [(n, mirror.fields[n][1]) for n in mirror.names], mirror.itemsize
    return [(f[0], getattr(mirror, f[0]).offset) for f in mirror._fields_], ctypes.sizeof(mirror)


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "trstmi.h"', "int main(void) {"]
    for cname, mirror in MIRRORS.items():
        lines.append(f'  printf("{cname} %zu\\n", sizeof({cname}));')
        for field, _ in _fields(mirror)[0]:
            lines.append(f'  printf("{cname}.{field} %zu\\n", offsetof({cname}, {field}));')
    lines += ["  return 0;", "}"]
    d = tmp_path_factory.mktemp("abi")
    src, exe = d / "layout.c", d / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), "-o", str(exe),
                           str(src)])
    out = subprocess.check_output([str(exe)], text=True)
    return {k: int(v) for k, v in (line.split() for line in out.splitlines())}


@pytest.mark.parametrize("cname", sorted(MIRRORS))
def test_binding_mirrors_the_header(cname, c_layout):
    fields, size = _fields(MIRRORS[cname])
    assert size == c_layout[cname], cname
    for field, offset in fields:
        assert offset == c_layout[f"{cname}.{field}"], (cname, field)
