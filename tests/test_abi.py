"""CPU-side checks of the C ABI: the library builds for sm_103a, loads, and
exports every function include/jag.h declares; ctypes mirrors match the
header's record sizes.  No GPU compute is called here."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2602_10258_gb300 import build_ext, datagen
from paper_2602_10258_gb300 import jag

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "jag.h")


@pytest.fixture(scope="module")
def lib():
    build_ext.build()
    return jag.load(build_if_missing=False)


def declared_functions():
    src = open(HEADER).read()
    return re.findall(r"JAG_API\s+[\w\s\*]+?\b(jag_\w+)\s*\(", src)


def test_header_declares_api():
    names = declared_functions()
    for n in ["jag_build", "jag_search", "jag_search_host", "jag_free", "jag_last_error"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", build_ext.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s+(\w+)", out))
    for n in declared_functions():
        assert n in exported, n
        assert hasattr(lib, n)
    assert set(jag.EXPORTED) == set(declared_functions())


def _c_layout(struct, fields):
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "jag.h"', "int main(void){"]
    lines.append('printf("size %%zu\\n", sizeof(%s));' % struct)
    for f in fields:
        lines.append('printf("%s %%zu\\n", offsetof(%s, %s));' % (f, struct, f))
    lines.append("return 0;}")
    p = "/tmp/jag_layout_%s.c" % struct
    open(p, "w").write("\n".join(lines))
    exe = p[:-2]
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-I", os.path.join(ROOT, "include"), p, "-o", exe],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([exe], capture_output=True, text=True).stdout.split()
    return {out[i]: int(out[i + 1]) for i in range(0, len(out), 2)}


@pytest.mark.parametrize("struct,cls", [("jag_build_params", jag.BuildParams),
                                        ("jag_search_args", jag.SearchArgs),
                                        ("jag_info", jag.Info),
                                        ("jag_policy", jag.PolicyStruct),
                                        ("jag_serve_params", jag.ServeParams),
                                        ("jag_serve_timing", jag.ServeTiming)])
def test_record_layouts_match_header(struct, cls):
    fields = [f for f, _ in cls._fields_]
    lay = _c_layout(struct, fields)
    assert lay["size"] == C.sizeof(cls)
    for f in fields:
        assert lay[f] == getattr(cls, f).offset, f


def test_filter_record_layout():
    assert datagen.FILTER_DTYPE.itemsize == 16
    lay = _c_layout("jag_filter", ["kind", "aux_off", "payload"])
    assert lay == {"size": 16, "kind": 0, "aux_off": 4, "payload": 8}
    assert [datagen.FILTER_DTYPE.fields[k][1] for k in ("kind", "aux_off", "payload")] == [0, 4, 8]


def test_last_error_and_version(lib):
    assert lib.jag_version().decode().startswith("jag-gb300")
    assert isinstance(lib.jag_last_error(), bytes)


def test_null_arguments_rejected_without_gpu(lib):
    # argument checks run before any device call
    assert lib.jag_build(None, None) == jag.JAG_EINVAL
    a = jag.SearchArgs()
    assert lib.jag_search(None, C.byref(a)) == jag.JAG_EINVAL
    p = jag.BuildParams()
    p.n, p.d = 10, 0
    h = C.c_void_p()
    assert lib.jag_build(C.byref(p), C.byref(h)) == jag.JAG_EINVAL
    assert b"d must be" in lib.jag_last_error()
    lib.jag_free(None)
    assert lib.jag_mlp_loss_grad(0, None, None, None, None, 1, 0.0, None, None, None) == jag.JAG_EINVAL
    assert lib.jag_mlp_export(17, None, None, None, None) == jag.JAG_EINVAL
    step = C.c_int64(0)
    assert lib.jag_mlp_train(9, None, None, None, C.byref(step), None, None, None, 1, 1, 1, 1e-3, 0.0, None,
                             None) == jag.JAG_EINVAL
    srv = C.c_void_p()
    assert lib.jag_serve_start(None, None, C.byref(srv)) == jag.JAG_EINVAL
    t = C.c_uint64(0)
    assert lib.jag_serve_submit(None, None, None, None, 0, 1, 0.0, C.byref(t)) == jag.JAG_EINVAL
    assert lib.jag_serve_wait(None, 1, None, None, None, 0.0) == jag.JAG_EINVAL
    assert lib.jag_serve_stop(None) == jag.JAG_OK
