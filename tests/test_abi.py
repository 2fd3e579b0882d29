"""The C-ABI library builds, loads on a machine without a GPU, exports every
entry point include/pod.h declares, and the binding's parameter struct has
the C layout.  No compute calls (CPU only)."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

from paper_1905_05107_gb300 import build, pod

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pod.h")


@pytest.fixture(scope="module")
def libpath():
    return build.build()


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"POD_API\s+[\w\s\*]*?\b(pod_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["pod_init", "pod_iterate", "pod_modes", "pod_backward", "pod_destroy", "pod_strerror"]:
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s+(pod_\w+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    assert set(pod.EXPORTED) == set(declared_functions())


def test_library_loads_and_strerror(libpath):
    L = pod.lib()
    assert L.pod_strerror(0) == b"ok"
    assert b"unsupported" in L.pod_strerror(pod.POD_EUNSUPPORTED)


def test_params_struct_layout_matches_c():
    fields = [f for f, _ in pod.PodParams._fields_]
    src = "#include <stdio.h>\n#include <stddef.h>\n#include \"pod.h\"\nint main(void){\n"
    src += 'printf("%zu\\n", sizeof(pod_params));\n'
    for f in fields:
        src += 'printf("%%zu\\n", offsetof(pod_params, %s));\n' % f
    src += "return 0;}\n"
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-I", os.path.dirname(HEADER), c, "-o", exe], check=True)
        vals = [int(v) for v in subprocess.run([exe], capture_output=True, text=True).stdout.split()]
    assert vals[0] == ctypes.sizeof(pod.PodParams)
    for f, off in zip(fields, vals[1:]):
        assert getattr(pod.PodParams, f).offset == off, f


def test_binding_refuses_cpu_tensors():
    import torch
    A = torch.zeros(4, 3).t().contiguous().t()
    with pytest.raises(ValueError):
        pod._check_colmajor(A)


def _good_params():
    p = pod.PodParams()
    p.m, p.n, p.lda = 1000, 200, 1000
    p.k, p.c = 5, 10
    p.tol = 1e-8
    return p


BAD_PARAMS = [
    ("m", 0), ("n", 0), ("lda", 999), ("k", 0), ("k", 201), ("c", 0), ("r", 3),
    ("dtype", 5), ("col_strategy", 7), ("criterion", 3), ("core", 9), ("rows", 2),
    ("row_strategy", 5), ("w", -1), ("block_trunc", 2), ("precision", 9), ("keep_tape", 2),
    ("reserved", 1), ("tol", float("nan")),
]


@pytest.mark.parametrize("field,value", BAD_PARAMS)
def test_init_rejects_bad_parameters(libpath, field, value):
    """pod_init validates every field before it touches a device, so these
    run without a GPU: each out-of-range field gives POD_EINVAL and no
    context."""
    p = _good_params()
    setattr(p, field, value)
    h = ctypes.c_void_p(123)
    st = pod.lib().pod_init(ctypes.byref(h), ctypes.byref(p), ctypes.c_void_p(0x1000), None)
    assert st == pod.POD_EINVAL, (field, value, st)
    assert not h.value


@pytest.mark.parametrize("field,value", [("c", 300), ("r", 250), ("keep_tape", 1)])
def test_init_rejects_unsupported_sizes(libpath, field, value):
    p = _good_params()
    setattr(p, field, value)
    if field == "r":
        p.c = 100            # r + c beyond the 320-wide core
    if field == "keep_tape":
        p.rows = 1           # the adjoint is built for ICS only
    h = ctypes.c_void_p(0)
    st = pod.lib().pod_init(ctypes.byref(h), ctypes.byref(p), ctypes.c_void_p(0x1000), None)
    assert st == pod.POD_EUNSUPPORTED, (field, value, st)


def test_null_arguments_are_einval(libpath):
    L = pod.lib()
    p = _good_params()
    assert L.pod_init(None, ctypes.byref(p), ctypes.c_void_p(0x1000), None) == pod.POD_EINVAL
    h = ctypes.c_void_p(0)
    assert L.pod_init(ctypes.byref(h), None, ctypes.c_void_p(0x1000), None) == pod.POD_EINVAL
    assert L.pod_init(ctypes.byref(h), ctypes.byref(p), None, None) == pod.POD_EINVAL
    assert L.pod_iterate(None, 1, None, None, None) == pod.POD_EINVAL
    assert L.pod_modes(None, None, None, None) == pod.POD_EINVAL
    assert L.pod_set_wait_limit(None, 1) == pod.POD_EINVAL
    assert L.pod_colnorms(None, 0, 10, 10, 10, None, None) == pod.POD_EINVAL
    assert L.pod_colnorms(ctypes.c_void_p(0x1000), 7, 10, 10, 10, ctypes.c_void_p(0x2000), None) == pod.POD_EINVAL
    assert L.pod_sample(None, None, 10, 1, 0, 0, 0, None, None, None) == pod.POD_EINVAL
    assert L.pod_sample_noalloc(ctypes.c_void_p(0x1000), ctypes.c_void_p(0x2000), 1 << 20, 4, 0, 0, 0,
                                ctypes.c_void_p(0x3000), ctypes.c_void_p(0x4000), None) == pod.POD_EUNSUPPORTED
    L.pod_destroy(None)


def test_strerror_covers_every_status(libpath):
    L = pod.lib()
    texts = [L.pod_strerror(s) for s in range(9)]
    assert len(set(texts)) == 9 and b"unknown" not in b"".join(texts)
    assert L.pod_strerror(99) == b"unknown status"
