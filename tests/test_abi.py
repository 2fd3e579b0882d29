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
