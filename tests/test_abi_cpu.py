"""CPU-side checks of the C ABI: the library builds for sm_103a, loads, and
exports every function include/helm.h declares; the Python binding knows each
one; calls that need no GPU behave as documented."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "helm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?(?:int|void|uint64_t|char)\s*\*?\s*(helm_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def built_lib():
    from paper_1712_08743_gb300 import _lib, build

    build.build()
    return _lib.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("helm_create_model", "helm_solve", "helm_adjoint_gradient", "helm_submit", "helm_poll",
                     "helm_release", "helm_ctx_create", "helm_destroy_model", "helm_ctx_destroy", "helm_strerror"):
        assert required in names


def test_library_exports_every_declared_symbol(built_lib):
    for name in declared_functions():
        assert hasattr(built_lib, name), name


def test_binding_covers_every_declared_symbol():
    from paper_1712_08743_gb300 import _lib

    assert set(declared_functions()) <= set(_lib.SIGNATURES)


def test_binding_constants_match_the_header():
    """Every enumerator of include/helm.h (status codes, options, kernel ids) has
    the same value in the binding."""
    from paper_1712_08743_gb300 import _lib

    src = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "helm.h")).read(), flags=re.S)
    enums = {k: int(v) for k, v in re.findall(r"\b(HELM_[A-Z0-9_]+)\s*=\s*(-?\d+)", src)}
    assert len(enums) >= 30
    for name, value in enums.items():
        assert getattr(_lib, name) == value, name


def test_calls_without_gpu(built_lib):
    from paper_1712_08743_gb300 import _lib

    o = _lib.helm_solve_opts()
    built_lib.helm_default_opts(C.byref(o))
    assert o.tol == 1e-6 and o.max_it == 5000 and (o.beta1, o.beta2) == (1.0, 0.5) and o.precision == 0
    assert built_lib.helm_strerror(_lib.HELM_E_NOT_CONVERGED).decode().startswith("tolerance")
    # null handles are rejected before any CUDA call
    assert built_lib.helm_solve(None, 1, None, None, None, None, None, None, None) == _lib.HELM_E_INVALID
    assert built_lib.helm_model_info(None, None, None, None) == _lib.HELM_E_INVALID
    assert built_lib.helm_poll(None, C.c_uint64(1), 0, None) == _lib.HELM_E_INVALID


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_1712_08743_gb300 import _lib

    monkeypatch.setattr(_lib, "_LIB", None)
    monkeypatch.setattr(_lib, "lib_path", lambda: str(tmp_path / "absent.so"))
    with pytest.raises(RuntimeError, match="not built"):
        _lib.load()


def test_kernels_compile_for_sm103a_without_spills():
    """ptxas report of the kernels translation unit: no register spills."""
    import subprocess

    from paper_1712_08743_gb300 import build

    src = os.path.join(build.CSRC, "helm_kernels.cu")
    r = subprocess.run([build._nvcc(), *build.ARCH, *build.FLAGS, "-Xptxas=-v", "-c", src, "-o", os.devnull],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    spills = re.findall(r"(\d+) bytes spill stores", r.stderr)
    assert spills and all(int(s) == 0 for s in spills)


def test_ctypes_structs_match_the_c_layout(tmp_path):
    """Every struct the binding mirrors has the C compiler's size and field
    offsets (include/helm.h compiled as plain C by gcc)."""
    import shutil
    import subprocess

    from paper_1712_08743_gb300 import _lib

    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no C compiler")
    structs = [_lib.helm_solve_opts, _lib.helm_solve_stats, _lib.helm_request, _lib.helm_result, _lib.helm_fwi_opts]
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "helm.h"', "int main(void) {"]
    for st in structs:
        lines.append(f'printf("{st.__name__} size %zu\\n", sizeof({st.__name__}));')
        for name, _ in st._fields_:
            lines.append(f'printf("{st.__name__} {name} %zu\\n", offsetof({st.__name__}, {name}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for st in structs:
        assert got[(st.__name__, "size")] == C.sizeof(st), st.__name__
        for name, _ in st._fields_:
            assert got[(st.__name__, name)] == getattr(st, name).offset, (st.__name__, name)
