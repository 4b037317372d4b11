"""The C-ABI library builds, loads, and exports every symbol include/bse.h
declares (CPU only: no compute call)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(bse_[a-z0-9_]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1904_05575_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_boundary():
    names = _declared()
    for required in ("bse_build_kernel", "bse_reduce", "bse_spectrum", "bse_last_error"):
        assert required in names


def test_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), f"libbse.so does not export {name}"


def test_version_and_error_without_gpu(lib):
    lib.bse_version.restype = ctypes.c_int
    assert lib.bse_version() >= 100
    lib.bse_last_error.restype = ctypes.c_char_p
    assert isinstance(lib.bse_last_error(), bytes)


def test_host_side_argument_errors(lib):
    """Argument checks run on the host before any CUDA call."""
    import paper_1904_05575_gb300 as bse
    lib2 = bse.load()
    # nprob = 0 is a no-op
    assert lib2.bse_build_kernel(None, 0, 0, None) == bse.BSE_OK
    # unknown precision / NULL probs / bad sizes are BSE_ERR_ARG
    assert lib2.bse_build_kernel(None, 1, 0, None) == bse.BSE_ERR_ARG
    p = bse.bse_problem(nk=0, nv=1, nc=1, ng=1, nq_w=1, omega_cell=1.0, ld=1)
    arr = (bse.bse_problem * 1)(p)
    assert lib2.bse_build_kernel(arr, 1, 0, None) == bse.BSE_ERR_ARG
    assert b"nk" in lib2.bse_last_error()
    assert lib2.bse_build_kernel(arr, 1, 99, None) == bse.BSE_ERR_ARG
    # a plan's wait limit: NULL plan or a limit outside (0, 60] s
    assert lib2.bse_plan_set_wait_limit(None, 1.0) == bse.BSE_ERR_ARG
    # a complex128 array that is not 16-byte aligned is refused before any launch
    q = bse.bse_problem(nk=1, nv=1, nc=1, ng=1, nq_w=1, omega_cell=1.0, ld=1, gamma_x=1.0,
                        gamma_c=0.0, coupling=0, e_v=0x1000, e_c=0x1000, m_x=0x1008,
                        v_bar=0x1000, A=0x2000)
    arr = (bse.bse_problem * 1)(q)
    assert lib2.bse_build_kernel(arr, 1, 0, None) == bse.BSE_ERR_ARG
    assert b"16-byte" in lib2.bse_last_error()
    # a k-row slab past nk is refused before any launch
    r = bse.bse_problem(nk=2, nv=1, nc=1, ng=1, nq_w=1, omega_cell=1.0, ld=2, k_begin=1, k_count=2)
    arr = (bse.bse_problem * 1)(r)
    assert lib2.bse_build_kernel(arr, 1, 0, None) == bse.BSE_ERR_ARG
    assert b"slab" in lib2.bse_last_error()
    assert lib2.bse_reduce(0, None, None, 1, None, None, None, None) == bse.BSE_ERR_ARG
    assert lib2.bse_spectrum(4, None, None, 2, None, 1.0, 1.0, 0, None, 0.1,
                             None, None, None, None) == bse.BSE_ERR_ARG


def test_header_is_c99_and_matches_the_binding(tmp_path):
    """include/bse.h compiles as strict C99, and bse_problem has the same size
    and field offsets in C as in the ctypes binding."""
    import shutil
    import subprocess
    import paper_1904_05575_gb300 as bse
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    inc = os.path.join(ROOT, "include")
    fields = [f for f, _ in bse.bse_problem._fields_]
    src = tmp_path / "layout.c"
    src.write_text(
        "#include <stdio.h>\n#include <stddef.h>\n#include \"bse.h\"\n"
        "int main(void) {\n  printf(\"%zu\\n\", sizeof(bse_problem));\n"
        + "".join(f"  printf(\"%zu\\n\", offsetof(bse_problem, {f}));\n" for f in fields)
        + "  return 0;\n}\n")
    exe = tmp_path / "layout"
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", inc,
                        str(src), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True,
                                          check=True).stdout.split()]
    assert out[0] == ctypes.sizeof(bse.bse_problem)
    for f, off in zip(fields, out[1:]):
        assert getattr(bse.bse_problem, f).offset == off, f


def test_problem_struct_shape_checks():
    """make_problem_struct checks every array's shape before taking pointers:
    problems as upload_problem lays them out (whole, k-row slab views, padded
    ld, TDA) pass the checks and only then meet the CUDA-tensor requirement
    (TypeError on the CPU); a mis-shaped array is a ValueError."""
    import bse_inputs as bi
    import paper_1904_05575_gb300 as bse
    torch = pytest.importorskip("torch")
    cfg = bi.BSEConfig("shapes", grid=2, nv=2, nc=3, ng=15, w_scale=0.1)
    d = bse.upload_problem(bi.make_problem(cfg), device="cpu", ld=50)
    slab = dict(d, m_vv=d["m_vv"][2:5], m_cc=d["m_cc"][2:5])
    for kw, dd in ((dict(), d), (dict(coupling=False), d), (dict(k_begin=2, k_count=3), slab)):
        with pytest.raises(TypeError):
            bse.make_problem_struct(dd, **kw)
    for name, bad in (("w", d["w"][:, :-1]), ("m_x", d["m_x"][..., :-1]), ("e_c", d["e_c"][:, :2]),
                      ("q_minus", d["q_minus"][:4]), ("v_bar", d["v_bar"][:-1]),
                      ("n_vc", d["n_vc"][..., :-1])):
        with pytest.raises(ValueError):
            bse.make_problem_struct(dict(d, **{name: bad}))
    # TDA does not read n_vc or q_plus
    with pytest.raises(TypeError):
        bse.make_problem_struct(dict(d, n_vc=d["n_vc"][..., :-1]), coupling=False)


def test_host_side_argument_errors_newer_entry_points(lib):
    """The eigensolve-free spectrum, the stage-2 shape query, the learned
    preconditioner's neighbour and feature calls and the input dtype all
    check their arguments on the host before any CUDA call."""
    import paper_1904_05575_gb300 as bse
    lib2 = bse.load()
    i32 = ctypes.c_int32
    assert lib2.bse_spectrum_lanczos(0, None, None, 1, None, 1.0, 1.0, 1, None, 0.1, 1e-8, 100,
                                     bse.BSE_PREC_FP64, None, None, None) == bse.BSE_ERR_ARG
    assert lib2.bse_spectrum_lanczos(4, None, None, 4, None, 1.0, 1.0, 1, None, 0.1, 1e-8, 100,
                                     bse.BSE_PREC_FP64, None, None, None) == bse.BSE_ERR_ARG
    assert b"NULL" in lib2.bse_last_error()
    t, st = i32(5), i32(5)
    assert lib2.bse_plan_stage2_shape(None, ctypes.byref(t), ctypes.byref(st)) == bse.BSE_ERR_ARG
    assert lib2.bse_mlp_set_neighbours(None, 4, 1, None, 0, None) == bse.BSE_ERR_ARG
    assert lib2.bse_mlp_features(None, 4, 1, None, None, None, None, None, 4, None, None, None,
                                 None) == bse.BSE_ERR_ARG
    # in_dtype outside {BSE_C128, BSE_C64}, and complex64 inputs not 8-byte aligned
    q = bse.bse_problem(nk=1, nv=1, nc=1, ng=1, nq_w=1, omega_cell=1.0, ld=1, gamma_x=1.0,
                        gamma_c=0.0, coupling=0, e_v=0x1000, e_c=0x1000, m_x=0x1000,
                        v_bar=0x1000, A=0x2000, in_dtype=7)
    assert lib2.bse_build_kernel((bse.bse_problem * 1)(q), 1, 0, None) == bse.BSE_ERR_ARG
    assert b"in_dtype" in lib2.bse_last_error()
    q.in_dtype = bse.BSE_C64
    q.m_x = 0x1004
    assert lib2.bse_build_kernel((bse.bse_problem * 1)(q), 1, 0, None) == bse.BSE_ERR_ARG
    assert b"8-byte" in lib2.bse_last_error()
