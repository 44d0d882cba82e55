"""CPU checks of the C ABI: the library builds/loads, exports every function
include/lbm.h declares, the ctypes struct mirrors lbm_params, and host-side
validation answers with error codes (no GPU needed, no kernel launched)."""
import ctypes
import os
import re

import pytest

from paper_2402_15752_gb300 import lbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbm.h")


@pytest.fixture(scope="module")
def L():
    from paper_2402_15752_gb300 import build
    build.build()
    return lbm.load_library()


def declared_functions():
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(lbm_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_every_declared_function_is_exported(L):
    names = declared_functions()
    assert len(names) >= 38
    for n in names:
        assert hasattr(L, n), n


def test_debug_build_exports_the_same_functions(L):
    """The debug build (kernels bounds-checked) loads without a GPU, exports every
    declared function and says which build it is; the release build says 0."""
    from paper_2402_15752_gb300 import build
    D = ctypes.CDLL(build.build(debug=True))
    for n in declared_functions():
        assert hasattr(D, n), n
    assert D.lbm_debug_build() == 1
    assert L.lbm_debug_build() == 0


def test_ctypes_struct_mirrors_the_header():
    text = open(HEADER).read()
    body = re.search(r"typedef struct \{(.*?)\} lbm_params;", text, flags=re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        ctype, names = decl.split(None, 1)
        for nm in names.split(","):
            fields.append((nm.strip(), ctype))
    mirror = [(n, t) for n, t in lbm.LBMParams._fields_]
    assert [n for n, _ in fields] == [n for n, _ in mirror]
    kinds = {"int32_t": ctypes.c_int32, "double": ctypes.c_double}
    for (n, ct), (_, pt) in zip(fields, mirror):
        assert kinds[ct] is pt, n


def test_workspace_size_and_validation(L):
    p = lbm.make_params(dict(nx=1024, ny=2048), "fp32")
    n = L.lbm_workspace_bytes(ctypes.byref(p))
    # two population buffers of 28 FP32 planes, 5 previous-step macro planes, small extras
    base = 2 * 28 * 4 * 1024 * 2048 + 5 * 4 * 1024 * 2048
    assert base <= n < base + 65536
    # 16-bit population storage: half the population bytes, FP32 macros, and
    # two planes of the writers' (p, phi, c1, c2) bases the populations are stored against
    for prec in ("bf16", "fp16"):
        p16 = lbm.make_params(dict(nx=1024, ny=2048), prec)
        n16 = L.lbm_workspace_bytes(ctypes.byref(p16))
        base16 = 2 * 28 * 2 * 1024 * 2048 + 5 * 4 * 1024 * 2048 + 2 * 12 * 1024 * 2048
        assert base16 <= n16 < base16 + 65536
    bad = [dict(nx=0, ny=4), dict(nx=4, ny=4, scalar_q=7), dict(nx=4, ny=4, rho1=-1.0),
           dict(nx=4, ny=4, D2=0.0), dict(nx=4, ny=4, M=0.0), dict(nx=4, ny=4, visc_model=5)]
    for b in bad:
        q = lbm.make_params(b, "fp32")
        assert L.lbm_workspace_bytes(ctypes.byref(q)) == 0, b
        assert L.lbm_last_error(None)
    q = lbm.make_params(dict(nx=4, ny=4, scalar_model=2), "fp32")
    assert L.lbm_workspace_bytes(ctypes.byref(q)) == 0
    q = lbm.make_params(dict(nx=4, ny=4, scalar_model=1), "bf16")  # one-scalar: FP64/FP32 only
    assert L.lbm_workspace_bytes(ctypes.byref(q)) == 0
    q = lbm.make_params(dict(nx=4, ny=4, scalar_model=1), "fp32")
    assert L.lbm_workspace_bytes(ctypes.byref(q)) > 0
    for code in (-1, 4):  # precision codes outside LBM_FP64 .. LBM_FP32_FP16STORE
        q = lbm.make_params(dict(nx=4, ny=4), code)
        assert L.lbm_workspace_bytes(ctypes.byref(q)) == 0
        assert b"precision" in L.lbm_last_error(None)


def test_create_rejects_bad_workspace_without_touching_a_gpu(L):
    p = lbm.make_params(dict(nx=16, ny=16), "fp32")
    h = ctypes.c_void_p()
    assert L.lbm_create(ctypes.byref(p), None, 1 << 20, None, ctypes.byref(h)) == lbm.LBM_ERR_WORKSPACE
    assert L.lbm_create(ctypes.byref(p), ctypes.c_void_p(0x1008), 1 << 20, None, ctypes.byref(h)) == lbm.LBM_ERR_WORKSPACE
    assert h.value is None
    q = lbm.make_params(dict(nx=16, ny=16, mu2=0.0), "fp32")
    assert L.lbm_create(ctypes.byref(q), None, 0, None, ctypes.byref(h)) == lbm.LBM_ERR_UNSTABLE_TAU
    assert L.lbm_create(ctypes.byref(p), None, 0, None, None) == lbm.LBM_ERR_ARG
    # calls on a NULL handle are argument errors
    assert L.lbm_step(None, 1) == lbm.LBM_ERR_ARG
    assert L.lbm_sync(None) == lbm.LBM_ERR_ARG
    assert L.lbm_time(None) == -1
    L.lbm_destroy(None)
