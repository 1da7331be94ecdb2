"""The C-ABI library builds, loads and exports every entry point of include/plam.h (no GPU needed).

Only calls that never reach the GPU are made: default parameters, version,
and argument validation that rejects a request before any CUDA call.
"""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "plam.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1810_03930_gb300 import _lib, build
    if not os.path.exists(_lib.LIB_PATH):
        build.build()
    return _lib.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:[\w\s\*]+?)\b((?:plam|pcal)_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("plam_create", "plam_step", "pcal_step", "plam_solve", "plam_orthonormalize",
                     "plam_destroy"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), name


def test_binding_covers_every_symbol():
    from paper_1810_03930_gb300 import _lib
    assert set(declared_functions()) <= set(_lib.SIGNATURES)


def test_default_params_are_the_papers(lib):
    from paper_1810_03930_gb300 import _lib
    prm = _lib.plam_default_params()
    assert prm.variant == _lib.PLAM_VARIANT_PCAL and prm.lambda_rule == _lib.PLAM_LAMBDA2
    assert prm.eta_rule == _lib.PLAM_ETA_ABB
    assert prm.tol == 1e-8 and prm.maxit == 3000 and prm.beta == 1.0   # Section 5.1
    assert _lib.plam_version() >= 100


def test_struct_layouts_match_header(tmp_path):
    """ctypes mirrors of the C structs have the sizes and field offsets the C compiler gives them."""
    import shutil
    import subprocess
    from paper_1810_03930_gb300 import _lib
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"plam_params_t": _lib.plam_params_t, "plam_info_t": _lib.plam_info_t,
               "plam_objective_t": _lib.plam_objective_t, "plam_comm_t": _lib.plam_comm_t,
               "plam_batch_problem_t": _lib.plam_batch_problem_t}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "plam.h"', "int main(void){"]
    expect = []
    for name, cls in structs.items():
        lines.append(f'printf("%zu\\n", sizeof({name}));')
        expect.append(C.sizeof(cls))
        for fname, _ in cls._fields_:
            lines.append(f'printf("%zu\\n", offsetof({name}, {fname}));')
            expect.append(getattr(cls, fname).offset)
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True,
                                          check=True).stdout.split()]
    assert got == expect


@pytest.mark.parametrize("n,p", [(10, 6), (0, 1), (5, 0)])
def test_create_rejects_bad_sizes_without_touching_the_gpu(lib, n, p):
    from paper_1810_03930_gb300 import _lib
    prm = _lib.plam_default_params()
    obj = _lib.plam_objective_t()
    obj.kind = _lib.PLAM_OBJ_HARTREE1D
    obj.alpha, obj.quad_scale = 1.0, 0.25
    h = C.c_void_p()
    st = lib.plam_create(C.byref(h), n, p, C.byref(obj), C.byref(prm), None)
    assert st == _lib.PLAM_ERR_INVALID and not h.value


def test_create_rejects_bad_params_and_objectives(lib):
    from paper_1810_03930_gb300 import _lib
    obj = _lib.plam_objective_t()
    obj.kind = _lib.PLAM_OBJ_HARTREE1D
    obj.alpha, obj.quad_scale = 1.0, 0.25
    for field, value in (("variant", 7), ("eta_rule", 9), ("precision", 5), ("beta", -1.0),
                         ("maxit", -1), ("final_orth", 3), ("eta_min", -1.0), ("eta_max", -2.0),
                         ("tensor_cores", 3), ("tensor_cores", 11)):
        prm = _lib.plam_default_params()
        setattr(prm, field, value)
        h = C.c_void_p()
        assert lib.plam_create(C.byref(h), 100, 5, C.byref(obj), C.byref(prm), None) == _lib.PLAM_ERR_INVALID
    prm = _lib.plam_default_params()
    prm.eta_min, prm.eta_max = 2.0, 1.0           # an empty step-size interval
    h = C.c_void_p()
    assert lib.plam_create(C.byref(h), 100, 5, C.byref(obj), C.byref(prm), None) == _lib.PLAM_ERR_INVALID
    assert prm.eta_min > 0 and _lib.plam_default_params().eta_min == 0.0
    prm = _lib.plam_default_params()
    bad = _lib.plam_objective_t()
    bad.kind = _lib.PLAM_OBJ_STENCIL3D
    bad.nx, bad.ny, bad.nz = 4, 4, 4          # 64 points for n = 100: inconsistent
    h = C.c_void_p()
    assert lib.plam_create(C.byref(h), 100, 5, C.byref(bad), C.byref(prm), None) == _lib.PLAM_ERR_INVALID
    bad.kind = _lib.PLAM_OBJ_DENSE            # no operator
    assert lib.plam_create(C.byref(h), 100, 5, C.byref(bad), C.byref(prm), None) == _lib.PLAM_ERR_INVALID
    bad.kind = 17
    assert lib.plam_create(C.byref(h), 100, 5, C.byref(bad), C.byref(prm), None) == _lib.PLAM_ERR_INVALID


def test_create_rejects_bad_block_and_linear_term(lib):
    """The 1D objective's block size and linear term (Section 5.4's Problems 1 and 2) are checked
    on the host before anything is allocated: a negative block, a Hartree term with blocks of more
    than 64 rows or with one block of n rows and a linear term, and a linear term whose leading
    dimension is short or whose address is not aligned to the storage type (the pointers are never
    dereferenced)."""
    from paper_1810_03930_gb300 import _lib
    prm = _lib.plam_default_params()          # FP64: 8-byte storage
    n, p = 500, 4
    cases = [dict(block=-1, alpha=0.0), dict(block=65, alpha=1.0),
             dict(block=0, alpha=1.0, lin=256, ldlin=n), dict(block=5, alpha=1.0, lin=256, ldlin=n - 1),
             dict(block=5, alpha=0.0, lin=260, ldlin=n)]
    for c in cases:
        obj = _lib.plam_objective_t()
        obj.kind = _lib.PLAM_OBJ_HARTREE1D
        obj.quad_scale = 0.5
        obj.alpha = c["alpha"]
        obj.block = c["block"]
        if "lin" in c:
            obj.lin, obj.ldlin = c["lin"], c["ldlin"]
        h = C.c_void_p()
        st = lib.plam_create(C.byref(h), n, p, C.byref(obj), C.byref(prm), None)
        assert st == _lib.PLAM_ERR_INVALID and not h.value, c


def test_sharded_create_rejects_bad_requests_without_touching_the_gpu(lib):
    """plam_create_sharded validates the rank layout and the objective before any CUDA call:
    no communicator, a rank outside [0, size), rows beyond n_global, a missing all-gather with
    several ranks, a slab that does not start on a z-plane, blocks that would cross ranks, and
    objectives whose gradient couples every row (one global Dirichlet L, a dense A)."""
    from paper_1810_03930_gb300 import _lib
    prm = _lib.plam_default_params()

    def stencil(nz):
        o = _lib.plam_objective_t()
        o.kind, o.nx, o.ny, o.nz = _lib.PLAM_OBJ_STENCIL3D, 8, 8, nz
        return o

    def comm(rank, size, row0, n_global, ag=True, ex=True):
        c = _lib.plam_comm_t()
        c.rank, c.size, c.row0, c.n_global = rank, size, row0, n_global
        if ag:
            c.allgather = _lib.plam_allgather_fn(lambda *a: 0)
        if ex:
            c.exchange = _lib.plam_exchange_fn(lambda *a: 0)
        return c

    cases = [
        (stencil(4), None, _lib.PLAM_ERR_INVALID),
        (stencil(4), comm(2, 2, 0, 512), _lib.PLAM_ERR_INVALID),
        (stencil(4), comm(1, 2, 300, 512), _lib.PLAM_ERR_INVALID),         # 300 + 256 > 512
        (stencil(4), comm(0, 2, 0, 512, ag=False), _lib.PLAM_ERR_INVALID),
        (stencil(4), comm(0, 2, 0, 512, ex=False), _lib.PLAM_ERR_INVALID),
        (stencil(4), comm(1, 2, 200, 512), _lib.PLAM_ERR_INVALID),         # not on a z-plane
    ]
    blk = _lib.plam_objective_t()
    blk.kind, blk.alpha, blk.quad_scale, blk.block = _lib.PLAM_OBJ_HARTREE1D, 1.0, 0.5, 5
    cases.append((blk, comm(0, 2, 0, 1000), _lib.PLAM_OK))                 # checked below
    one = _lib.plam_objective_t()
    one.kind, one.alpha, one.quad_scale, one.block = _lib.PLAM_OBJ_HARTREE1D, 1.0, 0.5, 0
    cases.append((one, comm(0, 2, 0, 1000), _lib.PLAM_ERR_UNSUPPORTED))
    dense = _lib.plam_objective_t()
    dense.kind, dense.A, dense.lda = _lib.PLAM_OBJ_DENSE, 256, 256
    cases.append((dense, comm(0, 2, 0, 512), _lib.PLAM_ERR_UNSUPPORTED))
    for obj, c, want in cases:
        if want == _lib.PLAM_OK:
            continue
        n = 256 if obj.kind != _lib.PLAM_OBJ_HARTREE1D else 500
        h = C.c_void_p()
        st = lib.plam_create_sharded(C.byref(h), n, 4, C.byref(obj), C.byref(prm),
                                     C.byref(c) if c is not None else None, None)
        assert st == want and not h.value, (obj.kind, st)
    # blocks of 5 must not cross ranks: 497 rows on rank 0 of 2
    h = C.c_void_p()
    st = lib.plam_create_sharded(C.byref(h), 497, 4, C.byref(blk), C.byref(prm),
                                 C.byref(comm(0, 2, 0, 1000)), None)
    assert st == _lib.PLAM_ERR_INVALID and not h.value


def test_null_handle_calls_are_rejected(lib):
    from paper_1810_03930_gb300 import _lib
    info = _lib.plam_info_t()
    assert lib.plam_step(None, None, 0, C.byref(info)) == _lib.PLAM_ERR_INVALID
    assert lib.pcal_step(None, None, 0, C.byref(info)) == _lib.PLAM_ERR_INVALID
    assert lib.plam_solve(None, None, 0, None, 0, C.byref(info)) == _lib.PLAM_ERR_INVALID
    assert lib.plam_destroy(None) == _lib.PLAM_ERR_INVALID
    assert lib.plam_last_iteration(None, None, 0, None, None, None) == _lib.PLAM_ERR_INVALID
    assert lib.plam_kernel_launches(None) == -1


def test_binding_fails_loudly_without_the_library(tmp_path, monkeypatch):
    """No CPU fallback: with the shared library absent the binding raises instead of computing
    anything (the loader is pointed at an empty directory in a fresh module state)."""
    from paper_1810_03930_gb300 import _lib
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        _lib.load(str(tmp_path / "libplam.so"))
