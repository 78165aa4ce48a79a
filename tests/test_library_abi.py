"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every function ``include/paro.h`` declares, and the ctypes structures of the
binding have the C layout."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "paro.h")
# a declaration: return type (one or more words, optional pointer), then the name
DECL = r"^\s*(?:const\s+)?(?:\w+\s+)*\w+\s*\*?\s*(paro_\w+)\s*"


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(DECL + r"\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_1405_0260_gb300 import binding

    if not os.path.exists(binding.LIB_PATH):
        import __graft_entry__

        __graft_entry__.build()
    return binding.lib()


def test_header_declares_the_entry_points():
    names = declared_functions()
    for f in ("paro_mesh_create", "paro_mesh_destroy", "paro_set_potential", "paro_orbital_solve",
              "paro_rayleigh_ritz", "paro_iterate", "paro_apply", "paro_last_error", "paro_default_params",
              "paro_density", "paro_ks_potential", "paro_scf_iterate", "paro_ks_density_in"):
        assert f in names


def test_library_exports_every_declared_function(lib):
    for f in declared_functions():
        assert hasattr(lib, f), f


def test_default_params_and_null_handle_errors(lib):
    from paper_1405_0260_gb300 import binding as B

    p = B.paro_default_params()
    assert p.tol == 1e-10 and p.solve_tol == 1e-12 and p.max_outer == 500 and p.profile == 0
    assert p.precond == B.PARO_PRECOND_JACOBI and p.mg_nu == 1 and p.mg_coarse_sweeps == 4
    assert p.hartree_precond == B.PARO_PRECOND_AUTO
    # argument errors are caught before any CUDA call
    h = ctypes.c_void_p()
    lo = (ctypes.c_double * 3)(-1, -1, -1)
    hi = (ctypes.c_double * 3)(1, 1, 1)
    rc = lib.paro_mesh_create(ctypes.byref(h), 1, 4, 4, lo, hi, 0, None)
    assert rc == -1 and "cells per axis" in B.paro_last_error(None)
    rc = lib.paro_mesh_create(ctypes.byref(h), 4, 4, 4, hi, lo, 0, None)
    assert rc == -1 and "lo < hi" in B.paro_last_error(None)
    rc = lib.paro_mesh_create(ctypes.byref(h), 4, 4, 4, lo, hi, 7, None)
    assert rc == -1
    assert lib.paro_mesh_destroy(None) == -1
    assert lib.paro_iterate(None, 1, None, None, None, None) == -1


def test_ctypes_structs_match_c_layout(lib):
    from paper_1405_0260_gb300 import binding as B

    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "paro.h"
int main(void) {
  printf("%zu %zu\n", sizeof(paro_params), sizeof(paro_stats));
  printf("%zu %zu %zu %zu\n", offsetof(paro_params, profile), offsetof(paro_stats, prof_ms),
         offsetof(paro_stats, prof_dof_orb), offsetof(paro_params, hartree_precond));
  printf("%zu %zu\n", offsetof(paro_params, wait_polls), offsetof(paro_stats, prof_dof_orb_active));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-I", os.path.dirname(HEADER), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    sizes = [int(v) for v in out]
    assert sizes[0] == ctypes.sizeof(B.paro_params)
    assert sizes[1] == ctypes.sizeof(B.paro_stats)
    assert sizes[2] == B.paro_params.profile.offset
    assert sizes[3] == B.paro_stats.prof_ms.offset
    assert sizes[4] == B.paro_stats.prof_dof_orb.offset
    assert sizes[5] == B.paro_params.hartree_precond.offset
    assert sizes[6] == B.paro_params.wait_polls.offset
    assert sizes[7] == B.paro_stats.prof_dof_orb_active.offset


def test_host_side_argument_checks_need_no_gpu(lib):
    # every one of these is rejected before any CUDA call, so it runs on a host
    # without a GPU; the batch calls keep their own host-side bookkeeping
    from paper_1405_0260_gb300 import binding as B

    assert B.paro_small_eig_static(0, 1, 1, 1, 1) == -1  # PARO_ERR_ARG
    assert B.paro_small_eig_static(129, 1, 1, 1, 1) == -1  # PARO_ERR_ARG
    assert B.paro_small_eig_static(4, 0, 1, 1, 1) == -1  # PARO_ERR_ARG
    b = ctypes.c_void_p()
    assert lib.paro_batch_create(ctypes.byref(b), 0) == -1
    assert lib.paro_batch_create(ctypes.byref(b), 257) == -1
    assert lib.paro_batch_create(ctypes.byref(b), 4) == 0
    assert lib.paro_batch_size(b) == 0
    assert lib.paro_batch_add(b, None, 4, None, None, None) == -1  # no handle
    rc = (ctypes.c_int * 1)()
    assert lib.paro_batch_iterate(b, rc, None) == 0  # an empty batch has nothing to do
    assert lib.paro_batch_iterate(None, rc, None) == -1
    assert lib.paro_batch_destroy(b) == 0
    assert lib.paro_batch_size(None) == -1
    assert lib.paro_interior_nodes(None) == -1
    assert lib.paro_set_potential(None, None, 0.0) == -1
    assert lib.paro_ks_density_in(None, None) == -1
    assert lib.paro_orbital_solve(None, 1, None, None, None, None, None) == -1
    assert lib.paro_rayleigh_ritz(None, 1, None, None, None, None) == -1
    # graded meshes: node coordinates must be finite and strictly increasing (checked on the host)
    h = ctypes.c_void_p()
    ok = (ctypes.c_double * 4)(0.0, 1.0, 2.0, 3.0)
    bad = (ctypes.c_double * 4)(0.0, 1.0, 1.0, 3.0)
    lib.paro_mesh_create_graded.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                            ctypes.c_void_p]
    assert lib.paro_mesh_create_graded(ctypes.byref(h), 3, 3, 3, ok, bad, ok, 0, None) == -1
    assert "strictly increasing" in B.paro_last_error(None)
    assert lib.paro_mesh_create_graded(ctypes.byref(h), 1, 3, 3, ok, ok, ok, 0, None) == -1
    assert lib.paro_mesh_create_graded(ctypes.byref(h), 3, 3, 3, None, ok, ok, 0, None) == -1
    t = ctypes.c_double(0.0)
    assert lib.paro_peak_fma(7, 1, ctypes.c_void_p(1), ctypes.byref(t), None) == -1  # unknown dtype
    assert lib.paro_peak_fma(0, 0, ctypes.c_void_p(1), ctypes.byref(t), None) == -1  # iters < 1


def test_binding_fails_loudly_without_the_library():
    # the package has no CPU fallback: with the library absent, loading it raises
    code = (
        "import sys; sys.path.insert(0, %r)\n"
        "from paper_1405_0260_gb300 import binding as B\n"
        "B.LIB_PATH = '/nonexistent/libparo.so'\n"
        "try:\n"
        "    B.lib()\n"
        "except RuntimeError as e:\n"
        "    print('raised', 'no CPU fallback' in str(e))\n" % ROOT
    )
    out = subprocess.run(["python", "-c", code], capture_output=True, text=True, timeout=120).stdout
    assert out.strip() == "raised True", out


def declared_arity():
    """{name: parameter count} of every function paro.h declares."""
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    out = {}
    for m in re.finditer(DECL + r"\(([^)]*)\)\s*;", text, flags=re.M | re.S):
        params = m.group(2).strip()
        out[m.group(1)] = 0 if params in ("", "void") else params.count(",") + 1
    return out


def test_binding_argument_lists_match_the_header(lib):
    from paper_1405_0260_gb300 import binding as B

    B.paro_small_eig_static(0, 1, 1, 1, 1)  # sets that function's argtypes (rejected: N = 0)
    arity = declared_arity()
    assert set(arity) == set(declared_functions())
    checked = 0
    for name, n in arity.items():
        argtypes = getattr(lib, name).argtypes
        if argtypes is not None:
            assert len(argtypes) == n, (name, len(argtypes), n)
            checked += 1
    assert checked >= len(arity) - 1  # every entry point the binding calls


def test_binding_constants_match_the_header():
    from paper_1405_0260_gb300 import binding as B

    text = open(HEADER).read()
    defines = {k: int(v) for k, v in re.findall(r"^#define\s+(PARO_\w+)\s+(-?\d+)", text, flags=re.M)}
    enum = {k: int(v) for k, v in re.findall(r"^\s*(PARO_(?:OK|ERR_\w+))\s*=\s*(-?\d+)", text, flags=re.M)}
    assert len(enum) == 9 and enum["PARO_OK"] == B.PARO_OK
    assert {v: k for k, v in enum.items()} == B.STATUS
    shared = [k for k in defines if hasattr(B, k)]
    assert len(shared) >= 10, shared
    for k in shared:
        assert getattr(B, k) == defines[k], k


def test_mesh_creation_without_a_gpu_returns_an_error(lib):
    # on a host without a usable GPU the library reports the CUDA failure through
    # its status and message: there is no host fallback to fall into
    from paper_1405_0260_gb300 import binding as B

    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    lo = (ctypes.c_double * 3)(-1, -1, -1)
    hi = (ctypes.c_double * 3)(1, 1, 1)
    rc = lib.paro_mesh_create(ctypes.byref(h), 4, 4, 4, lo, hi, 0, None)
    assert rc in (-2, -7) and h.value is None  # PARO_ERR_CUDA or PARO_ERR_OOM, no handle
    assert "cuda" in B.paro_last_error(None).lower()


def test_create_error_message_is_per_thread(lib):
    # two host threads whose creations fail for different reasons each read their own message
    import threading

    from paper_1405_0260_gb300 import binding as B

    lo = (ctypes.c_double * 3)(-1, -1, -1)
    hi = (ctypes.c_double * 3)(1, 1, 1)
    cases = {"cells": (1, lo, hi, "cells per axis"), "box": (4, hi, lo, "lo < hi")}
    seen = {}
    barrier = threading.Barrier(2)

    def run(name):
        n, a, b, want = cases[name]
        ok = True
        for _ in range(200):
            h = ctypes.c_void_p()
            rc = lib.paro_mesh_create(ctypes.byref(h), n, 4, 4, a, b, 0, None)
            if _ == 0:
                barrier.wait()
            ok &= rc == -1 and want in B.paro_last_error(None)
        seen[name] = ok

    ts = [threading.Thread(target=run, args=(k,)) for k in cases]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    assert seen == {"cells": True, "box": True}


def test_c_example_compiles_and_links_against_the_library(lib):
    # the C usage example stays in step with the header and the exports
    from paper_1405_0260_gb300 import binding as B

    c = os.path.join(ROOT, "tests", "abi_example.c")
    with tempfile.TemporaryDirectory() as d:
        so = os.path.join(d, "libex.so")
        subprocess.run(["gcc", "-shared", "-fPIC", "-Wall", "-Werror", "-I", os.path.dirname(HEADER), c, "-o", so,
                        "-L", os.path.dirname(B.LIB_PATH), "-lparo", "-Wl,--no-undefined", "-lm"],
                       check=True, capture_output=True, timeout=120)


def test_product_package_never_reaches_the_oracle():
    # the oracle is test infrastructure: the package and its CUDA sources neither
    # import nor include anything of it
    pkg = os.path.join(ROOT, "paper_1405_0260_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            path = os.path.join(dirpath, f)
            if f.endswith(".py"):
                text = open(path).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", text, flags=re.M), path
            elif f.endswith((".cu", ".cuh", ".h")):
                text = open(path).read()
                assert not re.search(r'#include\s+[<"][^>"]*oracle', text), path
