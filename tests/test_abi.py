"""CPU checks of the C ABI: the library builds, loads and exports every symbol
declared in include/su3.h, and host-side argument validation rejects bad input
before any CUDA call.  No compute call is made here (no GPU in this
environment)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import paper_0904_1179_gb300 as su3
from paper_0904_1179_gb300 import build as su3_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    su3_build.build()
    return su3.load_library()


def declared_symbols():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            names += re.findall(r"^SU3_API\s+[\w\s\*]+?\b(su3_\w+)\s*\(", text, flags=re.M)
    return names


def test_every_declared_symbol_is_exported(lib):
    names = declared_symbols()
    assert len(names) >= 16
    out = subprocess.run(["nm", "-D", "--defined-only", su3.library_path()], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (su3_\w+)$", out, flags=re.M))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    # the binding wraps exactly the declared entry points
    assert sorted(n for n, _, _ in su3.EXPORTS) == sorted(names)


def test_version(lib):
    assert "sm_103a" in su3.su3_version()


def _create(lib, dims, beta=5.7, start=0, prec=0):
    h = ctypes.c_void_p()
    rc = lib.su3_create_ex(*dims, beta, 1, start, prec, None, ctypes.byref(h))
    return rc, h


@pytest.mark.parametrize("dims", [(4, 4, 4, 5), (3, 4, 4, 4), (0, 4, 4, 4), (4, 4, -2, 4)])
def test_create_rejects_bad_extents(lib, dims):
    rc, h = _create(lib, dims)
    assert rc == su3.SU3_EINVAL and not h.value
    assert "extent" in su3.su3_last_error()


def test_create_rejects_oversized_volume(lib):
    rc, _ = _create(lib, (256, 256, 256, 256))
    assert rc == su3.SU3_EINVAL and "2^31" in su3.su3_last_error()


@pytest.mark.parametrize("beta", [0.0, -1.0, float("inf"), float("nan")])
def test_create_rejects_bad_beta(lib, beta):
    rc, _ = _create(lib, (4, 4, 4, 4), beta=beta)
    assert rc == su3.SU3_EINVAL and "beta" in su3.su3_last_error()


def test_create_rejects_bad_enums(lib):
    assert _create(lib, (4, 4, 4, 4), start=2)[0] == su3.SU3_EINVAL
    assert _create(lib, (4, 4, 4, 4), prec=7)[0] == su3.SU3_EINVAL
    assert lib.su3_create_ex(4, 4, 4, 4, 5.7, 1, 0, 0, None, None) == su3.SU3_EINVAL


@pytest.mark.parametrize("args", [(0, 2, 1), (5, 2, 1), (1, 0, 1), (1, 2, 0), (3, 4, 1), (2, 3, 1), (1, 2, 2)])
def test_decomp_create_rejects_bad_decompositions(lib, args):
    # ndmpi out of range, mpifactor < 1, exchange off with several
    # sublattices, parts of odd extent (12 / 4 = 3) or not dividing (8 / 3)
    h = ctypes.c_void_p()
    rc = lib.su3_decomp_create(8, 8, 12, 8, 5.7, 1, 0, 0, *args, None, ctypes.byref(h))
    assert rc == su3.SU3_EINVAL and not h.value
    assert "su3_decomp_create" in su3.su3_last_error()


def test_null_handle_calls(lib):
    assert lib.su3_destroy(None) == su3.SU3_OK
    assert lib.su3_sweep(None, 1) == su3.SU3_EINVAL
    assert lib.su3_half_sweep(None, 0, 0) == su3.SU3_EINVAL
    assert lib.su3_links_get(None, None, 0) == su3.SU3_EINVAL
    assert lib.su3_links_set(None, None, 0) == su3.SU3_EINVAL
    assert lib.su3_set_sweep_count(None, 0) == su3.SU3_EINVAL
    assert lib.su3_set_block_size(None, 64) == su3.SU3_EINVAL
    assert lib.su3_set_lanes(None, 1) == su3.SU3_EINVAL
    assert lib.su3_set_schedule(None, su3.SU3_SCHED_PHASES) == su3.SU3_EINVAL
    assert lib.su3_get_schedule(None, None) == su3.SU3_EINVAL
    assert lib.su3_sweep_debug(None, 1.0, -1) == su3.SU3_EINVAL
    # the product build has no bounds checks compiled in
    v = ctypes.c_uint(7)
    assert lib.su3_bounds_status(ctypes.byref(v), 0) == su3.SU3_EINVAL
    assert "without bounds checks" in su3.su3_last_error()
    v = lib.su3_plaquette(None)
    assert v != v


def test_binding_has_no_fallback_and_no_oracle():
    # the product path never imports the oracle
    pkg = os.path.join(ROOT, "paper_0904_1179_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, fn)).read()
                assert "import oracle" not in text and "su3_oracle" not in text, fn


def _halo_sites(L, nd, nf):
    """Ghost cells the staples read: both faces of every cut direction and the
    x + a - b edge of every ordered pair of cut directions, per sublattice."""
    l = [L[d] // nf if d < nd else L[d] for d in range(4)]
    vol = int(np.prod(l))
    faces = sum(2 * vol // l[d] for d in range(nd))
    edges = sum(vol // (l[a] * l[b]) for a in range(nd) for b in range(nd) if a != b)
    return (faces + edges) * nf ** nd


@pytest.mark.parametrize("L", [(8, 8, 8, 8), (12, 12, 12, 12), (16, 16, 16, 16), (8, 4, 12, 8), (32, 32, 32, 32)])
def test_decomp_plan_matches_closed_form(lib, L):
    # host-only: the gather lists of the boundary exchange, counted
    for nd in range(1, 5):
        for nf in (1, 2, 4):
            if any(L[d] % nf or (L[d] // nf) % 2 for d in range(nd)):
                with pytest.raises(su3.Su3Error):
                    su3.su3_decomp_plan(L, nd, nf)
                continue
            nsub, halo = su3.su3_decomp_plan(L, nd, nf)
            assert nsub == nf ** nd
            assert halo == 4 * _halo_sites(L, nd, nf), (L, nd, nf)
    assert su3.su3_decomp_plan(L, 1, 1, 0) == (1, 0)


def test_c_program_on_the_abi(lib, tmp_path):
    # the header compiles as C, and a C program linked against libsu3.so runs
    # the calls that need no GPU
    import shutil
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    libdir = os.path.dirname(su3._LIB_PATH)
    exe = str(tmp_path / "c_abi_host")
    src = os.path.join(os.path.dirname(__file__), "c_abi_host.c")
    inc = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include")
    subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", inc, src, "-L", libdir, "-lsu3", "-Wl,-rpath," + libdir,
                    "-o", exe], check=True)
    r = subprocess.run([exe], capture_output=True, text=True)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    assert "c abi ok" in r.stdout
