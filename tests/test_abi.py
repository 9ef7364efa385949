"""Host-side checks of the C ABI (no GPU): the library loads, exports every symbol the
header declares, returns the Figure 1 / Figure 2 tables, and rejects bad arguments on
the host before any CUDA work."""
import ctypes
import os
import re

import pytest

import paper_1605_01078_gb300 as sg
from paper_1605_01078_gb300 import _binding
from oracle import tables

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"^\s*(?:STRASSEN_API\s+)?(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+\**([a-z_][a-z0-9_]*)\s*\(",
                             src, flags=re.M):
            names.append(m.group(1))
    return names


def test_library_exports_every_declared_symbol():
    lib = sg.load_library()
    names = declared_functions()
    assert "strassen_gemm" in names and "classical_gemm" in names
    for name in names:
        assert hasattr(lib, name), name
        assert name in _binding.SIGNATURES, f"binding lacks {name}"


@pytest.mark.parametrize("levels", [0, 1, 2, 3])
def test_plan_table_matches_oracle_tables(levels):
    assert sg.strassen_plan_table(levels) == tables.table(levels)


def test_plan_table_rejects_levels():
    with pytest.raises(sg.StrassenError):
        sg.strassen_plan_table(4)


P = 0x1000  # a non-null dummy pointer: these calls must fail before touching it


@pytest.mark.parametrize("args,status", [
    ((-1, 4, 4, P, 4, P, 4, P, 4), -1),
    ((4, 4, 4, 0, 4, P, 4, P, 4), -3),
    ((4, 4, 4, P, 3, P, 4, 2 * P, 4), -2),
    ((4, 4, 4, P, 4, P, 3, 2 * P, 4), -2),
    ((4, 4, 4, P, 4, P, 4, 2 * P, 3), -2),
    ((4, 4, 4, P, 4, 3 * P, 4, P + 8, 4), -9),   # C overlaps A
    ((0, 4, 4, 0, 4, 0, 4, 0, 4), 0),             # empty: no-op
    ((4, 4, 0, 0, 0, 0, 4, 0, 4), 0),
])
def test_argument_checks(args, status):
    st = sg.strassen_gemm(*args, 1, sg.STRASSEN_ABC, sg.STRASSEN_F64, 0)
    assert st == status, sg.strassen_status_string(st)
    st2 = sg.classical_gemm(*args, 0)
    assert st2 == status


def test_levels_and_enums_checked():
    a = (4, 4, 4, P, 4, 2 * P, 4, 3 * P, 4)
    assert sg.strassen_gemm(*a, 4, 0, 0, 0) == -4
    assert sg.strassen_gemm(*a, -2, 0, 0, 0) == -4
    assert sg.strassen_gemm(*a, 1, 7, 0, 0) == -5
    assert sg.strassen_gemm(*a, 1, 0, 9, 0) == -5


def test_workspace_sizes():
    f = sg.strassen_workspace_size
    assert f(1024, 1024, 1024, 1, sg.STRASSEN_ABC, 0) == 0
    assert f(1024, 1024, 1024, 0, sg.STRASSEN_AB, 0) == 0
    assert f(1024, 1024, 1024, 1, sg.STRASSEN_AB, 0) == 8 * 512 * 512
    assert f(1000, 998, 7, 2, sg.STRASSEN_NAIVE, 0) == 8 * (250 * 2 + 2 * 250 + 250 * 250)
    # hybrid: the outer blocks of the L-level partition, 2^(L-1) ceil(d / 2^L)
    assert f(1000, 998, 7, 2, sg.STRASSEN_HYBRID, 0) == 8 * (2 * 250) * (2 * 250)
    assert f(1001, 999, 64, 3, sg.STRASSEN_HYBRID, 0) == 8 * (4 * 126) * (4 * 125)
    assert f(1024, 1024, 1024, 1, sg.STRASSEN_HYBRID, 0) == 8 * 512 * 512
    assert f(-1, 4, 4, 1, 0, 0) == -1
    assert f(4, 4, 4, 5, 0, 0) == -4
    assert f(4, 4, 4, 1, 5, 0) == -5


def test_status_strings():
    assert sg.strassen_status_string(0) == "ok"
    assert "dimension" in sg.strassen_status_string(-1)
    assert sg.strassen_status_string(12345) == "unknown status"


def test_select_fixed_rule_without_model():
    lv, var, tile = sg.strassen_select(8192, 8192, 8192, 0)
    assert lv in (0, 1, 2, 3) and var in (0, 1, 2) and tile >= 0


def test_analytic_model_counts():
    """The analytic model's arithmetic terms (Section 4.2's T_a restated for the GPU
    tile): on tile-aligned sizes the products cost 7/8 (one level) and 49/64 (two
    levels) of the classical multiply-adds, plus the staging additions."""
    f = sg.strassen_model_seconds
    n = 8192
    t0 = f(n, n, n, 0, sg.STRASSEN_ABC)
    fma_rate = 2.0 * 152 * 2.07e9
    assert abs(t0 - (n ** 3 / fma_rate + 4e-6)) / t0 < 1e-9
    t1 = f(n, n, n, 1, sg.STRASSEN_ABC)
    t2 = f(n, n, n, 2, sg.STRASSEN_ABC)
    # ABC one level: 7 products of (n/2)^3 FMAs; its staging sums run on the integer pipe
    fma1 = 7 * (n // 2) ** 3
    assert abs(t1 - (fma1 / fma_rate + 4e-6)) / t1 < 1e-9
    assert t2 < t1 < t0
    # Naive pays FP64 additions, extra memory passes and launches on top of the products
    assert f(n, n, n, 2, sg.STRASSEN_NAIVE) > t2
    assert f(256, 256, 256, 2, sg.STRASSEN_NAIVE) > f(256, 256, 256, 0, sg.STRASSEN_ABC)
    assert f(0, 4, 4, 1, 0) == -1.0


def test_dgemm_argument_checks_on_the_host():
    """strassen_dgemm rejects bad transposes, leading dimensions that do not cover the
    stored (transposed) operands, and overlaps, before any CUDA work."""
    f = sg.strassen_dgemm
    assert f(2, 0, 8, 4, 4, 1.0, P, 8, 2 * P, 4, 1.0, 3 * P, 4, 1, 0, 0, 0) == -9
    assert f(1, 0, 8, 4, 4, 1.0, P, 4, 2 * P, 4, 1.0, 3 * P, 4, 1, 0, 0, 0) == -2   # A^T is 4 x 8: lda >= 8
    assert f(0, 1, 8, 4, 6, 1.0, P, 6, 2 * P, 4, 1.0, 3 * P, 4, 1, 0, 0, 0) == -2   # B^T is 4 x 6: ldb >= 6
    assert f(0, 0, 4, 4, 4, 1.0, P, 4, 2 * P, 4, 1.0, P + 8, 4, 1, 0, 0, 0) == -9   # C overlaps A
    assert f(0, 0, -1, 4, 4, 1.0, P, 4, 2 * P, 4, 1.0, 3 * P, 4, 1, 0, 0, 0) == -1
    assert f(0, 0, 0, 4, 4, 1.0, 0, 4, 0, 4, 1.0, 0, 4, 1, 0, 0, 0) == 0             # empty: no-op
    assert f(0, 0, 4, 4, 4, 1.0, P, 4, 2 * P, 4, 1.0, 3 * P, 4, 5, 0, 0, 0) == -4


def test_dgemm_ex_flags_checked_on_the_host():
    """strassen_dgemm_ex takes only the flags it defines; its argument checks are those
    of strassen_dgemm."""
    f = sg.strassen_dgemm_ex
    assert sg.STRASSEN_FLAG_DETERMINISTIC == 1
    assert f(0, 0, 4, 4, 4, 1.0, P, 4, 2 * P, 4, 1.0, 3 * P, 4, 1, 0, 0, 2, 0) == -9
    assert f(0, 0, 4, 4, 4, 1.0, P, 4, 2 * P, 4, 1.0, 3 * P, 4, 1, 0, 0, 0x80000000, 0) == -9
    assert f(0, 0, -1, 4, 4, 1.0, P, 4, 2 * P, 4, 1.0, 3 * P, 4, 1, 0, 0, 1, 0) == -1
    assert f(1, 0, 8, 4, 4, 1.0, P, 4, 2 * P, 4, 1.0, 3 * P, 4, 1, 0, 0, 1, 0) == -2
    assert f(0, 0, 0, 4, 4, 1.0, 0, 4, 0, 4, 1.0, 0, 4, 1, 0, 0, 1, 0) == 0


def test_batched_rejects_unfused_variants_on_the_host():
    """A batched problem asking for AB or Naive with one or more levels is refused
    (the persistent launch runs the fused form only); no device work is attempted."""
    for variant, levels in ((sg.STRASSEN_AB, 1), (sg.STRASSEN_NAIVE, 2), (sg.STRASSEN_AB, -1)):
        arr = (sg.strassen_problem * 1)()
        arr[0] = sg.strassen_problem(8, 8, 8, P, 2 * P, 3 * P, 8, 8, 8, levels, variant)
        assert sg.strassen_gemm_batched(1, arr, 0, 0) == -5


def test_dsyrk_argument_checks_on_the_host():
    f = sg.strassen_dsyrk
    assert f(2, 0, 8, 4, 1.0, P, 4, 1.0, 2 * P, 8, 1, 0, 0) == -9        # uplo
    assert f(0, 2, 8, 4, 1.0, P, 4, 1.0, 2 * P, 8, 1, 0, 0) == -9        # trans
    assert f(0, 0, 8, 4, 1.0, P, 4, 1.0, 2 * P, 8, 1, 4, 0) == -9        # flags
    assert f(0, 0, -1, 4, 1.0, P, 4, 1.0, 2 * P, 8, 1, 0, 0) == -1
    assert f(0, 0, 8, 4, 1.0, P, 3, 1.0, 2 * P, 8, 1, 0, 0) == -2        # lda < k
    assert f(0, 1, 8, 4, 1.0, P, 4, 1.0, 2 * P, 8, 1, 0, 0) == -2        # A stored 4 x 8: lda >= 8
    assert f(0, 0, 8, 4, 1.0, P, 4, 1.0, 2 * P, 7, 1, 0, 0) == -2        # ldc < n
    assert f(0, 0, 8, 4, 1.0, P, 4, 1.0, P + 8, 8, 1, 0, 0) == -9        # C overlaps A
    assert f(0, 0, 8, 4, 1.0, P, 4, 1.0, 2 * P, 8, 4, 0, 0) == -4
    assert f(0, 0, 0, 4, 1.0, 0, 4, 1.0, 0, 8, 1, 0, 0) == 0             # empty


def test_plain_c_client_compiles_and_runs(tmp_path):
    """The header is plain C (extern "C", C types only): a C99 program includes it, links
    the library and calls its host-side entry points."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("needs gcc")
    sg.load_library()
    libdir = os.path.dirname(_binding.LIB_PATH)
    exe = tmp_path / "abi_client"
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                           os.path.join(ROOT, "tests", "native", "abi_client.c"), "-o", str(exe),
                           "-L", libdir, "-lstrassen_gb300", f"-Wl,-rpath,{libdir}"])
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and "abi client ok" in r.stdout, r.stdout + r.stderr
