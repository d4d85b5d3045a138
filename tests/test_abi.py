"""The C-ABI library loads and exports every symbol include/bmm.h declares
(no compute calls: these run without a GPU)."""
import os
import re
import subprocess

import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "bmm.h")
LIB = os.path.join(ROOT, "paper_1909_01554_gb300", "libbmm.so")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(bmm_[a-z0-9_]+)\s*\(",
                       src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def built_lib():
    if not os.path.exists(LIB):
        from paper_1909_01554_gb300 import build

        build.build()
    return LIB


def test_header_declares_the_product_calls():
    names = declared_functions()
    for required in ("bmm_gf2", "bmm_bool", "bmm_gf2_batched", "bmm_bool_batched",
                     "bmm_base_product", "bmm_transpose", "bmm_basis_change"):
        assert required in names


def test_library_exports_every_declared_symbol(built_lib):
    out = subprocess.run(["nm", "-D", "--defined-only", built_lib], capture_output=True,
                         text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, missing


def test_library_loads_and_binding_names_match(built_lib):
    import paper_1909_01554_gb300 as bmm

    L = bmm.lib()
    for name in declared_functions():
        assert hasattr(L, name)
    assert set(bmm.EXPORTED) <= set(declared_functions())
    assert L.bmm_status_string(bmm.ERR_TIMEOUT) == b"BMM_ERR_TIMEOUT"


def test_argument_checks_need_no_gpu(built_lib):
    """Invalid sizes and null pointers are rejected before any CUDA call."""
    import paper_1909_01554_gb300 as bmm

    L = bmm.lib()
    assert L.bmm_gf2(0, 0, 0, 64, 64, 64, None) == bmm.ERR_INVALID
    assert L.bmm_gf2(16, 32, 4096, 100, 64, 64, None) == bmm.ERR_INVALID
    assert L.bmm_bool(16, 32, 4096, 64, 0, 64, None) == bmm.ERR_INVALID
    assert L.bmm_gf2(8, 32 << 20, 64 << 20, 64, 64, 64, None) == bmm.ERR_ALIGN
    # C overlapping A
    assert L.bmm_gf2(1 << 20, 32 << 20, (1 << 20) + 256, 64, 64, 64, None) == bmm.ERR_INVALID
    assert L.bmm_transpose(0, 16, 64, 64, None) == bmm.ERR_INVALID
    assert L.bmm_basis_change(1, 0, 16, 96, 128, 1, None) == bmm.ERR_INVALID
    assert L.bmm_basis_change(7, 0, 16, 128, 128, 1, None) == bmm.ERR_INVALID


def test_autotune_argument_checks_need_no_gpu(built_lib):
    """The autotuner rejects bad operations, sizes and flags before any CUDA call."""
    import ctypes

    import paper_1909_01554_gb300 as bmm

    L = bmm.lib()
    r = bmm.TuneResult()
    assert L.bmm_autotune(2, 64, 64, 64, 0, None, ctypes.byref(r)) == bmm.ERR_INVALID
    assert L.bmm_autotune(0, 96, 64, 64, 0, None, ctypes.byref(r)) == bmm.ERR_INVALID
    assert L.bmm_autotune(1, 64, 0, 64, 0, None, ctypes.byref(r)) == bmm.ERR_INVALID
    assert L.bmm_autotune(0, 64, 64, 64, 4, None, ctypes.byref(r)) == bmm.ERR_INVALID
    assert L.bmm_autotune(0, 64, 64, 64, 0, None, None) == bmm.ERR_INVALID
    L.bmm_autotune_clear()


def test_batched_plan_argument_checks_need_no_gpu(built_lib):
    """A batch plan rejects an unknown base-case path, a null plan pointer and
    bad problem sizes before any CUDA call; the 8-bit integer path does not
    exist on sm_103a."""
    import ctypes

    import paper_1909_01554_gb300 as bmm

    L = bmm.lib()
    one = lambda t, v: (t * 1)(v)  # noqa: E731
    ops = one(ctypes.c_int32, 0)
    ptr = one(ctypes.c_void_p, 1 << 20)
    sz = one(ctypes.c_int64, 64)
    bad = one(ctypes.c_int64, 96)
    h = ctypes.c_void_p(0)
    args = (1, ops, ptr, ptr, ptr, sz, sz, sz)
    assert L.bmm_batched_plan_create_ex(*args, 99, ctypes.byref(h)) == bmm.ERR_INVALID
    assert L.bmm_batched_plan_create_ex(*args, -1, ctypes.byref(h)) == bmm.ERR_INVALID
    assert L.bmm_batched_plan_create_ex(*args, bmm.PATH_TC_I8,
                                        ctypes.byref(h)) == bmm.ERR_UNSUPPORTED
    assert L.bmm_batched_plan_create_ex(*args, bmm.PATH_AUTO, None) == bmm.ERR_INVALID
    assert L.bmm_batched_plan_create_ex(1, ops, ptr, ptr, ptr, bad, sz, sz, bmm.PATH_AUTO,
                                        ctypes.byref(h)) == bmm.ERR_INVALID
    assert h.value is None
    p = ctypes.c_int32(0)
    assert L.bmm_batched_plan_path(None, ctypes.byref(p)) == bmm.ERR_INVALID


def test_host_product_argument_checks_need_no_gpu(built_lib):
    """Host-memory products reject bad sizes, null, misaligned and overlapping
    arrays, host Strassen levels for the Boolean product and bad options
    before any CUDA call."""
    import ctypes

    import numpy as np

    import paper_1909_01554_gb300 as bmm

    L = bmm.lib()
    A = np.zeros(64 * 64 // 64 + 2, dtype=np.uint64)
    a = A.ctypes.data
    o = bmm.host_opts(device_bytes=1 << 30)
    ob = bmm.host_opts(device_bytes=1 << 30, host_depth=1)
    for f in (L.bmm_gf2_host, L.bmm_bool_host):
        assert f(a, a, 0, 64, 64, 64, ctypes.byref(o), None) == bmm.ERR_INVALID
        assert f(a, a, a + 4096, 96, 64, 64, ctypes.byref(o), None) == bmm.ERR_INVALID
        assert f(a + 8, a, a + 4096, 64, 64, 64, ctypes.byref(o), None) == bmm.ERR_ALIGN
        assert f(a, a, a, 64, 64, 64, ctypes.byref(o), None) == bmm.ERR_INVALID  # C overlaps A
    assert L.bmm_bool_host(a, a, a + 4096, 64, 64, 64, ctypes.byref(ob), None) == bmm.ERR_INVALID
    bad = bmm.host_opts(device_bytes=1 << 30, host_depth=-2)
    assert L.bmm_gf2_host(a, a, a + 4096, 64, 64, 64, ctypes.byref(bad), None) == bmm.ERR_INVALID
    info = bmm.HostPlanInfo()
    assert L.bmm_host_plan(2, 64, 64, 64, ctypes.byref(o), ctypes.byref(info)) == bmm.ERR_INVALID
    assert L.bmm_host_plan(0, 64, 64, 64, ctypes.byref(o), None) == bmm.ERR_INVALID


def test_kernel_level_plans_need_no_gpu(built_lib):
    """With the innermost Strassen level inside the CUDA-core kernel, the XOR
    passes run one level fewer: the plan's scratch is that of the plan one
    level shallower (no leaf operands or products of the last level), its
    depth-first levels are capped one lower, and the option is refused where
    it cannot apply."""
    import paper_1909_01554_gb300 as bmm

    m = k = n = 8192
    for d in (1, 2, 3, 4):
        kl = bmm.plan(bmm.GF2, m, k, n, path=bmm.PATH_POPC, depth=d, kernel_level=1)
        assert kl["kernel_level"] == 1 and kl["strassen_depth"] == d
        assert kl["leaves"] == 7 ** d
        flat = bmm.plan(bmm.GF2, m, k, n, path=bmm.PATH_POPC, depth=d - 1,
                        serial=kl["serial_depth"])
        assert kl["workspace_bytes"] == flat["workspace_bytes"]
        assert kl["serial_depth"] <= d - 1
        # the same depth-first split with every level in XOR passes needs more
        whole = bmm.plan(bmm.GF2, m, k, n, path=bmm.PATH_POPC, depth=d,
                         serial=kl["serial_depth"])
        assert whole["kernel_level"] == 0
        if whole["serial_depth"] == kl["serial_depth"]:  # else XOR passes merge too few
            assert kl["workspace_bytes"] < whole["workspace_bytes"]
    # depth 1: the only scratch is B^T
    assert bmm.plan(bmm.GF2, m, k, n, path=bmm.PATH_POPC, depth=1,
                    kernel_level=1)["workspace_bytes"] == k * n // 8
    # nothing to move: cubic plans and the Boolean product ignore it
    assert bmm.plan(bmm.GF2, m, k, n, path=bmm.PATH_POPC, depth=0,
                    kernel_level=1)["kernel_level"] == 0
    assert bmm.plan(bmm.BOOL, m, k, n, path=bmm.PATH_POPC, kernel_level=1)["kernel_level"] == 0
    L = bmm.lib()
    info = bmm.PlanInfo()
    for bad in (-1, 2):
        o = bmm.opts(path=bmm.PATH_POPC, depth=2, kernel_level=bad)
        assert L.bmm_plan(bmm.GF2, m, k, n, ctypes_ref(o), ctypes_ref(info)) == bmm.ERR_INVALID
    # every depth-first level would leave none for the kernel
    o = bmm.opts(path=bmm.PATH_POPC, depth=2, serial=2, kernel_level=1)
    assert L.bmm_plan(bmm.GF2, m, k, n, ctypes_ref(o), ctypes_ref(info)) == bmm.ERR_INVALID
    # the e4m3 tensor kernels have no in-kernel level (the e2m1 SM-pair kernel
    # has one, where the device has that path)
    for path in bmm.TENSOR_PATHS:
        if path == bmm.PATH_TC_FP4_PAIR and bmm.device_supported():
            continue
        o = bmm.opts(path=path, depth=2, kernel_level=1)
        assert L.bmm_plan(bmm.GF2, m, k, n, ctypes_ref(o),
                          ctypes_ref(info)) == bmm.ERR_UNSUPPORTED


def ctypes_ref(x):
    import ctypes

    return ctypes.byref(x)


def test_batched_plan_arguments_need_no_gpu(built_lib):
    """Per-problem path requests and the plan queries are checked before any
    CUDA call: unknown paths, two different tensor paths in one plan, the
    integer tensor path sm_103a lacks, null plans and out-of-range problems."""
    import ctypes

    import paper_1909_01554_gb300 as bmm

    L = bmm.lib()
    a = 1 << 20  # never dereferenced: every case fails its argument checks first
    P = ctypes.c_void_p * 2
    I64 = ctypes.c_int64 * 2
    I32 = ctypes.c_int32 * 2
    ops, A, B, C = I32(0, 1), P(a, a), P(a, a), P(a + 4096, a + 8192)
    sz = I64(64, 64)
    h = ctypes.c_void_p(0)
    for paths, want in (((9, bmm.PATH_AUTO), bmm.ERR_INVALID),
                        ((bmm.PATH_TC_FP4_PAIR, bmm.PATH_TC_FP8_PAIR), bmm.ERR_INVALID),
                        ((bmm.PATH_TC_I8, bmm.PATH_POPC), bmm.ERR_UNSUPPORTED)):
        assert L.bmm_batched_plan_create_paths(2, ops, A, B, C, sz, sz, sz, I32(*paths),
                                               ctypes.byref(h)) == want
        assert not h.value
    assert L.bmm_batched_plan_create_paths(2, ops, A, B, C, sz, sz, sz, None,
                                           ctypes.byref(h)) == bmm.ERR_INVALID
    assert L.bmm_batched_plan_create_paths(2, ops, A, B, C, I64(64, 100), sz, sz,
                                           I32(0, 0), ctypes.byref(h)) == bmm.ERR_INVALID
    assert L.bmm_batched_plan_choice(None, 0, ctypes.byref(bmm.BatchedChoice())) == bmm.ERR_INVALID
    assert L.bmm_batched_plan_stats(None, ctypes.byref(bmm.BatchedStats())) == bmm.ERR_INVALID
    assert L.bmm_batched_model(9, ctypes.byref(bmm.BatchedModel())) == bmm.ERR_INVALID
    assert L.bmm_batched_model(bmm.PATH_TC_I8, ctypes.byref(bmm.BatchedModel())) == \
        bmm.ERR_UNSUPPORTED


def test_plan_pass_bytes_closed_form(built_lib):
    """The plan's streaming bytes against the closed form of a breadth-first
    plan (Secs. 3.9 and 3.11 with d levels merged): the transpose reads and
    writes k n / 8; each operand's expansion reads its matrix once and writes
    (7/4)^d of it; the compression reads the 7^d leaf products, (7/4)^d m n / 8,
    and writes C once. Cubic plans move only the transpose."""
    import paper_1909_01554_gb300 as bmm

    for m, k, n in ((4096, 4096, 4096), (2048, 8192, 1024), (1536, 512, 3072)):
        cubic = bmm.plan(bmm.GF2, m, k, n, path=bmm.PATH_POPC, depth=0)
        assert cubic["pass_bytes"] == 2 * k * n // 8 and cubic["kp"] == k
        for d in (1, 2):
            pl = bmm.plan(bmm.GF2, m, k, n, path=bmm.PATH_POPC, depth=d, serial=0)
            assert (pl["strassen_depth"], pl["serial_depth"]) == (d, 0)
            grow = 7 ** d / 4 ** d
            want = (2 * k * n + m * k * (1 + grow) + k * n * (1 + grow) + m * n * (1 + grow)) / 8
            assert pl["pass_bytes"] == want, (m, k, n, d)
