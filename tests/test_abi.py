"""CPU checks of the C-ABI boundary: the library builds, loads without a GPU
and exports every function include/pdot.h declares; the ctypes structs match
the header's field lists.  No compute call is made here."""
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pdot.h")


def _declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pdot_[a-z_]+)\s*\(", src)))


def _struct_fields(name):
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    bodies = dict((nm, body) for body, nm in re.findall(r"typedef struct \{([^}]*)\}\s*(\w+);", src))
    body = bodies[name]
    fields = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        for part in decl.split(","):
            fields.append(re.search(r"(\w+)\s*$", part).group(1))
    return fields


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2407_19689_gb300 import _build, pdot
    _build.build()
    return pdot.load()


def test_every_declared_symbol_is_exported(lib):
    from paper_2407_19689_gb300 import pdot
    names = _declared_functions()
    assert sorted(pdot.DECLARED) == names
    for name in names:
        assert hasattr(lib, name), name


@pytest.mark.parametrize("cname,pyname", [("pdot_options", "Options"), ("pdot_result", "Result"),
                                          ("pdot_kkt_parts", "KktParts"), ("pdot_request", "Request"),
                                          ("pdot_points_cost", "PointsCostDesc"), ("pdot_start", "Start")])
def test_ctypes_structs_follow_header(cname, pyname):
    from paper_2407_19689_gb300 import pdot
    py = [f for f, _ in getattr(pdot, pyname)._fields_]
    assert py == _struct_fields(cname)


def test_default_options_and_status_strings(lib):
    from paper_2407_19689_gb300 import pdot
    o = pdot.pdot_default_options()
    assert o.tol == 1e-4 and o.restart_check_every == 64 and o.beta_suff == 0.1 and o.beta_nec == 0.9
    assert o.beta_art == 0.36 and o.theta == 0.5 and o.omega0 == 1.0 and o.adaptive_step == 1
    assert pdot.status_str(pdot.OK) == "PDOT_OK" and pdot.status_str(pdot.BUSY) == "PDOT_BUSY"


def test_null_handle_is_rejected_without_gpu(lib):
    from paper_2407_19689_gb300 import pdot
    st, _ = pdot.pdot_solve(None, 4, 4, 0, pdot.F32, 4, 0, 0, 1e-4)
    assert st == pdot.ERR_ARG
    st, _ = pdot.pdot_dual_bound(None, 4, 4, 0, pdot.F32, 4, 0, 0, 0)
    assert st == pdot.ERR_ARG
    assert pdot.pdot_destroy(None) == pdot.OK


def test_dtype_and_distance_codes_follow_header():
    from paper_2407_19689_gb300 import pdot
    src = open(HEADER).read()
    for name, val in [("PDOT_F32", pdot.F32), ("PDOT_BF16", pdot.BF16), ("PDOT_F64", pdot.F64),
                      ("PDOT_POINTS", pdot.POINTS)]:
        assert re.search(rf"\b{name}\s*=\s*{val}\b", src), name
    for dist, val in pdot.DIST.items():
        assert re.search(rf"\bPDOT_DIST_{dist.upper()}\s*=\s*{val}\b", src), dist


def test_watchdog_selftest_rejects_bad_arguments_before_any_cuda_call(lib):
    import ctypes
    from paper_2407_19689_gb300 import pdot
    out = ctypes.c_int32(-1)
    assert lib.pdot_watchdog_selftest(0, 0, ctypes.byref(out)) == pdot.ERR_ARG
    assert lib.pdot_watchdog_selftest(0, (1 << 24) + 1, ctypes.byref(out)) == pdot.ERR_ARG
    assert lib.pdot_watchdog_selftest(0, 4096, None) == pdot.ERR_ARG
    assert out.value == -1


def test_unknown_solver_option_is_rejected_before_any_cuda_call():
    from paper_2407_19689_gb300 import pdot
    with pytest.raises(TypeError, match="beta_artt"):
        pdot.Solver(device=0, beta_artt=0.5)


def test_state_bytes_needs_no_gpu(lib):
    """pdot_state_bytes: a 1 KB header, then three plans of m x ldx (ldx = n
    rounded up to 4) and three vector sets of 2(m + n) doubles, each piece
    256-byte aligned; 0 for invalid arguments."""
    from paper_2407_19689_gb300 import pdot

    def al(b):
        return (b + 255) // 256 * 256

    for m, n, xt, xs in [(300, 517, pdot.F32, 4), (1, 1, pdot.F64, 8), (4096, 4096, pdot.F32, 4)]:
        ldx = (n + 3) // 4 * 4
        assert pdot.pdot_state_bytes(m, n, xt) == 1024 + 3 * al(m * ldx * xs) + 3 * al(16 * (m + n))
    assert pdot.pdot_state_bytes(0, 5, pdot.F32) == 0
    assert pdot.pdot_state_bytes(5, 5, pdot.BF16) == 0


def test_option_ranges_are_checked_before_any_cuda_call(lib):
    """pdot_create rejects a pass_kernel outside 0..3, a compensated_cost
    outside 0..2 and a resident flag outside 0..1 (PDOT_ERR_ARG) before it
    touches a device; the defaults are the autotuner's kernel, the
    size-dependent compensation and the tile kernels."""
    import ctypes
    from paper_2407_19689_gb300 import pdot
    o = pdot.pdot_default_options()
    assert o.pass_kernel == 0 and o.compensated_cost == 2 and o.resident == 0
    for field, bad in (("pass_kernel", 4), ("pass_kernel", -1), ("compensated_cost", 3), ("resident", 2)):
        o = pdot.pdot_default_options()
        setattr(o, field, bad)
        h = ctypes.c_void_p()
        assert lib.pdot_create(ctypes.byref(o), 0, None, ctypes.byref(h)) == pdot.ERR_ARG
        assert not h.value


def test_resident_fit_rule_needs_no_gpu(lib):
    """pdot_resident_fits: a plan and its average's deviation at 4 B each per
    entry, split over the 8 CTAs of a cluster, must fit one CTA's shared
    memory (with the FP64 partial sums): about 190k entries for square plans."""
    from paper_2407_19689_gb300 import pdot
    assert pdot.pdot_resident_fits(1, 1) == 1
    assert pdot.pdot_resident_fits(430, 430) == 1
    assert pdot.pdot_resident_fits(700, 700) == 0
    assert pdot.pdot_resident_fits(60, 2100) == 1
    assert pdot.pdot_resident_fits(0, 5) == 0 and pdot.pdot_resident_fits(5, -1) == 0
    # monotone in each dimension
    for n in (1, 100, 1000, 5000):
        fits = [pdot.pdot_resident_fits(m, n) for m in range(1, 3000, 37)]
        assert fits == sorted(fits, reverse=True)
