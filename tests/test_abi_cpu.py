"""C-ABI checks that need no GPU: the library loads, exports every declared entry point, the
Python binding declares exactly the header's functions, and host-side validation answers with
the documented status codes before any device work."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

import synthetic as syn

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    names = set()
    for path in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(path).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*[A-Za-z_][\w\s\*]*?\b(ms3?_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2608_26875_b300 import _native
    from paper_2608_26875_b300.build import build
    if not os.path.exists(_native.LIB_PATH):
        build()
    return _native.lib()


def test_header_declares_the_boundary_calls():
    names = header_functions()
    for required in ("ms_setup", "ms_apply", "ms_solve", "ms_fields", "ms_rhs", "ms_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in header_functions():
        assert hasattr(lib, name), name


def test_binding_matches_header():
    from paper_2608_26875_b300 import _native
    assert set(_native.SIGNATURES) == header_functions()


def test_status_strings(lib):
    assert lib.ms_status_string(0) == b"ok"
    assert b"1.1" in lib.ms_status_string(-3)
    assert lib.ms_status_string(12345) == b"unknown status"


def test_default_options(lib):
    import paper_2608_26875_b300 as P
    o = P.default_options()
    assert (o.n_panels, o.nodes_per_panel, o.t_max, o.restart) == (32, 16, 20.0, 50)
    assert (o.use_fmm, o.leaf_target, o.depth, o.grade, o.tensor_cores) == (1, 10, 0.5, 0, 1)
    assert o.inner_tol == 0.0 and o.tc_wait_test == 0 and o.block_krylov == 1 and o.cuda_graph == 1
    assert ctypes.sizeof(o) == 88      # the C struct: 14 int32, 3 doubles, padding


def test_timeout_status_string(lib):
    assert b"tensor-core" in lib.ms_status_string(-12)


@pytest.mark.parametrize("case", ["overlap", "not_buried", "bad_bc", "bad_p", "bad_omega", "bad_radius"])
def test_setup_validation_on_host(lib, case):
    import paper_2608_26875_b300 as P
    wl = syn.config1()
    c, r, bc = wl.centres.copy(), wl.radius.copy(), wl.bc.copy()
    omega, p = wl.omega, wl.p
    want = P._native.MS_ERR_ARG
    if case == "overlap":
        c[1] = c[0] + np.array([0.5, 0.0])
        want = P._native.MS_ERR_OVERLAP
    elif case == "not_buried":
        c[3, 1] = -0.4
        want = P._native.MS_ERR_NOT_BURIED
    elif case == "bad_bc":
        bc[2] = 7
    elif case == "bad_p":
        p = 31
    elif case == "bad_omega":
        omega = 0.0
    elif case == "bad_radius":
        r[0] = -1.0
    with pytest.raises(P.MsError) as e:
        P.Solver(c, r, bc, wl.media, omega, p)
    assert e.value.status == want


def test_separation_rule_boundary_is_exact(lib):
    """Two discs exactly at 1.1 (R_l + R_m) are accepted by the validation (no device work is
    reached because the second, buried-check failure is planted after it)."""
    import paper_2608_26875_b300 as P
    c = np.array([[0.0, -5.0], [1.1 * 1.0 + 1e-12, -5.0], [3.0, 0.5]])
    r = np.array([0.5, 0.5, 0.3])
    with pytest.raises(P.MsError) as e:
        P.Solver(c, r, np.zeros(3, np.int32), syn.MEDIA_STD, 2.0, 4)
    assert e.value.status == P._native.MS_ERR_NOT_BURIED


def test_perturbed_truth_keeps_the_separation_rule():
    wl = syn.config4(M=300, nrhs=1)
    c = syn.perturb_centres(wl.centres, wl.radius, 0.05, 3001)
    assert np.abs(c - wl.centres).max() > 0.05
    d = np.sqrt(((c[:, None, :] - c[None, :, :]) ** 2).sum(-1))
    lim = syn.SEP * (wl.radius[:, None] + wl.radius[None, :])
    np.fill_diagonal(d, np.inf)
    assert np.all(d >= lim)
    assert np.all(c[:, 1] + syn.SEP * wl.radius <= 0.0)


def _raw_setup(lib, case):
    """ms_setup through ctypes with one field of config1's arguments made invalid; returns
    (status, handle pointer value)."""
    from paper_2608_26875_b300 import _native as nat
    wl = syn.config1()
    c = np.ascontiguousarray(wl.centres, dtype=np.float64)
    r = np.ascontiguousarray(wl.radius, dtype=np.float64)
    bc = np.ascontiguousarray(wl.bc, dtype=np.int32)
    proto = np.full(wl.M, -1, dtype=np.int32)
    g = nat.Geometry()
    g.M = wl.M
    g.centres, g.radius, g.bc = c.ctypes.data_as(nat.c_dp), r.ctypes.data_as(nat.c_dp), bc.ctypes.data_as(nat.c_ip)
    md = nat.Media(wl.media.lam_u, wl.media.mu_u, wl.media.lam_l, wl.media.mu_l)
    o = nat.Options()
    lib.ms_default_options(ctypes.byref(o))
    omega, p = wl.omega, wl.p
    field, _, value = case.partition("=")
    if field in ("tensor_cores", "leaf_target", "restart", "max_iters", "n_panels", "nodes_per_panel", "grade",
                 "store_near", "precond_group"):
        setattr(o, field, int(value))
    elif field in ("inner_tol", "t_max", "depth"):
        setattr(o, field, float(value))
    elif field in ("mu_u", "mu_l", "lam_l"):
        setattr(md, field, float(value))
    elif field == "M":
        g.M = int(value)
    elif field == "centre":
        c[4, 0] = float(value)
    elif field == "proto":
        proto[5] = int(value)                  # an index with no prototype table behind it
        g.proto = proto.ctypes.data_as(nat.c_ip)
    elif field == "n_proto":
        g.n_proto = int(value)                 # tables announced, none passed
    elif field == "p":
        p = int(value)
    elif field == "omega":
        omega = float(value)
    elif field == "radius":
        r[3] = float(value)
    else:
        raise AssertionError(case)
    h = ctypes.c_void_p(12345)
    st = lib.ms_setup(ctypes.byref(g), ctypes.byref(md), float(omega), int(p), ctypes.byref(o), ctypes.byref(h))
    return st, h.value


@pytest.mark.parametrize("case", [
    "tensor_cores=2", "tensor_cores=-1", "inner_tol=1.0", "inner_tol=-0.001", "inner_tol=nan",
    "leaf_target=0", "restart=0", "max_iters=0", "n_panels=0", "nodes_per_panel=0", "t_max=0",
    "depth=0", "depth=nan", "grade=-1", "grade=31", "mu_u=0", "mu_l=-1", "lam_l=-1.5", "M=0",
    "centre=nan", "centre=inf", "proto=0", "proto=-2", "n_proto=2", "p=-1", "store_near=-1",
    "store_near=1025", "precond_group=-1", "precond_group=65", "t_max=inf", "omega=inf", "omega=nan",
    "radius=inf", "nodes_per_panel=65536"])
def test_invalid_options_and_media_are_refused_before_device_work(lib, case):
    """Every ms_options field, the media and the geometry arrays are checked on the host: an
    invalid value returns MS_ERR_ARG and leaves the handle NULL (the call never reaches CUDA, so
    this runs without a device)."""
    from paper_2608_26875_b300 import _native as nat
    st, h = _raw_setup(lib, case)
    assert st == nat.MS_ERR_ARG, (case, st)
    assert h is None


def test_setup_refuses_a_null_handle_slot(lib):
    from paper_2608_26875_b300 import _native as nat
    assert lib.ms_setup(None, None, 1.0, 4, None, None) == nat.MS_ERR_ARG


def test_every_handle_call_refuses_a_null_handle(lib):
    """Each entry point that takes a handle answers MS_ERR_ARG to a NULL one (all other pointers
    NULL, sizes 1) without touching memory; ms_destroy(NULL) is a no-op and ms_last_cuda_error(NULL)
    is 0."""
    from paper_2608_26875_b300 import _native as nat
    skip = {"ms_default_options", "ms_setup", "ms_status_string", "ms_destroy", "ms_last_cuda_error",
            "ms_tensor_peak", "ms3_default_options", "ms3_setup", "ms3_destroy"}
    checked = 0
    for name, (restype, argtypes) in nat.SIGNATURES.items():
        if name in skip:
            continue
        assert argtypes[0] is ctypes.c_void_p, name          # the handle comes first
        args = []
        for t in argtypes:
            if t in (ctypes.c_int, ctypes.c_int32, ctypes.c_int64):
                args.append(1)
            elif t is ctypes.c_double:
                args.append(1e-8)
            else:
                args.append(None)
        assert getattr(lib, name)(*args) == nat.MS_ERR_ARG, name
        checked += 1
    assert checked == 21         # apply, apply_adjoint, operator, rhs, rhs_point, solve, solve_rhs, fields,
    #                              fields_upper, time_reversal, grad, fields_noalloc, autotune, info, work,
    #                              near_stored; ms3_: apply, operator, rhs, solve, info
    lib.ms_destroy(None)
    assert lib.ms_last_cuda_error(None) == 0


def test_every_declared_status_has_its_own_message(lib):
    src = open(os.path.join(ROOT, "include", "ms_b300.h")).read()
    codes = {int(v): k for k, v in re.findall(r"^#define\s+(MS_(?:OK|NOT_CONVERGED|ERR_\w+))\s+(-?\d+)", src, re.M)}
    assert len(codes) >= 12
    msgs = {c: lib.ms_status_string(c) for c in codes}
    for c, m in msgs.items():
        assert m and m != b"unknown status", (codes[c], m)
    assert len(set(msgs.values())) == len(msgs)


def test_tensor_peak_refuses_invalid_arguments(lib):
    """ms_tensor_peak takes no handle; it refuses an unknown operand kind, a non-positive count and a
    NULL output before touching the device."""
    import ctypes as ct
    from paper_2608_26875_b300 import _native as nat
    out = ct.c_double()
    assert lib.ms_tensor_peak(0, 10, ct.byref(out), None) == nat.MS_ERR_ARG      # FP64 has no tensor kind here
    assert lib.ms_tensor_peak(1, 0, ct.byref(out), None) == nat.MS_ERR_ARG
    assert lib.ms_tensor_peak(1, 10, None, None) == nat.MS_ERR_ARG


@pytest.mark.parametrize("case", ["p=0", "p=11", "not_buried", "overlap", "bc=2", "panels", "M=0", "nan",
                                  "omega=inf", "t_max=inf", "alpha=nan", "radius=inf", "nodes"])
def test_3d_setup_refuses_invalid_input_before_device_work(lib, case):
    """ms3_setup validates geometry, order and rule on the host (no device needed)."""
    from paper_2608_26875_b300 import _native as nat
    c = np.array([[0.0, 0.0, -2.0], [2.0, 0.0, -2.5]])
    r = np.array([0.4, 0.4])
    bc = np.array([0, 1], dtype=np.int32)
    p = 4
    o = nat.Options3()
    lib.ms3_default_options(ctypes.byref(o))
    M = 2
    want = nat.MS_ERR_ARG
    if case == "p=0":
        p = 0
    elif case == "p=11":
        p = 11
    elif case == "not_buried":
        c[1, 2] = -0.3
        want = nat.MS_ERR_NOT_BURIED
    elif case == "overlap":
        c[1] = [0.5, 0.0, -2.0]
        want = nat.MS_ERR_OVERLAP
    elif case == "bc=2":
        bc[0] = 2
    elif case == "panels":
        o.n_panels = 3                   # does not divide n_r = 128
    elif case == "M=0":
        M = 0
    elif case == "nan":
        c[0, 0] = np.nan
    elif case == "t_max=inf":
        o.t_max = np.inf
    elif case == "alpha=nan":
        o.alpha = np.nan
    elif case == "radius=inf":
        r[0] = np.inf
    elif case == "nodes":
        o.n_r, o.n_theta = 1024, 512     # 2^19 Sommerfeld nodes, above the 2^18 limit
    omega = np.inf if case == "omega=inf" else 2.0
    g = nat.Geometry3(M, c.ctypes.data_as(nat.c_dp), r.ctypes.data_as(nat.c_dp), bc.ctypes.data_as(nat.c_ip))
    md = nat.Media(1.0, 0.5, 2.0, 1.0)
    h = ctypes.c_void_p()
    st = lib.ms3_setup(ctypes.byref(g), ctypes.byref(md), omega, p, ctypes.byref(o), ctypes.byref(h))
    assert st == want, (case, st)
    assert not h.value


def test_3d_default_options(lib):
    from paper_2608_26875_b300 import _native as nat
    o = nat.Options3()
    lib.ms3_default_options(ctypes.byref(o))
    assert (o.n_r, o.n_theta, o.n_panels, o.t_max, o.alpha, o.beta) == (128, 64, 4, 10.0, 1.0, 1.0)
    assert ctypes.sizeof(o) == 48
