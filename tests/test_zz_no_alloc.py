"""The allocation-free receiver-field call (ms_fields_noalloc) against ms_fields.

ms_fields_noalloc exists for callers that cannot call cudaMalloc -- real-time loops that must not
wait on the allocator, processes whose device memory is owned by a pool sized in advance.  It keeps
its scratch in fixed device arrays instead.  This file
is collected last so that a failure here comes after every other test has run; it also passes on
its own in a fresh process.
"""
import numpy as np
import pytest

import synthetic as syn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("CUDA device required", allow_module_level=True)

import paper_2608_26875_b300 as P  # noqa: E402

# the receiver-field tolerance used by the parity tests (relative l2)
TOL = 1e-10


def _fields_both(solver, gamma, rx_host):
    ref = solver.fields(gamma, rx_host)
    rx = torch.as_tensor(np.ascontiguousarray(rx_host, dtype=np.float64), device="cuda")
    out = torch.full(ref.shape, complex(np.nan, np.nan), dtype=torch.complex128, device="cuda")
    got = solver.fields_noalloc(gamma, rx, out)
    torch.cuda.synchronize()
    return ref.cpu().numpy(), got.cpu().numpy()


def test_noalloc_fields_match_ms_fields_on_two_calls_in_a_row():
    wl = syn.config1()
    s = P.Solver.from_workload(wl)
    for seed, nrhs in ((301, 3), (302, 5)):
        g = torch.as_tensor(syn.random_coeffs(seed, wl.M, wl.p, nrhs), device="cuda")
        ref, got = _fields_both(s, g, wl.receivers)
        assert np.all(np.isfinite(got))
        e = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert e <= TOL, (seed, e)


def test_noalloc_fields_on_a_larger_geometry_and_solution():
    wl = syn.small_case(303, 40, 12, omega=3.0, nrhs=4, box=(-20.0, 20.0, -12.0, -1.0))
    s = P.Solver.from_workload(wl)
    g, info = s.solve(wl.inc_kind, wl.inc_angle, tol=1e-10, prec=P.MS_PREC_FP64)
    for _ in range(2):
        ref, got = _fields_both(s, g, wl.receivers)
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= TOL


def test_noalloc_rejects_requests_beyond_its_fixed_scratch():
    wl = syn.config1()
    s = P.Solver.from_workload(wl)
    g = torch.zeros((wl.M, 2, wl.nc, 64), dtype=torch.complex128, device="cuda")
    rx = torch.as_tensor(wl.receivers, device="cuda")
    out = torch.empty((64, rx.shape[0], 2), dtype=torch.complex128, device="cuda")
    with pytest.raises(P.MsError) as e:
        s.fields_noalloc(g, rx, out)
    assert e.value.status == P._native.MS_ERR_TOO_LARGE


def test_noalloc_rejects_receiver_inside_a_particle():
    wl = syn.config1()
    s = P.Solver.from_workload(wl)
    g = torch.zeros((wl.M, 2, wl.nc, 1), dtype=torch.complex128, device="cuda")
    rx = torch.as_tensor(np.ascontiguousarray(wl.centres[:2]), device="cuda")
    out = torch.empty((1, 2, 2), dtype=torch.complex128, device="cuda")
    with pytest.raises(P.MsError) as e:
        s.fields_noalloc(g, rx, out)
    assert e.value.status == P._native.MS_ERR_RECEIVER_INSIDE
