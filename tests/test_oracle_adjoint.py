"""Pins of the oracle's adjoint gradient (oracle/adjoint.py) against central finite differences of
the oracle's own loss: a forward solve at perturbed centres, radii and frequency, independent of
every derivative formula in the adjoint."""
import copy

import numpy as np
import pytest

import synthetic as syn
from oracle import adjoint
from oracle.system import Problem

H = 1e-6


@pytest.fixture(scope="module")
def case():
    wl = syn.small_case(401, 3, 5, omega=2.0, nrhs=2)      # particles 0, 2 rigid; 1 traction-free
    rx = wl.receivers[::6]
    rng = np.random.default_rng(0)
    d = 0.1 * (rng.standard_normal((2, rx.shape[0], 2)) + 1j * rng.standard_normal((2, rx.shape[0], 2)))
    return wl, rx, d, adjoint.gradient(wl, wl.inc_kind, wl.inc_angle, rx, d)


def _loss(wl, rx, d):
    return adjoint.loss(Problem(wl), wl.inc_kind, wl.inc_angle, rx, d)


def _fd(wl, rx, d, edit):
    wp, wm = copy.deepcopy(wl), copy.deepcopy(wl)
    edit(wp, +H)
    edit(wm, -H)
    return (_loss(wp, rx, d) - _loss(wm, rx, d)) / (2 * H)


@pytest.mark.parametrize("m,axis", [(0, 0), (0, 1), (1, 0), (1, 1), (2, 1)])
def test_centre_gradient_matches_central_differences(case, m, axis):
    wl, rx, d, (L, gc, gr, gw) = case

    def edit(w, s):
        w.centres = w.centres.copy()
        w.centres[m, axis] += s
    fd = _fd(wl, rx, d, edit)
    assert abs(gc[m, axis] - fd) <= 1e-7 * max(1.0, abs(fd))


@pytest.mark.parametrize("m", [0, 1])
def test_radius_gradient_matches_central_differences(case, m):
    wl, rx, d, (L, gc, gr, gw) = case

    def edit(w, s):
        w.radius = w.radius.copy()
        w.radius[m] += s
    fd = _fd(wl, rx, d, edit)
    assert abs(gr[m] - fd) <= 1e-7 * max(1.0, abs(fd))


def test_frequency_gradient_matches_central_differences(case):
    wl, rx, d, (L, gc, gr, gw) = case
    hw = H * wl.omega
    wp, wm = copy.deepcopy(wl), copy.deepcopy(wl)
    wp.omega += hw
    wm.omega -= hw
    fd = (_loss(wp, rx, d) - _loss(wm, rx, d)) / (2 * hw)
    assert abs(gw - fd) <= 1e-7 * max(1.0, abs(fd))


def test_loss_value_is_the_misfit(case):
    wl, rx, d, (L, gc, gr, gw) = case
    assert L == pytest.approx(_loss(wl, rx, d), rel=1e-12)


def test_planted_source_side_translation_sign_is_caught(monkeypatch):
    """Dropping the source-side term of dT/dc (a plausible slip) must break the FD agreement."""
    wl = syn.small_case(402, 2, 4, omega=2.0, nrhs=1)
    rx = wl.receivers[::8]
    d = np.zeros((1, rx.shape[0], 2), dtype=complex)
    orig = adjoint._dT
    calls = {"n": 0}

    def half(p, k, v, axis):
        calls["n"] += 1
        D = orig(p, k, v, axis)
        return D if calls["n"] % 2 == 1 else 0 * D          # zero every source-side block
    monkeypatch.setattr(adjoint, "_dT", half)
    L, gc, gr, gw = adjoint.gradient(wl, wl.inc_kind, wl.inc_angle, rx, d)
    monkeypatch.setattr(adjoint, "_dT", orig)

    def edit(w, s):
        w.centres = w.centres.copy()
        w.centres[0, 0] += s
    fd = _fd(wl, rx, d, edit)
    assert abs(gc[0, 0] - fd) > 1e-4 * abs(fd)
