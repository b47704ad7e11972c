"""Pins of the sphere-cutoff oracle (oracle/cutoff.py) to closed forms and
theorems, not to itself.

  * set membership against a plain enumeration of integer frequency
    triples with |G|^2/2 <= ecut;
  * the projector: idempotent and symmetric; a cosine planewave inside the
    sphere is kept exactly and one outside is removed;
  * free electrons: the Galerkin eigenvalues are the lowest |G|^2/2 of the
    set, with their multiplicities;
  * a sphere holding the whole grid gives the full-grid eigenvalues;
  * Cauchy interlacing for the compression of H to an N_set-dimensional
    subspace: lambda_i <= mu_i <= lambda_{i + N_g - N_set}, and the
    eigenvalues do not increase with ecut;
  * the eigenvectors lie in the set and solve the projected problem.
"""

import dataclasses
import itertools

import numpy as np
import pytest

import synth
from oracle import cutoff as oc
from oracle import hamiltonian as H


def _box0():
    return synth.cutoff_boxes([0])[0]


def _shells(n, L, ecut):
    """|G|^2/2 of every integer triple (f_x, f_y, f_z), f_d in
    [-n_d/2, n_d/2), inside the sphere: plain loops, no FFT helpers."""
    out = []
    for fx, fy, fz in itertools.product(*[range(-(nd // 2), nd - nd // 2) for nd in n]):
        e = 0.5 * sum((2.0 * np.pi * f / ld) ** 2 for f, ld in zip((fx, fy, fz), L))
        if e <= ecut:
            out.append(e)
    return np.sort(np.array(out))


def _ecut(el, frac=0.9):
    ec = frac * oc.ngecut_ecut(el.n, el.L)
    gap = np.min(np.abs(H.kinetic_symbol(el.n, el.L) - ec))
    assert gap > 1e-8 * ec  # no frequency on the sphere: membership is not a rounding decision
    return ec


def _cos_wave(el, f):
    h = np.asarray(el.L) / np.asarray(el.n)
    z, y, x = np.meshgrid(*[np.arange(el.n[d]) * h[d] for d in (2, 1, 0)], indexing="ij")
    g = [2.0 * np.pi * f[d] / el.L[d] for d in range(3)]
    return np.cos(g[0] * x + g[1] * y + g[2] * z).reshape(1, -1)


def test_ngecut_is_the_inscribed_sphere():
    el = _box0()
    ec = oc.ngecut_ecut(el.n, el.L)
    # Eq. Ngecut: n_d = sqrt(2 Ecut) L_d / pi on the axis with the smallest Nyquist frequency
    d = int(np.argmin([nd / ld for nd, ld in zip(el.n, el.L)]))
    assert abs(np.sqrt(2.0 * ec) * el.L[d] / np.pi - el.n[d]) < 1e-12 * el.n[d]


@pytest.mark.parametrize("frac", [0.3, 0.9, 1.7])
def test_set_membership_matches_enumeration(frac):
    el = _box0()
    ec = _ecut(el, frac)
    mask = oc.cutoff_mask(el.n, el.L, ec)
    assert mask.sum() == len(_shells(el.n, el.L, ec))
    assert np.max(np.abs(np.sort(H.kinetic_symbol(el.n, el.L)[mask]) - _shells(el.n, el.L, ec))) <= 1e-12 * ec


def test_projector_properties():
    el = _box0()
    ec = _ecut(el)
    gen = np.random.default_rng(5)
    x = gen.standard_normal((3, el.ng))
    y = gen.standard_normal((3, el.ng))
    px = oc.project(x, el.n, el.L, ec)
    assert np.max(np.abs(oc.project(px, el.n, el.L, ec) - px)) < 1e-12
    assert np.max(np.abs(oc.project(y, el.n, el.L, ec) @ x.T - y @ px.T)) < 1e-9
    inside = _cos_wave(el, (1, -2, 1))
    assert 0.5 * sum((2 * np.pi * f / L) ** 2 for f, L in zip((1, -2, 1), el.L)) < ec
    assert np.max(np.abs(oc.project(inside, el.n, el.L, ec) - inside)) < 1e-12
    corner = tuple(nd // 2 for nd in el.n)  # Nyquist corner, outside the inscribed sphere
    outside = _cos_wave(el, corner)
    assert np.max(np.abs(oc.project(outside, el.n, el.L, ec))) < 1e-12


def test_free_electrons_closed_form():
    el = _box0()
    free = dataclasses.replace(el, veff=np.zeros_like(el.veff), proj_row_ptr=np.zeros(1, np.int64),
                               proj_idx=np.zeros(0, np.int32), proj_val=np.zeros(0),
                               proj_gamma=np.zeros(0))
    ec = _ecut(el, 0.45)
    k = 30
    theta, _ = oc.galerkin_eigenpairs(free, ec, k)
    assert np.max(np.abs(theta - _shells(el.n, el.L, ec)[:k])) < 1e-11


def test_whole_grid_sphere_is_the_grid_problem():
    el = _box0()
    ec = 1.01 * float(np.max(H.kinetic_symbol(el.n, el.L)))
    assert oc.cutoff_mask(el.n, el.L, ec).all()
    mu, _ = oc.galerkin_eigenpairs(el, ec, el.m)
    lam, _ = oc.full_eigenpairs(el, el.m)
    assert np.max(np.abs(mu - lam)) < 1e-10


def test_interlacing_and_monotone_in_ecut():
    el = _box0()
    k = el.m
    lam_all = np.linalg.eigvalsh(0.5 * (lambda h: h + h.T)(H.apply_h(np.eye(el.ng), el)))
    prev = None
    gaps = {}
    for frac in (0.6, 0.9, 1.3):
        ec = _ecut(el, frac)
        nset = int(oc.cutoff_mask(el.n, el.L, ec).sum())
        mu, vec = oc.galerkin_eigenpairs(el, ec, k)
        shift = el.ng - nset
        assert np.all(mu >= lam_all[:k] - 1e-10)
        assert np.all(mu <= lam_all[shift:shift + k] + 1e-10)
        if prev is not None:
            assert np.all(mu <= prev + 1e-10)
        prev = mu
        gaps[frac] = float(np.max(mu - lam_all[:k]))
        # eigenvectors: orthonormal, inside the set, P (H v - mu v) = 0
        assert np.max(np.abs(vec @ vec.T - np.eye(k))) < 1e-10
        assert np.max(np.abs(oc.project(vec, el.n, el.L, ec) - vec)) < 1e-10
        r = oc.project(H.apply_h(vec, el) - mu[:, None] * vec, el.n, el.L, ec)
        assert np.max(np.linalg.norm(r, axis=1)) < 1e-9
    # the sphere changes the problem: inside Eq. Ngecut's sphere the
    # eigenvalues lie measurably above the grid's
    assert gaps[0.9] > 1e-6


def test_teter_keeps_the_set():
    """The Galerkin iteration relies on the Teter multiplier being diagonal in
    G: T(P r) lies in the set, so W = T(P R) needs no projection of its own."""
    from oracle import teter
    el = _box0()
    ec = _ecut(el)
    gen = np.random.default_rng(11)
    r = gen.standard_normal((4, el.ng))
    x = gen.standard_normal((4, el.ng))
    w = teter.precondition(oc.project(r, el.n, el.L, ec), x, el.n, el.L)
    assert np.max(np.abs(oc.project(w, el.n, el.L, ec) - w)) < 1e-12 * np.max(np.abs(w))
    # and T commutes with P
    tp = teter.precondition(oc.project(r, el.n, el.L, ec), x, el.n, el.L)
    pt = oc.project(teter.precondition(r, x, el.n, el.L), el.n, el.L, ec)
    assert np.max(np.abs(tp - pt)) < 1e-12 * np.max(np.abs(pt))
