"""Pins of the FP64 CPU oracle to closed forms, brute force and invariants.

Each test ties an oracle function to something other than itself:
  * kinetic operator: the closed-form periodic spectral second-derivative
    matrix (Trefethen, Spectral Methods in MATLAB, ch. 3) and the analytic
    Laplacian of a smooth periodic function;
  * free electrons: eigenvalues (2 pi / L)^2 |n|^2 / 2 with shell
    degeneracies 1, 6, 12 (tests/golden/free_electron_L10.txt);
  * separable potential: product spectrum from 1-D dense eigensolves;
  * full H (local + Kleinman-Bylander): explicit Kronecker-sum assembly;
  * LOBPCG: dense diagonalisation, Ritz monotonicity, Cauchy interlacing,
    orthonormality, Hermiticity; the warm-started fixed-iteration run (the
    SCF-mode reference) against the dense Rayleigh-Ritz of its start block;
  * Teter: limits of the rational function and plane-wave eigenfunctions;
  * restriction/SVD: orthonormality, span equality, E_K = Q_K; the element's
    index map against the points picked by their coordinates.
"""

import os

import numpy as np
import pytest

import synth
from oracle import alb, hamiltonian as H, lobpcg as L, teter as T
from synth.workloads import ElementInput

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def d2_matrix(n: int, length: float) -> np.ndarray:
    """Closed-form periodic spectral second-derivative matrix (even n)."""
    h = 2.0 * np.pi / n
    j = np.arange(n)
    d = j[:, None] - j[None, :]
    with np.errstate(divide="ignore"):
        s = -((-1.0) ** d) / (2.0 * np.sin(d * h / 2.0) ** 2)
    s[j, j] = -np.pi ** 2 / (3.0 * h * h) - 1.0 / 6.0
    return s * (2.0 * np.pi / length) ** 2


def make_element(n, L_, veff=None, proj=None, m=8, J=8, tol=1e-10):
    ng = int(np.prod(n))
    v = np.zeros((n[2], n[1], n[0])) if veff is None else veff
    if proj is None:
        proj = (np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0), np.zeros(0))
    rp, idx, val, gam = proj
    return ElementInput(n=tuple(n), L=tuple(L_), veff=v, proj_row_ptr=rp, proj_idx=idx,
                        proj_val=val, proj_gamma=gam, e_lo=(0, 0, 0), e_hi=tuple(n),
                        m=m, J=J, tol=tol, seed_key=(9, 9))


def kron_kinetic(n, L_):
    """-1/2 Lap as a Kronecker sum of 1-D closed-form matrices (x fastest)."""
    ix, iy, iz = (np.eye(k) for k in n)
    dx, dy, dz = (d2_matrix(k, l) for k, l in zip(n, L_))
    lap = (np.kron(iz, np.kron(iy, dx)) + np.kron(iz, np.kron(dy, ix))
           + np.kron(dz, np.kron(iy, ix)))
    return -0.5 * lap


def random_projectors(n, L_, n_proj, gen):
    """Random sparse unit rows with gamma in [0.5, 2] (test input only)."""
    ng = int(np.prod(n))
    rp, idx, val = [0], [], []
    for _ in range(n_proj):
        pts = np.sort(gen.choice(ng, size=min(20, ng), replace=False)).astype(np.int32)
        v = gen.standard_normal(len(pts))
        v /= np.linalg.norm(v)
        idx.append(pts)
        val.append(v)
        rp.append(rp[-1] + len(pts))
    return (np.asarray(rp, np.int64), np.concatenate(idx), np.concatenate(val),
            gen.uniform(0.5, 2.0, n_proj))


# ---------------------------------------------------------------- kinetic

def test_kinetic_matches_closed_form_differentiation_matrix():
    n, L_ = (8, 6, 4), (7.0, 5.0, 3.0)
    dense = H.apply_kinetic(np.eye(int(np.prod(n))), n, L_).T
    np.testing.assert_allclose(dense, kron_kinetic(n, L_), atol=1e-12)


def test_kinetic_analytic_laplacian_of_smooth_function():
    n, L_ = (32, 24, 20), (9.0, 7.0, 6.0)
    x = np.arange(n[0]) * L_[0] / n[0]
    y = np.arange(n[1]) * L_[1] / n[1]
    z = np.arange(n[2]) * L_[2] / n[2]
    zz, yy, xx = np.meshgrid(z, y, x, indexing="ij")
    kx, ky, kz = (2 * np.pi / l for l in L_)
    f = np.exp(np.sin(kx * xx)) * np.cos(ky * yy) * np.exp(0.5 * np.cos(kz * zz))
    # analytic second derivatives of each factor
    ax = np.exp(np.sin(kx * xx)) * (kx ** 2) * (np.cos(kx * xx) ** 2 - np.sin(kx * xx))
    az = np.exp(0.5 * np.cos(kz * zz)) * (kz ** 2) * (0.25 * np.sin(kz * zz) ** 2
                                                       - 0.5 * np.cos(kz * zz))
    lap = (ax * np.cos(ky * yy) * np.exp(0.5 * np.cos(kz * zz))
           - ky ** 2 * f
           + np.exp(np.sin(kx * xx)) * np.cos(ky * yy) * az)
    out = H.apply_kinetic(f.reshape(1, -1), n, L_).reshape(f.shape)
    np.testing.assert_allclose(out, -0.5 * lap, atol=1e-9 * np.abs(lap).max())


def test_free_electron_spectrum_golden():
    data = np.loadtxt(os.path.join(GOLDEN, "free_electron_L10.txt"))
    n, L_ = (8, 8, 8), (10.0, 10.0, 10.0)
    ev = np.linalg.eigvalsh(H.apply_kinetic(np.eye(512), n, L_))
    # golden rows: eigenvalue, multiplicity (lowest three shells)
    k = 0
    for val, mult in data:
        np.testing.assert_allclose(ev[k:k + int(mult)], val, atol=5e-6)
        k += int(mult)
    assert ev[k] > data[-1, 0] + 0.1


# ------------------------------------------------------------- full H

def test_full_hamiltonian_equals_explicit_assembly():
    gen = np.random.default_rng(11)
    n, L_ = (6, 4, 8), (5.0, 4.0, 6.0)
    v = gen.uniform(-3, 1, size=(n[2], n[1], n[0]))
    proj = random_projectors(n, L_, 5, gen)
    el = make_element(n, L_, v, proj)
    ref = kron_kinetic(n, L_) + np.diag(v.reshape(-1))
    rp, idx, val, gam = proj
    for p in range(len(gam)):
        b = np.zeros(el.ng)
        b[idx[rp[p]:rp[p + 1]]] = val[rp[p]:rp[p + 1]]
        ref += gam[p] * np.outer(b, b)
    np.testing.assert_allclose(H.dense_h(el), ref, atol=1e-11)


def test_hermiticity_16cubed():
    el = synth.config1()
    gen = np.random.default_rng(5)
    el.proj_row_ptr, el.proj_idx, el.proj_val, el.proj_gamma = random_projectors(
        el.n, el.L, 6, gen)
    x, y = gen.standard_normal((2, el.ng))
    lhs = x @ H.apply_h(y[None], el)[0]
    rhs = y @ H.apply_h(x[None], el)[0]
    assert abs(lhs - rhs) <= 1e-13 * np.linalg.norm(x) * np.linalg.norm(H.apply_h(y[None], el))


def test_separable_potential_product_spectrum():
    n, L_ = (12, 10, 8), (8.0, 7.0, 6.0)
    gen = np.random.default_rng(3)
    coords = [np.arange(k) * l / k for k, l in zip(n, L_)]
    v1 = -2.0 * np.exp(-((coords[0] - 4.0) ** 2))
    v2 = 0.5 * np.cos(2 * np.pi * coords[1] / L_[1])
    v3 = -1.0 * np.exp(-((coords[2] - 3.0) ** 2) / 2.0)
    v = v3[:, None, None] + v2[None, :, None] + v1[None, None, :]
    spectra = [np.linalg.eigvalsh(-0.5 * d2_matrix(k, l) + np.diag(vd))
               for k, l, vd in zip(n, L_, (v1, v2, v3))]
    sums = np.sort((spectra[2][:, None, None] + spectra[1][None, :, None]
                    + spectra[0][None, None, :]).reshape(-1))
    el = make_element(n, L_, v, m=10, J=10, tol=1e-9)
    x0 = gen.standard_normal((10, el.ng))
    out = L.lobpcg(el, x0)
    assert out["converged"]
    np.testing.assert_allclose(out["theta"][:7], sums[:7], atol=1e-10)


# -------------------------------------------------------------- Teter

def test_teter_function_limits():
    assert T.teter_k(0.0) == 1.0
    for s in (1e-2, 1e-3):  # 1 - K = (16 s^4 / 27)(1 - 2 s / 3 + O(s^2))
        assert abs((1.0 - T.teter_k(s)) * 27.0 / (16.0 * s ** 4) - 1.0) < s
    big = np.array([1e3, 1e4, 1e5])
    np.testing.assert_allclose(T.teter_k(big) * 2 * big, 1.0, rtol=2e-3)
    grid = np.linspace(0, 50, 2001)
    k = T.teter_k(grid)
    assert np.all(k > 0) and np.all(k <= 1) and np.all(np.diff(k) <= 0)


def test_teter_plane_wave_eigenfunctions():
    n, L_ = (16, 12, 10), (10.0, 8.0, 6.0)
    coords = [np.arange(k) * l / k for k, l in zip(n, L_)]
    zz, yy, xx = np.meshgrid(coords[2], coords[1], coords[0], indexing="ij")
    g_x = 2 * np.pi * 2 / L_[0]
    g_r = (2 * np.pi * 3 / L_[1], 2 * np.pi * 1 / L_[2])
    x = np.cos(g_x * xx).reshape(1, -1)            # kinetic energy g_x^2 / 2
    r = np.cos(g_r[0] * yy + g_r[1] * zz).reshape(1, -1)
    w = T.precondition(r, x, n, L_)
    s = (g_r[0] ** 2 + g_r[1] ** 2) / g_x ** 2
    expect = (27 + 18 * s + 12 * s * s + 8 * s ** 3) / (27 + 18 * s + 12 * s * s + 8 * s ** 3
                                                       + 16 * s ** 4)
    np.testing.assert_allclose(w, expect * r, atol=1e-12)
    np.testing.assert_allclose(T.kinetic_energy(x, n, L_), [0.5 * g_x ** 2], rtol=1e-12)


# ------------------------------------------------------------ LOBPCG

def test_free_electron_lobpcg_shells():
    n, L_ = (16, 16, 16), (10.0, 10.0, 10.0)
    gen = np.random.default_rng(0)
    el = make_element(n, L_, m=7, J=7, tol=1e-9)
    out = L.lobpcg(el, gen.standard_normal((7, el.ng)))
    assert out["converged"]
    data = np.loadtxt(os.path.join(GOLDEN, "free_electron_L10.txt"))
    np.testing.assert_allclose(out["theta"][0], data[0, 0], atol=1e-9)
    np.testing.assert_allclose(out["theta"][1:7], data[1, 0], atol=1e-9)
    # the 7-dim subspace is exactly {1, cos/sin(2 pi x_d / L)}
    coords = np.arange(16) * 10.0 / 16
    zz, yy, xx = np.meshgrid(coords, coords, coords, indexing="ij")
    k = 2 * np.pi / 10.0
    basis = np.stack([np.ones_like(xx)] + [f(k * c) for c in (xx, yy, zz)
                                           for f in (np.cos, np.sin)]).reshape(7, -1)
    assert alb.sin_max_angle(basis, out["X"]) < 1e-7


def test_lobpcg_matches_dense_small_with_projectors():
    gen = np.random.default_rng(21)
    n, L_ = (8, 8, 8), (6.0, 6.0, 6.0)
    v = gen.uniform(-4, 0, size=(8, 8, 8))
    el = make_element(n, L_, v, random_projectors(n, L_, 6, gen), m=12, J=10, tol=1e-10)
    exact = np.linalg.eigh(kron_kinetic(n, L_) + np.diag(v.reshape(-1))
                           + H.nonlocal_matrix(el).T @ np.diag(el.proj_gamma)
                           @ H.nonlocal_matrix(el))
    out = L.lobpcg(el, gen.standard_normal((12, el.ng)))
    assert out["converged"]
    np.testing.assert_allclose(out["theta"][:10], exact[0][:10], atol=1e-10)
    gap = exact[0][10] - exact[0][9]
    assert alb.sin_max_angle(exact[1][:, :10].T, out["X"][:10]) < 1e-9 / gap * 10
    # Ritz values never increase and never fall below the exact eigenvalues
    th = np.array(out["history"]["theta"])
    assert np.all(np.diff(th, axis=0) <= 1e-12)
    assert np.all(th >= exact[0][None, :12] - 1e-12)
    # orthonormality of the Ritz block
    np.testing.assert_allclose(out["X"] @ out["X"].T, np.eye(12), atol=1e-12)


def test_lobpcg_fixed_iterations_from_warm_block():
    # the SCF-mode reference: a block converged for V0, three iterations under
    # V1 = V0 + a smooth field.  Pinned to dense diagonalisation of the
    # explicitly assembled H1: the first Ritz values are the Rayleigh-Ritz of
    # the warm block under H1, Ritz values never increase, never fall below
    # H1's eigenvalues, and move toward them
    gen = np.random.default_rng(23)
    n, L_ = (8, 8, 8), (6.0, 6.0, 6.0)
    v0 = gen.uniform(-4, 0, size=(8, 8, 8))
    proj = random_projectors(n, L_, 6, gen)
    el0 = make_element(n, L_, v0, proj, m=10, J=8, tol=1e-11)
    x0 = L.lobpcg(el0, gen.standard_normal((10, el0.ng)))["X"]
    z, y, x = np.meshgrid(*(np.arange(8) / 8.0,) * 3, indexing="ij")
    v1 = v0 + 0.3 * np.cos(2 * np.pi * x) * np.sin(2 * np.pi * (y + z))
    el1 = make_element(n, L_, v1, proj, m=10, J=8, tol=1e-11)
    nl = H.nonlocal_matrix(el1)
    h1 = kron_kinetic(n, L_) + np.diag(v1.reshape(-1)) + nl.T @ np.diag(el1.proj_gamma) @ nl
    exact = np.linalg.eigvalsh(h1)[:10]
    out = L.lobpcg(el1, x0, tol=0.0, maxit=3)
    th = np.array(out["history"]["theta"])
    assert out["iterations"] == 3 and th.shape == (4, 10)
    q, _ = np.linalg.qr(x0.T)
    np.testing.assert_allclose(th[0], np.linalg.eigvalsh(q.T @ h1 @ q), atol=1e-10)
    assert np.all(np.diff(th, axis=0) <= 1e-12)
    assert np.all(th >= exact[None, :] - 1e-12)
    assert np.sum(th[-1] - exact) < 0.1 * np.sum(th[0] - exact)


def test_config1_golden_eigenvalues():
    el = synth.config1()
    data = np.loadtxt(os.path.join(GOLDEN, "config1_eigenvalues.txt"))
    out = L.lobpcg(el, synth.initial_block(el))
    assert out["converged"] and out["res"].max() <= 1e-8
    np.testing.assert_allclose(out["theta"], data, atol=1e-9)


# ------------------------------------------------- restriction + SVD

def test_restriction_orthonormalisation():
    gen = np.random.default_rng(8)
    n = (12, 9, 6)
    el = make_element(n, (6.0, 5.0, 4.0), m=6, J=5)
    el.e_lo, el.e_hi = synth.element_box(n)
    x = L.cholesky_qr(gen.standard_normal((6, el.ng)))
    phi = alb.orthonormalise(alb.restrict(x, el), el.dv)
    np.testing.assert_allclose(phi @ phi.T * el.dv, np.eye(5), atol=1e-12)
    assert alb.sin_max_angle(alb.restrict(x, el), phi) < 1e-12
    # an explicit Gram-Schmidt of the restricted rows spans the same space
    q = alb.restrict(x, el).copy()
    for i in range(5):
        for j in range(i):
            q[i] -= (q[i] @ q[j]) * q[j]
        q[i] /= np.linalg.norm(q[i])
    assert alb.sin_max_angle(q, phi) < 1e-12
    assert phi.shape[1] == 4 * 3 * 6   # E_K = [4,8) x [3,6) x [0,6): zero elsewhere


def points_in_box_by_coordinates(n, L_, lo_frac, hi_frac):
    """Flat indices (x fastest) of the grid points whose coordinates x_a =
    i_a L_a / n_a satisfy lo_frac[a] L_a <= x_a < hi_frac[a] L_a, found by
    visiting every point in z, y, x order (exact rational comparison)."""
    from fractions import Fraction
    out = []
    for k in range(n[2]):
        for j in range(n[1]):
            for i in range(n[0]):
                inside = all(Fraction(lo_frac[a]) <= Fraction(idx, n[a]) < Fraction(hi_frac[a])
                             for a, idx in enumerate((i, j, k)))
                if inside:
                    out.append(i + n[0] * (j + n[1] * k))
    return np.array(out)


@pytest.mark.parametrize("n", [(12, 9, 5), (48, 64, 40), (20, 15, 9), (10, 14, 6)])
def test_element_indices_from_coordinates(n):
    """E_K is the set of points with coordinate in [L/3, 2L/3) along x and y,
    all z (the reading of the element inside its extended element): the
    oracle's index map (from synth's grid-index box) must list exactly those
    points, in x-fastest order.  Non-cubic grids catch an x/y swap."""
    from fractions import Fraction
    L_ = (7.0, 9.0, 4.0)
    el = make_element(n, L_, m=2, J=2)
    el.e_lo, el.e_hi = synth.element_box(n)
    got = alb.element_indices(el)
    ref = points_in_box_by_coordinates(n, L_, (Fraction(1, 3), Fraction(1, 3), 0), (Fraction(2, 3), Fraction(2, 3), 1))
    np.testing.assert_array_equal(got, ref)


def test_element_indices_asymmetric_box():
    """An arbitrary grid-index box with different bounds on every axis: the
    index map equals the brute-force list of points inside it."""
    from fractions import Fraction
    n = (11, 7, 6)
    el = make_element(n, (5.0, 6.0, 7.0), m=2, J=2)
    el.e_lo, el.e_hi = (2, 1, 3), (9, 4, 5)
    got = alb.element_indices(el)
    ref = points_in_box_by_coordinates(n, (5.0, 6.0, 7.0), tuple(Fraction(l, d) for l, d in zip(el.e_lo, n)),
                                       tuple(Fraction(h, d) for h, d in zip(el.e_hi, n)))
    np.testing.assert_array_equal(got, ref)
    assert len(got) == 7 * 3 * 2


def test_restriction_whole_box_reproduces_span():
    gen = np.random.default_rng(9)
    el = make_element((8, 6, 4), (5.0, 4.0, 3.0), m=5, J=5)
    x = L.cholesky_qr(gen.standard_normal((5, el.ng)))
    phi = alb.orthonormalise(alb.restrict(x, el), el.dv)
    assert alb.sin_max_angle(x, phi) < 1e-13
    np.testing.assert_allclose(phi @ phi.T * el.dv, np.eye(5), atol=1e-12)


def test_orthonormalise_top_keeps_the_largest_singular_directions():
    """The restriction variant (all k vectors restricted, the J left singular
    vectors of the largest singular values kept), on a block built from
    known singular vectors and values: the kept rows span exactly the first
    J of them, are orthonormal in the dV inner product, and with J = k span
    the same space as the paper's procedure."""
    from oracle import alb
    gen = np.random.default_rng(3)
    ne, k, J, dv = 500, 12, 8, 0.3
    u0, _ = np.linalg.qr(gen.standard_normal((ne, k)))
    v0, _ = np.linalg.qr(gen.standard_normal((k, k)))
    s = np.geomspace(10.0, 0.01, k)
    phit = ((u0 * s) @ v0.T).T  # (k, ne): rows are the restricted vectors
    phi = alb.orthonormalise_top(phit, dv, J)
    np.testing.assert_allclose(phi @ phi.T * dv, np.eye(J), atol=1e-12)
    assert alb.sin_max_angle(u0[:, :J].T, phi) < 1e-10
    assert alb.sin_max_angle(alb.orthonormalise(phit, dv), alb.orthonormalise_top(phit, dv, k)) < 1e-10
