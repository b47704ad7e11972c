"""Pins of the DG-assembly oracle (oracle/dg.py) against closed forms.

Each check ties a piece of Eq. DGHamiltonian's evaluation (Sec. II.B: LGL
quadrature and differentiation, the three groups of terms) to mathematics
the oracle does not compute itself:
  * LGL nodes and weights: the closed forms for 3, 4 and 5 points, exactness
    of the quadrature to degree 2n - 3, and its known value 2 / N for P_N^2;
  * differentiation matrices: exact on polynomials of degree < n;
  * trigonometric interpolation: the identity at the grid, and the values of
    numpy's FFT coefficients summed at the same points;
  * the penalty term: a piecewise-constant basis gives alpha times the
    face-area graph Laplacian of the element partition;
  * consistency of the face terms: for a smooth periodic u, a(u, v) equals
    <-1/2 Lap u + c u, v> on each element (closed-form integrals of
    products of cosines), which fixes the signs of both jump/average terms;
  * the whole pipeline (interpolation, LGL orthonormalisation, gradients,
    volume and face terms): built from the lowest plane waves of the cell,
    the DG matrix has eigenvalues 1/2 |G|^2;
  * the KB term: with the constant function, sum_p gamma_p (int b_p)^2 over
    the elements the projector is cut into, against the integral over the
    ball (radial quadrature);
  * symmetry H_{K,K'} = H_{K',K}^T with every term present;
  * the density (Eq. density): it integrates to the number of states with
    every term present, and from the lowest plane waves of the cell it is
    the uniform n / V (all 7 states) or 1 / V (the ground state alone).
"""

import numpy as np
import pytest
from scipy import integrate

import synth.dg as sdg
from oracle import dg


def test_lgl_closed_forms():
    x, w = dg.lgl_nodes_weights(3)
    assert np.allclose(x, [-1, 0, 1], atol=1e-15) and np.allclose(w, [1 / 3, 4 / 3, 1 / 3])
    x, w = dg.lgl_nodes_weights(4)
    a = 1 / np.sqrt(5)
    assert np.allclose(x, [-1, -a, a, 1]) and np.allclose(w, [1 / 6, 5 / 6, 5 / 6, 1 / 6])
    x, w = dg.lgl_nodes_weights(5)
    b = np.sqrt(3 / 7)
    assert np.allclose(x, [-1, -b, 0, b, 1], atol=1e-15)
    assert np.allclose(w, [1 / 10, 49 / 90, 32 / 45, 49 / 90, 1 / 10])


@pytest.mark.parametrize("n", [6, 12, 16, 42, 80])
def test_lgl_quadrature_degree(n):
    x, w = dg.lgl_nodes_weights(n)
    assert np.all(np.diff(x) > 0) and abs(w.sum() - 2) < 1e-13
    for k in range(2 * n - 2):
        exact = 2 / (k + 1) if k % 2 == 0 else 0.0
        assert abs(np.sum(w * x ** k) - exact) < 1e-13
    # degree 2n - 2 is not integrated exactly (LGL, not Gauss): the rule
    # gives 2 / N for P_N^2 (N = n - 1), whose integral is 2 / (2N + 1)
    from numpy.polynomial import legendre as leg
    N = n - 1
    c = np.zeros(N + 1)
    c[N] = 1
    assert abs(np.sum(w * leg.legval(x, c) ** 2) - 2 / N) < 1e-12


@pytest.mark.parametrize("n", [5, 16, 42, 80])
def test_diff_matrix_exact_on_polynomials(n):
    x, _ = dg.lgl_nodes_weights(n)
    D = dg.diff_matrix(x)
    # Legendre polynomials P_k, k < n, and their derivatives (numpy series)
    from numpy.polynomial import legendre as leg
    for k in range(n):
        c = np.zeros(k + 1)
        c[k] = 1
        f = leg.legval(x, c)
        df = leg.legval(x, leg.legder(c)) if k else np.zeros_like(x)
        assert np.max(np.abs(D @ f - df)) < 1e-10 * max(1, k * k)


@pytest.mark.parametrize("n", [9, 16, 24])
def test_trig_interp(n):
    L = 7.3
    grid = np.arange(n) * L / n
    T = dg.trig_interp_matrix(n, L, grid)
    assert np.allclose(T, np.eye(n), atol=1e-13)
    f = np.random.default_rng(n).standard_normal(n)
    pts = np.random.default_rng(n + 1).uniform(-L, 2 * L, 17)
    # FFT route: sum the coefficients (Nyquist term as its real cosine)
    F = np.fft.fft(f) / n
    m = np.fft.fftfreq(n, d=1.0 / n)
    vals = np.zeros(len(pts))
    for c, mm in zip(F, m):
        if n % 2 == 0 and abs(mm) == n // 2:
            vals += (c * np.cos(2 * np.pi * (n // 2) * pts / L)).real
        else:
            vals += (c * np.exp(2j * np.pi * mm * pts / L)).real
    assert np.allclose(dg.trig_interp_matrix(n, L, pts) @ f, vals, atol=1e-12)


def _empty(dom):
    e = (np.zeros(0, np.int32), np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0))
    return {k: e for k in range(dom.n_elem)}


@pytest.mark.parametrize("make", [sdg.dg_small_cube, sdg.dg_small_layer])
def test_penalty_is_face_graph_laplacian(make):
    dom = make()
    ne = dom.n_elem
    phis = {k: np.ones((1, dom.n_lgl)) for k in range(ne)}
    v = {k: np.zeros(dom.n_lgl) for k in range(ne)}
    A = dg.Assembly(dom, phis, v, _empty(dom), np.zeros(0), alpha=dom.alpha)
    le = dom.le
    area = [le[1] * le[2], le[0] * le[2], le[0] * le[1]]
    for k in range(ne):
        row = A.row(k)
        exp = {kk: 0.0 for kk in row}
        for d in range(3):
            for s in (-1, 1):
                c = list(dom.coords(k))
                c[d] += s
                nb = dom.index(*c)
                if nb != k:  # a face to itself has no jump
                    exp[k] += dom.alpha * area[d]
                    exp[nb] -= dom.alpha * area[d]
        for kk in row:
            assert abs(row[kk][0, 0] - exp[kk]) < 1e-10 * dom.alpha * max(area)


def _cos_int(k1, p1, k2, p2, a, b):
    """int_a^b cos(k1 x + p1) cos(k2 x + p2) dx."""
    def prim(kk, pp, x):
        return (np.sin(kk * x + pp) / kk) if kk != 0 else x * np.cos(pp)
    return 0.5 * (prim(k1 - k2, p1 - p2, b) - prim(k1 - k2, p1 - p2, a)
                  + prim(k1 + k2, p1 + p2, b) - prim(k1 + k2, p1 + p2, a))


def _separable_funcs(dom, n_fun, seed):
    gen = np.random.default_rng(seed)
    out = []
    for _ in range(n_fun):
        m = gen.integers(0, 2, size=3)  # modes 0 and 1: LGL error ~1e-10 at 12-16 points
        out.append((2 * np.pi * m / np.asarray(dom.cell), gen.uniform(0, 2 * np.pi, 3)))
    return out


def _eval_separable(f, g):
    (k, p) = f
    fx = np.cos(k[0] * g.cell_pts[0] + p[0])
    fy = np.cos(k[1] * g.cell_pts[1] + p[1])
    fz = np.cos(k[2] * g.cell_pts[2] + p[2])
    return (fz[:, None, None] * fy[None, :, None] * fx[None, None, :]).reshape(-1)


@pytest.mark.parametrize("make", [sdg.dg_small_cube, sdg.dg_small_layer])
def test_face_terms_consistent_for_smooth_u(make):
    """a(u, phi_{K,j}) = int_{E_K} (-1/2 Lap u + c u) phi_{K,j} for u = f_0,
    basis phi_{K,j} = f_j restricted to E_K (not orthonormalised)."""
    dom = make()
    funcs = _separable_funcs(dom, 4, 11)
    c0 = 0.37
    grids = {k: dg.ElementGrid(dom, k) for k in range(dom.n_elem)}
    phis = {k: np.stack([_eval_separable(f, grids[k]) for f in funcs]) for k in grids}
    v = {k: np.full(dom.n_lgl, c0) for k in grids}
    A = dg.Assembly(dom, phis, v, _empty(dom), np.zeros(0), alpha=dom.alpha)
    k0, p0 = funcs[0]
    lap = float(np.sum(k0 ** 2))
    for k in range(dom.n_elem):
        row = A.row(k)
        lhs = sum(blk[:, 0] for blk in row.values())  # coefficient 1 on f_0 everywhere
        lo = dom.corner(k)
        hi = lo + dom.le
        for j, (kj, pj) in enumerate(funcs):
            ov = np.prod([_cos_int(k0[d], p0[d], kj[d], pj[d], lo[d], hi[d]) for d in range(3)])
            # measured: 2e-10 (cube) and 7e-13 (layer) on values up to ~100
            assert abs(lhs[j] - (0.5 * lap + c0) * ov) < 1e-9 * (0.5 * lap + c0) * np.prod(dom.le), (k, j)


def _planewaves(dom, n):
    """The n lowest real plane waves of the cell (complete shells):
    list of (G, phase)."""
    ms = [(a, b, c) for a in range(-2, 3) for b in range(-2, 3) for c in range(-2, 3)]
    g2 = lambda m: sum((2 * np.pi * mm / L) ** 2 for mm, L in zip(m, dom.cell))
    ms.sort(key=lambda m: (g2(m), m))
    out = []
    for m in ms:
        if m == (0, 0, 0):
            out.append((np.zeros(3), 0.0))
        elif m > (0, 0, 0):
            G = 2 * np.pi * np.asarray(m) / np.asarray(dom.cell)
            out += [(G, 0.0), (G, -np.pi / 2)]
        if len(out) >= n:
            return out[:n]
    return out


def test_planewave_spectrum_through_whole_pipeline():
    """Q_K = the cell: the lowest plane waves sampled on Q_K's grid are the
    input columns; interpolation, LGL orthonormalisation, gradients, volume
    and face terms must give a DG matrix whose spectrum holds 1/2 |G|^2."""
    dom = sdg.dg_small_cube(J=7)
    waves = _planewaves(dom, dom.J)
    phis = {}
    for k in range(dom.n_elem):
        qo = dom.corner(k) - dom.e_off
        ax = [qo[d] + np.arange(dom.nq[d]) * dom.lq[d] / dom.nq[d] for d in range(3)]
        z = np.stack([
            (np.cos(G[2] * ax[2][:, None, None] + G[1] * ax[1][None, :, None]
                    + G[0] * ax[0][None, None, :] + ph)).reshape(-1) for G, ph in waves])
        phis[k] = dg.alb_on_lgl(dom, k, z)
        g = dg.ElementGrid(dom, k)
        assert np.allclose((phis[k] * g.w) @ phis[k].T, np.eye(dom.J), atol=1e-12)
    v = {k: np.zeros(dom.n_lgl) for k in range(dom.n_elem)}
    A = dg.Assembly(dom, phis, v, _empty(dom), np.zeros(0), alpha=dom.alpha)
    n = dom.n_elem * dom.J
    H = np.zeros((n, n))
    for k in range(dom.n_elem):
        for kk, blk in A.row(k).items():
            H[k * dom.J:(k + 1) * dom.J, kk * dom.J:(kk + 1) * dom.J] = blk
    assert np.allclose(H, H.T, atol=1e-10)
    ev = np.linalg.eigvalsh(H)
    exact = np.sort([0.5 * float(G @ G) for G, _ in waves])
    assert np.max(np.abs(ev[:dom.J] - exact)) < 1e-9, (ev[:dom.J], exact)


def test_kb_term_of_constant_function():
    """sum over elements of <b_p, 1> (each element's LGL quadrature of its
    piece) squared and weighted -> sum_p gamma_p (int_ball b_p)^2."""
    dom = sdg.dg_small_cube(J=1)
    gam = sdg.gamma_table(dom)
    phis, projs = {}, {}
    for k in range(dom.n_elem):
        g = dg.ElementGrid(dom, k)
        phis[k] = np.ones((1, dom.n_lgl))
        projs[k] = sdg.projectors_at(dom, *g.cell_pts)
    v = {k: np.zeros(dom.n_lgl) for k in range(dom.n_elem)}
    A = dg.Assembly(dom, phis, v, projs, gam, alpha=0.0)
    total = sum(sum(blk[0, 0] for blk in A.row(k).values()) for k in range(dom.n_elem))
    s2 = 0.5 ** 2
    ns = sdg._kb_norms()[0]
    ball = ns * integrate.quad(lambda r: 4 * np.pi * r * r * np.exp(-r * r / (2 * s2)), 0, 2.0,
                               epsabs=0, epsrel=1e-12)[0]
    exact = sum(gam[2 * a] for a in range(len(dom.atoms))) * ball ** 2  # p: int b_p = 0
    # LGL quadrature of the cut Gaussians (a 3e-4 step at r_c): measured 1.2e-5
    assert abs(total - exact) < 1e-4 * exact, (total, exact)


def test_blocks_symmetric_with_every_term():
    dom = sdg.dg_small_layer()
    gam = sdg.gamma_table(dom)
    phis, v, projs = {}, {}, {}
    for k in range(dom.n_elem):
        g = dg.ElementGrid(dom, k)
        phis[k] = dg.alb_on_lgl(dom, k, sdg.smooth_block(dom, k))
        v[k] = sdg.potential_at(dom, *g.cell_pts)
        projs[k] = sdg.projectors_at(dom, *g.cell_pts)
    A = dg.Assembly(dom, phis, v, projs, gam, alpha=dom.alpha)
    rows = {k: A.row(k) for k in range(dom.n_elem)}
    for k, row in rows.items():
        assert len(row) == 9  # 3 x 3 x 1 periodic neighbourhood
        for kk, blk in row.items():
            assert np.allclose(blk, rows[kk][k].T, atol=1e-10 * np.max(np.abs(blk)))


def test_density_integrates_to_states():
    dom = sdg.dg_small_layer()
    gam = sdg.gamma_table(dom)
    phis, v, projs = {}, {}, {}
    for k in range(dom.n_elem):
        g = dg.ElementGrid(dom, k)
        phis[k] = dg.alb_on_lgl(dom, k, sdg.smooth_block(dom, k))
        v[k] = sdg.potential_at(dom, *g.cell_pts)
        projs[k] = sdg.projectors_at(dom, *g.cell_pts)
    A = dg.Assembly(dom, phis, v, projs, gam, alpha=dom.alpha)
    H = dg.dense_matrix(dom, {k: A.row(k) for k in range(dom.n_elem)}, dom.J)
    for n_occ in (1, 10, dom.n_elem * dom.J):
        lam, rho = dg.density(dom, phis, H, n_occ, dom.J)
        total = sum(float(A.g(k).w @ rho[k]) for k in range(dom.n_elem))
        assert abs(total - n_occ) < 1e-10 * n_occ
        assert np.all(np.diff(lam) >= 0) and all(np.all(r >= 0) for r in rho.values())


def test_density_of_planewaves_is_uniform():
    dom = sdg.dg_small_cube(J=7)
    waves = _planewaves(dom, dom.J)
    phis = {}
    for k in range(dom.n_elem):
        qo = dom.corner(k) - dom.e_off
        ax = [qo[d] + np.arange(dom.nq[d]) * dom.lq[d] / dom.nq[d] for d in range(3)]
        z = np.stack([
            (np.cos(G[2] * ax[2][:, None, None] + G[1] * ax[1][None, :, None]
                    + G[0] * ax[0][None, None, :] + ph)).reshape(-1) for G, ph in waves])
        phis[k] = dg.alb_on_lgl(dom, k, z)
    v = {k: np.zeros(dom.n_lgl) for k in range(dom.n_elem)}
    A = dg.Assembly(dom, phis, v, _empty(dom), np.zeros(0), alpha=dom.alpha)
    H = dg.dense_matrix(dom, {k: A.row(k) for k in range(dom.n_elem)}, dom.J)
    vol = float(np.prod(dom.cell))
    for n_occ, level in ((1, 1.0), (dom.J, float(dom.J))):
        lam, rho = dg.density(dom, phis, H, n_occ, dom.J)
        for r in rho.values():
            assert np.allclose(r, level / vol, rtol=1e-8, atol=0)
