"""DG Hamiltonian assembly (Eq. DGHamiltonian) on the GPU against the oracle.

The GPU assembles every block row from J columns per element; the oracle
(oracle/dg.py) does the same from the same columns, each side with its own
LGL nodes, differentiation and interpolation tables, and V_eff / projectors
evaluated by synth at its own nodes.  The LGL-orthonormal basis is unique
given the columns (Cholesky), so blocks are compared element by element.

Cases: the two small domains (every block), the 576-atom monolayer at full
size (J = 40, 32 x 42 x 80 LGL points; sampled block rows), the blocks built
from a real ALB solve, the plane-wave spectrum through the GPU path (a closed
form), batching and host/device input invariance, and the error for a mass
matrix that is not positive definite.

Density (Eq. density, dense diagonalisation of H^DG): eigenvalues and rho
against the oracle on the small layer at an occupation with a spectral gap
(rho is unique there), rho integrating to the number of states, and the
closed-form uniform density of the lowest plane waves.
"""

import numpy as np
import pytest

import synth.dg as sdg
from oracle import dg as odg
from paper_1506_08147_gb300 import binding as B

pytestmark = pytest.mark.gpu

# FP64 on the oracle's side, FP64 or double-float pairs (dfloat) on the
# GPU's; differences come from summation order, from the two sides' own
# tables (LGL nodes, differentiation and interpolation matrices agree to
# ~1e-14 relative) and from the pair arithmetic's ~2^-48 per operation,
# amplified by the mass matrix's conditioning in the orthonormalisation.
H_RTOL = 1e-9
UNIT = {False: np.finfo(float).eps, True: 2.0 ** -44}  # rounding unit of the GPU's contractions
ARITH = [pytest.param(False, id="fp64"), pytest.param(True, id="dfloat")]


def make_dg(dom, **kw):
    return B.DG(dom.ne, dom.cell, dom.q_span, dom.nq, dom.nl, dom.J, dom.alpha,
                2 * len(dom.atoms), **kw)


def load_inputs(d, dom, elems=None):
    d.dgdft_dg_set_gamma(sdg.gamma_table(dom))
    for k in (range(dom.n_elem) if elems is None else elems):
        pts = d.dgdft_dg_lgl_points(k)
        d.dgdft_dg_set_potential(k, np.ascontiguousarray(sdg.potential_at(dom, *pts).reshape(-1)))
        pid, rp, idx, val = sdg.projectors_at(dom, *pts)
        d.dgdft_dg_set_projectors(k, pid, rp, idx, val)


class OracleDG:
    """Oracle assembly with lazily computed per-element bases."""

    def __init__(self, dom, blocks):
        self.dom = dom
        self.blocks = blocks
        phis, v, projs = _Lazy(self._phi), _Lazy(self._v), _Lazy(self._proj)
        self.A = odg.Assembly(dom, phis, v, projs, sdg.gamma_table(dom), dom.alpha)

    def _phi(self, k):
        return odg.alb_on_lgl(self.dom, k, self.blocks[k])

    def _v(self, k):
        g = self.A.g(k)
        return sdg.potential_at(self.dom, *g.cell_pts).reshape(-1)

    def _proj(self, k):
        g = self.A.g(k)
        return sdg.projectors_at(self.dom, *g.cell_pts)

    def row(self, k):
        return self.A.row(k)


class _Lazy(dict):
    def __init__(self, fn):
        super().__init__()
        self.fn = fn

    def __missing__(self, k):
        v = self.fn(k)
        self[k] = v
        return v


def compare_invariants(d, ora, rows, tag, rtol):
    """Quantities of a block row fixed by the spans of the two elements'
    ALBs alone: eigenvalues of H_KK, singular values of H_KK'."""
    worst, scale = 0.0, 0.0
    for k in rows:
        got = d.dgdft_dg_get_row(k)
        exp = ora.row(k)
        for kk in exp:
            scale = max(scale, np.max(np.abs(exp[kk])))
            if kk == k:
                a = np.linalg.eigvalsh(0.5 * (got[kk] + got[kk].T))
                b = np.linalg.eigvalsh(0.5 * (exp[kk] + exp[kk].T))
            else:
                a = np.linalg.svd(got[kk], compute_uv=False)
                b = np.linalg.svd(exp[kk], compute_uv=False)
            worst = max(worst, np.max(np.abs(a - b)))
    print(f"{tag}: max invariant difference {worst:.2e} of max |H| {scale:.2e}")
    assert worst <= rtol * scale


def compare_rows(d, ora, rows, tag, rtol=H_RTOL):
    worst, scale = 0.0, 0.0
    for k in rows:
        got = d.dgdft_dg_get_row(k)
        exp = ora.row(k)
        assert sorted(got) == sorted(exp)
        for kk in exp:
            scale = max(scale, np.max(np.abs(exp[kk])))
            worst = max(worst, np.max(np.abs(got[kk] - exp[kk])))
    print(f"{tag}: max |H_gpu - H_oracle| {worst:.2e} of max |H| {scale:.2e}")
    assert worst <= rtol * scale


@pytest.mark.parametrize("make", [sdg.dg_small_layer, sdg.dg_small_cube])
def test_lgl_basis_matches_oracle(make):
    dom = make()
    d = make_dg(dom)
    for k in (0, dom.n_elem - 1):
        z = sdg.smooth_block(dom, k)
        got = d.dgdft_dg_lgl_basis(k, z)
        exp = odg.alb_on_lgl(dom, k, z)
        err = np.max(np.abs(got - exp)) / np.max(np.abs(exp))
        print(f"{dom.ne} element {k}: LGL basis relative error {err:.2e}")
        assert err < 1e-11
    d.close()


@pytest.mark.parametrize("dfloat", ARITH)
@pytest.mark.parametrize("make", [sdg.dg_small_layer, sdg.dg_small_cube])
def test_assemble_small_domains_every_block(make, dfloat):
    dom = make()
    blocks = [sdg.smooth_block(dom, k) for k in range(dom.n_elem)]
    d = make_dg(dom, dfloat=dfloat)
    load_inputs(d, dom)
    d.dgdft_dg_assemble(blocks)
    compare_rows(d, OracleDG(dom, blocks), range(dom.n_elem), f"{dom.ne} dfloat={dfloat}")
    # the assembled matrix is symmetric across block rows
    rows = {k: d.dgdft_dg_get_row(k) for k in range(dom.n_elem)}
    for k, row in rows.items():
        for kk, blk in row.items():
            assert np.allclose(blk, rows[kk][k].T, rtol=0, atol=1e-11 * np.max(np.abs(blk)))
    timing, launches = d.dgdft_dg_last_timing()
    assert launches > 0 and all(v >= 0 for v in timing.values())
    d.close()


def test_batches_and_host_device_inputs_agree():
    torch = pytest.importorskip("torch")
    dom = sdg.dg_small_cube()
    blocks = [sdg.smooth_block(dom, k) for k in range(dom.n_elem)]
    d1 = make_dg(dom)
    load_inputs(d1, dom)
    d1.dgdft_dg_assemble(blocks)
    ref = {k: d1.dgdft_dg_get_row(k) for k in range(dom.n_elem)}
    d1.close()
    # batches of about two elements (scratch cap), device-resident columns
    d2 = make_dg(dom, hbm_cap_bytes=2 * 8 * (dom.J * (dom.ng_q + 5 * dom.n_lgl) + 40 * dom.J ** 2))
    load_inputs(d2, dom)
    dev = [torch.from_numpy(np.ascontiguousarray(z)).cuda() for z in blocks]
    d2.dgdft_dg_assemble(dev)
    for k in range(dom.n_elem):
        got = d2.dgdft_dg_get_row(k)
        for kk in ref[k]:
            assert np.array_equal(got[kk], ref[k][kk])
    d2.close()


@pytest.mark.parametrize("dfloat", ARITH)
def test_planewave_spectrum_on_gpu(dfloat):
    """Q_K = the cell, V = 0, no projectors: the DG matrix from the lowest
    plane waves has eigenvalues 1/2 |G|^2 (complete shells)."""
    dom = sdg.dg_small_cube(J=7)
    waves = []
    ms = sorted([(a, b, c) for a in range(-1, 2) for b in range(-1, 2) for c in range(-1, 2)],
                key=lambda m: (sum(v * v for v in m), m))
    for m in ms:
        G = 2 * np.pi * np.asarray(m) / np.asarray(dom.cell)
        if m == (0, 0, 0):
            waves.append((G, 0.0))
        elif m > (0, 0, 0):
            waves += [(G, 0.0), (G, -np.pi / 2)]
    waves = waves[:dom.J]
    blocks = []
    for k in range(dom.n_elem):
        qo = dom.corner(k) - dom.e_off
        ax = [qo[d] + np.arange(dom.nq[d]) * dom.lq[d] / dom.nq[d] for d in range(3)]
        blocks.append(np.stack([np.cos(G[2] * ax[2][:, None, None] + G[1] * ax[1][None, :, None]
                                       + G[0] * ax[0][None, None, :] + ph).reshape(-1) for G, ph in waves]))
    d = B.DG(dom.ne, dom.cell, dom.q_span, dom.nq, dom.nl, dom.J, dom.alpha, 0, dfloat=dfloat)
    d.dgdft_dg_assemble(blocks)
    n = dom.n_elem * dom.J
    H = np.zeros((n, n))
    for k in range(dom.n_elem):
        for kk, blk in d.dgdft_dg_get_row(k).items():
            H[k * dom.J:(k + 1) * dom.J, kk * dom.J:(kk + 1) * dom.J] = blk
    ev = np.linalg.eigvalsh(0.5 * (H + H.T))
    exact = np.sort([0.5 * float(G @ G) for G, _ in waves])
    err = np.max(np.abs(ev[:dom.J] - exact))
    print(f"plane-wave spectrum (dfloat={dfloat}): max error {err:.2e} Ha")
    assert err < 1e-9
    d.close()


def test_zero_column_reports_enotconv():
    dom = sdg.dg_small_cube()
    blocks = [sdg.smooth_block(dom, k) for k in range(dom.n_elem)]
    blocks[5][2] = 0.0
    d = make_dg(dom)
    load_inputs(d, dom)
    with pytest.raises(B.DgdftError) as ex:
        d.dgdft_dg_assemble(blocks)
    assert ex.value.status == B.DGDFT_ENOTCONV and "element 5" in str(ex.value)
    with pytest.raises(B.DgdftError) as ex:
        d.dgdft_dg_get_row(0)
    assert ex.value.status == B.DGDFT_ESTATE
    d.close()


@pytest.mark.parametrize("dfloat", ARITH)
def test_assemble_monolayer_full_size_sampled_rows(dfloat):
    """The 576-atom monolayer: 36 elements, J = 40, 32 x 42 x 80 LGL points,
    smooth seeded columns on the 48 x 64 x 40 grids; rows 0 and 7 against the
    oracle."""
    dom = sdg.dg_config2()
    blocks = [sdg.smooth_block(dom, k) for k in range(dom.n_elem)]
    d = make_dg(dom, dfloat=dfloat)
    load_inputs(d, dom)
    d.dgdft_dg_assemble(blocks)
    timing, launches = d.dgdft_dg_last_timing()
    print("stage ms:", {k: round(v, 3) for k, v in timing.items()}, "launches", launches)
    compare_rows(d, OracleDG(dom, blocks), [0, 7], f"monolayer dfloat={dfloat}")
    d.close()


@pytest.mark.parametrize("dfloat", ARITH)
def test_assemble_from_alb_solve(dfloat):
    """Blocks from a real ALB solve of the 36-element workload (the lowest J
    Ritz vectors of each element) handed over on the device; rows 0 and 7
    against the oracle from the same columns."""
    torch = pytest.importorskip("torch")
    import synth
    els = synth.config2()
    # no keep_block: the blocks are read from the resident wave on the device
    ctx = B.Context([B.element_dict(e) for e in els], precision=B.DGDFT_PREC_MIXED, tol=1e-6, maxit=600)
    for k, e in enumerate(els):
        B.load_element(ctx, k, e, synth.initial_block(e))
    st, rep = ctx.dgdft_alb_solve()
    assert st == B.DGDFT_OK
    dom = sdg.dg_config2()
    ng = dom.ng_q
    dev = []
    for k in range(dom.n_elem):
        x = torch.empty(els[k].m * ng, dtype=torch.float64, device="cuda")
        ctx.dgdft_alb_get_block(k, out=x)
        dev.append(x[:dom.J * ng])
    ctx.close()
    d = make_dg(dom, dfloat=dfloat)
    load_inputs(d, dom)
    d.dgdft_dg_assemble(dev)
    host = [t.view(dom.J, ng).cpu().numpy() for t in dev]
    # The lowest J Ritz vectors restricted to E_K are nearly dependent: the
    # mass matrix of Eq. orthonormal has condition kappa ~1e12, so both sides'
    # bases (and spans) are fixed only to rounding amplified by kappa^(1/2)
    # in their weak directions, times the length of the sums (interpolation
    # over 40-64 terms per pass, quadrature over 1e5 points): the tolerance
    # is 1e3 u kappa_max^(1/2) relative (u the unit of the GPU's arithmetic),
    # kappa_max over every element the two block rows touch.
    ora = OracleDG(dom, host)
    touched = sorted({kk for k in (0, 7) for kk in odg.neighbours(dom, k)})
    kappa = 0.0
    for k in touched:
        g = ora.A.g(k)
        pt = odg.interpolate_to_lgl(dom, g, host[k])
        kappa = max(kappa, np.linalg.cond((pt * g.w) @ pt.T))
    rtol = 1e3 * UNIT[dfloat] * np.sqrt(kappa)
    print(f"max cond(mass matrix) {kappa:.2e} over {len(touched)} elements: rtol {rtol:.1e}")
    compare_rows(d, ora, [0, 7], f"monolayer ALBs dfloat={dfloat}", rtol)
    compare_invariants(d, ora, [0, 7], "monolayer ALBs", rtol)
    d.close()


def _gap_occupation(lam, lo, hi):
    """An occupation in [lo, hi) with the largest gap above it."""
    gaps = lam[lo:hi] - lam[lo - 1:hi - 1]
    n = lo + int(np.argmax(gaps))
    return n, float(lam[n] - lam[n - 1])


def test_density_small_layer_matches_oracle():
    dom = sdg.dg_small_layer()
    blocks = [sdg.smooth_block(dom, k) for k in range(dom.n_elem)]
    d = make_dg(dom)
    load_inputs(d, dom)
    d.dgdft_dg_assemble(blocks)
    ora = OracleDG(dom, blocks)
    H = odg.dense_matrix(dom, {k: ora.row(k) for k in range(dom.n_elem)}, dom.J)
    lam_all = np.linalg.eigvalsh(0.5 * (H + H.T))
    n_occ, gap = _gap_occupation(lam_all, 10, 40)
    eig, rho = d.dgdft_dg_density(blocks, n_occ)
    lam, rho_o = odg.density(dom, ora.A.phis, H, n_occ, dom.J)
    e_err = np.max(np.abs(eig - lam)) / np.max(np.abs(lam))
    r_err = max(np.max(np.abs(rho[k] - rho_o[k])) for k in range(dom.n_elem)) / max(
        np.max(rho_o[k]) for k in range(dom.n_elem))
    total = sum(float(ora.A.g(k).w @ rho[k]) for k in range(dom.n_elem))
    timing, _ = d.dgdft_dg_last_timing()
    print(f"density n_occ {n_occ} (gap {gap:.2e} Ha): eigenvalue rel error {e_err:.2e}, rho rel error "
          f"{r_err:.2e}, integral {total:.12f}; ms {timing['density_eigensolve']:.2f} + "
          f"{timing['density_evaluation']:.2f}")
    assert e_err < 1e-11
    # rho is the projector onto the lowest n_occ states: its error scales
    # with rounding / gap
    assert r_err < 1e-10 * max(1.0, 1.0 / gap)
    assert abs(total - n_occ) < 1e-9 * n_occ
    d.close()


def test_density_of_planewaves_on_gpu():
    dom = sdg.dg_small_cube(J=7)
    ms = sorted([(a, b, c) for a in range(-1, 2) for b in range(-1, 2) for c in range(-1, 2)],
                key=lambda m: (sum(v * v for v in m), m))
    waves = []
    for m in ms:
        G = 2 * np.pi * np.asarray(m) / np.asarray(dom.cell)
        if m == (0, 0, 0):
            waves.append((G, 0.0))
        elif m > (0, 0, 0):
            waves += [(G, 0.0), (G, -np.pi / 2)]
    waves = waves[:dom.J]
    blocks = []
    for k in range(dom.n_elem):
        qo = dom.corner(k) - dom.e_off
        ax = [qo[d] + np.arange(dom.nq[d]) * dom.lq[d] / dom.nq[d] for d in range(3)]
        blocks.append(np.stack([np.cos(G[2] * ax[2][:, None, None] + G[1] * ax[1][None, :, None]
                                       + G[0] * ax[0][None, None, :] + ph).reshape(-1) for G, ph in waves]))
    d = B.DG(dom.ne, dom.cell, dom.q_span, dom.nq, dom.nl, dom.J, dom.alpha, 0)
    d.dgdft_dg_assemble(blocks)
    vol = float(np.prod(dom.cell))
    for n_occ, level in ((1, 1.0), (dom.J, float(dom.J))):
        eig, rho = d.dgdft_dg_density(blocks, n_occ)
        err = np.max(np.abs(rho * vol / level - 1.0))
        print(f"plane waves, {n_occ} states: max |rho V / n - 1| = {err:.2e}")
        assert err < 1e-9
    d.close()


def test_density_eigensolver_monolayer_scale():
    """n = 36 x 40 = 1440: the GPU eigenvalues of the assembled H^DG against
    numpy's dense eigvalsh of the same (GPU) blocks, and rho integrating to
    n_occ under the quadrature."""
    dom = sdg.dg_config2()
    blocks = [sdg.smooth_block(dom, k) for k in range(dom.n_elem)]
    d = make_dg(dom)
    load_inputs(d, dom)
    d.dgdft_dg_assemble(blocks)
    rows = {k: d.dgdft_dg_get_row(k) for k in range(dom.n_elem)}
    H = odg.dense_matrix(dom, rows, dom.J)
    lam = np.linalg.eigvalsh(0.5 * (H + H.T))
    n_occ = dom.n_elem * dom.J // 2
    eig, rho = d.dgdft_dg_density(blocks, n_occ)
    timing, _ = d.dgdft_dg_last_timing()
    err = np.max(np.abs(eig - lam[:n_occ])) / np.max(np.abs(lam))
    total = sum(float(odg.ElementGrid(dom, k).w @ rho[k]) for k in range(dom.n_elem))
    sweeps = d.dgdft_dg_density_info()
    print(f"n = {H.shape[0]}, n_occ = {n_occ}: eigenvalue error {err:.2e} of max |lambda| "
          f"{np.max(np.abs(lam)):.1f}; integral {total:.10f}; eigensolve {timing['density_eigensolve']:.1f} ms, "
          f"{sweeps} Jacobi sweeps")
    assert 0 < sweeps < 40
    assert err < 1e-12
    assert abs(total - n_occ) < 1e-8 * n_occ
    d.close()


def test_assemble_large_monolayer_row():
    """The 3,456-atom monolayer: 216 elements, J = 120, 32 x 42 x 96 LGL
    points (~800 MB of scratch per element, so the assembly runs in several
    memory-capped batches).  Every element gets the same seeded columns (V_eff
    and the projectors differ); block row 100 against the oracle."""
    dom = sdg.dg_config5()
    z = sdg.smooth_block(dom, 0)
    blocks = [z] * dom.n_elem
    d = make_dg(dom)
    load_inputs(d, dom)
    d.dgdft_dg_assemble(blocks)
    timing, launches = d.dgdft_dg_last_timing()
    print("large monolayer stage ms:", {k: round(v, 1) for k, v in timing.items() if not k.startswith("density")},
          "launches", launches)
    assert launches > 17  # more than one batch
    compare_rows(d, OracleDG(dom, blocks), [100], "large monolayer")
    d.close()
