"""The DG step's inputs (synth/dg.py) against the ALB step's own inputs.

The DG assembly evaluates V_eff and the KB projection functions at LGL points
through synth/dg.py, the ALB solve tabulates them on the extended elements'
uniform grids through synth/workloads.py.  Both must describe the same
functions:
  * V_eff at an extended element's uniform grid points equals that
    element's tabulated V_eff;
  * the KB functions at those points have the tabulated projectors' shapes
    (the two normalise differently: unit norm over the cut ball here, unit
    grid norm there);
  * the KB normalisation: integral of b^2 over the ball is 1 by a fine
    Cartesian quadrature (independent of the radial integral synth uses).
"""

import numpy as np

import synth
import synth.dg as sdg
from synth import fields


def test_potential_matches_alb_input():
    dom = sdg.dg_config2()
    el = synth.config2(elems=[7])[0]
    qo = dom.corner(7) - dom.e_off
    ax = [np.mod(qo[d], dom.cell[d]) + np.arange(dom.nq[d]) * dom.lq[d] / dom.nq[d] for d in range(3)]
    v = sdg.potential_at(dom, *ax)
    assert np.max(np.abs(v - el.veff)) < 1e-10 * np.max(np.abs(el.veff))


def test_projector_shapes_match_alb_input():
    dom = sdg.dg_config2()
    el = synth.config2(elems=[7])[0]
    qo = dom.corner(7) - dom.e_off
    ax = [np.mod(qo[d], dom.cell[d]) + np.arange(dom.nq[d]) * dom.lq[d] / dom.nq[d] for d in range(3)]
    pid, rp, idx, val = sdg.projectors_at(dom, *ax)
    dg_rows = {}
    for r in range(len(pid)):
        dg_rows.setdefault(tuple(idx[rp[r]:rp[r + 1]]), []).append(val[rp[r]:rp[r + 1]])
    matched = 0
    for r in range(el.n_proj):
        key = tuple(el.proj_idx[el.proj_row_ptr[r]:el.proj_row_ptr[r + 1]])
        alb = el.proj_val[el.proj_row_ptr[r]:el.proj_row_ptr[r + 1]]
        for cand in dg_rows.get(key, []):
            # proportional: one constant per projector
            c = cand @ alb / (alb @ alb)
            if np.max(np.abs(cand - c * alb)) <= 1e-12 * np.max(np.abs(cand)):
                matched += 1
                break
    # the ALB step keeps atoms with centres inside Q_K and drops points
    # outside it; those projectors appear at the same points here
    assert matched == el.n_proj


def test_kb_normalisation_on_fine_grid():
    ns, npn = sdg._kb_norms()
    h = 0.04
    x = np.arange(-fields.RCUT_KB, fields.RCUT_KB + h / 2, h)
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    r2 = X * X + Y * Y + Z * Z
    inside = r2 <= fields.RCUT_KB ** 2
    g = np.exp(-r2 / (2 * fields.SIGMA_KB ** 2)) * inside
    s_int = np.sum((ns * g) ** 2) * h ** 3
    p_int = np.sum((npn * Z * g) ** 2) * h ** 3
    assert abs(s_int - 1.0) < 2e-3 and abs(p_int - 1.0) < 2e-3
