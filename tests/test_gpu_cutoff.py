"""Sphere-cutoff planewave set (dgdft_alb_config.ecut) on the GPU.

Against the dense Galerkin oracle (oracle/cutoff.py) on two small boxes with
projectors, batched together (two grids: the runtime-planned transforms):
eigenvalues, the returned vectors inside the set, the projected residual
recomputed by the oracle, and the span of the kept vectors against the
oracle's eigenvectors within the Davis-Kahan bound.  On one monolayer element
(48 x 64 x 40, the transforms specialised for that grid): the projection
step against the oracle, and a solve whose vectors lie in the set, whose
projected residuals meet the tolerance and whose Ritz values lie above the
grid problem's (Courant-Fischer).  The chosen mixed form (FP32 stage with its
FP32 mask, FP64 check and iterations) on both: against the oracle, and on
the monolayer element against the FP64 cutoff solve.  Sizes of the set are chosen with no
frequency on the sphere, so membership is never a rounding decision.
"""

import numpy as np
import pytest

import synth
from oracle import alb as OA
from oracle import cutoff as oc
from oracle import hamiltonian as H
from paper_1506_08147_gb300 import binding as B

pytestmark = pytest.mark.gpu


def _ecut(els, frac):
    ec = frac * min(oc.ngecut_ecut(e.n, e.L) for e in els)
    for e in els:
        assert np.min(np.abs(H.kinetic_symbol(e.n, e.L) - ec)) > 1e-6 * ec
    return ec


def _ctx(els, ec, tol, precision=B.DGDFT_PREC_FP64, **kw):
    ctx = B.Context([B.element_dict(e) for e in els], precision=precision, tol=tol, maxit=800,
                    keep_block=True, ecut=ec, **kw)
    for i, e in enumerate(els):
        B.load_element(ctx, i, e, synth.initial_block(e))
    return ctx


@pytest.fixture(scope="module")
def boxes():
    return synth.cutoff_boxes()


def test_projection_step_small_box(boxes):
    el = boxes[0]
    ec = _ecut([el], 0.9)
    ctx = _ctx([el], ec, 1e-8)
    x = np.random.default_rng(3).standard_normal((5, el.ng))
    got = ctx.dgdft_alb_project_cutoff(0, x)
    ctx.close()
    ref = oc.project(x, el.n, el.L, ec)
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(x))


@pytest.mark.parametrize("frac", [0.6, 0.9])
def test_solve_matches_galerkin_oracle(boxes, frac):
    ec = _ecut(boxes, frac)
    ctx = _ctx(boxes, ec, 1e-8)
    st, rep = ctx.dgdft_alb_solve()
    assert st == B.DGDFT_OK, rep
    for i, el in enumerate(boxes):
        J = el.J
        phi, eig, res = ctx.dgdft_alb_get_basis(i)
        x = ctx.dgdft_alb_get_block(i)[:J]
        mu, vec = oc.galerkin_eigenpairs(el, ec, el.m)
        lam, _ = oc.full_eigenpairs(el, J)
        print(f"box {i} ecut {ec:.3f} Ha: iterations {rep[i]['iterations']}, max |theta - oracle| "
              f"{np.max(np.abs(eig - mu[:J])):.2e}, above the grid problem by up to {np.max(eig - lam):.3e} Ha")
        assert np.max(res) <= 1e-8
        assert np.max(np.abs(eig - mu[:J])) <= 1e-11
        # not the grid problem
        assert np.max(eig - lam) > 1e-4
        # inside the set, and the projected residual from the oracle's H
        assert np.max(np.abs(oc.project(x, el.n, el.L, ec) - x)) <= 1e-12 * np.max(np.abs(x))
        r = oc.project(H.apply_h(x, el) - eig[:, None] * x, el.n, el.L, ec)
        assert np.max(np.linalg.norm(r, axis=1) / np.linalg.norm(x, axis=1)) <= 1.05e-8
        # span of the kept Ritz vectors: Davis-Kahan with the oracle's gap
        gap = mu[J] - mu[J - 1]
        bound = np.sqrt(J) * 1.05e-8 / gap
        assert OA.sin_max_angle(x, vec[:J]) <= max(bound, 1e-10), (gap, bound)
        # the ALBs span the restricted Ritz vectors
        assert OA.sin_max_angle(phi, OA.restrict(x, el, J)) <= 1e-10
    ctx.close()


def test_monolayer_element_cutoff():
    el = synth.config2(elems=[0])[0]
    ec = _ecut([el], 0.91)
    ctx = _ctx([el], ec, el.tol)
    x0 = np.random.default_rng(4).standard_normal((4, el.ng))
    got = ctx.dgdft_alb_project_cutoff(0, x0)
    assert np.max(np.abs(got - oc.project(x0, el.n, el.L, ec))) <= 1e-13 * np.max(np.abs(x0))
    st, rep = ctx.dgdft_alb_solve()
    assert st == B.DGDFT_OK, rep
    _, eig, res = ctx.dgdft_alb_get_basis(0)
    x = ctx.dgdft_alb_get_block(0)[:el.J]
    ctx.close()
    grid = _ctx([el], 0.0, el.tol)
    st, rep_g = grid.dgdft_alb_solve()
    assert st == B.DGDFT_OK
    _, eig_g, _ = grid.dgdft_alb_get_basis(0)
    grid.close()
    t_cut = rep[0]["seconds"] / rep[0]["iterations"]
    t_grid = rep_g[0]["seconds"] / rep_g[0]["iterations"]
    print(f"monolayer element, ecut {ec:.3f} Ha ({int(oc.cutoff_mask(el.n, el.L, ec).sum())} of {el.ng} "
          f"planewaves): {rep[0]['iterations']} iterations, {1e3 * t_cut:.2f} ms each; grid problem "
          f"{rep_g[0]['iterations']} iterations, {1e3 * t_grid:.2f} ms each; Ritz values above the grid's "
          f"by {np.min(eig - eig_g):.2e} .. {np.max(eig - eig_g):.2e} Ha")
    assert np.max(res) <= el.tol
    assert np.max(np.abs(oc.project(x, el.n, el.L, ec) - x)) <= 1e-12 * np.max(np.abs(x))
    r = oc.project(H.apply_h(x, el) - eig[:, None] * x, el.n, el.L, ec)
    assert np.max(np.linalg.norm(r, axis=1) / np.linalg.norm(x, axis=1)) <= 1.05 * el.tol
    # Courant-Fischer: the Galerkin eigenvalues lie above the grid's (both
    # sides' Ritz values are within res^2 / gap of their eigenvalues)
    assert np.all(eig >= eig_g - 1e-8)


def test_scf_step_stays_in_the_set(boxes):
    """SCF-mode steps of the cutoff solve: box 0 restarts from a block with
    out-of-set noise (the step projects it), box 1 from its resident block."""
    ec = _ecut(boxes, 0.9)
    ctx = _ctx(boxes, ec, 1e-8)
    st, _ = ctx.dgdft_alb_solve()
    assert st == B.DGDFT_OK
    el0 = boxes[0]
    x0 = ctx.dgdft_alb_get_block(0)
    noise = np.random.default_rng(9).standard_normal(x0.shape)
    ctx.dgdft_alb_set_initial(0, np.ascontiguousarray(x0 + 1e-4 * noise))
    st, rep = ctx.dgdft_alb_scf_step(3)
    assert st in (B.DGDFT_OK, B.DGDFT_ENOTCONV)
    for i, el in enumerate(boxes):
        _, eig, _ = ctx.dgdft_alb_get_basis(i)
        x = ctx.dgdft_alb_get_block(i)[:el.J]
        mu, _ = oc.galerkin_eigenpairs(el, ec, el.J)
        assert np.max(np.abs(oc.project(x, el.n, el.L, ec) - x)) <= 1e-12 * np.max(np.abs(x))
        # Ritz values of a subspace of range(P) lie above the Galerkin eigenvalues
        assert np.all(eig >= mu - 1e-11)
        assert np.max(eig - mu) <= (1e-4 if i == 0 else 1e-11)
    ctx.close()


def test_mixed_form_small_boxes(boxes):
    ec = _ecut(boxes, 0.9)
    ctx = _ctx(boxes, ec, 1e-6, precision=B.DGDFT_PREC_MIXED)
    st, rep = ctx.dgdft_alb_solve()
    assert st == B.DGDFT_OK, rep
    for i, el in enumerate(boxes):
        J = el.J
        phi, eig, res = ctx.dgdft_alb_get_basis(i)
        x = ctx.dgdft_alb_get_block(i)[:J]
        mu, _ = oc.galerkin_eigenpairs(el, ec, J)
        print(f"mixed, box {i}: iterations {rep[i]['iterations']} (FP32 {rep[i]['iterations_bulk']}), "
              f"max |theta - oracle| {np.max(np.abs(eig - mu)):.2e}")
        assert np.max(res) <= 1e-6
        assert np.max(np.abs(eig - mu)) <= 1e-9
        assert np.max(np.abs(oc.project(x, el.n, el.L, ec) - x)) <= 1e-12 * np.max(np.abs(x))
        r = oc.project(H.apply_h(x, el) - eig[:, None] * x, el.n, el.L, ec)
        assert np.max(np.linalg.norm(r, axis=1) / np.linalg.norm(x, axis=1)) <= 1.05e-6
        assert OA.sin_max_angle(phi, OA.restrict(x, el, J)) <= 1e-10
    ctx.close()


def test_mixed_form_monolayer_element():
    el = synth.config2(elems=[0])[0]
    ec = _ecut([el], 0.91)
    out = {}
    for name, prec in (("fp64", B.DGDFT_PREC_FP64), ("mixed", B.DGDFT_PREC_MIXED)):
        ctx = _ctx([el], ec, el.tol, precision=prec)
        st, rep = ctx.dgdft_alb_solve()
        assert st == B.DGDFT_OK, rep
        _, eig, res = ctx.dgdft_alb_get_basis(0)
        out[name] = (eig, res, ctx.dgdft_alb_get_block(0)[:el.J], rep[0])
        ctx.close()
    eig, res, x, rep = out["mixed"]
    print(f"mixed, monolayer element with the cutoff: {rep['iterations']} iterations "
          f"(FP32 {rep['iterations_bulk']}) in {rep['seconds']:.3f} s; FP64: {out['fp64'][3]['iterations']} "
          f"in {out['fp64'][3]['seconds']:.3f} s; max |theta_mixed - theta_fp64| "
          f"{np.max(np.abs(eig - out['fp64'][0])):.2e}")
    assert np.max(res) <= el.tol
    assert np.max(np.abs(eig - out["fp64"][0])) <= 1e-8
    assert np.max(np.abs(oc.project(x, el.n, el.L, ec) - x)) <= 1e-12 * np.max(np.abs(x))
    r = oc.project(H.apply_h(x, el) - eig[:, None] * x, el.n, el.L, ec)
    assert np.max(np.linalg.norm(r, axis=1) / np.linalg.norm(x, axis=1)) <= 1.05 * el.tol

