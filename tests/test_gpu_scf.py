"""SCF-mode steps: a fixed number of LOBPCG iterations from a warm start under
an updated potential (Sec. II.B: every SCF iteration refines the ALBs with a
few LOBPCG iterations started from those of the previous SCF step).

Parity: the oracle runs the same number of iterations from the same block
(its own converged block for the old potential, given to the GPU through
set_initial) under the same new potential; Ritz values and residuals are
compared.  A warm start from the GPU's own resident block is checked against
the oracle's H (residuals recomputed from the returned block).
"""

import dataclasses

import numpy as np
import pytest

import __graft_entry__ as entry
import synth
from oracle import alb, hamiltonian as H, lobpcg as OL
from paper_1506_08147_gb300 import binding as B

pytestmark = pytest.mark.gpu

N_ITER = 3


@pytest.fixture(scope="module", autouse=True)
def _built():
    entry.build()


def small_element():
    # 16 x 12 x 10 periodic box, 6 atoms: local potential + 12 projectors
    return synth.random_element(9, 0, (16, 12, 10), 6, J=8, m=10, tol=1e-9)


def perturbed(el, amp=0.05, seed=11):
    """The element under an SCF-like update of its potential: a smooth seeded
    field of amplitude amp Ha added to V_eff."""
    gen = np.random.default_rng(seed)
    nx, ny, nz = el.n
    z, y, x = np.meshgrid(np.arange(nz) / nz, np.arange(ny) / ny, np.arange(nx) / nx, indexing="ij")
    ph = gen.uniform(0, 2 * np.pi, size=3)
    dv = amp * (np.cos(2 * np.pi * x + ph[0]) * np.cos(2 * np.pi * y + ph[1]) + np.sin(2 * np.pi * z + ph[2]))
    return dataclasses.replace(el, veff=el.veff + dv.reshape(el.veff.shape))


@pytest.fixture(scope="module")
def warm_case():
    el0 = small_element()
    x0 = OL.lobpcg(el0, synth.initial_block(el0), tol=1e-10, maxit=400)["X"]
    el1 = perturbed(el0)
    ref = OL.lobpcg(el1, x0, tol=0.0, maxit=N_ITER)
    return el0, el1, x0, ref


def check_block(c, el, rep):
    phi, eig, res = c.dgdft_alb_get_basis(0)
    x = c.dgdft_alb_get_block(0)
    assert rep["status"] == B.DGDFT_OK and rep["iterations"] == N_ITER
    # the reported residuals are those of the returned block under the new H
    r = H.apply_h(x[:el.J], el) - eig[:, None] * x[:el.J]
    got = np.linalg.norm(r, axis=1) / np.linalg.norm(x[:el.J], axis=1)
    np.testing.assert_allclose(res, got, rtol=1e-3, atol=1e-12)
    np.testing.assert_allclose(phi @ phi.T * el.dv, np.eye(el.J), atol=1e-12)
    xr = alb.restrict(x, el)
    sv = np.linalg.svd(xr, compute_uv=False)
    assert alb.sin_max_angle(xr, phi) < max(1e-10, 1e-14 * sv[0] / sv[-1])
    return eig, res


@pytest.mark.parametrize("prec", [B.DGDFT_PREC_FP64, B.DGDFT_PREC_MIXED])
def test_scf_step_matches_oracle(prec, warm_case):
    _, el1, x0, ref = warm_case
    c = B.Context([B.element_dict(el1)], precision=prec, keep_block=True)
    B.load_element(c, 0, el1, x0)
    st, reps = c.dgdft_alb_scf_step(N_ITER)
    assert st == B.DGDFT_OK, reps
    eig, res = check_block(c, el1, reps[0])
    J = el1.J
    if prec == B.DGDFT_PREC_FP64:
        # the same iteration in FP64 from the same block: Ritz values agree to
        # rounding propagated through three Rayleigh-Ritz steps, residuals
        # to a few percent
        np.testing.assert_allclose(eig, ref["theta"][:J], rtol=0, atol=1e-9)
        assert np.max(res) <= 1.05 * np.max(ref["res"][:J]) + 1e-10
    else:
        # FP32 iterations: Ritz values within FP32 rounding of the H apply,
        # residuals no worse than the FP64 run or the FP32 floor
        np.testing.assert_allclose(eig, ref["theta"][:J], rtol=0, atol=1e-5)
        assert np.max(res) <= max(1.5 * np.max(ref["res"][:J]), 5e-6)
    c.close()


def test_scf_step_warm_from_previous_solve(warm_case):
    # solve under the old potential, update the potential, step from the
    # resident block (converged like the oracle's, so the step matches the
    # oracle's three iterations from its own block); then a second step
    # continues from the first
    el0, el1, _, ref = warm_case
    el2 = perturbed(el0, amp=0.07, seed=12)
    c = B.Context([B.element_dict(el0)], precision=B.DGDFT_PREC_FP64, tol=1e-9, keep_block=True)
    B.load_element(c, 0, el0, synth.initial_block(el0))
    st, _ = c.dgdft_alb_solve()
    assert st == B.DGDFT_OK
    # residual of the solved block under the new potential (Rayleigh quotients)
    xs = c.dgdft_alb_get_block(0)[:el1.J]
    hx = H.apply_h(xs, el1)
    th = np.einsum("ij,ij->i", xs, hx) / np.einsum("ij,ij->i", xs, xs)
    start_res = np.max(np.linalg.norm(hx - th[:, None] * xs, axis=1) / np.linalg.norm(xs, axis=1))
    c.dgdft_alb_set_potential(0, np.ascontiguousarray(el1.veff.reshape(-1)))
    st, reps = c.dgdft_alb_scf_step(N_ITER)
    assert st == B.DGDFT_OK
    _, res1 = check_block(c, el1, reps[0])
    assert np.max(res1) < start_res
    assert np.max(res1) <= 1.05 * np.max(ref["res"][:el1.J]) + 1e-8
    c.dgdft_alb_set_potential(0, np.ascontiguousarray(el2.veff.reshape(-1)))
    st, reps = c.dgdft_alb_scf_step(N_ITER)
    assert st == B.DGDFT_OK
    check_block(c, el2, reps[0])
    c.close()


def start_ritz(x, el, J):
    """Ritz values of the block x (rows) under el's H, and the largest
    residual |H y - theta y| of its lowest J Ritz vectors y."""
    q, _ = np.linalg.qr(x.T)
    hq = H.apply_h(q.T, el)
    th, z = np.linalg.eigh(0.5 * (hq @ q + (hq @ q).T))
    y = z[:, :J].T @ q.T
    r = z[:, :J].T @ hq - th[:J, None] * y
    return th, float(np.max(np.linalg.norm(r, axis=1)))


def test_scf_step_monolayer_mixed():
    # monolayer elements: mixed-form solve, potential update, SCF step (FP32
    # iterations).  The returned block's residuals are recomputed with the
    # oracle's H; each kept Ritz value is at or below the same-index Ritz
    # value of the starting block under the new H (the step's subspace
    # contains the starting block), up to the FP32 rounding of the
    # iterations, and their sum drops.  The oracle runs the same three
    # iterations from the same block: Ritz values agree to FP32 rounding and
    # the residuals are no worse than the oracle's (a residual may grow over
    # a step: a state from outside the starting block can enter the kept J).
    # Two elements, so that the two half batches of the FP32 stage both run.
    els0 = synth.config2(elems=[0, 32])
    els1 = [perturbed(e, amp=0.02) for e in els0]
    c = B.Context([B.element_dict(e) for e in els0], precision=B.DGDFT_PREC_MIXED, keep_block=True)
    for k, e in enumerate(els0):
        B.load_element(c, k, e, synth.initial_block(e))
    st, _ = c.dgdft_alb_solve()
    assert st == B.DGDFT_OK
    blocks = [c.dgdft_alb_get_block(k) for k in range(len(els0))]
    for k, e in enumerate(els1):
        c.dgdft_alb_set_potential(k, np.ascontiguousarray(e.veff.reshape(-1)))
    st, reps = c.dgdft_alb_scf_step(N_ITER)
    assert st == B.DGDFT_OK
    for k, e in enumerate(els1):
        th0, r0 = start_ritz(blocks[k], e, e.J)
        ref = OL.lobpcg(e, blocks[k], tol=0.0, maxit=N_ITER)
        phi, eig, res = c.dgdft_alb_get_basis(k)
        x = c.dgdft_alb_get_block(k)
        assert reps[k]["status"] == B.DGDFT_OK and reps[k]["iterations"] == N_ITER
        assert reps[k]["restarts"] == 0
        r = H.apply_h(x[:e.J], e) - eig[:, None] * x[:e.J]
        got = np.linalg.norm(r, axis=1) / np.linalg.norm(x[:e.J], axis=1)
        np.testing.assert_allclose(res, got, rtol=1e-3, atol=1e-12)
        np.testing.assert_allclose(phi @ phi.T * e.dv, np.eye(e.J), atol=1e-12)
        assert np.all(eig <= th0[:e.J] + 1e-6)
        assert np.sum(th0[:e.J] - eig) > 1e-4
        np.testing.assert_allclose(eig, ref["theta"][:e.J], rtol=0, atol=1e-5)
        print(f"SCF step, element {[0, 32][k]}: max residual of the starting Ritz pairs {r0:.3e}, "
              f"after {np.max(got):.3e} (oracle {np.max(ref['res'][:e.J]):.3e})")
        assert np.max(got) <= max(1.5 * np.max(ref["res"][:e.J]), 5e-6)
    # the same step again from the same block and potential: the iteration
    # graphs captured by the first step are launched again and give bitwise
    # the same ALBs, eigenvalues and residuals
    first = [c.dgdft_alb_get_basis(k) for k in range(len(els0))]
    for k in range(len(els0)):
        c.dgdft_alb_set_initial(k, np.ascontiguousarray(blocks[k]))
    st, reps2 = c.dgdft_alb_scf_step(N_ITER)
    assert st == B.DGDFT_OK
    for k in range(len(els0)):
        for a, b in zip(first[k], c.dgdft_alb_get_basis(k)):
            assert np.array_equal(a, b)
    c.close()


def test_scf_steps_monolayer_workload():
    """The 36-element monolayer in the launch configuration of the benchmark
    (mixed form, both half batches): a solve, then SCF steps under a
    potential that alternates between V_eff + a smooth 0.02 Ha field and
    V_eff.  n_iter = 0 first gives the FP64 residuals of the starting block's
    Ritz pairs under the new potential.  No element may restart (a restart
    perturbs the block by 3 % and leaves residuals near 0.3 Ha after three
    iterations); the worst element of the last step and element 32 are
    checked against the oracle's three iterations from the same block.  The
    largest kept residual is not required to drop over a step: from a warm
    start under a 0.02 Ha change the vectors near the J cut mix with states
    from the guard set, and the oracle's own three iterations leave it 2-4x
    above the starting Ritz residual on these elements."""
    els = synth.config2()
    c = B.Context([B.element_dict(e) for e in els], precision=B.DGDFT_PREC_MIXED, keep_block=True)
    for k, e in enumerate(els):
        B.load_element(c, k, e, synth.initial_block(e))
    st, _ = c.dgdft_alb_solve()
    assert st == B.DGDFT_OK
    pert = [perturbed(e, amp=0.02, seed=20 + k) for k, e in enumerate(els)]
    for step in range(3):
        cur = pert if step % 2 == 0 else els
        for k, e in enumerate(cur):
            c.dgdft_alb_set_potential(k, np.ascontiguousarray(e.veff.reshape(-1)))
        st, before = c.dgdft_alb_scf_step(0)
        assert st == B.DGDFT_OK
        assert all(r["iterations"] == 0 for r in before)
        start = {k: c.dgdft_alb_get_block(k) for k in range(len(els))}
        st, after = c.dgdft_alb_scf_step(N_ITER)
        assert st == B.DGDFT_OK
        r0 = np.array([r["max_resid"] for r in before])
        r1 = np.array([r["max_resid"] for r in after])
        print(f"step {step}: max residual before {r0.max():.3e}, after {r1.max():.3e}")
        assert all(r["restarts"] == 0 for r in after)
    for k in sorted({32, int(np.argmax(r1))}):
        e = cur[k]
        ref = OL.lobpcg(e, start[k], tol=0.0, maxit=N_ITER)
        _, eig, res = c.dgdft_alb_get_basis(k)
        x = c.dgdft_alb_get_block(k)
        r = H.apply_h(x[:e.J], e) - eig[:, None] * x[:e.J]
        got = np.linalg.norm(r, axis=1)
        np.testing.assert_allclose(res, got, rtol=1e-3, atol=1e-12)
        np.testing.assert_allclose(eig, ref["theta"][:e.J], rtol=0, atol=1e-5)
        assert np.max(got) <= max(1.5 * np.max(ref["res"][:e.J]), 5e-6)
    c.close()


def test_scf_step_errors():
    el = small_element()
    c = B.Context([B.element_dict(el)], precision=B.DGDFT_PREC_FP64)
    B.load_element(c, 0, el)
    # no previous solve and no set_initial: nothing to start from
    st = c.lib.dgdft_alb_scf_step(c.h, N_ITER, None)
    assert st == B.DGDFT_ESTATE
    assert c.lib.dgdft_alb_scf_step(c.h, -1, None) == B.DGDFT_EINVAL
    c.close()
