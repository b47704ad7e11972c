"""Bounded device waits: a wait that runs out is reported, not hung on.

The tensor-core Gram kernel of the FP32 stage waits on mbarriers for its TMA
copies, its split warps, its MMAs and its tensor-memory read-out.  Every
wait is bounded (config device_wait_polls; about a second by default).  A
bound of one poll makes the first waits run out before the first copy has
landed: the kernel records the timeout on the element, waits (with the
default bound) for its copies and MMAs in flight, frees tensor memory and
returns.  Nothing traps or hangs: the call returns DGDFT_ETIMEOUT and the
device stays usable.
"""

import numpy as np
import pytest

import __graft_entry__ as entry
import synth
from oracle import hamiltonian as H
from paper_1506_08147_gb300 import binding as B

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    entry.build()


def test_gram_wait_timeout_is_reported():
    el = synth.config2(elems=[3])[0]
    gen = np.random.default_rng(5)
    blk = gen.standard_normal((6, el.m, el.ng))
    c = B.Context([B.element_dict(el)], precision=B.DGDFT_PREC_MIXED, device_wait_polls=1)
    B.load_element(c, 0, el)
    with pytest.raises(B.DgdftError) as ei:
        c.dgdft_alb_lobpcg_gram(0, blk, True, stage=0)
    assert ei.value.status == B.DGDFT_ETIMEOUT
    c.close()
    # the same products with the default bound, on the same device
    c = B.Context([B.element_dict(el)], precision=B.DGDFT_PREC_MIXED)
    B.load_element(c, 0, el)
    a, b, xtw = c.dgdft_alb_lobpcg_gram(0, blk, True)
    c.close()
    b32 = blk.astype(np.float32).astype(np.float64)
    s = np.vstack(b32[:3])
    assert np.max(np.abs(b[:el.m, :el.m] - s[:el.m] @ s[:el.m].T)) < 1e-5 * el.ng


def test_solve_with_timeouts_reports_and_recovers():
    """Every FP32-stage Gram launch times out: each element is stopped in
    that stage and marked; the FP64 stage (no device waits) then converges
    it from the FP32 block.  The solve returns DGDFT_ETIMEOUT and every
    report says so, while the returned Ritz pairs still meet the tolerance
    under the oracle's H."""
    els = synth.config2(elems=[0, 7])
    c = B.Context([B.element_dict(e) for e in els], precision=B.DGDFT_PREC_MIXED, tol=1e-6, maxit=600,
                  keep_block=True, device_wait_polls=1)
    for k, e in enumerate(els):
        B.load_element(c, k, e, synth.initial_block(e))
    st, reps = c.dgdft_alb_solve()
    assert st == B.DGDFT_ETIMEOUT
    assert all(r["status"] == B.DGDFT_ETIMEOUT for r in reps)
    assert all(r["iterations_bulk"] <= 1 for r in reps)
    for k, e in enumerate(els):
        _, eig, res = c.dgdft_alb_get_basis(k)
        x = c.dgdft_alb_get_block(k)
        r = H.apply_h(x[:e.J], e) - eig[:, None] * x[:e.J]
        assert np.max(np.linalg.norm(r, axis=1)) <= 1.05e-6
    c.close()
