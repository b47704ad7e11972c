"""GPU kernels of the learned preconditioner against the FP64 oracle.

The GPU stores weights in BF16 and accumulates in FP32, so the oracle runs on
the same BF16-rounded weights; tolerances then cover FP32 accumulation only.
Training pairs come from the plain FP64 solver: the CG targets must satisfy
(H - sigma I) t = r, checked with the oracle's H apply.
"""

import numpy as np
import pytest

import __graft_entry__ as entry
import synth
from oracle import convnet as N
from oracle import hamiltonian as H
from paper_1506_08147_gb300 import binding as B

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    entry.build()


def bf16_round(x):
    """Round float32 values to the nearest bfloat16 (ties to even)."""
    u = np.ascontiguousarray(x, np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def flat_params(params):
    return np.concatenate([np.concatenate([w.reshape(-1), b]) for w, b in params]).astype(np.float32)


def gpu_params(params):
    """Oracle parameters with weights rounded as the GPU stores them."""
    return [(bf16_round(w).astype(np.float64), b.astype(np.float32).astype(np.float64)) for w, b in params]


def small_ctx():
    el = synth.random_element(9, 0, (16, 12, 10), 6, J=8, m=10, tol=1e-9)
    c = B.Context([B.element_dict(el)])
    B.load_element(c, 0, el)
    return c, el


def test_forward_matches_oracle():
    gen = np.random.default_rng(31)
    params = N.init_params(gen)
    params = [(w, gen.standard_normal(b.shape) * 0.1) for w, b in params]
    c, _ = small_ctx()
    c.dgdft_alb_precond_set_params(flat_params(params))
    inp = gen.standard_normal((3, 2, 10, 12, 16)).astype(np.float32)
    got = c.dgdft_alb_precond_forward(inp)
    ref = np.stack([N.forward(gpu_params(params), inp[b].astype(np.float64))[0] for b in range(3)])
    assert np.max(np.abs(got - ref)) <= 2e-5 * np.max(np.abs(ref))
    c.close()


def test_loss_and_gradients_match_oracle():
    gen = np.random.default_rng(32)
    params = N.init_params(gen)
    params = [(w, gen.standard_normal(b.shape) * 0.05) for w, b in params]
    c, _ = small_ctx()
    c.dgdft_alb_precond_set_params(flat_params(params))
    Bn, n = 2, 14
    inp = gen.standard_normal((Bn, 2, n, n, n)).astype(np.float32)
    tgt = gen.standard_normal((Bn, 1, n, n, n)).astype(np.float32)
    lo, hi = 4, n - 4
    loss, grads = c.dgdft_alb_precond_loss_grad(inp, tgt, lo, hi)
    gp = gpu_params(params)
    ref_loss = 0.0
    ref_g = None
    cnt = Bn * (hi - lo) ** 3
    for b in range(Bn):
        out, acts = N.forward(gp, inp[b].astype(np.float64))
        d = np.zeros_like(out)
        sl = (slice(None), slice(lo, hi), slice(lo, hi), slice(lo, hi))
        d[sl] = (out - tgt[b])[sl]
        ref_loss += float(np.sum(d * d)) / cnt
        g = N.backward(gp, acts, 2.0 * d / cnt)
        fg = np.concatenate([np.concatenate([gw.reshape(-1), gb]) for gw, gb in g])
        ref_g = fg if ref_g is None else ref_g + fg
    assert abs(loss - ref_loss) <= 1e-5 * abs(ref_loss)
    assert np.max(np.abs(grads - ref_g)) <= 1e-4 * np.max(np.abs(ref_g))
    c.close()


def test_training_targets_and_loss_decrease(tmp_path):
    import torch
    c, el = small_ctx()
    r, t, sig, cg = c.dgdft_alb_precond_make_data(0, [3, 8])
    assert np.all(cg < 1000)
    m = el.m
    rr = r.cpu().numpy().reshape(2 * m, -1).astype(np.float64)
    tt = t.cpu().numpy().reshape(2 * m, -1).astype(np.float64)
    for q in range(2):
        rows = slice(q * m, (q + 1) * m)
        res = H.apply_h(tt[rows], el) - sig[q] * tt[rows] - rr[rows]
        rel = np.linalg.norm(res, axis=1) / np.linalg.norm(rr[rows], axis=1)
        assert np.max(rel) < 1e-5  # float32 storage of r and t
    v = torch.from_numpy(np.broadcast_to(el.veff.astype(np.float32), r.shape).copy()).cuda()
    c.dgdft_alb_precond_init(7)
    l0, l1 = c.dgdft_alb_precond_train(r, v, t, crop=10, batch=8, steps=200, lr=2e-3, seed=3)
    assert np.isfinite(l0) and np.isfinite(l1) and l1 < 0.7 * l0
    path = str(tmp_path / "w.bin")
    c.dgdft_alb_precond_save(path)
    p = c.dgdft_alb_precond_get_params()
    c.dgdft_alb_precond_init(99)
    c.dgdft_alb_precond_load(path)
    np.testing.assert_array_equal(c.dgdft_alb_precond_get_params(), p)
    c.close()


def _scaled_error(a, b):
    """Mean over fields of min_s |s a - b| / |b|: how well a approximates b up
    to the column scale LOBPCG ignores."""
    import torch
    dims = tuple(range(1, a.dim()))
    s = torch.sum(a * b, dim=dims) / torch.clamp(torch.sum(a * a, dim=dims), min=1e-30)
    err = torch.sqrt(torch.sum((s.view(-1, *([1] * (a.dim() - 1))) * a - b) ** 2, dim=dims)) / \
        torch.sqrt(torch.sum(b * b, dim=dims))
    return float(torch.mean(err))


def test_learned_preconditioner_held_out(capsys):
    """The network is trained on (residual, exact correction) pairs of one
    system and evaluated on another it has not seen: on the held-out pairs
    its output, rescaled by rms(r), must approximate the exact correction
    t = (H - sigma I)^-1 r better than the untrained network and better than
    the residual itself (W = R, no preconditioner), each up to the best
    scale per field -- what the preconditioner is trained for.  Then the
    held-out system is solved with Teter and with the network: both reach
    the tolerance with the same eigenvalues; the FP32-stage iteration counts
    are printed, not asserted (on this small system they differ by a few
    iterations either way)."""
    import torch
    train_el = synth.random_element(9, 5, (24, 24, 24), 10, J=16, m=24, tol=1e-6)
    test_el = synth.random_element(17, 5, (24, 24, 24), 10, J=16, m=24, tol=1e-6)

    def pairs(el):
        cc = B.Context([B.element_dict(el)], precision=B.DGDFT_PREC_FP64)
        B.load_element(cc, 0, el, synth.initial_block(el))
        r, t, _, _ = cc.dgdft_alb_precond_make_data(0, [4, 12, 30])
        cc.close()
        v = torch.from_numpy(np.broadcast_to(el.veff.astype(np.float32), r.shape).copy()).cuda()
        return r, t, v

    r, t, v = pairs(train_el)
    rh, th, vh = pairs(test_el)
    c = B.Context([B.element_dict(train_el)], precision=B.DGDFT_PREC_FP64)
    c.dgdft_alb_precond_init(11)

    def held_out_error():
        rms = torch.sqrt(torch.mean(rh * rh, dim=(1, 2, 3), keepdim=True))
        out = c.dgdft_alb_precond_forward(torch.stack([rh / rms, vh], dim=1).contiguous())[:, 0] * rms
        return _scaled_error(out, th)

    e_untrained = held_out_error()
    # ~20 s: with a tenth of the steps the network only learns to output ~0
    l0, l1 = c.dgdft_alb_precond_train(r, v, t, crop=20, batch=8, steps=3000, lr=1e-3, seed=5)
    e_net = held_out_error()
    e_res = _scaled_error(rh, th)
    params = c.dgdft_alb_precond_get_params()
    c.close()
    assert l1 < l0
    with capsys.disabled():
        print(f"\nheld-out error of the correction (best scale per field): network {e_net:.3f}, "
              f"untrained {e_untrained:.3f}, residual itself {e_res:.3f}; train loss {l0:.3e} -> {l1:.3e}")
    assert e_net < e_untrained and e_net < e_res
    out = {}
    for mode in (B.DGDFT_PRECOND_TETER, B.DGDFT_PRECOND_LEARNED):
        cc = B.Context([B.element_dict(test_el)], precision=B.DGDFT_PREC_MIXED, tol=1e-6, maxit=400,
                       precond=mode, keep_block=True)
        if mode == B.DGDFT_PRECOND_LEARNED:
            cc.dgdft_alb_precond_set_params(params)
        B.load_element(cc, 0, test_el, synth.initial_block(test_el))
        st, rep = cc.dgdft_alb_solve()
        assert st == B.DGDFT_OK, rep
        _, eig, res = cc.dgdft_alb_get_basis(0)
        x = cc.dgdft_alb_get_block(0)
        cc.close()
        rr = H.apply_h(x[:test_el.J], test_el) - eig[:, None] * x[:test_el.J]
        assert np.max(np.linalg.norm(rr, axis=1)) <= 1.05e-6
        out[mode] = (rep[0], eig)
    np.testing.assert_allclose(out[B.DGDFT_PRECOND_LEARNED][1], out[B.DGDFT_PRECOND_TETER][1], atol=1e-6)
    with capsys.disabled():
        print(f"held-out solve: FP32-stage iterations {out[1][0]['iterations_bulk']} with the network "
              f"(Teter {out[0][0]['iterations_bulk']}), total {out[1][0]['iterations']} "
              f"(Teter {out[0][0]['iterations']}), Teter fallbacks {out[1][0]['fallbacks']}")
