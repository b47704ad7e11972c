"""Pins of the learned-preconditioner network oracle (oracle/convnet.py).

* conv3d equals a brute-force 7-deep loop over taps with explicit modulo
  indexing on tiny grids (and a scipy periodic correlation on a larger one);
* every gradient matches central finite differences of the loss;
* the network is equivariant under periodic translation of its inputs and
  the preconditioner output scales linearly with the residual.
"""

import numpy as np
import scipy.ndimage as ndi

from oracle import convnet as N


def brute_conv(x, w, b):
    ci, nz, ny, nx = x.shape
    co = w.shape[0]
    out = np.zeros((co, nz, ny, nx))
    for o in range(co):
        for z in range(nz):
            for y in range(ny):
                for xx in range(nx):
                    s = b[o]
                    for i in range(ci):
                        for dz in range(3):
                            for dy in range(3):
                                for dx in range(3):
                                    s += w[o, i, dz, dy, dx] * x[i, (z + dz - 1) % nz, (y + dy - 1) % ny,
                                                                  (xx + dx - 1) % nx]
                    out[o, z, y, xx] = s
    return out


def test_conv3d_brute_force():
    gen = np.random.default_rng(0)
    x = gen.standard_normal((2, 4, 3, 5))
    w = gen.standard_normal((3, 2, 3, 3, 3))
    b = gen.standard_normal(3)
    np.testing.assert_allclose(N.conv3d(x, w, b), brute_conv(x, w, b), atol=1e-12)


def test_conv3d_matches_scipy_periodic_correlation():
    gen = np.random.default_rng(1)
    x = gen.standard_normal((1, 8, 6, 10))
    w = gen.standard_normal((1, 1, 3, 3, 3))
    ref = ndi.correlate(x[0], w[0, 0], mode="wrap")
    np.testing.assert_allclose(N.conv3d(x, w, np.zeros(1))[0], ref, atol=1e-12)


def test_gradients_finite_differences():
    gen = np.random.default_rng(2)
    params = N.init_params(gen, channels=(2, 3, 3, 1))
    params = [(w, gen.standard_normal(b.shape) * 0.1) for w, b in params]
    r = gen.standard_normal((4, 5, 6))
    v = gen.standard_normal((4, 5, 6))
    t = gen.standard_normal((4, 5, 6))
    loss, grads = N.loss_and_grads(params, r, v, t)
    h = 1e-6
    for k in range(len(params)):
        for which in (0, 1):
            arr = params[k][which]
            flat = arr.reshape(-1)
            for idx in gen.choice(flat.size, size=min(6, flat.size), replace=False):
                old = flat[idx]
                flat[idx] = old + h
                lp, _ = N.loss_and_grads(params, r, v, t)
                flat[idx] = old - h
                lm, _ = N.loss_and_grads(params, r, v, t)
                flat[idx] = old
                fd = (lp - lm) / (2 * h)
                an = grads[k][which].reshape(-1)[idx]
                assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)), (k, which, idx, fd, an)


def test_input_gradient_finite_differences():
    gen = np.random.default_rng(3)
    x = gen.standard_normal((2, 3, 4, 5))
    w = gen.standard_normal((2, 2, 3, 3, 3))
    g = gen.standard_normal((2, 3, 4, 5))
    gx, _, _ = N.conv3d_backward(x, w, g)
    h = 1e-6
    for idx in [(0, 0, 0, 0), (1, 2, 3, 4), (0, 1, 2, 3)]:
        xp = x.copy()
        xp[idx] += h
        xm = x.copy()
        xm[idx] -= h
        fd = (np.sum(g * N.conv3d(xp, w, np.zeros(2))) - np.sum(g * N.conv3d(xm, w, np.zeros(2)))) / (2 * h)
        assert abs(fd - gx[idx]) < 1e-7


def test_translation_equivariance_and_scaling():
    gen = np.random.default_rng(4)
    params = N.init_params(gen)
    r = gen.standard_normal((6, 5, 4))
    v = gen.standard_normal((6, 5, 4))
    w0 = N.precondition(params, r, v)
    sh = (2, 1, 3)
    w1 = N.precondition(params, np.roll(r, sh, axis=(0, 1, 2)), np.roll(v, sh, axis=(0, 1, 2)))
    np.testing.assert_allclose(w1, np.roll(w0, sh, axis=(0, 1, 2)), atol=1e-12)
    np.testing.assert_allclose(N.precondition(params, 3.5 * r, v), 3.5 * w0, atol=1e-11)
