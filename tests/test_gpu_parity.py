"""GPU parity of every step of the hot path against the FP64 CPU oracle.

All calls go through the C-ABI (include/dgdft_alb.h, dgdft_alb_steps.h).
Tolerances: FP64 steps to ~1e-12 relative; the mixed form's FP32 steps to
a few units of FP32 rounding times the step's conditioning (stated per
test).  Full solves: FP64 eigenvalues within 1e-8 Ha and subspace sine
within 1e-7 (where the spectral gap allows, Davis-Kahan); mixed form within
1e-6 Ha and 1e-5.
"""

import os

import numpy as np
import pytest
import scipy.linalg as sla

import __graft_entry__ as entry
import synth
import oracle_compare as OC
from oracle import alb, hamiltonian as H, lobpcg as OL, teter as T
from paper_1506_08147_gb300 import binding as B

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
PRECS = [B.DGDFT_PREC_FP64, B.DGDFT_PREC_MIXED]
# (precision, stage) of the H apply: plain FP64, the mixed form's FP32 stage,
# and its FP64 stage (FP64 vectors, transforms in double-float arithmetic)
H_KINDS = [(B.DGDFT_PREC_FP64, 0), (B.DGDFT_PREC_MIXED, 0), (B.DGDFT_PREC_MIXED, 1)]
H_TOL = {(B.DGDFT_PREC_FP64, 0): 1e-12, (B.DGDFT_PREC_MIXED, 0): 2e-6, (B.DGDFT_PREC_MIXED, 1): 1e-11}


@pytest.fixture(scope="module", autouse=True)
def _built():
    entry.build()


def small_kb_element():
    # 16 x 12 x 10 periodic box with 6 atoms: local potential + 12 projectors
    return synth.random_element(9, 0, (16, 12, 10), 6, J=8, m=10, tol=1e-9)


def cfg2_element(k=0):
    return synth.config2(elems=[k])[0]


def element_of(which):
    # small: general kernels (runtime plans); cfg2 / cfg5: the monolayer
    # grids 48 x 64 x 40 and 48 x 64 x 48 (register-resident FP32 kernels in
    # the mixed form, compile-time FP64 kernels otherwise)
    if which == "small":
        return small_kb_element()
    if which == "cfg2":
        return cfg2_element()
    return synth.config5(elems=[100])[0]


def ctx_for(el, prec, **kw):
    c = B.Context([B.element_dict(el)], precision=prec, **kw)
    B.load_element(c, 0, el)
    return c


def rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


# ------------------------------------------------------------ H apply

@pytest.mark.parametrize("prec,stage", H_KINDS)
@pytest.mark.parametrize("which", ["small", "cfg2", "cfg5"])
def test_apply_h(prec, stage, which):
    el = element_of(which)
    gen = np.random.default_rng(1)
    k = 5 if which == "small" else 3
    x = gen.standard_normal((k, el.ng))
    c = ctx_for(el, prec)
    got = c.dgdft_alb_apply_h(0, x, stage=stage)
    ref = H.apply_h(x, el)
    # FP32: the r2c/c2r FFTs carry ~1e-7 relative error, amplified by the
    # kinetic symbol relative to |H x| (rough white-noise inputs);
    # double-float transforms: ~2^-46 per operation over ~log2(N_g) stages
    print(f"{which} prec={prec} stage={stage}: relative error {rel(got, ref):.1e}")
    assert rel(got, ref) < H_TOL[(prec, stage)]
    c.close()


@pytest.mark.parametrize("prec,stage", H_KINDS)
@pytest.mark.parametrize("grid,freq", [((16, 12, 10), (8, 2, 5)), ((48, 64, 40), (24, 7, 20)),
                                       ((48, 64, 48), (5, 32, 24))])
def test_apply_h_plane_wave_eigenvalue(prec, stage, grid, freq):
    # a single plane wave cos(G.r) in a potential-free box: H x = |G|^2/2 x,
    # including the Nyquist frequency (|n/2|, the reading of the planewave set)
    el = synth.random_element(9, 1, grid, 4, J=4, m=4)
    el.veff[:] = 0.0
    el.proj_row_ptr = np.zeros(1, np.int64)
    el.proj_idx = np.zeros(0, np.int32)
    el.proj_val = np.zeros(0)
    el.proj_gamma = np.zeros(0)
    coords = [np.arange(n) * l / n for n, l in zip(el.n, el.L)]
    zz, yy, xx = np.meshgrid(coords[2], coords[1], coords[0], indexing="ij")
    gx, gy, gz = (2 * np.pi * f / l for f, l in zip(freq, el.L))
    x = np.cos(gx * xx + gy * yy + gz * zz).reshape(1, -1)
    c = ctx_for(el, prec)
    got = c.dgdft_alb_apply_h(0, x, stage=stage)
    lam = 0.5 * (gx * gx + gy * gy + gz * gz)
    tol = {0: 1e-12, 1: 1e-6}[prec] if stage == 0 else 1e-11
    assert rel(got, lam * x) < tol
    c.close()


# ------------------------------------------------------------- Teter

@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("which", ["small", "cfg2", "cfg5"])
def test_teter(prec, which):
    el = element_of(which)
    gen = np.random.default_rng(2)
    x = gen.standard_normal((4, el.ng))
    r = gen.standard_normal((4, el.ng))
    t = T.kinetic_energy(x, el.n, el.L)
    c = ctx_for(el, prec)
    got = c.dgdft_alb_apply_teter(0, r, t)
    ref = T.precondition(r, x, el.n, el.L)
    tol = 1e-12 if prec == B.DGDFT_PREC_FP64 else 2e-6
    assert rel(got, ref) < tol
    c.close()


# -------------------------------------------------------------- Gram

GRAM_KINDS = [B.DGDFT_PREC_FP64, B.DGDFT_PREC_MIXED]


@pytest.mark.parametrize("prec", GRAM_KINDS)
@pytest.mark.parametrize("shape", [(1000, 7, 5), (122880, 48, 48), (70001, 130, 70), (4096, 288, 144)])
def test_gram(prec, shape):
    ng, p, q = shape
    gen = np.random.default_rng(3)
    u = gen.standard_normal((p, ng))
    v = gen.standard_normal((q, ng))
    el = small_kb_element()
    c = ctx_for(el, prec)
    got = c.dgdft_alb_gram(u, v)
    ref = u @ v.T
    scale = np.sqrt(ng)  # typical |u_i| |v_j| / sqrt(ng) for random rows
    err = np.max(np.abs(got - ref)) / (np.sqrt(ng) * scale)
    tol = 1e-14 if prec == B.DGDFT_PREC_FP64 else 1e-6
    assert err < tol
    c.close()


@pytest.mark.parametrize("ng,q", [(122880, 48), (122880, 144), (70000, 70)])
def test_gram_accumulation_one_signed(ng, q):
    """Rows of one sign make every partial sum grow, the worst case for
    accumulation rounding.  Measured against the exact product of the
    FP32-rounded inputs, relative to sum_k |u_k| |v_k|: the compensated SIMT
    kernel within a few FP32 units."""
    p = 48
    gen = np.random.default_rng(4)
    u = 1.0 + np.abs(gen.standard_normal((p, ng)))
    v = 1.0 + np.abs(gen.standard_normal((q, ng)))
    u32 = u.astype(np.float32).astype(np.float64)
    v32 = v.astype(np.float32).astype(np.float64)
    el = small_kb_element()
    c = ctx_for(el, B.DGDFT_PREC_MIXED)
    got = c.dgdft_alb_gram(u, v)
    ref = u32 @ v32.T
    err = np.max(np.abs(got - ref) / ref)
    assert err < 2e-8, err
    c.close()


def ragged_element():
    # N_g = 20 * 15 * 9 = 2700: a multiple of 4 (16-byte columns) but not of
    # the tensor-core kernel's 32-row stage; m = 40 < 48 leaves zero-filled
    # columns in every 48-column slot
    return synth.random_element(9, 2, (20, 15, 9), 5, J=30, m=40)


def lobpcg_blocks(el, gen, kind):
    """Six (m, N_g) blocks X, W, P, HX, HW, HP.  kind 'random': independent
    normal rows; 'ortho': X orthonormal and W, P orthogonal to X, so X^T W
    and X^T P are zero up to rounding (sums that cancel), with H-images that
    are near multiples of their blocks as in a converging LOBPCG."""
    m, ng = el.m, el.ng
    if kind == "random":
        return gen.standard_normal((6, m, ng))
    q, _ = np.linalg.qr(gen.standard_normal((ng, 3 * m)))
    x, w, p = q[:, :m].T, q[:, m:2 * m].T, q[:, 2 * m:].T * 1e-3
    th = np.sort(gen.uniform(-6.0, -4.0, m))
    hx = th[:, None] * x + 1e-4 * gen.standard_normal((m, ng)) / np.sqrt(ng)
    hw = 5.0 * w + gen.standard_normal((m, ng)) / np.sqrt(ng)
    hp = -5.0 * p + 1e-3 * gen.standard_normal((m, ng)) / np.sqrt(ng)
    return np.stack([x, w, p, hx, hw, hp])


# (precision, SIMT Gram, stage): the plain FP64 kernels, the compensated
# FP32 SIMT kernel, the tensor-core TF32-split kernel (default of the mixed
# form), and the mixed form's double-float FP64-stage kernel
LOBPCG_GRAM_KINDS = [(B.DGDFT_PREC_FP64, False, 0), (B.DGDFT_PREC_MIXED, True, 0), (B.DGDFT_PREC_MIXED, False, 0),
                     (B.DGDFT_PREC_MIXED, False, 1)]


@pytest.mark.parametrize("prec,simt,stage", LOBPCG_GRAM_KINDS)
@pytest.mark.parametrize("which", ["small", "ragged", "cfg2"])
@pytest.mark.parametrize("has_p", [True, False])
@pytest.mark.parametrize("kind", ["random", "ortho"])
def test_lobpcg_gram(prec, simt, stage, which, has_p, kind):
    """The Gram products of one LOBPCG iteration through the solver's own
    kernels, against NumPy FP64 products of the same (working-precision)
    inputs, entry by entry relative to sum_k |a_k| |b_k| (the scale of the
    rounding of any summation order): FP64 to 1e-13, double-float to 4e-12
    (~2^-44 per product plus the FP32 rounding of the low parts' running
    sums, renormalised every 16 rows), the compensated SIMT kernel to 2e-7,
    the TF32-split tensor-core
    kernel to 2^-20 (two TF32
    parts carry ~2^-22 of each value) except on one-signed sums (the
    diagonals of the diagonal blocks, x^T x and x^T (H x) of a near
    eigenvector): there the tensor core's FP32 accumulation, which does not
    round to nearest, loses ~1/2 unit of the running sum per MMA and leaves
    a bias below 4e-6."""
    el = {"small": small_kb_element, "ragged": ragged_element, "cfg2": cfg2_element}[which]()
    gen = np.random.default_rng(31)
    blk = lobpcg_blocks(el, gen, kind)
    c = ctx_for(el, prec, simt_gram=simt)
    a, b, xtw = c.dgdft_alb_lobpcg_gram(0, blk, has_p, stage=stage)
    c.close()
    fp32 = prec == B.DGDFT_PREC_MIXED and stage == 0
    if fp32:
        blk = blk.astype(np.float32).astype(np.float64)
    x, w, p, hx, hw, hp = blk
    m = el.m
    s_ = np.vstack([x, w, p])
    hs = np.vstack([hx, hw, hp])
    ref_a, ref_b = hs @ s_.T, s_ @ s_.T
    sc_a, sc_b = np.abs(hs) @ np.abs(s_).T, np.abs(s_) @ np.abs(s_).T
    nb = 3 if has_p else 2
    tol = 1e-13 if prec == B.DGDFT_PREC_FP64 else (4e-12 if stage == 1 else (2e-7 if simt else 2.0 ** -20))
    worst = worst_diag = 0.0
    for bi in range(3):
        for bj in range(3):
            rs, cs = slice(bi * m, bi * m + m), slice(bj * m, bj * m + m)
            if bi > bj or bi >= nb or bj >= nb:
                assert np.all(a[rs, cs] == 0.0) and np.all(b[rs, cs] == 0.0)
                continue
            for got, ref, sc in ((a, ref_a, sc_a), (b, ref_b, sc_b)):
                e = np.abs(got[rs, cs] - ref[rs, cs]) / sc[rs, cs]
                if bi == bj and fp32 and not simt:
                    diag = float(np.max(np.diag(e)))
                    worst_diag = max(worst_diag, diag)
                    assert diag < 4e-6
                    e = e - np.diag(np.diag(e))
                worst = max(worst, float(np.max(e)))
    e_xtw = float(np.max(np.abs(xtw - x @ w.T) / (np.abs(x) @ np.abs(w).T)))
    print(f"{which} {kind} has_p={has_p} prec={prec} simt={simt} stage={stage}: pencil {worst:.2e} "
          f"(one-signed diagonals {worst_diag:.2e}), X^T W {e_xtw:.2e}")
    assert worst < tol and e_xtw < tol


# ---------------------------------------------------- block updates

# (precision, update kernels, stage): plain FP64; the mixed form's FP32 stage
# with SIMT updates (default) and with tensor-core updates (bulk_kernels = 2);
# the mixed form's double-float FP64 stage
LOBPCG_UPDATE_KINDS = [(B.DGDFT_PREC_FP64, "simt", 0), (B.DGDFT_PREC_MIXED, "simt", 0),
                       (B.DGDFT_PREC_MIXED, "tc", 0), (B.DGDFT_PREC_MIXED, "simt", 1)]
# worst-case bounds relative to sum_k |s_k| |y_k| over K <= 3m = 144 terms:
# FP64 and double-float as for the Gram; FP32 with round-to-nearest
# accumulation K 2^-24; TF32 split (3 2^-22 per product) plus the tensor
# core's FP32 accumulation, which does not round to nearest (K 2^-23)
UPDATE_TOL = {(B.DGDFT_PREC_FP64, "simt", 0): 1e-13, (B.DGDFT_PREC_MIXED, "simt", 0): 144 * 2.0 ** -24,
              (B.DGDFT_PREC_MIXED, "tc", 0): 3 * 2.0 ** -22 + 144 * 2.0 ** -23,
              (B.DGDFT_PREC_MIXED, "simt", 1): 4e-12}


@pytest.mark.parametrize("prec,kernels,stage", LOBPCG_UPDATE_KINDS)
@pytest.mark.parametrize("which", ["small", "ragged", "cfg2"])
@pytest.mark.parametrize("has_p", [True, False])
def test_lobpcg_update(prec, kernels, stage, which, has_p):
    """X' = [X W P] Y, P' = [W P] Y_wp and HP' = [HW HP] Y_wp (the paper's
    Phi C products) through the solver's own kernels, against NumPy FP64
    products of the same working-precision inputs, entry by entry relative
    to sum_k |s_k| |y_k| (UPDATE_TOL); without P the P terms are dropped."""
    el = {"small": small_kb_element, "ragged": ragged_element, "cfg2": cfg2_element}[which]()
    gen = np.random.default_rng(41)
    m = el.m
    blk = gen.standard_normal((6, m, el.ng))
    y = gen.standard_normal((3 * m, m))
    c = ctx_for(el, prec, tc_update=(kernels == "tc"))
    out = c.dgdft_alb_lobpcg_update(0, blk, y, has_p, stage=stage)
    c.close()
    if prec == B.DGDFT_PREC_MIXED and stage == 0:
        blk = blk.astype(np.float32).astype(np.float64)
        y = y.astype(np.float32).astype(np.float64)
    k = 3 if has_p else 2
    s_x = np.vstack(blk[:k])
    s_wp, s_hwp = np.vstack(blk[1:k]), np.vstack(blk[4:3 + k])
    y_x, y_wp = y[:k * m], y[m:k * m]
    worst = 0.0
    for got, yy, ss in ((out[0], y_x, s_x), (out[1], y_wp, s_wp), (out[2], y_wp, s_hwp)):
        ref = yy.T @ ss
        scale = np.abs(yy).T @ np.abs(ss)
        worst = max(worst, float(np.max(np.abs(got - ref) / scale)))
    print(f"{which} has_p={has_p} prec={prec} {kernels} stage={stage}: max error {worst:.2e} of sum |s||y|")
    assert worst <= UPDATE_TOL[(prec, kernels, stage)]


# ---------------------------------------------------- Rayleigh-Ritz

def spd(n, gen, cond=1e3):
    q, _ = np.linalg.qr(gen.standard_normal((n, n)))
    return (q * np.logspace(0, np.log10(cond), n)) @ q.T


# The Rayleigh-Ritz entry point in both arithmetics a solve uses: FP64
# (stage 1, and every stage of an FP64 context) and the FP32 stage's
# double-float reduction (stage 0 of a mixed-precision context; pencils
# beyond 160 x 160 or 64 wanted pairs fall back to FP64).  Both are checked
# against LAPACK's generalized symmetric eigensolver.
RR_ARITH = {"fp64": (B.DGDFT_PREC_FP64, 1), "dfloat": (B.DGDFT_PREC_MIXED, 0)}


def rr_context(arith):
    prec, stage = RR_ARITH[arith]
    return ctx_for(small_kb_element(), prec), stage


@pytest.mark.parametrize("arith", sorted(RR_ARITH))
@pytest.mark.parametrize("n,m", [(20, 5), (96, 48), (144, 48), (30, 30), (160, 64), (180, 60)])
def test_rayleigh_ritz(n, m, arith):
    gen = np.random.default_rng(n + m)
    a = gen.standard_normal((n, n))
    a = a + a.T
    b = spd(n, gen)
    c, stage = rr_context(arith)
    theta, y = c.dgdft_alb_rayleigh_ritz(a, b, m, stage=stage)
    c.close()
    ref = sla.eigh(a, b, eigvals_only=True)[:m]
    np.testing.assert_allclose(theta, ref, atol=1e-10 * np.max(np.abs(ref)))
    np.testing.assert_allclose(y.T @ b @ y, np.eye(m), atol=1e-10)
    assert np.max(np.abs(a @ y - b @ y * theta)) < 1e-9 * np.max(np.abs(a))


@pytest.mark.parametrize("arith", sorted(RR_ARITH))
def test_rayleigh_ritz_degenerate_shells(arith):
    # exactly degenerate clusters (free-electron-like multiplicities 1, 6, 12)
    gen = np.random.default_rng(7)
    n, m = 60, 19
    q, _ = np.linalg.qr(gen.standard_normal((n, n)))
    ev = np.r_[0.0, np.full(6, 0.2), np.full(12, 0.4), np.linspace(0.6, 3, 41)]
    a = (q * ev) @ q.T
    c, stage = rr_context(arith)
    theta, y = c.dgdft_alb_rayleigh_ritz(a, np.eye(n), m, stage=stage)
    c.close()
    # FP64: rounding of eps |A| n; double-float: 2^-46 |A| n
    tol = 1e-12 if arith == "fp64" else 1e-11
    np.testing.assert_allclose(theta, ev[:m], atol=tol)
    np.testing.assert_allclose(y.T @ y, np.eye(m), atol=10 * tol)
    assert alb.sin_max_angle(q[:, :m].T, y.T) < 100 * tol


@pytest.mark.parametrize("arith", sorted(RR_ARITH))
@pytest.mark.parametrize("seed", range(12))
def test_rayleigh_ritz_close_pairs(seed, arith):
    """Pencils shaped like the FP32 stage's: the lowest 48 of 144 eigenvalues
    near zero in close pairs (gaps 1e-7 to 1e-3 of the norm), the rest spread
    up to ~30.  Eigenvalue estimates from bisection are good to roughly the
    cluster threshold here, so two close eigenvalues can be taken as
    isolated; the eigenvectors must still come out B-orthonormal (two copies
    of one eigenvector would make the next LOBPCG block rank deficient)."""
    gen = np.random.default_rng(100 + seed)
    n, m = 144, 48
    low = np.sort(gen.uniform(-0.4, 0.4, m // 2))
    gaps = 30.0 * 10.0 ** gen.uniform(-7, -3, m // 2)
    ev = np.sort(np.r_[low, low + gaps, gen.uniform(1.0, 30.0, n - m)])
    q, _ = np.linalg.qr(gen.standard_normal((n, n)))
    b = spd(n, gen, cond=1e2) if seed % 2 else np.eye(n)
    lb = np.linalg.cholesky(b)
    a = lb @ (q * ev) @ q.T @ lb.T
    a = 0.5 * (a + a.T)
    c, stage = rr_context(arith)
    theta, y = c.dgdft_alb_rayleigh_ritz(a, b, m, stage=stage)
    c.close()
    np.testing.assert_allclose(theta, ev[:m], atol=1e-10 * 30.0)
    np.testing.assert_allclose(y.T @ b @ y, np.eye(m), atol=1e-9)
    assert np.max(np.abs(a @ y - b @ y * theta)) < 1e-8 * 30.0


@pytest.mark.parametrize("arith", sorted(RR_ARITH))
def test_rayleigh_ritz_rejects_indefinite_b(arith):
    n = 10
    a = np.eye(n)
    b = np.eye(n)
    b[3, 3] = -1.0
    c, stage = rr_context(arith)
    with pytest.raises(B.DgdftError):
        c.dgdft_alb_rayleigh_ritz(a, b, 3, stage=stage)
    c.close()


def test_rayleigh_ritz_rejects_bad_stage():
    c, _ = rr_context("dfloat")
    with pytest.raises(B.DgdftError):
        c.dgdft_alb_rayleigh_ritz(np.eye(4), np.eye(4), 2, stage=2)
    c.close()


# ------------------------------------------ restriction + orthonormalisation

@pytest.mark.parametrize("which", ["small", "cfg2"])
def test_restrict_orthonormalise(which):
    el = small_kb_element() if which == "small" else cfg2_element()
    if which == "small":
        el.e_lo, el.e_hi = synth.element_box(el.n)
    gen = np.random.default_rng(4)
    k, J = (10, 8) if which == "small" else (48, 40)
    x = OL.cholesky_qr(gen.standard_normal((k, el.ng)))
    c = ctx_for(el, B.DGDFT_PREC_FP64)
    phi = c.dgdft_alb_restrict_orthonormalise(0, x, J)
    ref = alb.orthonormalise(alb.restrict(x, el, J), el.dv)
    np.testing.assert_allclose(phi @ phi.T * el.dv, np.eye(J), atol=1e-12)
    assert alb.sin_max_angle(ref, phi) < 1e-11
    c.close()


@pytest.mark.parametrize("which", ["small", "cfg2"])
def test_restrict_orthonormalise_top(which):
    """The restriction variant (restrict_all = 1): all k columns restricted,
    the J left singular vectors of the largest singular values kept, against
    the oracle's SVD.  The angle tolerance follows the gap between the J-th
    and (J+1)-th singular values of the restricted block (the GPU works on
    its Gram, sigma^2, in FP64)."""
    el = small_kb_element() if which == "small" else cfg2_element()
    if which == "small":
        el.e_lo, el.e_hi = synth.element_box(el.n)
    gen = np.random.default_rng(5)
    k, J = (10, 6) if which == "small" else (48, 40)
    x = OL.cholesky_qr(gen.standard_normal((k, el.ng)))
    c = ctx_for(el, B.DGDFT_PREC_FP64, restrict_all=True)
    phi = c.dgdft_alb_restrict_orthonormalise(0, x, J)
    c.close()
    phit = alb.restrict(x, el, k)
    ref = alb.orthonormalise_top(phit, el.dv, J)
    sv = np.linalg.svd(phit, compute_uv=False)
    rel_gap = (sv[J - 1] ** 2 - sv[J] ** 2) / sv[0] ** 2
    ang = alb.sin_max_angle(ref, phi)
    print(f"{which}: sin(angle) {ang:.1e}, relative sigma^2 gap at J {rel_gap:.2e}")
    np.testing.assert_allclose(phi @ phi.T * el.dv, np.eye(J), atol=1e-12)
    assert ang < max(1e-11, 1e-13 / rel_gap)


def test_solve_restrict_all_variant():
    """A mixed-form solve of a monolayer element with restrict_all = 1: the
    returned ALBs are orthonormal and span the oracle's top-J left singular
    subspace of the GPU's own restricted Ritz block (all m columns)."""
    e = cfg2_element(0)
    c = B.Context([B.element_dict(e)], precision=B.DGDFT_PREC_MIXED, tol=1e-6, maxit=600, keep_block=True,
                  restrict_all=True)
    B.load_element(c, 0, e, synth.initial_block(e))
    st, rep = c.dgdft_alb_solve()
    assert st == B.DGDFT_OK, rep
    phi, eig, res = c.dgdft_alb_get_basis(0)
    x = c.dgdft_alb_get_block(0)
    c.close()
    assert np.max(res) <= 1e-6
    np.testing.assert_allclose(phi @ phi.T * e.dv, np.eye(e.J), atol=1e-12)
    phit = alb.restrict(x, e, e.m)
    ref = alb.orthonormalise_top(phit, e.dv, e.J)
    sv = np.linalg.svd(phit, compute_uv=False)
    rel_gap = (sv[e.J - 1] ** 2 - sv[e.J] ** 2) / sv[0] ** 2
    ang = alb.sin_max_angle(ref, phi)
    print(f"restrict_all solve: sin(angle) to the oracle's top-J subspace {ang:.1e}, "
          f"relative sigma^2 gap at J {rel_gap:.2e}")
    assert ang < max(1e-11, 1e-13 / rel_gap)


# -------------------------------------------------------------- full solves

def _gap_ok(gap, tol, bound):
    return gap >= tol / bound


@pytest.mark.parametrize("prec", PRECS)
def test_solve_config1(prec):
    el = synth.config1()
    gold = np.loadtxt(os.path.join(GOLDEN, "config1_eigenvalues.txt"))
    c = B.Context([B.element_dict(el)], precision=prec, tol=1e-8, maxit=800, keep_block=True)
    B.load_element(c, 0, el, synth.initial_block(el))
    st, rep = c.dgdft_alb_solve()
    assert st == B.DGDFT_OK, rep
    phi, eig, res = c.dgdft_alb_get_basis(0)
    x = c.dgdft_alb_get_block(0)
    c.close()
    eig_tol = 1e-8 if prec == B.DGDFT_PREC_FP64 else 1e-6
    np.testing.assert_allclose(eig, gold, atol=eig_tol)
    # FP64 residual of the returned vectors, recomputed by the oracle
    r = H.apply_h(x[:16], el) - eig[:, None] * x[:16]
    assert np.max(np.linalg.norm(r, axis=1)) <= 1.05e-8
    np.testing.assert_allclose(phi @ phi.T * el.dv, np.eye(16), atol=1e-12)
    # subspace against the exact invariant subspace (dense eigh at 16^3)
    w, v = np.linalg.eigh(H.dense_h(el))
    gap = w[16] - w[15]
    bound = 1.05e-8 / gap
    assert alb.sin_max_angle(v[:, :16].T, x[:16]) <= max(bound, 1e-12) * 1.5
    assert alb.sin_max_angle(v[:, :16].T, phi) <= max(bound, 1e-12) * 1.5


@pytest.mark.parametrize("prec,simt", [(B.DGDFT_PREC_FP64, False), (B.DGDFT_PREC_MIXED, False),
                                       (B.DGDFT_PREC_MIXED, True)])
def test_solve_config2_elements(prec, simt):
    els = synth.config2(elems=[0, 7])
    c = B.Context([B.element_dict(e) for e in els], precision=prec, tol=1e-6, maxit=600,
                  keep_block=True, simt_gram=simt)
    for k, e in enumerate(els):
        B.load_element(c, k, e, synth.initial_block(e))
    st, rep = c.dgdft_alb_solve()
    assert st == B.DGDFT_OK, rep
    for k, e in enumerate(els):
        phi, eig, res = c.dgdft_alb_get_basis(k)
        x = c.dgdft_alb_get_block(k)
        assert np.max(res) <= 1e-6
        r = H.apply_h(x[:e.J], e) - eig[:, None] * x[:e.J]
        assert np.max(np.linalg.norm(r, axis=1)) <= 1.05e-6
        np.testing.assert_allclose(phi @ phi.T * e.dv, np.eye(e.J), atol=1e-12)
        assert alb.sin_max_angle(alb.restrict(x, e), phi) < 1e-10
        # eigenvalues against the oracle's (error ~ residual^2 / gap, below
        # the tolerance); the subspace through its Davis-Kahan bound, reported
        # with the gap at J (at residual 1e-6 it does not reach 1e-5 here:
        # see test_solve_config2_tight_subspace)
        gth, gres = OC.ritz_golden(f"config2_elem{[0, 7][k]}")
        np.testing.assert_allclose(eig, gth[:e.J], rtol=0,
                                   atol=1e-6 if prec == B.DGDFT_PREC_MIXED else 1e-8)
        bound, gap = OC.angle_bound(x, eig, e, gth, gres)
        print(f"config-2 element {[0, 7][k]} (prec {prec}, simt {simt}): max |eig - oracle| "
              f"{np.max(np.abs(eig - gth[:e.J])):.1e} Ha; sin(angle) to the oracle's subspace <= {bound:.1e} "
              f"(gap at J {gap:.2e} Ha)")
    c.close()


def test_solve_config2_workload():
    """All 36 monolayer elements in one solve, in the launch configuration the
    benchmark times (mixed form, tensor-core Gram, two half batches): every
    element converges with orthonormal ALBs; sampled elements' Ritz pairs are
    re-checked with the oracle's H, and elements 0 and 7 against the
    oracle's eigenvalues."""
    els = synth.config2()
    c = B.Context([B.element_dict(e) for e in els], precision=B.DGDFT_PREC_MIXED, tol=1e-6, maxit=600,
                  keep_block=True)
    for k, e in enumerate(els):
        B.load_element(c, k, e, synth.initial_block(e))
    st, rep = c.dgdft_alb_solve()
    assert st == B.DGDFT_OK, rep
    assert all(r["restarts"] == 0 for r in rep)
    for k, e in enumerate(els):
        phi, eig, res = c.dgdft_alb_get_basis(k)
        assert np.max(res) <= 1e-6
        np.testing.assert_allclose(phi @ phi.T * e.dv, np.eye(e.J), atol=1e-12)
        if k in (0, 7, 17, 35):
            x = c.dgdft_alb_get_block(k)
            r = H.apply_h(x[:e.J], e) - eig[:, None] * x[:e.J]
            assert np.max(np.linalg.norm(r, axis=1)) <= 1.05e-6
        if k in (0, 7):
            gth, _ = OC.ritz_golden(f"config2_elem{k}")
            np.testing.assert_allclose(eig, gth[:e.J], rtol=0, atol=1e-6)
    print("iterations (mean / max):", np.mean([r["iterations"] for r in rep]), max(r["iterations"] for r in rep))
    c.close()


@pytest.mark.parametrize("prec,tol,angle_tol", [(B.DGDFT_PREC_FP64, 1e-10, 1e-7), (B.DGDFT_PREC_MIXED, 1e-9, 1e-5)])
def test_solve_config2_tight_subspace(prec, tol, angle_tol):
    """The subspace tolerances (FP64 1e-7, mixed 1e-5) need residual <~
    gap x tolerance; with the 4.6 mHa gap at J of monolayer element 0 that is
    a tighter solve.  Both forms get there (the mixed form through its FP64
    stage) and the Davis-Kahan bound then proves the angle to the oracle's
    subspace within tolerance; eigenvalues within 1e-8 Ha."""
    e = cfg2_element(0)
    c = B.Context([B.element_dict(e)], precision=prec, tol=tol, maxit=1200, keep_block=True)
    B.load_element(c, 0, e, synth.initial_block(e))
    st, rep = c.dgdft_alb_solve()
    assert st == B.DGDFT_OK, rep
    _, eig, res = c.dgdft_alb_get_basis(0)
    x = c.dgdft_alb_get_block(0)
    c.close()
    gth, gres = OC.ritz_golden("config2_elem0")
    np.testing.assert_allclose(eig, gth[:e.J], rtol=0, atol=1e-8)
    bound, gap = OC.angle_bound(x, eig, e, gth, gres)
    print(f"tight solve (prec {prec}, tol {tol:g}): sin(angle) <= {bound:.2e}, gap at J {gap:.2e} Ha")
    assert bound <= angle_tol


def test_nonfinite_potential_rejected():
    el = small_kb_element()
    c = B.Context([B.element_dict(el)])
    v = el.veff.reshape(-1).copy()
    v[5] = np.nan
    with pytest.raises(B.DgdftError) as ei:
        c.dgdft_alb_set_potential(0, v)
    assert ei.value.status == B.DGDFT_EINVAL
    with pytest.raises(B.DgdftError) as ei:
        c.dgdft_alb_get_basis(0)
    assert ei.value.status == B.DGDFT_ESTATE
    c.close()
