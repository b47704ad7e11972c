"""DG Hamiltonian assembly from the ALBs (oracle, FP64).

TEST INFRASTRUCTURE, like the rest of ``oracle``: only the tests, smoke()
and the benchmark's CPU leg may use it.

Eq. DGHamiltonian gives H^DG in three groups: (1) kinetic and V_eff volume
integrals over each element (diagonal blocks), (2) the KB nonlocal term
sum_p gamma_p <phi', b_p> <b_p, phi> (diagonal and off-diagonal blocks of
elements the projector touches), (3) the interior-penalty face terms
-1/2 <[phi'], {grad phi}> - 1/2 <{grad phi'}, [phi]> + alpha <[phi'], [phi]>
on faces shared by neighbouring elements.  Sec. II.B ("Construction of the
DG Hamiltonian") evaluates every integral by Legendre-Gauss-Lobatto (LGL)
quadrature on each element and the gradients by LGL differentiation
matrices; Sec. III sets the LGL points per direction to twice the uniform
grid's.

Readings where the paper is silent (each listed in the design notes):
  * ALB functions off the uniform grid: the ALBs of E_K are spanned by the
    real trigonometric interpolants over the periodic box Q_K of J columns on
    Q_K's grid (Nyquist mode as a cosine, as in the planewave set of the
    local problem), restricted to E_K.
  * Eq. orthonormal is imposed with the LGL quadrature: the interpolated
    block Phi~ with mass matrix M = Phi~^T W Phi~ = L L^T (Cholesky) gives
    Phi = Phi~ L^-T, so <phi_i, phi_j> = delta_ij under the quadrature and
    the basis is unique given the J columns.
  * Faces: the face between element a and its +e_d neighbour b uses a's
    last LGL plane along d and b's first (the two coincide in space); jump
    [u] = (u_a - u_b) e_d, average {d_d u} = (d_d u_a + d_d u_b) / 2, face
    weights the product of the other two directions' LGL weights.  With one
    element along d the face joins the element to itself through the
    periodic boundary.
  * Blocks are H_{K,K'} (rows: basis of K) for K' in the 3 x 3 x 3 periodic
    neighbourhood of K; coinciding neighbours are merged.
  * Density (Eq. density) of the lowest n_occ eigenvectors of H^DG, one
    electron per state as the equation is written (no spin factor).
"""

from __future__ import annotations

import numpy as np
from numpy.polynomial import legendre as leg


# ---------------------------------------------------------------- 1-D pieces

def lgl_nodes_weights(n: int):
    """The n >= 2 LGL nodes on [-1, 1] (ascending) and their weights: the end
    points and the roots of P'_{n-1}; w_i = 2 / (n (n - 1) P_{n-1}(x_i)^2)."""
    N = n - 1
    cN = np.zeros(N + 1)
    cN[N] = 1.0
    if n == 2:
        x = np.array([-1.0, 1.0])
    else:
        d1 = leg.legder(cN)
        d2 = leg.legder(d1)
        r = np.sort(leg.legroots(d1).real)
        for _ in range(4):  # Newton on P'_N
            r = r - leg.legval(r, d1) / leg.legval(r, d2)
        x = np.concatenate([[-1.0], r, [1.0]])
    w = 2.0 / (N * (N + 1) * leg.legval(x, cN) ** 2)
    return x, w


def diff_matrix(x: np.ndarray) -> np.ndarray:
    """Differentiation matrix of the polynomial interpolant through the nodes
    x (barycentric form): D_ij = (lam_j / lam_i) / (x_i - x_j) for i != j,
    lam_j = 1 / prod_{k != j} (x_j - x_k), rows summing to zero."""
    n = len(x)
    diff = x[:, None] - x[None, :]
    np.fill_diagonal(diff, 1.0)
    lam = 1.0 / np.prod(diff, axis=1)
    D = (lam[None, :] / lam[:, None]) / diff
    np.fill_diagonal(D, 0.0)
    D[np.arange(n), np.arange(n)] = -D.sum(axis=1)
    return D


def trig_interp_matrix(n: int, length: float, pts: np.ndarray) -> np.ndarray:
    """(len(pts), n) matrix taking the n samples at k * length / n to the real
    trigonometric interpolant's values at pts: the cosine sum over the modes
    of the periodic grid, weights 1 (m = 0), 2 (0 < m < n/2), 1 (m = n/2 for
    even n), divided by n."""
    pts = np.asarray(pts, float)
    t = pts[:, None] - np.arange(n)[None, :] * (length / n)
    out = np.ones((len(pts), n))
    for m in range(1, (n - 1) // 2 + 1):
        out += 2.0 * np.cos(2.0 * np.pi * m * t / length)
    if n % 2 == 0:
        out += np.cos(np.pi * n * t / length)
    return out / n


# ---------------------------------------------------------------- per element

class ElementGrid:
    """LGL tensor grid of one element box (lower corner `corner`, sides le)."""

    def __init__(self, dom, k: int):
        self.k = k
        self.nl = dom.nl
        self.le = dom.le
        self.corner = dom.corner(k)
        self.ref = [lgl_nodes_weights(n) for n in self.nl]
        # nodes in the element frame [0, le_d], and in the cell
        self.local = [(xr + 1.0) * (l / 2.0) for (xr, _), l in zip(self.ref, self.le)]
        self.cell_pts = [c + p for c, p in zip(self.corner, self.local)]
        self.w1 = [wr * (l / 2.0) for (_, wr), l in zip(self.ref, self.le)]
        self.D = [diff_matrix(xr) * (2.0 / l) for (xr, _), l in zip(self.ref, self.le)]
        wz, wy, wx = self.w1[2], self.w1[1], self.w1[0]
        self.w = (wz[:, None, None] * wy[None, :, None] * wx[None, None, :]).reshape(-1)

    @property
    def shape(self):
        return (self.nl[2], self.nl[1], self.nl[0])


def interpolate_to_lgl(dom, g: ElementGrid, z: np.ndarray) -> np.ndarray:
    """Rows of z (J, N_gQ) on Q_K's grid -> their trigonometric interpolants
    over Q_K at E_K's LGL nodes, (J, n_LGL)."""
    mats = [trig_interp_matrix(dom.nq[d], dom.lq[d], dom.e_off[d] + g.local[d]) for d in range(3)]
    zz = z.reshape(z.shape[0], dom.nq[2], dom.nq[1], dom.nq[0])
    out = np.einsum("ai,jkbi->jkba", mats[0], zz, optimize=True)
    out = np.einsum("by,jkya->jkba", mats[1], out, optimize=True)
    out = np.einsum("ck,jkba->jcba", mats[2], out, optimize=True)
    return out.reshape(z.shape[0], -1)


def orthonormalise_lgl(phi_t: np.ndarray, w: np.ndarray) -> np.ndarray:
    """Eq. orthonormal under the LGL quadrature: M = Phi~ W Phi~^T = L L^T,
    Phi = L^-1 Phi~ (rows)."""
    m = (phi_t * w[None, :]) @ phi_t.T
    lo = np.linalg.cholesky(m)
    return np.linalg.solve(lo, phi_t)


def gradients(g: ElementGrid, phi: np.ndarray):
    """d/dx, d/dy, d/dz of the rows of phi by the LGL differentiation
    matrices applied along each axis."""
    f = phi.reshape(phi.shape[0], *g.shape)
    gx = np.einsum("ai,jcbi->jcba", g.D[0], f, optimize=True)
    gy = np.einsum("bi,jcia->jcba", g.D[1], f, optimize=True)
    gz = np.einsum("ci,jiba->jcba", g.D[2], f, optimize=True)
    return [a.reshape(phi.shape) for a in (gx, gy, gz)]


def volume_block(g: ElementGrid, phi, grads, v_lgl) -> np.ndarray:
    """First group of Eq. DGHamiltonian: 1/2 <grad phi', grad phi> + <phi', V phi>."""
    w = g.w
    a = sum(0.5 * ((gd * w[None, :]) @ gd.T) for gd in grads)
    return a + (phi * (w * v_lgl.reshape(-1))[None, :]) @ phi.T


def kb_coefficients(g: ElementGrid, phi, proj) -> dict:
    """<b_p, phi_j> by LGL quadrature for every projector touching E_K:
    {pid: (J,)}; proj = (pid, row_ptr, idx, val) at the element's nodes."""
    pid, rp, idx, val = proj
    out = {}
    for r, p in enumerate(pid):
        sl = slice(rp[r], rp[r + 1])
        i = idx[sl]
        out[int(p)] = phi[:, i] @ (g.w[i] * val[sl])
    return out


def face_traces(g: ElementGrid, phi, grads, d: int, high: bool):
    """Values and normal derivatives of the rows of phi on the element's
    low (high=False) or high face normal to axis d: (J, n_face) each."""
    sel = [slice(None)] * 3
    sel[2 - d] = g.nl[d] - 1 if high else 0  # array axes are (z, y, x)
    sel = (slice(None), *sel)
    f = phi.reshape(phi.shape[0], *g.shape)[sel].reshape(phi.shape[0], -1)
    df = grads[d].reshape(phi.shape[0], *g.shape)[sel].reshape(phi.shape[0], -1)
    return f, df


def face_weights(g: ElementGrid, d: int) -> np.ndarray:
    """Quadrature weights of a face normal to axis d (the other two
    directions' LGL weights, in array order)."""
    others = [e for e in (2, 1, 0) if e != d]  # array order: slow to fast
    return (g.w1[others[0]][:, None] * g.w1[others[1]][None, :]).reshape(-1)


# ---------------------------------------------------------------- assembly

def neighbours(dom, k: int):
    """Distinct elements of the 3 x 3 x 3 periodic neighbourhood of K, sorted."""
    ix, iy, iz = dom.coords(k)
    out = {dom.index(ix + a, iy + b, iz + c)
           for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)}
    return sorted(out)


class Assembly:
    """H^DG blocks for a set of elements, computed lazily per element.

    phis: {K: (J, n_LGL) basis rows on E_K's LGL grid} (already orthonormal
    or not: the assembly uses them as given); v: {K: V_eff at the nodes};
    projs: {K: projector tuple at the nodes}; gamma[pid]."""

    def __init__(self, dom, phis, v, projs, gamma, alpha):
        self.dom, self.phis, self.v, self.projs = dom, phis, v, projs
        self.gamma, self.alpha = gamma, alpha
        self.grid = {}
        self._grads, self._kb = {}, {}

    def g(self, k):
        if k not in self.grid:
            self.grid[k] = ElementGrid(self.dom, k)
        return self.grid[k]

    def grads(self, k):
        if k not in self._grads:
            self._grads[k] = gradients(self.g(k), self.phis[k])
        return self._grads[k]

    def kb(self, k):
        if k not in self._kb:
            self._kb[k] = kb_coefficients(self.g(k), self.phis[k], self.projs[k])
        return self._kb[k]

    def face_terms(self, a: int, d: int) -> dict:
        """Face between a and its +e_d neighbour b: contributions to the
        blocks (K, K') for K, K' in {a, b}."""
        dom = self.dom
        ix = list(dom.coords(a))
        ix[d] += 1
        b = dom.index(*ix)
        ga = self.g(a)
        wf = face_weights(ga, d)
        fa, dfa = face_traces(ga, self.phis[a], self.grads(a), d, high=True)
        fb, dfb = face_traces(self.g(b), self.phis[b], self.grads(b), d, high=False)
        jump, avg = {}, {}
        for k in {a, b}:
            jmp = np.zeros_like(fa)
            av = np.zeros_like(fa)
            if k == a:
                jmp += fa
                av += 0.5 * dfa
            if k == b:
                jmp -= fb
                av += 0.5 * dfb
            jump[k], avg[k] = jmp, av
        out = {}
        for k1 in jump:
            for k2 in jump:
                blk = (-0.5 * (jump[k1] * wf) @ avg[k2].T
                       - 0.5 * (avg[k1] * wf) @ jump[k2].T
                       + self.alpha * (jump[k1] * wf) @ jump[k2].T)
                out[(k1, k2)] = blk
        return out

    def row(self, k: int) -> dict:
        """Block row K: {K': H_{K,K'}}."""
        dom = self.dom
        J = self.phis[k].shape[0]
        nb = neighbours(dom, k)
        out = {kk: np.zeros((J, self.phis[kk].shape[0])) for kk in nb}
        # (1) volume
        out[k] += volume_block(self.g(k), self.phis[k], self.grads(k), self.v[k])
        # (2) KB: projectors shared by K and K'
        ck = self.kb(k)
        for kk in nb:
            ckk = self.kb(kk)
            for p, c in ck.items():
                if p in ckk:
                    out[kk] += self.gamma[p] * np.outer(c, ckk[p])
        # (3) faces of K: the +e_d face (K low side) and the -e_d face
        ixyz = dom.coords(k)
        for d in range(3):
            lower = list(ixyz)
            lower[d] -= 1
            faces = {k, dom.index(*lower)}  # faces whose low side is K or K - e_d
            for a in sorted(faces):
                for (k1, k2), blk in self.face_terms(a, d).items():
                    if k1 == k:
                        out[k2] += blk
        return out


def alb_on_lgl(dom, k: int, z: np.ndarray, orthonormalise: bool = True) -> np.ndarray:
    """ALB rows of element K on its LGL grid from the J columns z (J, N_gQ)."""
    g = ElementGrid(dom, k)
    phi = interpolate_to_lgl(dom, g, z)
    return orthonormalise_lgl(phi, g.w) if orthonormalise else phi


# ---------------------------------------------------------------- density

def dense_matrix(dom, rows: dict, J: int) -> np.ndarray:
    """H^DG as one dense matrix (element-major: row K * J + j) from the
    block rows {K: {K': H_{K,K'}}}."""
    n = dom.n_elem * J
    H = np.zeros((n, n))
    for k, row in rows.items():
        for kk, blk in row.items():
            H[k * J:(k + 1) * J, kk * J:(kk + 1) * J] = blk
    return H


def density(dom, phis: dict, H: np.ndarray, n_occ: int, J: int):
    """Eq. ELeq and Eq. density by dense diagonalisation (the DIAG route):
    the lowest n_occ eigenpairs of the symmetric H^DG (orthonormal basis, so
    a standard problem) and rho(x) = sum_i |psi_i(x)|^2 on every element's
    LGL grid, psi_i = sum_{K,j} c_{i;K,j} phi_{K,j}.  Returns (eigenvalues,
    {K: rho_K})."""
    lam, c = np.linalg.eigh(0.5 * (H + H.T))
    c = c[:, :n_occ]
    rho = {k: np.sum((c[k * J:(k + 1) * J].T @ phis[k]) ** 2, axis=0) for k in range(dom.n_elem)}
    return lam[:n_occ], rho
