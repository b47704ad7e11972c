"""ctypes binding of the C-ABI in include/dgdft_alb.h, dgdft_alb_steps.h and
dgdft_dg.h.

Argument marshalling only: every step of ALB generation runs in the CUDA
library.  Functions keep the C names.  Arrays may be NumPy (host) or torch
CUDA tensors (device, passed by data pointer with on_device = 1).  Loading
fails loudly when the shared library has not been built; there is no
fallback.
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

DGDFT_OK, DGDFT_EINVAL, DGDFT_ENOMEM, DGDFT_ECUDA, DGDFT_ENOTCONV, DGDFT_ETIMEOUT, DGDFT_ESTATE = range(7)
STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "ECUDA", "ENOTCONV", "ETIMEOUT", "ESTATE"]
DGDFT_PREC_FP64, DGDFT_PREC_MIXED = 0, 1
DGDFT_PRECOND_TETER, DGDFT_PRECOND_LEARNED = 0, 1


class dgdft_element_desc(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("Lx", C.c_double), ("Ly", C.c_double), ("Lz", C.c_double),
                ("e_lo", C.c_int * 3), ("e_hi", C.c_int * 3),
                ("n_compute", C.c_int), ("n_keep", C.c_int)]


class dgdft_alb_config(C.Structure):
    _fields_ = [("precision", C.c_int), ("precond", C.c_int), ("tol", C.c_double),
                ("maxit", C.c_int), ("check_every", C.c_int), ("hbm_cap_bytes", C.c_size_t),
                ("cuda_stream", C.c_void_p), ("device", C.c_int), ("keep_block", C.c_int),
                ("bulk_kernels", C.c_int), ("h_fp64_forward", C.c_int),
                ("autotune_cache", C.c_char_p), ("precond_weights", C.c_char_p),
                ("device_wait_polls", C.c_int), ("restrict_all", C.c_int), ("ecut", C.c_double)]


class dgdft_solve_report(C.Structure):
    _fields_ = [("status", C.c_int), ("iterations", C.c_int), ("max_resid", C.c_double),
                ("fallbacks", C.c_int), ("wave", C.c_int), ("seconds", C.c_double),
                ("iterations_bulk", C.c_int), ("resid_bulk", C.c_double), ("graph_kernels", C.c_longlong),
                ("restarts", C.c_int)]


class dgdft_dg_config(C.Structure):
    _fields_ = [("ne", C.c_int * 3), ("cell", C.c_double * 3), ("q_span", C.c_int * 3),
                ("nq", C.c_int * 3), ("nl", C.c_int * 3), ("J", C.c_int), ("alpha", C.c_double),
                ("n_proj", C.c_int), ("cuda_stream", C.c_void_p), ("device", C.c_int),
                ("hbm_cap_bytes", C.c_size_t), ("arith", C.c_int)]


_P = C.c_void_p
_SIGS = {
    "dgdft_alb_config_init": (None, [C.POINTER(dgdft_alb_config)]),
    "dgdft_alb_create": (C.c_int, [C.POINTER(dgdft_alb_config), C.c_int,
                                   C.POINTER(dgdft_element_desc), C.POINTER(_P)]),
    "dgdft_alb_set_potential": (C.c_int, [_P, C.c_int, _P, C.c_int]),
    "dgdft_alb_set_projectors": (C.c_int, [_P, C.c_int, C.c_int, _P, _P, _P, _P]),
    "dgdft_alb_set_initial": (C.c_int, [_P, C.c_int, _P, C.c_int]),
    "dgdft_alb_solve": (C.c_int, [_P, C.POINTER(dgdft_solve_report)]),
    "dgdft_alb_scf_step": (C.c_int, [_P, C.c_int, C.POINTER(dgdft_solve_report)]),
    "dgdft_alb_get_basis": (C.c_int, [_P, C.c_int, _P, _P, _P, C.c_int]),
    "dgdft_alb_last_error": (C.c_char_p, [_P]),
    "dgdft_alb_destroy": (None, [_P]),
    "dgdft_alb_apply_h": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, _P, _P, C.c_int]),
    "dgdft_alb_apply_teter": (C.c_int, [_P, C.c_int, C.c_int, _P, _P, _P, C.c_int]),
    "dgdft_alb_project_cutoff": (C.c_int, [_P, C.c_int, C.c_int, _P, _P, C.c_int]),
    "dgdft_alb_gram": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, _P, _P, _P, C.c_int]),
    "dgdft_alb_rayleigh_ritz": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, _P, _P, _P, _P]),
    "dgdft_alb_lobpcg_gram": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, _P, _P, _P, _P, C.c_int]),
    "dgdft_alb_lobpcg_update": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, _P, _P, _P, C.c_int]),
    "dgdft_alb_restrict_orthonormalise": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, _P, _P,
                                                    C.c_int]),
    "dgdft_alb_get_block": (C.c_int, [_P, C.c_int, _P, C.c_int]),
    "dgdft_alb_time_stage": (C.c_int, [_P, C.c_int, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_int),
                                       C.POINTER(C.c_int)]),
    "dgdft_alb_gram_noalloc": (C.c_int, [C.c_int, C.c_int, C.c_int, _P, _P, _P, _P]),
    "dgdft_alb_precond_init": (C.c_int, [_P, C.c_uint64]),
    "dgdft_alb_precond_set_params": (C.c_int, [_P, _P]),
    "dgdft_alb_precond_get_params": (C.c_int, [_P, _P]),
    "dgdft_alb_precond_save": (C.c_int, [_P, C.c_char_p]),
    "dgdft_alb_precond_load": (C.c_int, [_P, C.c_char_p]),
    "dgdft_alb_precond_forward": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, C.c_int, _P, _P, C.c_int]),
    "dgdft_alb_precond_loss_grad": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, _P, _P,
                                              C.POINTER(C.c_double), _P, C.c_int]),
    "dgdft_alb_precond_train": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, C.c_int, _P, _P, _P, C.c_int, C.c_int,
                                          C.c_int, C.c_double, C.c_uint64, C.POINTER(C.c_double),
                                          C.POINTER(C.c_double)]),
    "dgdft_alb_precond_make_data": (C.c_int, [_P, C.c_int, C.c_int, _P, _P, _P, _P, _P]),
    "dgdft_dg_create": (C.c_int, [C.POINTER(dgdft_dg_config), C.POINTER(_P)]),
    "dgdft_dg_lgl_points": (C.c_int, [_P, C.c_int, _P, _P, _P]),
    "dgdft_dg_set_potential": (C.c_int, [_P, C.c_int, _P, C.c_int]),
    "dgdft_dg_set_gamma": (C.c_int, [_P, _P]),
    "dgdft_dg_set_projectors": (C.c_int, [_P, C.c_int, C.c_int, _P, _P, _P, _P]),
    "dgdft_dg_assemble": (C.c_int, [_P, _P, C.c_int]),
    "dgdft_dg_neighbours": (C.c_int, [_P, C.c_int, _P, _P]),
    "dgdft_dg_get_row": (C.c_int, [_P, C.c_int, _P, C.c_int]),
    "dgdft_dg_lgl_basis": (C.c_int, [_P, C.c_int, _P, C.c_int, _P, C.c_int]),
    "dgdft_dg_density": (C.c_int, [_P, _P, C.c_int, C.c_int, _P, _P, C.c_int]),
    "dgdft_dg_density_info": (C.c_int, [_P, _P]),
    "dgdft_dg_last_timing": (C.c_int, [_P, _P, C.c_int, _P]),
    "dgdft_dg_last_error": (C.c_char_p, [_P]),
    "dgdft_dg_destroy": (None, [_P]),
}

PRECOND_PARAMS = 15169

_lib = None


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load libdgdft_alb.so (built in-tree by build.py) and bind every symbol."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build the CUDA library first "
                           "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class DgdftError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 7 else status}: {msg}")
        self.status = status


def _ptr(a):
    """(pointer, on_device) of a NumPy array or a torch tensor."""
    if a is None:
        return None, 0
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data_as(C.c_void_p), 0
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return C.c_void_p(a.data_ptr()), 1 if a.is_cuda else 0
    raise TypeError(type(a))


class Context:
    """Owns one dgdft_alb_ctx; methods mirror the C entry points."""

    def __init__(self, elems, precision=DGDFT_PREC_FP64, tol=1e-6, maxit=400, check_every=4,
                 stream=None, keep_block=False, hbm_cap_bytes=0, precond=DGDFT_PRECOND_TETER,
                 precond_weights=None, simt_gram=False, h_fp64_forward=False, device_wait_polls=0,
                 tc_update=False, restrict_all=False, autotune_cache=None, ecut=0.0):
        self.lib = load()
        cfg = dgdft_alb_config()
        self.lib.dgdft_alb_config_init(C.byref(cfg))
        cfg.precision = precision
        cfg.precond = precond
        cfg.tol = tol
        cfg.maxit = maxit
        cfg.check_every = check_every
        cfg.keep_block = int(keep_block)
        cfg.bulk_kernels = 1 if simt_gram else (2 if tc_update else 0)
        cfg.device_wait_polls = int(device_wait_polls)
        cfg.restrict_all = int(bool(restrict_all))
        cfg.ecut = float(ecut)
        cfg.h_fp64_forward = int(h_fp64_forward)
        cfg.hbm_cap_bytes = int(hbm_cap_bytes)
        cfg.cuda_stream = stream
        self._weights = precond_weights.encode() if precond_weights else None
        cfg.precond_weights = self._weights
        self._tune = str(autotune_cache).encode() if autotune_cache else None
        cfg.autotune_cache = self._tune
        self.cfg = cfg
        n = len(elems)
        arr = (dgdft_element_desc * n)()
        for i, e in enumerate(elems):
            d = arr[i]
            d.nx, d.ny, d.nz = e["n"]
            d.Lx, d.Ly, d.Lz = e["L"]
            for a in range(3):
                d.e_lo[a] = int(e["e_lo"][a])
                d.e_hi[a] = int(e["e_hi"][a])
            d.n_compute, d.n_keep = int(e["m"]), int(e["J"])
        self.descs = arr
        h = C.c_void_p()
        st = self.lib.dgdft_alb_create(C.byref(cfg), n, arr, C.byref(h))
        if st != DGDFT_OK:
            raise DgdftError(st, "dgdft_alb_create failed")
        self.h = h
        self.n = n

    def _check(self, st, what):
        if st not in (DGDFT_OK,):
            msg = self.lib.dgdft_alb_last_error(self.h)
            raise DgdftError(st, f"{what}: {msg.decode() if msg else ''}")

    def close(self):
        if getattr(self, "h", None):
            self.lib.dgdft_alb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def dgdft_alb_set_potential(self, elem, veff):
        p, dev = _ptr(veff)
        self._check(self.lib.dgdft_alb_set_potential(self.h, elem, p, dev), "set_potential")

    def dgdft_alb_set_projectors(self, elem, row_ptr, idx, val, gamma):
        n_proj = len(row_ptr) - 1
        rp = np.ascontiguousarray(row_ptr, np.int64)
        ix = np.ascontiguousarray(idx, np.int32)
        vv = np.ascontiguousarray(val, np.float64)
        gg = np.ascontiguousarray(gamma, np.float64)
        self._check(self.lib.dgdft_alb_set_projectors(self.h, elem, n_proj, _ptr(rp)[0], _ptr(ix)[0],
                                                      _ptr(vv)[0], _ptr(gg)[0]), "set_projectors")

    def dgdft_alb_set_initial(self, elem, x0):
        p, dev = _ptr(x0)
        self._check(self.lib.dgdft_alb_set_initial(self.h, elem, p, dev), "set_initial")

    @staticmethod
    def _reports(reps):
        return [dict(status=r.status, iterations=r.iterations, max_resid=r.max_resid,
                     fallbacks=r.fallbacks, wave=r.wave, seconds=r.seconds,
                     iterations_bulk=r.iterations_bulk, resid_bulk=r.resid_bulk,
                     graph_kernels=r.graph_kernels, restarts=r.restarts) for r in reps]

    def dgdft_alb_solve(self, check=False):
        reps = (dgdft_solve_report * self.n)()
        st = self.lib.dgdft_alb_solve(self.h, reps)
        if st not in (DGDFT_OK, DGDFT_ENOTCONV, DGDFT_ETIMEOUT) or (check and st != DGDFT_OK):
            self._check(st, "solve")
        return st, self._reports(reps)

    def dgdft_alb_scf_step(self, n_iter=3):
        reps = (dgdft_solve_report * self.n)()
        st = self.lib.dgdft_alb_scf_step(self.h, int(n_iter), reps)
        if st not in (DGDFT_OK, DGDFT_ENOTCONV, DGDFT_ETIMEOUT):
            self._check(st, "scf_step")
        return st, self._reports(reps)

    def dgdft_alb_get_basis(self, elem, phi=None, eig=None, resid=None):
        d = self.descs[elem]
        ne = (d.e_hi[0] - d.e_lo[0]) * (d.e_hi[1] - d.e_lo[1]) * (d.e_hi[2] - d.e_lo[2])
        J = d.n_keep
        phi = np.zeros((J, ne)) if phi is None else phi
        eig = np.zeros(J) if eig is None else eig
        resid = np.zeros(J) if resid is None else resid
        pp, dev = _ptr(phi)
        self._check(self.lib.dgdft_alb_get_basis(self.h, elem, pp, _ptr(eig)[0], _ptr(resid)[0], dev),
                    "get_basis")
        return phi, eig, resid

    def dgdft_alb_get_block(self, elem, out=None):
        """The Ritz block as (m, N_g) rows; with out (a contiguous device
        tensor of N_g * m doubles) the copy goes there instead."""
        d = self.descs[elem]
        x = np.zeros((d.n_compute, d.nx * d.ny * d.nz)) if out is None else out
        p, dev = _ptr(x)
        self._check(self.lib.dgdft_alb_get_block(self.h, elem, p, dev), "get_block")
        return x

    def dgdft_alb_time_stage(self, stage, reps=10):
        """(ms per launch, elements, working-precision bytes) of one kernel stage."""
        ms = C.c_double()
        ne = C.c_int()
        rb = C.c_int()
        self._check(self.lib.dgdft_alb_time_stage(self.h, stage, reps, C.byref(ms), C.byref(ne),
                                                  C.byref(rb)), "time_stage")
        return ms.value, ne.value, rb.value

    # learned preconditioner ---------------------------------------------
    def dgdft_alb_precond_init(self, seed=0):
        self._check(self.lib.dgdft_alb_precond_init(self.h, seed), "precond_init")

    def dgdft_alb_precond_set_params(self, params):
        p = np.ascontiguousarray(params, np.float32)
        assert p.size == PRECOND_PARAMS
        self._check(self.lib.dgdft_alb_precond_set_params(self.h, _ptr(p)[0]), "precond_set_params")

    def dgdft_alb_precond_get_params(self):
        p = np.zeros(PRECOND_PARAMS, np.float32)
        self._check(self.lib.dgdft_alb_precond_get_params(self.h, _ptr(p)[0]), "precond_get_params")
        return p

    def dgdft_alb_precond_save(self, path):
        self._check(self.lib.dgdft_alb_precond_save(self.h, path.encode()), "precond_save")

    def dgdft_alb_precond_load(self, path):
        self._check(self.lib.dgdft_alb_precond_load(self.h, path.encode()), "precond_load")

    def dgdft_alb_precond_forward(self, inp):
        """inp: (B, 2, nz, ny, nx) float32 (NumPy or CUDA tensor)."""
        B, _, nz, ny, nx = inp.shape
        if isinstance(inp, np.ndarray):
            inp = np.ascontiguousarray(inp, np.float32)
            out = np.zeros((B, 1, nz, ny, nx), np.float32)
        else:
            import torch
            out = torch.zeros((B, 1, nz, ny, nx), dtype=torch.float32, device=inp.device)
        pi, dev = _ptr(inp)
        self._check(self.lib.dgdft_alb_precond_forward(self.h, B, nz, ny, nx, pi, _ptr(out)[0], dev),
                    "precond_forward")
        return out

    def dgdft_alb_precond_loss_grad(self, inp, tgt, lo, hi):
        inp = np.ascontiguousarray(inp, np.float32)
        tgt = np.ascontiguousarray(tgt, np.float32)
        B, _, nz, ny, nx = inp.shape
        loss = C.c_double()
        g = np.zeros(PRECOND_PARAMS, np.float32)
        self._check(self.lib.dgdft_alb_precond_loss_grad(self.h, B, nz, ny, nx, lo, hi, _ptr(inp)[0],
                                                         _ptr(tgt)[0], C.byref(loss), _ptr(g)[0], 0),
                    "precond_loss_grad")
        return loss.value, g

    def dgdft_alb_precond_train(self, r, v, t, crop=32, batch=8, steps=100, lr=1e-3, seed=0):
        """r, v, t: CUDA float32 tensors (nfields, nz, ny, nx)."""
        nf, nz, ny, nx = r.shape
        l0 = C.c_double()
        l1 = C.c_double()
        self._check(self.lib.dgdft_alb_precond_train(self.h, nf, nz, ny, nx, _ptr(r)[0], _ptr(v)[0], _ptr(t)[0],
                                                     crop, batch, steps, lr, seed, C.byref(l0), C.byref(l1)),
                    "precond_train")
        return l0.value, l1.value

    def dgdft_alb_precond_make_data(self, elem, snap_iters):
        """(r, t, sigma, cg_iters): CUDA float32 tensors (nsnap * m, nz, ny, nx)."""
        import torch
        d = self.descs[elem]
        ns = len(snap_iters)
        shape = (ns * d.n_compute, d.nz, d.ny, d.nx)
        r = torch.zeros(shape, dtype=torch.float32, device="cuda")
        t = torch.zeros(shape, dtype=torch.float32, device="cuda")
        it = np.ascontiguousarray(snap_iters, np.int32)
        sig = np.zeros(ns)
        cg = np.zeros(ns, np.int32)
        self._check(self.lib.dgdft_alb_precond_make_data(self.h, elem, ns, _ptr(it)[0], _ptr(r)[0], _ptr(t)[0],
                                                         _ptr(sig)[0], _ptr(cg)[0]), "precond_make_data")
        return r, t, sig, cg

    # step entry points -------------------------------------------------
    def dgdft_alb_apply_h(self, elem, x, stage=0):
        x = np.ascontiguousarray(x, np.float64)
        out = np.zeros_like(x)
        self._check(self.lib.dgdft_alb_apply_h(self.h, elem, int(stage), x.shape[0], _ptr(x)[0], _ptr(out)[0], 0),
                    "apply_h")
        return out

    def dgdft_alb_apply_teter(self, elem, r, t_kin):
        r = np.ascontiguousarray(r, np.float64)
        t = np.ascontiguousarray(t_kin, np.float64)
        out = np.zeros_like(r)
        self._check(self.lib.dgdft_alb_apply_teter(self.h, elem, r.shape[0], _ptr(r)[0], _ptr(t)[0],
                                                   _ptr(out)[0], 0), "apply_teter")
        return out

    def dgdft_alb_project_cutoff(self, elem, x):
        """x: (k, N_g) rows; returns P x (the context's sphere-cutoff set)."""
        x = np.ascontiguousarray(x, np.float64)
        out = np.zeros_like(x)
        self._check(self.lib.dgdft_alb_project_cutoff(self.h, elem, x.shape[0], _ptr(x)[0], _ptr(out)[0], 0),
                    "project_cutoff")
        return out

    def dgdft_alb_gram(self, u, v):
        """u: (p, ng), v: (q, ng) rows = columns of the column-major blocks."""
        u = np.ascontiguousarray(u, np.float64)
        v = np.ascontiguousarray(v, np.float64)
        p, ng = u.shape
        q = v.shape[0]
        c = np.zeros((q, p))  # column-major p x q
        self._check(self.lib.dgdft_alb_gram(self.h, ng, p, q, _ptr(u)[0], _ptr(v)[0], _ptr(c)[0], 0),
                    "gram")
        return c.T.copy()

    def dgdft_alb_lobpcg_gram(self, elem, blocks, has_p=True, stage=0):
        """blocks: (6, m, N_g) rows X, W, P, HX, HW, HP.  Returns (a, b, xtw)
        with a, b the 3m x 3m pencil blocks (upper block triangle) and xtw =
        X^T W, as row-major NumPy arrays of the matrices.  stage 0: the bulk
        stage's kernels, 1: the FP64 stage's."""
        blk = np.ascontiguousarray(blocks, np.float64)
        m = blk.shape[1]
        a = np.zeros((3 * m, 3 * m))
        b = np.zeros((3 * m, 3 * m))
        xtw = np.zeros((m, m))
        self._check(self.lib.dgdft_alb_lobpcg_gram(self.h, elem, int(stage), int(bool(has_p)), _ptr(blk)[0],
                                                   _ptr(a)[0], _ptr(b)[0], _ptr(xtw)[0], 0), "lobpcg_gram")
        # column-major out -> matrices
        return a.T.copy(), b.T.copy(), xtw.T.copy()

    def dgdft_alb_lobpcg_update(self, elem, blocks, y, has_p=True, stage=0):
        """blocks: (6, m, N_g) rows X, W, P, HX, HW, HP; y: the 3m x m
        coefficient matrix.  Returns (3, m, N_g): X', P', HP' as rows."""
        blk = np.ascontiguousarray(blocks, np.float64)
        m, ng = blk.shape[1], blk.shape[2]
        ycm = np.ascontiguousarray(np.asarray(y, np.float64).T)  # column-major 3m x m
        out = np.zeros((3, m, ng))
        self._check(self.lib.dgdft_alb_lobpcg_update(self.h, elem, int(stage), int(bool(has_p)), _ptr(blk)[0],
                                                     _ptr(ycm)[0], _ptr(out)[0], 0), "lobpcg_update")
        return out

    def dgdft_alb_rayleigh_ritz(self, a, b, m, stage=1):
        """Lowest m eigenpairs of a y = theta b y; stage 0 is the FP32 stage's
        reduction (double-float in a mixed-precision context), 1 is FP64."""
        n = a.shape[0]
        a = np.ascontiguousarray(np.asarray(a, np.float64).T)
        b = np.ascontiguousarray(np.asarray(b, np.float64).T)
        theta = np.zeros(m)
        y = np.zeros((m, n))
        self._check(self.lib.dgdft_alb_rayleigh_ritz(self.h, int(stage), n, m, _ptr(a)[0], _ptr(b)[0],
                                                     _ptr(theta)[0], _ptr(y)[0]), "rayleigh_ritz")
        return theta, y.T.copy()

    def dgdft_alb_restrict_orthonormalise(self, elem, x, J):
        x = np.ascontiguousarray(x, np.float64)
        d = self.descs[elem]
        ne = (d.e_hi[0] - d.e_lo[0]) * (d.e_hi[1] - d.e_lo[1]) * (d.e_hi[2] - d.e_lo[2])
        phi = np.zeros((J, ne))
        self._check(self.lib.dgdft_alb_restrict_orthonormalise(self.h, elem, x.shape[0], J, _ptr(x)[0],
                                                               _ptr(phi)[0], 0), "restrict")
        return phi


def element_dict(el) -> dict:
    """Descriptor fields of a synthetic element (duck-typed: n, L, e_lo, e_hi, m, J)."""
    return dict(n=tuple(int(v) for v in el.n), L=tuple(float(v) for v in el.L),
                e_lo=tuple(el.e_lo), e_hi=tuple(el.e_hi), m=el.m, J=el.J)


def load_element(ctx: Context, k: int, el, x0=None):
    """Copy one element's potential, projectors and optional initial block in."""
    ctx.dgdft_alb_set_potential(k, np.ascontiguousarray(el.veff.reshape(-1), np.float64))
    if el.n_proj:
        ctx.dgdft_alb_set_projectors(k, el.proj_row_ptr, el.proj_idx, el.proj_val, el.proj_gamma)
    if x0 is not None:
        ctx.dgdft_alb_set_initial(k, np.ascontiguousarray(x0, np.float64))


STAGES = {"xy_fwd": 0, "z_mult": 1, "xy_inv": 2, "gram": 3, "update": 4, "rayleigh_ritz": 5,
          "residual": 6}


DG_STAGES = ("interpolation", "orthonormalise_gradients", "volume", "traces_kb", "faces", "blocks",
             "density_eigensolve", "density_evaluation")


class DG:
    """Owns one dgdft_dg handle (include/dgdft_dg.h); methods mirror the C
    entry points.  Arrays may be NumPy (host) or torch CUDA tensors."""

    def __init__(self, ne, cell, q_span, nq, nl, J, alpha, n_proj, stream=None, device=0,
                 hbm_cap_bytes=0, dfloat=False):
        self.lib = load()
        c = dgdft_dg_config()
        c.ne[:] = [int(v) for v in ne]
        c.cell[:] = [float(v) for v in cell]
        c.q_span[:] = [int(v) for v in q_span]
        c.nq[:] = [int(v) for v in nq]
        c.nl[:] = [int(v) for v in nl]
        c.J, c.alpha, c.n_proj = int(J), float(alpha), int(n_proj)
        c.cuda_stream = stream
        c.device = int(device)
        c.hbm_cap_bytes = int(hbm_cap_bytes)
        c.arith = 1 if dfloat else 0
        self.cfg = c
        self.J = int(J)
        self.nl = tuple(int(v) for v in nl)
        self.n_lgl = int(np.prod(self.nl))
        self.n_elem = int(np.prod(ne))
        self.h = C.c_void_p()
        st = self.lib.dgdft_dg_create(C.byref(c), C.byref(self.h))
        if st != DGDFT_OK:
            msg = self.lib.dgdft_dg_last_error(self.h).decode()
            self.lib.dgdft_dg_destroy(self.h)
            self.h = None
            raise DgdftError(st, msg)

    def _check(self, st, what):
        if st != DGDFT_OK:
            raise DgdftError(st, f"{what}: {self.lib.dgdft_dg_last_error(self.h).decode()}")

    def close(self):
        if self.h:
            self.lib.dgdft_dg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def dgdft_dg_lgl_points(self, elem):
        out = [np.zeros(n) for n in self.nl]
        self._check(self.lib.dgdft_dg_lgl_points(self.h, elem, *[_ptr(a)[0] for a in out]), "lgl_points")
        return out

    def dgdft_dg_set_potential(self, elem, v):
        p, dev = _ptr(v)
        self._check(self.lib.dgdft_dg_set_potential(self.h, elem, p, dev), "set_potential")

    def dgdft_dg_set_gamma(self, gamma):
        g = np.ascontiguousarray(gamma, np.float64)
        self._check(self.lib.dgdft_dg_set_gamma(self.h, _ptr(g)[0]), "set_gamma")

    def dgdft_dg_set_projectors(self, elem, pid, row_ptr, idx, val):
        pid = np.ascontiguousarray(pid, np.int32)
        rp = np.ascontiguousarray(row_ptr, np.int64)
        idx = np.ascontiguousarray(idx, np.int32)
        val = np.ascontiguousarray(val, np.float64)
        self._check(self.lib.dgdft_dg_set_projectors(self.h, elem, len(pid), _ptr(pid)[0], _ptr(rp)[0],
                                                     _ptr(idx)[0], _ptr(val)[0]), "set_projectors")

    def _block_ptrs(self, blocks):
        ptrs = (C.c_void_p * self.n_elem)()
        keep = []
        dev = None
        for k, z in enumerate(blocks):
            if isinstance(z, np.ndarray):
                z = np.ascontiguousarray(z, np.float64)
            keep.append(z)
            p, d = _ptr(z)
            if dev is None:
                dev = d
            elif dev != d:
                raise ValueError("blocks must all be on the host or all on the device")
            ptrs[k] = p
        return ptrs, int(dev or 0), keep

    def dgdft_dg_assemble(self, blocks):
        """blocks[K]: the J columns of element K on Q_K's grid, as (J, N_gQ)
        rows (NumPy) or a contiguous N_gQ x J column-major device tensor."""
        ptrs, dev, keep = self._block_ptrs(blocks)
        self._check(self.lib.dgdft_dg_assemble(self.h, ptrs, dev), "assemble")

    def dgdft_dg_density(self, blocks, n_occ, out=None):
        """(eigenvalues, rho (n_elem, n_LGL)) of the lowest n_occ states of the
        assembled H^DG; blocks as for assemble; out: an optional device tensor
        of n_elem * n_LGL doubles for rho."""
        ptrs, dev, keep = self._block_ptrs(blocks)
        eig = np.zeros(int(n_occ))
        rho = np.zeros((self.n_elem, self.n_lgl)) if out is None else out
        p, rdev = _ptr(rho)
        self._check(self.lib.dgdft_dg_density(self.h, ptrs, dev, int(n_occ), _ptr(eig)[0], p, rdev), "density")
        return eig, rho

    def dgdft_dg_neighbours(self, elem):
        nb = np.zeros(27, np.int32)
        n = C.c_int()
        self._check(self.lib.dgdft_dg_neighbours(self.h, elem, _ptr(nb)[0], C.byref(n)), "neighbours")
        return [int(v) for v in nb[:n.value]]

    def dgdft_dg_get_row(self, elem):
        """{K': H_{elem, K'} (J x J, rows = basis of elem)}."""
        nb = self.dgdft_dg_neighbours(elem)
        out = np.zeros((len(nb), self.J, self.J))
        self._check(self.lib.dgdft_dg_get_row(self.h, elem, _ptr(out)[0], 0), "get_row")
        return {k: out[s] for s, k in enumerate(nb)}

    def dgdft_dg_lgl_basis(self, elem, z):
        """Orthonormal ALBs on the LGL grid as (J, n_LGL) rows."""
        z = np.ascontiguousarray(z, np.float64)
        phi = np.zeros((self.J, self.n_lgl))
        self._check(self.lib.dgdft_dg_lgl_basis(self.h, elem, _ptr(z)[0], 0, _ptr(phi)[0], 0), "lgl_basis")
        return phi

    def dgdft_dg_density_info(self):
        """Sweeps of the Jacobi eigensolver in the last density call."""
        n = C.c_int()
        self._check(self.lib.dgdft_dg_density_info(self.h, C.byref(n)), "density_info")
        return n.value

    def dgdft_dg_last_timing(self):
        ms = np.zeros(8)
        n = C.c_int()
        self._check(self.lib.dgdft_dg_last_timing(self.h, _ptr(ms)[0], 8, C.byref(n)), "last_timing")
        return dict(zip(DG_STAGES, ms.tolist())), n.value
