"""Host-side checks of the C-ABI library (no GPU needed).

* the in-tree shared library builds and exports every function that
  include/*.h declares;
* argument validation happens before any device work (bad descriptors give
  DGDFT_EINVAL) and, without a usable sm_103a device, create() fails with
  DGDFT_ECUDA instead of falling back to the CPU.
"""

import ctypes as C
import os
import re

import pytest

import __graft_entry__ as entry
from paper_1506_08147_gb300 import binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if not f.endswith(".h"):
            continue
        text = open(os.path.join(inc, f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(dgdft_(?:alb|dg)_\w+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    entry.build()
    return B.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15 and any(n.startswith("dgdft_dg_") for n in names)
    for n in names:
        assert hasattr(lib, n), n
        assert n in B._SIGS, f"binding lacks {n}"


def test_config_defaults(lib):
    cfg = B.dgdft_alb_config()
    lib.dgdft_alb_config_init(C.byref(cfg))
    assert cfg.precision == B.DGDFT_PREC_FP64 and cfg.tol == 1e-6 and cfg.maxit == 400
    assert cfg.check_every == 4 and cfg.device == -1 and cfg.keep_block == 0


def _desc(**kw):
    d = B.dgdft_element_desc()
    d.nx, d.ny, d.nz = kw.get("n", (16, 16, 16))
    d.Lx = d.Ly = d.Lz = 10.0
    lo, hi = kw.get("box", ((0, 0, 0), (16, 16, 16)))
    for a in range(3):
        d.e_lo[a], d.e_hi[a] = lo[a], hi[a]
    d.n_compute, d.n_keep = kw.get("mj", (16, 16))
    return d


@pytest.mark.parametrize("kw", [
    dict(n=(14, 16, 16)),            # 14/2 = 7 is not a product of 2, 3, 5
    dict(n=(15, 16, 16)),            # odd nx
    dict(mj=(8, 16)),                # J > m
    dict(box=((0, 0, 0), (17, 16, 16))),  # E_K outside Q_K
    dict(box=((4, 4, 4), (4, 8, 8))),     # empty E_K
])
def test_invalid_descriptors_rejected(lib, kw):
    cfg = B.dgdft_alb_config()
    lib.dgdft_alb_config_init(C.byref(cfg))
    arr = (B.dgdft_element_desc * 1)(_desc(**kw))
    h = C.c_void_p()
    assert lib.dgdft_alb_create(C.byref(cfg), 1, arr, C.byref(h)) == B.DGDFT_EINVAL


@pytest.mark.parametrize("kw", [
    dict(ecut=-1.0),                                  # negative cutoff
    dict(ecut=float("nan")),                          # not finite
    dict(ecut=1.0, precond=B.DGDFT_PRECOND_LEARNED),  # the cutoff needs the Teter preconditioner
    dict(ecut=0.5),                                   # 19 planewaves < 3 m = 48
])
def test_invalid_cutoff_rejected(lib, kw):
    cfg = B.dgdft_alb_config()
    lib.dgdft_alb_config_init(C.byref(cfg))
    for k, v in kw.items():
        setattr(cfg, k, v)
    arr = (B.dgdft_element_desc * 1)(_desc())
    h = C.c_void_p()
    assert lib.dgdft_alb_create(C.byref(cfg), 1, arr, C.byref(h)) == B.DGDFT_EINVAL


def test_valid_cutoff_passes_validation(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    # 16^3 on a 10 bohr box: |G|^2/2 <= 1 Ha holds 57 planewaves >= 3 m = 48,
    # so create() gets as far as the device check
    cfg = B.dgdft_alb_config()
    lib.dgdft_alb_config_init(C.byref(cfg))
    cfg.ecut = 1.0
    arr = (B.dgdft_element_desc * 1)(_desc())
    h = C.c_void_p()
    assert lib.dgdft_alb_create(C.byref(cfg), 1, arr, C.byref(h)) == B.DGDFT_ECUDA
    assert lib.dgdft_alb_project_cutoff(None, 0, 1, None, None, 0) == B.DGDFT_EINVAL


@pytest.mark.parametrize("ecut", [0.7, 1.0, 1.9])
def test_cutoff_set_size_matches_oracle(lib, ecut):
    """The library's count of planewaves in the sphere, seen through create()'s
    3 m check, equals the oracle mask's count: m = count / 3 passes
    validation, one more column is rejected."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from oracle import cutoff as oc
    count = int(oc.cutoff_mask((16, 16, 16), (10.0, 10.0, 10.0), ecut).sum())
    for m, want in ((count // 3, B.DGDFT_ECUDA), (count // 3 + 1, B.DGDFT_EINVAL)):
        cfg = B.dgdft_alb_config()
        lib.dgdft_alb_config_init(C.byref(cfg))
        cfg.ecut = ecut
        arr = (B.dgdft_element_desc * 1)(_desc(mj=(m, 1)))
        h = C.c_void_p()
        assert lib.dgdft_alb_create(C.byref(cfg), 1, arr, C.byref(h)) == want, (ecut, count, m)


def test_no_cpu_fallback_without_device(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    cfg = B.dgdft_alb_config()
    lib.dgdft_alb_config_init(C.byref(cfg))
    arr = (B.dgdft_element_desc * 1)(_desc())
    h = C.c_void_p()
    assert lib.dgdft_alb_create(C.byref(cfg), 1, arr, C.byref(h)) == B.DGDFT_ECUDA
    assert not h.value


def test_null_context_rejected(lib):
    # entry points validate their arguments before touching a device
    assert lib.dgdft_alb_solve(None, None) == B.DGDFT_EINVAL
    assert lib.dgdft_alb_scf_step(None, 3, None) == B.DGDFT_EINVAL
    assert lib.dgdft_alb_set_initial(None, 0, None, 0) == B.DGDFT_EINVAL
    assert lib.dgdft_alb_get_basis(None, 0, None, None, None, 0) == B.DGDFT_EINVAL


def _dg_cfg(**kw):
    c = B.dgdft_dg_config()
    c.ne[:] = kw.get("ne", (3, 3, 1))
    c.cell[:] = (18.0, 18.0, 24.0)
    c.q_span[:] = kw.get("q_span", (3, 3, 1))
    c.nq[:] = kw.get("nq", (24, 24, 30))
    c.nl[:] = kw.get("nl", (16, 16, 60))
    c.J = kw.get("J", 8)
    c.alpha = kw.get("alpha", 20.0)
    c.n_proj = 4
    return c


@pytest.mark.parametrize("kw", [
    dict(ne=(0, 3, 1)),
    dict(q_span=(2, 3, 1)),          # Q_K spans 3 elements, or the cell (1 with ne = 1)
    dict(q_span=(1, 3, 1)),          # q_span 1 with ne = 3
    dict(nl=(1, 16, 60)),
    dict(nl=(16, 16, 200)),          # above 128 LGL points
    dict(J=0),
    dict(J=200),
    dict(alpha=-1.0),
])
def test_dg_invalid_configs_rejected(lib, kw):
    h = C.c_void_p()
    assert lib.dgdft_dg_create(C.byref(_dg_cfg(**kw)), C.byref(h)) == B.DGDFT_EINVAL
    assert lib.dgdft_dg_last_error(h)
    lib.dgdft_dg_destroy(h)


def test_dg_no_cpu_fallback_without_device(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = C.c_void_p()
    assert lib.dgdft_dg_create(C.byref(_dg_cfg()), C.byref(h)) == B.DGDFT_ECUDA
    lib.dgdft_dg_destroy(h)


def test_dg_null_handle_rejected(lib):
    assert lib.dgdft_dg_assemble(None, None, 0) == B.DGDFT_EINVAL
    assert lib.dgdft_dg_get_row(None, 0, None, 0) == B.DGDFT_EINVAL
    assert lib.dgdft_dg_set_gamma(None, None) == B.DGDFT_EINVAL
