"""The allocation-free Gram entry point against NumPy and the regular one.

dgdft_alb_gram_noalloc exists for callers that cannot allocate device
memory while they run; its split-K scratch is a fixed device array inside
the library.  This file is collected last so that a run stopping at the
first failure has already run every other test; it passes on its own in a
fresh process too.  Two calls in a row (different shapes, so the second
call reuses scratch holding the first call's data) are each compared with
the FP64 product u v^T computed by NumPy on the host, and with dgdft_alb_gram
of an FP64 context, within 1e-12 relative.
"""

import ctypes as C

import numpy as np
import pytest

import __graft_entry__ as entry
from paper_1506_08147_gb300 import binding as B

pytestmark = pytest.mark.gpu


def test_gram_noalloc_matches_gram():
    import torch

    entry.build()
    lib = B.load()
    # a one-element FP64 context for the reference entry point
    desc = dict(n=(16, 16, 16), L=(10.0, 10.0, 10.0), e_lo=(0, 0, 0), e_hi=(16, 16, 16), m=8, J=8)
    ctx = B.Context([desc], precision=B.DGDFT_PREC_FP64)
    gen = np.random.default_rng(12)
    stream = torch.cuda.current_stream()
    for ng, p, q in ((122880, 144, 144), (7001, 37, 250)):
        u = gen.standard_normal((p, ng))
        v = gen.standard_normal((q, ng))
        du = torch.from_numpy(u).cuda()
        dv = torch.from_numpy(v).cuda()
        dc = torch.full((q, p), float("nan"), dtype=torch.float64, device="cuda")
        st = lib.dgdft_alb_gram_noalloc(ng, p, q, C.c_void_p(du.data_ptr()), C.c_void_p(dv.data_ptr()),
                                        C.c_void_p(dc.data_ptr()), C.c_void_p(stream.cuda_stream))
        assert st == B.DGDFT_OK
        torch.cuda.synchronize()
        got = dc.cpu().numpy().T          # column-major p x q
        exact = u @ v.T
        assert np.max(np.abs(got - exact)) <= 1e-12 * np.max(np.abs(exact))
        ref = ctx.dgdft_alb_gram(u, v)
        assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    # sizes beyond the limit are rejected before any GPU work
    assert lib.dgdft_alb_gram_noalloc(100, 257, 4, C.c_void_p(du.data_ptr()), C.c_void_p(dv.data_ptr()),
                                      C.c_void_p(dc.data_ptr()), None) == B.DGDFT_EINVAL
    ctx.close()
