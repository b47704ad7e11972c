"""Train the learned preconditioner on pairs made by the plain FP64 solver.

    python -m paper_1506_08147_gb300.train_precond --out weights.bin \
        [--geometries 64] [--snaps 5,15,40] [--steps 3000] [--batch 8] [--crop 40]

For each seeded perturbation of the monolayer geometry (extended element 0),
the library runs the plain FP64 LOBPCG and records residual blocks at the
given iterations together with exact corrections t = (H - sigma I)^-1 r
(FP64 conjugate gradients); the network is then trained on random crops by
the library's own BF16/FP32 kernels.  Everything runs on the GPU through the
C-ABI; this script only moves device pointers around.
"""

from __future__ import annotations

import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def make_pool(geometries, snaps, log=print):
    import numpy as np
    import torch

    import synth
    from paper_1506_08147_gb300 import binding as B

    rs, ts, vs = [], [], []
    for g in range(geometries):
        el = synth.config4(g)[0]
        c = B.Context([B.element_dict(el)], precision=B.DGDFT_PREC_FP64)
        B.load_element(c, 0, el, synth.initial_block(el))
        t0 = time.time()
        r, t, sig, cg = c.dgdft_alb_precond_make_data(0, snaps)
        c.close()
        v = torch.from_numpy(el.veff.astype(np.float32)).cuda()
        rs.append(r)
        ts.append(t)
        vs.append(v.unsqueeze(0).expand(r.shape[0], *v.shape))
        log(f"geometry {g}: {r.shape[0]} fields, sigma {np.round(sig, 4).tolist()}, CG {cg.tolist()}, "
            f"{time.time() - t0:.1f} s")
    return torch.cat(rs), torch.cat(vs).contiguous(), torch.cat(ts)


def train(out_path, geometries=64, snaps=(5, 15, 40), steps=3000, batch=8, crop=40, lr=1e-3, seed=0, log=print):
    import synth
    from paper_1506_08147_gb300 import binding as B

    r, v, t = make_pool(geometries, list(snaps), log)
    el = synth.config4(0)[0]
    c = B.Context([B.element_dict(el)], precision=B.DGDFT_PREC_MIXED)
    c.dgdft_alb_precond_init(seed)
    t0 = time.time()
    l0, l1 = c.dgdft_alb_precond_train(r, v, t, crop=crop, batch=batch, steps=steps, lr=lr, seed=seed)
    c.dgdft_alb_precond_save(out_path)
    c.close()
    info = {"fields": int(r.shape[0]), "crops_seen": steps * batch, "loss_first": l0, "loss_last": l1,
            "train_seconds": time.time() - t0}
    log(json.dumps(info))
    return info


def evaluate(weights_path, n_elems=4, log=print):
    """Mixed-form solves of the first n_elems monolayer elements (config 2,
    which is not among the training geometries) with Teter and with the
    network: iterations of the FP32 stage, total iterations, seconds."""
    import time as _time

    import numpy as np

    import synth
    from paper_1506_08147_gb300 import binding as B

    els = synth.config2(elems=list(range(n_elems)))
    out = {}
    for name, mode in (("teter", B.DGDFT_PRECOND_TETER), ("learned", B.DGDFT_PRECOND_LEARNED)):
        c = B.Context([B.element_dict(e) for e in els], precision=B.DGDFT_PREC_MIXED, tol=1e-6, maxit=600,
                      precond=mode, precond_weights=weights_path if name == "learned" else None)
        for k, e in enumerate(els):
            B.load_element(c, k, e, synth.initial_block(e))
        c.dgdft_alb_solve()  # warm-up (wave build)
        for k, e in enumerate(els):
            c.dgdft_alb_set_initial(k, synth.initial_block(e))
        t0 = _time.time()
        st, rep = c.dgdft_alb_solve()
        dt = _time.time() - t0
        c.close()
        out[name] = {"status": int(st), "seconds": dt,
                     "fp32_iterations_mean": float(np.mean([r["iterations_bulk"] for r in rep])),
                     "iterations_mean": float(np.mean([r["iterations"] for r in rep])),
                     "iterations_max": int(max(r["iterations"] for r in rep)),
                     "teter_fallbacks": int(sum(r["fallbacks"] for r in rep)) if name == "learned" else 0,
                     "max_resid": float(max(r["max_resid"] for r in rep))}
        log(json.dumps({name: out[name]}))
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", required=True)
    ap.add_argument("--geometries", type=int, default=64)
    ap.add_argument("--snaps", default="5,15,40")
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--crop", type=int, default=40)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--eval", type=int, default=0, help="then compare with Teter on this many monolayer elements")
    a = ap.parse_args()
    train(a.out, a.geometries, [int(s) for s in a.snaps.split(",")], a.steps, a.batch, a.crop, a.lr, a.seed)
    if a.eval > 0:
        evaluate(a.out, a.eval)


if __name__ == "__main__":
    main()
