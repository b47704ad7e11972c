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
    a = ap.parse_args()
    train(a.out, a.geometries, [int(s) for s in a.snaps.split(",")], a.steps, a.batch, a.crop, a.lr, a.seed)


if __name__ == "__main__":
    main()
