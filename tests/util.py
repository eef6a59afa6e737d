"""Helpers shared by the GPU tests: block-relative errors of effective tensors."""
import numpy as np


def block_rel_err(E, Eref, N, d):
    """max over points and blocks of ||dE_blk||_F / ||Eref_blk||_F for the exchange block
    (N x N), the two cross blocks and the permeability block (Nd x Nd)."""
    E = np.asarray(E).reshape(-1, *np.asarray(E).shape[-2:])
    Eref = np.asarray(Eref).reshape(E.shape)
    sl = [slice(0, N), slice(N, N * (1 + d))]
    worst = 0.0
    for a in sl:
        for b in sl:
            num = np.linalg.norm(E[:, a, b] - Eref[:, a, b], axis=(1, 2))
            den = np.linalg.norm(Eref[:, a, b], axis=(1, 2))
            ok = den > 0
            if ok.any():
                worst = max(worst, float((num[ok] / den[ok]).max()))
            if (~ok).any():
                worst = max(worst, float(num[~ok].max()))
    return worst
