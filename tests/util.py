"""Helpers shared by the GPU tests: block-relative errors of effective tensors."""
import numpy as np


def block_rel_err(E, Eref, N, d):
    """max over points and blocks of ||dE_blk||_F / scale_blk for the exchange block
    (N x N), the two cross blocks and the permeability block (Nd x Nd).

    The scale of a diagonal block is its own norm ||Eref_aa||_F. A cross block of the Gram
    matrix E is bounded by Cauchy-Schwarz (|E_rs| <= sqrt(E_rr E_ss)), and on media with a
    mirror symmetry its exact value vanishes, so its own norm is round-off; its scale is
    sqrt(||Eref_aa||_F ||Eref_bb||_F)."""
    E = np.asarray(E).reshape(-1, *np.asarray(E).shape[-2:])
    Eref = np.asarray(Eref).reshape(E.shape)
    sl = [slice(0, N), slice(N, N * (1 + d))]
    diag = [np.linalg.norm(Eref[:, a, a], axis=(1, 2)) for a in sl]
    worst = 0.0
    for i, a in enumerate(sl):
        for j, b in enumerate(sl):
            num = np.linalg.norm(E[:, a, b] - Eref[:, a, b], axis=(1, 2))
            den = diag[i] if i == j else np.sqrt(diag[i] * diag[j])
            ok = den > 0
            if ok.any():
                worst = max(worst, float((num[ok] / den[ok]).max()))
            if (~ok).any():
                worst = max(worst, float(num[~ok].max()))
    return worst


def entry_rel_err(E, Eref):
    """max over points and entries of |dE_rs| / sqrt(Eref_rr Eref_ss): every entry of the
    (symmetric positive definite) Gram matrix against its Cauchy-Schwarz bound |E_rs| <=
    sqrt(E_rr E_ss), so that a small entry inside a block is checked on its own."""
    E = np.asarray(E).reshape(-1, *np.asarray(E).shape[-2:])
    Eref = np.asarray(Eref).reshape(E.shape)
    d = np.sqrt(np.abs(np.einsum("pii->pi", Eref)))
    scale = d[:, :, None] * d[:, None, :]
    return float((np.abs(E - Eref) / scale).max())
