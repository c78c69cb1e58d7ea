"""N = 256 (the slice is distributed over a 4-CTA cluster): the phase-screen GSM workload
(N = 256, dxi = 20 um, lambda = 633 nm, z = 0.5 m, unit-modulus screen with 3 px correlation)
against the oracle's row probes, plus Hermiticity, power and trace conservation (GPU)."""
import numpy as np
import pytest

import oracle as O
import workloads as WL

pytestmark = pytest.mark.gpu


def test_phase_screen_n256():
    import torch
    import paper_2203_02734_gb300 as pw

    cfg = WL.PHASE_SCREEN_N256
    N, dxi, lam, z = cfg["N"], cfg["dxi"], cfg["lam"], cfg["z"]
    mask = WL.to_c64(WL.phase_screen(N, seed=WL.SEED, corr_px=cfg["corr_px"]))
    c = pw.CSD(N, dxi, lam)
    mt = torch.from_numpy(mask).cuda()
    c.source_gsm(cfg["sigma_S"], cfg["sigma_mu"], cfg["A"])
    c.source_mask(mt)
    c.propagate_fresnel(z)
    S = c.spectral_density()
    pw.pw_csd_check(c.h)
    torch.cuda.synchronize()
    rows = [cfg["P1"], (120, 137), (140, 122)]
    Wrows = [c.W[a, b].cpu().numpy().astype(np.complex128) for a, b in rows]
    S = S.cpu().numpy().astype(np.float64)
    dx = c.sampling()
    # Hermiticity on sampled columns
    wref = np.linalg.norm(Wrows[0])
    for (a, b) in [(128, 128), (131, 125), (10, 250)]:
        col = c.W[:, :, a, b].cpu().numpy().astype(np.complex128)
        rowv = c.W[a, b].cpu().numpy().astype(np.complex128)
        assert np.linalg.norm(col - np.conj(rowv)) < 1e-6 * wref
    # power (float64 accumulation in chunks) and trace
    flat = c.W.view(-1)
    p2 = 0.0
    for k in range(0, flat.numel(), 1 << 27):
        p2 += float(torch.sum(torch.abs(flat[k:k + (1 << 27)]).double() ** 2))
    c.close()
    x, _ = O.axis_coords(N, dxi)
    g = np.exp(-(x[:, None] ** 2 + x[None, :] ** 2) / (4 * cfg["sigma_S"] ** 2)
               - (x[:, None] - x[None, :]) ** 2 / (2 * cfg["sigma_mu"] ** 2))
    m = mask.astype(np.complex128)
    w2 = np.abs(m) ** 2
    p0 = np.einsum("ab,ac,bd,cd->", w2, g ** 2, g ** 2, w2, optimize=True) * dxi ** 4
    assert abs(p2 * dx ** 4 / p0 - 1) < 1e-5
    S0 = np.einsum("aa,bb,ab->ab", g, g, w2)
    assert abs(S.sum() * dx ** 2 / (S0.sum() * dxi ** 2) - 1) < 1e-5
    assert S.min() > -1e-6 * S.max()

    probe = O.propagate_rows_gsm(m, N, dxi, lam, z, cfg["sigma_S"], cfg["sigma_mu"], cfg["A"], rows)
    for r, (a, b) in enumerate(rows):
        err = np.linalg.norm(Wrows[r] - probe[r]) / np.linalg.norm(probe[r])
        assert err < 1e-5, (a, b, err)
        assert abs(S[a, b] - probe[r][a, b].real) < 1e-5 * np.abs(probe[0]).max()


def test_n256_rejects_general_array():
    import torch
    import paper_2203_02734_gb300 as pw
    c = pw.CSD(256, 20e-6, 633e-9)
    with pytest.raises(pw.PwError, match="PW_EUNSUPPORTED"):
        pw.pw_source_array(c.h, c.W.data_ptr(), False)
        pw.pw_propagate_fresnel(c.h, 0.5)
    c.close()
