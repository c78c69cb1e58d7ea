"""The paper's worked examples on the GPU, against their closed forms (Sec. 5.1 and 5.2): physics
pins of the CUDA path that do not go through the oracle.

- Fresnel "dark spot" of a perfectly coherent square source (Sec. 5.1): S at the distance
  R = a^2/(2 pi lambda) against the Fresnel-integral intensity of a square aperture.
- Far field of a perfectly incoherent annular source (Sec. 5.2): mu(0, x) against the van
  Cittert-Zernike theorem.

The discrete sources are pixelated (a square of N_a pixels, an annulus of pixels with the
half-weight boundary of the paper's circ function), so they differ from the continuous ones of
the closed forms by their sampling: measured on the FP64 oracle with the same parameters, the
normalised profiles differ by up to 0.019 (dark spot) and 0.027 (annulus); the bars below are
0.03 and 0.04."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

D, LAM = 20e-6, 633e-9


def test_fresnel_dark_spot_coherent_square():
    sp = pytest.importorskip("scipy.special")
    import torch
    import paper_2203_02734_gb300 as pw
    N = 64
    Na = int(round(np.sqrt(2 * np.pi * N)))  # Eq. Na: the output sampling equals the source's
    R = (Na * D) ** 2 / (2 * np.pi * LAM)    # Eq. darkspot
    i0 = N // 2 - Na // 2
    m = np.zeros((N, N), np.complex64)
    m[i0:i0 + Na, i0:i0 + Na] = 1.0
    c = pw.CSD(N, D, LAM)
    c.source_gsm(1e3, 1e3, 1.0)  # coherence widths of a kilometre: G = 1, a perfectly coherent source
    c.source_mask(torch.from_numpy(m).cuda())
    c.propagate_fresnel(R)
    S = c.spectral_density().cpu().numpy().astype(np.float64)
    dx = c.sampling()
    c.close()
    x, _ = O.axis_coords(N, D)
    X, Y = O.axis_coords(N, dx)
    lo, hi = x[i0] - D / 2, x[i0 + Na - 1] + D / 2  # the square's outer pixel edges
    s = np.sqrt(2 / (LAM * R))

    def factor(u):  # Fresnel-integral intensity factor of one axis (Eq. I_square_fresnel)
        S1, C1 = sp.fresnel(s * (lo - u))
        S2, C2 = sp.fresnel(s * (hi - u))
        return 0.5 * ((C2 - C1) ** 2 + (S2 - S1) ** 2)
    I = factor(X)[:, None] * factor(-Y)[None, :]  # second axis: y = (N/2 - j) dx = -x
    Sn, In = S / S.max(), I / I.max()
    assert np.abs(Sn - In).max() < 0.03
    cidx = N // 2
    assert Sn[cidx, cidx] < 0.5 * Sn[cidx, cidx + 3]  # the dark spot: a minimum at the centre


def test_annulus_far_field_van_cittert_zernike():
    sp = pytest.importorskip("scipy.special")
    import torch
    import paper_2203_02734_gb300 as pw
    N, z, No, Ni = 64, 2.0, 12, 5
    x, y = O.axis_coords(N, D)
    r2 = np.rint((x[:, None] ** 2 + y[None, :] ** 2) / D ** 2)

    def circ(n):  # 1 inside, 1/2 on the boundary, 0 outside (Sec. 5.2)
        return np.where(r2 < n * n, 1.0, np.where(r2 == n * n, 0.5, 0.0))
    dsrc = (circ(No) - circ(Ni)).astype(np.float32)
    c = pw.CSD(N, D, LAM)
    dd = torch.from_numpy(dsrc).cuda()
    pw.pw_source_diagonal(c.h, dd.data_ptr(), 1.0)
    c.propagate_farfield(z)
    P1 = (N // 2, N // 2)
    mu = c.degree_of_coherence(*P1).cpu().numpy().astype(np.complex128)
    dx = c.sampling()
    c.close()
    X, Y = O.axis_coords(N, dx)
    k = 2 * np.pi / LAM
    rho2 = X[:, None] ** 2 + Y[None, :] ** 2
    b = np.sqrt(rho2)
    # mu(0, x) carries the output propagator q(x) = exp(i pi |x|^2/(lambda z)); without it mu is real
    mr = mu * np.exp(-1j * k * rho2 / (2 * z))
    assert np.abs(mr.imag).max() < 1e-5

    def jinc(u):
        u = np.asarray(u, dtype=np.float64)
        safe = np.where(u == 0, 1.0, u)
        return np.where(u == 0, 1.0, 2 * sp.j1(safe) / safe)
    ao, ai = No * D, Ni * D
    mu_t = (ao ** 2 * jinc(k * ao * b / z) - ai ** 2 * jinc(k * ai * b / z)) / (ao ** 2 - ai ** 2)
    assert np.abs(mr.real - mu_t).max() < 0.04
