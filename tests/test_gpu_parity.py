"""CUDA path vs the FP64 oracle, element by element, through the C ABI (GPU only).

Bar: relative L2 error <= 1e-5 for W, S and mu (mu where S >= 1e-4 max S), complex64 on
the GPU against complex128 in the oracle."""
import numpy as np
import pytest

import oracle as O
import workloads as WL
from gpu_cases import check_s_mu, gpu_run, oracle_run, rel

pytestmark = pytest.mark.gpu

DXI, LAM, SS, SM = 20e-6, 633e-9, 0.1e-3, 0.05e-3
TOL = 1e-5


def _mask(N, seed):
    u = WL.uniform01(seed, 2 * N * N).reshape(2, N, N)
    return (0.5 + 0.5 * u[0]) * np.exp(2j * np.pi * u[1])


def test_config_gsm_n32_fresnel():
    """Plain GSM, N = 32, dxi = 20 um, lambda = 633 nm, z = 0.5 m, P1 = (16, 16)."""
    cfg = WL.GSM_N32
    gsm = (cfg["sigma_S"], cfg["sigma_mu"], cfg["A"])
    out = gpu_run(32, cfg["dxi"], cfg["lam"], [("fresnel", cfg["z"])], gsm=gsm, P1=cfg["P1"])
    ref, dx = oracle_run(32, cfg["dxi"], cfg["lam"], [("fresnel", cfg["z"])], gsm=gsm)
    assert rel(out["W"], ref) < TOL
    assert abs(out["dx"] - dx) <= 1e-15 * dx
    check_s_mu(out, ref, cfg["P1"], name="gsm_n32_fresnel")
    # the discrete separable reference (no FFT) agrees too
    sep = O.gsm_separable_quadrature(32, cfg["dxi"], cfg["lam"], cfg["z"], *gsm)
    assert rel(out["W"], sep) < TOL


@pytest.mark.parametrize("N", [2, 4, 6, 8, 12, 16, 24, 32, 48, 64])
@pytest.mark.parametrize("kind", ["fresnel", "farfield"])
def test_masked_gsm_all_plans(N, kind):
    """GSM x aperture x thin lens x random complex mask; every radix plan, both regimes."""
    src = dict(gsm=(SS, SM, 1.3), aperture=0.37 * N * DXI, lens_f=0.25, mask=_mask(N, 100 + N))
    z = 0.4
    out = gpu_run(N, DXI, LAM, [(kind, z)], **src)
    ref, _ = oracle_run(N, DXI, LAM, [(kind, z)], **src)
    assert rel(out["W"], ref) < TOL
    check_s_mu(out, ref, (N // 2, N // 2), name="masked_gsm_n%d_%s" % (N, kind))


def test_amplitude_mask_n96():
    """N = 96 (radix 8 x 4 x 3), z = 1 m, amplitude mask uniform in [0.5, 1]."""
    cfg = WL.INVERSE_N96
    src = dict(gsm=(cfg["sigma_S"], cfg["sigma_mu"], 1.0), mask=WL.amplitude_mask(96))
    out = gpu_run(96, cfg["dxi"], cfg["lam"], [("fresnel", cfg["z"])], P1=cfg["P1"], **src)
    ref, _ = oracle_run(96, cfg["dxi"], cfg["lam"], [("fresnel", cfg["z"])], **src)
    assert rel(out["W"], ref) < TOL
    check_s_mu(out, ref, cfg["P1"], name="amplitude_mask_n96")


@pytest.mark.parametrize("N", [8, 16])
def test_uploaded_hermitian_csda(N):
    W0 = WL.random_csd(N, seed=5 + N, n_modes=3)
    out = gpu_run(N, DXI, LAM, [("fresnel", 0.3)], array=W0, hermitian=True)
    ref, _ = oracle_run(N, DXI, LAM, [("fresnel", 0.3)], array=W0)
    assert rel(out["W"], ref) < TOL
    check_s_mu(out, ref, (N // 2, N // 2))


@pytest.mark.parametrize("N", [8, 12])
def test_uploaded_general_array(N):
    """A non-Hermitian array takes the general (strided-store) second pass."""
    rng = np.random.default_rng(N)
    W0 = rng.standard_normal((N,) * 4) + 1j * rng.standard_normal((N,) * 4)
    out = gpu_run(N, DXI, LAM, [("farfield", 0.6)], array=W0, hermitian=False)
    ref, _ = oracle_run(N, DXI, LAM, [("farfield", 0.6)], array=W0)
    assert rel(out["W"], ref) < TOL


def test_two_planes():
    """Propagate, then propagate the result again (the output plane becomes the source)."""
    N = 32
    src = dict(gsm=(SS, SM, 1.0), aperture=0.3e-3)
    steps = [("fresnel", 0.2), ("farfield", 1.5)]
    out = gpu_run(N, DXI, LAM, steps, **src)
    ref, d = oracle_run(N, DXI, LAM, steps, **src)
    assert rel(out["W"], ref) < TOL
    assert abs(out["dx"] - d) <= 1e-14 * d
    check_s_mu(out, ref, (N // 2, N // 2))


def test_lens_identity_on_gpu():
    """Fresnel over z = f behind a thin lens equals far field without the lens (Eq. qprop3)."""
    N = 32
    a = gpu_run(N, DXI, LAM, [("fresnel", 0.3)], gsm=(SS, SM, 1.0), aperture=0.25e-3, lens_f=0.3)
    b = gpu_run(N, DXI, LAM, [("farfield", 0.3)], gsm=(SS, SM, 1.0), aperture=0.25e-3)
    assert rel(a["W"], b["W"]) < 1e-6


@pytest.mark.parametrize("src", ["gsm", "array"])
def test_source_plane_s_mu(src):
    N = 16
    if src == "gsm":
        kw = dict(gsm=(SS, SM, 2.0), aperture=0.11e-3, mask=_mask(N, 3))
    else:
        kw = dict(array=WL.random_csd(N, seed=9), lens_f=0.4)
    out = gpu_run(N, DXI, LAM, [], P1=(5, 9), **kw)
    W0 = oracle_run(N, DXI, LAM, [], **kw)[0]
    check_s_mu(out, W0, (5, 9))


def test_degenerate_point_source_and_zero_mask():
    N = 16
    # an aperture admitting only the centre pixel: a coherent point source, |mu| = 1
    out = gpu_run(N, DXI, LAM, [("fresnel", 0.5)], gsm=(SS, SM, 1.0), aperture=0.2 * DXI)
    ref, _ = oracle_run(N, DXI, LAM, [("fresnel", 0.5)], gsm=(SS, SM, 1.0), aperture=0.2 * DXI)
    assert rel(out["W"], ref) < TOL
    assert np.allclose(np.abs(out["mu"]), 1.0, atol=1e-5)
    # an all-zero mask: W = 0, S = 0, mu := 0
    z = gpu_run(N, DXI, LAM, [("fresnel", 0.5)], gsm=(SS, SM, 1.0), mask=np.zeros((N, N)))
    assert np.abs(z["W"]).max() == 0 and np.abs(z["S"]).max() == 0 and np.abs(z["mu"]).max() == 0


def test_invariants_full_size_n128():
    """N = 128 workload (GSM x 0.8 mm aperture x f = 0.3 m lens, Fresnel z = 0.3 m): sampled
    rows against the oracle's row probes, plus Hermiticity, power and trace conservation."""
    cfg = WL.GSM_APERTURE_LENS_N128
    N, dxi, lam, z = cfg["N"], cfg["dxi"], cfg["lam"], cfg["z"]
    src = dict(gsm=(cfg["sigma_S"], cfg["sigma_mu"], cfg["A"]), aperture=cfg["aperture"], lens_f=cfg["lens_f"])
    out = gpu_run(N, dxi, lam, [("fresnel", z)], P1=cfg["P1"], **src)
    W = out["W"]
    from gpu_cases import source_mask
    m = source_mask(N, dxi, lam, cfg["aperture"], cfg["lens_f"])
    x, _ = O.axis_coords(N, dxi)
    g = np.exp(-(x[:, None] ** 2 + x[None, :] ** 2) / (4 * cfg["sigma_S"] ** 2)
               - (x[:, None] - x[None, :]) ** 2 / (2 * cfg["sigma_mu"] ** 2))

    def slice_fn(a, b):
        return np.conj(m[a, b]) * g[a][:, None] * g[b][None, :] * m
    # rows in the beam core (the far-field pattern is ~8 px wide here) and one in the tail,
    # where W ~ 1e-19 and only the absolute error (relative to max |W|) is meaningful
    rows = [cfg["P1"], (60, 70), (72, 57), (40, 90)]
    probe = O.propagate_rows(slice_fn, N, dxi, lam, z, rows)
    wmax = np.abs(probe[0]).max()
    for r, (a, b) in enumerate(rows[:3]):
        assert rel(W[a, b], probe[r]) < TOL
        assert abs(out["S"][a, b] - probe[r][a, b].real) < 1e-5 * wmax
    assert np.linalg.norm(W[40, 90] - probe[3]) < 1e-6 * np.linalg.norm(probe[0])
    # Hermiticity (sampled blocks), power and trace
    wref = np.linalg.norm(W[64, 64])
    for (a, b) in [(3, 70), (64, 64), (60, 70), (120, 1)]:
        assert np.linalg.norm(W[:, :, a, b] - np.conj(W[a, b])) < 1e-6 * wref
    dx = out["dx"]
    w2 = np.abs(m) ** 2
    p0 = np.einsum("ab,ac,bd,cd->", w2, g ** 2, g ** 2, w2) * dxi ** 4
    assert abs(np.sum(np.abs(W) ** 2) * dx ** 4 / p0 - 1) < 1e-5
    S0 = np.einsum("aa,bb,ab->ab", g, g, w2)
    assert abs(out["S"].sum() * dx ** 2 / (S0.sum() * dxi ** 2) - 1) < 1e-5
    assert out["S"].min() > -1e-6 * out["S"].max()
    assert np.abs(out["mu"]).max() <= 1 + 1e-5


@pytest.mark.parametrize("kind", ["fresnel", "farfield"])
def test_output_is_hermitian_non_negative_definite(kind):
    """A CSD is a Hermitian non-negative definite kernel (Sec. 3.3): the propagated N^2 x N^2 matrix
    of a random PSD source keeps both properties up to FP32 rounding."""
    N = 16
    W0 = WL.random_csd(N, seed=31, n_modes=4)
    out = gpu_run(N, DXI, LAM, [(kind, 0.35)], array=W0, hermitian=True)
    M = out["W"].reshape(N * N, N * N)
    scale = np.abs(M).max()
    assert np.abs(M - M.conj().T).max() <= 1e-6 * scale
    ev = np.linalg.eigvalsh(0.5 * (M + M.conj().T))
    assert ev.min() >= -1e-5 * ev.max()
    # rank: four modes in, four significant eigenvalues out (propagation is unitary up to scale)
    assert np.sum(ev > 1e-4 * ev.max()) == 4


def test_general_array_n96():
    """Non-Hermitian rank-2 CSDA at N = 96: the register-resident pass A with the general
    (strided-store) pass B, against the oracle's row probes (Eq. W_fresnel row by row)."""
    N = 96
    f = [WL.to_c64((0.5 + 0.5 * WL.uniform01(400 + k, N * N).reshape(N, N))
                   * np.exp(2j * np.pi * WL.uniform01(500 + k, N * N).reshape(N, N))) for k in range(4)]
    W0 = (f[0].reshape(-1, 1) * f[1].reshape(1, -1) + f[2].reshape(-1, 1) * f[3].reshape(1, -1))
    W0 = W0.astype(np.complex64).reshape(N, N, N, N)
    out = gpu_run(N, DXI, LAM, [("fresnel", 0.45)], array=W0, hermitian=False)
    rows = [(48, 48), (5, 90), (77, 13)]
    probe = O.propagate_rows(lambda a, b: W0[a, b].astype(np.complex128), N, DXI, LAM, 0.45, rows)
    for r, (a, b) in enumerate(rows):
        assert rel(out["W"][a, b], probe[r]) < TOL
        assert abs(out["S"][a, b] - probe[r][a, b].real) <= 1e-5 * np.abs(probe[r]).max()
