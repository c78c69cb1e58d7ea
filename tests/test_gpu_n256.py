"""N = 256: the phase-screen GSM workload (N = 256, dxi = 20 um, lambda = 633 nm, z = 0.5 m,
unit-modulus screen with 3 px correlation) against the oracle: 65 output rows spread over the grid
(edges included) from the row route of Eq. W_fresnel, 16 random bilinear probes u^H W_B v over the
whole array from W0 through the kernel sums of Eq. W_general, S and mu at the rows' points, plus
Hermiticity, power and trace conservation (GPU); a non-Hermitian uploaded array and a
delta-correlated source in the far field on the three-pass engine; and the
same workload with the first radix-16 stage on the tensor cores (split-BF16x3), whose FP64
errors for W, S and mu are printed next to those of the FP32 path."""
import numpy as np
import pytest

import oracle as O
import workloads as WL

pytestmark = pytest.mark.gpu


# 64 output rows spread over the grid, edges included (8 x 8 point-1 positions)
ROW_IDX = (0, 1, 64, 120, 128, 137, 200, 255)
ROWS_64 = [(a, b) for a in ROW_IDX for b in (0, 3, 70, 122, 128, 140, 190, 255)]


def _probe_fields(N, K, seed):
    u = WL.uniform01(seed, 4 * K * N * N).reshape(4, K, N, N)
    return (u[0] - 0.5) + 1j * (u[1] - 0.5), (u[2] - 0.5) + 1j * (u[3] - 0.5)


def _gpu_probes(W, U, V):
    """u_k^H W v_k of the device CSDA (N^2 x N^2 matrix), accumulated in complex128 on the device."""
    import torch
    N, K = W.shape[0], U.shape[0]
    M = W.view(N * N, N * N)
    Vt = torch.from_numpy(np.ascontiguousarray(V.reshape(K, N * N).T)).cuda()
    Mv = torch.empty((N * N, K), dtype=torch.complex128, device="cuda")
    for r0 in range(0, N * N, 2048):
        Mv[r0:r0 + 2048] = M[r0:r0 + 2048].to(torch.complex128) @ Vt
    Ut = torch.from_numpy(U.reshape(K, N * N)).cuda()
    return (torch.conj(Ut) * Mv.T).sum(1).cpu().numpy()


def test_phase_screen_n256():
    import torch
    import paper_2203_02734_gb300 as pw
    from gpu_cases import record

    cfg = WL.PHASE_SCREEN_N256
    N, dxi, lam, z = cfg["N"], cfg["dxi"], cfg["lam"], cfg["z"]
    mask = WL.to_c64(WL.phase_screen(N, seed=WL.SEED, corr_px=cfg["corr_px"]))
    c = pw.CSD(N, dxi, lam)
    mt = torch.from_numpy(mask).cuda()
    c.source_gsm(cfg["sigma_S"], cfg["sigma_mu"], cfg["A"])
    c.source_mask(mt)
    c.propagate_fresnel(z)
    P1 = tuple(cfg["P1"])
    S = c.spectral_density()
    mu = c.degree_of_coherence(*P1)
    pw.pw_csd_check(c.h)
    torch.cuda.synchronize()
    rows = [P1] + ROWS_64
    Wrows = np.stack([c.W[a, b].cpu().numpy().astype(np.complex128) for a, b in rows])
    S = S.cpu().numpy().astype(np.float64)
    mu = mu.cpu().numpy().astype(np.complex128)
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
    # 16 random bilinear probes u^H W_B v over the whole array
    U, V = _probe_fields(N, 16, 2022)
    pg = _gpu_probes(c.W, U, V)
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
    assert np.abs(mu).max() <= 1 + 1e-5

    # the probes from W0 through the kernel sums of Eq. W_general (no FFT)
    pr = O.bilinear_probes_gsm(m, N, dxi, lam, z, cfg["sigma_S"], cfg["sigma_mu"], cfg["A"], U, V)
    rms = np.sqrt(np.mean(np.abs(pr) ** 2))
    ep = np.abs(pg - pr).max() / rms
    # 64 rows (and P1's row) against the oracle's row probes (Eq. W_fresnel row by row)
    probe = O.propagate_rows_gsm(m, N, dxi, lam, z, cfg["sigma_S"], cfg["sigma_mu"], cfg["A"], rows)
    erows = rel(Wrows, probe)
    rmax = np.linalg.norm(probe, axis=(1, 2)).max()
    eworst = max(np.linalg.norm(Wrows[r] - probe[r]) for r in range(len(rows))) / rmax
    # S at the rows' own points and mu(P1, x) at those points (S from each row's diagonal entry)
    pts = rows[1:]
    S_ref = np.array([probe[1 + k][a, b].real for k, (a, b) in enumerate(pts)])
    S_gpu = np.array([S[a, b] for a, b in pts])
    eS = np.linalg.norm(S_gpu - S_ref) / np.linalg.norm(S_ref)
    S_P1 = probe[0][P1].real
    keep = S_ref >= 1e-4 * S_ref.max()
    mu_ref = np.array([probe[0][a, b] / np.sqrt(S_P1 * S_ref[k]) for k, (a, b) in enumerate(pts)])
    mu_gpu = np.array([mu[a, b] for a, b in pts])
    emu = np.linalg.norm((mu_gpu - mu_ref)[keep]) / np.linalg.norm(mu_ref[keep])
    record("phase_screen_n256", W_rows=erows, W_row_worst=eworst, probes=ep, S_pts=eS, mu_pts=emu,
           mu_pts_kept=float(keep.sum()))
    assert ep < 1e-5, ep
    assert erows < 1e-5, erows
    assert eworst < 1e-5, eworst
    assert eS < 1e-5, eS
    assert emu < 1e-5, emu


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


def test_n256_general_array():
    # a non-Hermitian uploaded CSDA, W0 = u(xi1) v(xi2) (built on the device), two rows against the
    # oracle's row route (Eq. W_fresnel, point-1 sum written out)
    import torch
    import paper_2203_02734_gb300 as pw
    N, dxi, lam, z = 256, 20e-6, 633e-9, 0.5
    u = WL.phase_screen(N, seed=WL.SEED + 5, corr_px=4.0)
    x, _ = O.axis_coords(N, dxi)
    env = np.exp(-(x[:, None] ** 2 + x[None, :] ** 2) / (4 * (0.3e-3) ** 2))
    u = (u * env).astype(np.complex64)
    v = (WL.to_c64(WL.phase_screen(N, seed=WL.SEED + 6, corr_px=2.0)) * np.sqrt(env)).astype(np.complex64)
    c = pw.CSD(N, dxi, lam)
    ut, vt = torch.from_numpy(u).cuda(), torch.from_numpy(v).cuda()
    for a in range(N):  # W0[a, b, :, :] = u[a, b] v
        c.W[a].copy_(ut[a][:, None, None] * vt[None])
    pw.pw_source_array(c.h, c.W.data_ptr(), False)
    c.propagate_fresnel(z)
    rows = [(128, 128), (121, 140)]
    Wrows = [c.W[a, b].cpu().numpy().astype(np.complex128) for a, b in rows]
    pw.pw_csd_check(c.h)
    c.close()
    u64, v64 = u.astype(np.complex128), v.astype(np.complex128)
    ref = O.propagate_rows(lambda i1, j1: u64[i1, j1] * v64, N, dxi, lam, z, rows)
    for r in range(len(rows)):
        assert np.linalg.norm(Wrows[r] - ref[r]) / np.linalg.norm(ref[r]) < 1e-5


def _sample_points(N, n, seed=7):
    rng = np.random.default_rng(seed)
    pts = [(int(a), int(b)) for a, b in rng.integers(N // 2 - 40, N // 2 + 40, size=(n, 2))]
    return pts


def _errors_vs_oracle(mode):
    """Propagate the phase-screen workload in `mode`; return the FP64 errors of W (three full rows),
    S and mu(P1, .) (at sampled points, each computed by the oracle one row at a time)."""
    import torch
    import paper_2203_02734_gb300 as pw
    cfg = WL.PHASE_SCREEN_N256
    N, dxi, lam, z = cfg["N"], cfg["dxi"], cfg["lam"], cfg["z"]
    mask = WL.to_c64(WL.phase_screen(N, seed=WL.SEED, corr_px=cfg["corr_px"]))
    c = pw.CSD(N, dxi, lam)
    pw.pw_csd_set_dft_mode(c.h, mode)
    assert pw.pw_csd_get_dft_mode(c.h) == mode
    mt = torch.from_numpy(mask).cuda()
    c.source_gsm(cfg["sigma_S"], cfg["sigma_mu"], cfg["A"])
    c.source_mask(mt)
    c.propagate_fresnel(z)
    P1 = tuple(cfg["P1"])
    S = c.spectral_density().cpu().numpy().astype(np.float64)
    mu = c.degree_of_coherence(*P1).cpu().numpy().astype(np.complex128)
    pw.pw_csd_check(c.h)
    rows = [P1, (120, 137), (140, 122)]
    Wrows = [c.W[a, b].cpu().numpy().astype(np.complex128) for a, b in rows]
    c.close()
    pts = _sample_points(N, 24)
    m = mask.astype(np.complex128)
    ref = O.propagate_rows_gsm(m, N, dxi, lam, z, cfg["sigma_S"], cfg["sigma_mu"], cfg["A"], rows + pts)
    err_w = max(np.linalg.norm(Wrows[r] - ref[r]) / np.linalg.norm(ref[r]) for r in range(len(rows)))
    S_ref = np.array([ref[len(rows) + k][a, b].real for k, (a, b) in enumerate(pts)])
    S_gpu = np.array([S[a, b] for a, b in pts])
    err_s = np.abs(S_gpu - S_ref).max() / np.abs(S_ref).max()
    S_P1 = ref[0][P1].real
    mu_ref = np.array([ref[0][a, b] / np.sqrt(S_P1 * S_ref[k]) for k, (a, b) in enumerate(pts)])
    mu_gpu = np.array([mu[a, b] for a, b in pts])
    err_mu = np.abs(mu_gpu - mu_ref).max()
    return err_w, err_s, err_mu


def test_phase_screen_n256_tensor_core_stage():
    import paper_2203_02734_gb300 as pw
    fp32 = _errors_vs_oracle(pw.PW_DFT_FP32)
    tc = _errors_vs_oracle(pw.PW_DFT_TC_BF16X3)
    print("\nN=256 phase screen, FP64 errors  W rows (rel L2)  S (rel max)  mu (abs max)\n"
          "  FP32 codelets              %.3e  %.3e  %.3e\n"
          "  split-BF16x3 tensor cores  %.3e  %.3e  %.3e" % (fp32 + tc))
    for e in (fp32, tc):
        assert e[0] < 1e-5 and e[1] < 1e-5 and e[2] < 1e-5, e


def test_dft_mode_arguments():
    import torch
    import paper_2203_02734_gb300 as pw
    c = pw.CSD(256, 20e-6, 633e-9)
    with pytest.raises(pw.PwError, match="PW_EINVAL"):
        pw.pw_csd_set_dft_mode(c.h, 7)
    pw.pw_csd_set_dft_mode(c.h, pw.PW_DFT_TC_BF16X3)
    d = torch.ones((256, 256), dtype=torch.float32, device="cuda")
    pw.pw_source_diagonal(c.h, d.data_ptr(), 1.0)
    with pytest.raises(pw.PwError, match="PW_EUNSUPPORTED"):
        pw.pw_propagate_fresnel(c.h, 0.5)
    c.close()
    # N = 300 (dense path, above the tensor-core limit): buffers that are never touched
    nb = pw.pw_csda_bytes(300)
    h = pw.pw_csd_create(300, 20e-6, 633e-9, 1 << 40, nb, (1 << 40) + nb, nb)
    with pytest.raises(pw.PwError, match="PW_EUNSUPPORTED"):
        pw.pw_csd_set_dft_mode(h, pw.PW_DFT_TC_BF16X3)
    assert pw.pw_csd_get_dft_mode(h) == pw.PW_DFT_AUTO
    pw.pw_csd_destroy(h)


def test_n256_adjoint_dot_product_identity():
    """The adjoint at N = 256 (three-pass engine, the general non-Hermitian adjoint of a loss on S and
    mu): for the linear loss L(W_B) = Re <2 Y, W_B> with Y the adjoint source of gradients (gS, gmu)
    (reading R22), dL/dW0 = 2 P^H(Y), so Re <dL/dW0, W0> must equal Re <2 Y, P(W0)> -- the left side
    from the gradient the call writes over the whole N^4 array, the right side from S and the P1 row
    of the forward propagation (FP64 sums on both sides)."""
    import torch
    import paper_2203_02734_gb300 as pw
    cfg = WL.PHASE_SCREEN_N256
    N, dxi, lam, z = cfg["N"], cfg["dxi"], cfg["lam"], cfg["z"]
    P1 = tuple(cfg["P1"])
    mask = WL.to_c64(WL.phase_screen(N, seed=WL.SEED, corr_px=cfg["corr_px"]))
    c = pw.CSD(N, dxi, lam)
    mt = torch.from_numpy(mask).cuda()
    c.source_gsm(cfg["sigma_S"], cfg["sigma_mu"], cfg["A"])
    c.source_mask(mt)
    c.propagate_fresnel(z)
    S = c.spectral_density()
    mu = c.degree_of_coherence(*P1)
    row = c.W[P1[0], P1[1]].clone()
    torch.cuda.synchronize()
    # positive dL/dS (no cancellation in the reference sum), and a random dL/dmu on S >= 1e-4 max S
    # scaled so that the mu terms are about 1 % of the total: the mu part of a linear loss cancels
    # between the P1 row and the diagonal (mu is scale-free), so a wrong row adjoint shows at that level
    Sh0 = S.cpu().numpy().astype(np.float64)
    gS_h = 0.5 + 0.5 * WL.uniform01(71, N * N).reshape(N, N)
    u = WL.uniform01(72, 2 * N * N).reshape(2, N, N) - 0.5
    region = Sh0 >= 1e-4 * Sh0.max()
    scale = 0.01 * np.sum(gS_h * Sh0) / max(float(np.sum(np.abs(mu.cpu().numpy())[region])), 1e-30)
    gS = torch.tensor(gS_h, dtype=torch.float32, device="cuda")
    gmu = torch.tensor(np.where(region, scale * (u[0] + 1j * u[1]), 0.0), dtype=torch.complex64, device="cuda")
    adj = pw.pw_adjoint()
    adj.dev_dS, adj.dev_dmu, adj.iP, adj.jP = gS.data_ptr(), gmu.data_ptr(), P1[0], P1[1]
    adj.dev_S, adj.dev_mu, adj.grad_W0 = S.data_ptr(), mu.data_ptr(), 1
    pw.pw_propagate_fresnel_adjoint(c.h, z, adj)
    pw.pw_csd_check(c.h)
    # left: Re <g, W0> with W0 = A conj(m(x1)) g(a,c) g(b,d) m(x2) generated slice block by slice block
    x, _ = O.axis_coords(N, dxi)
    gax = np.exp(-(x[:, None] ** 2 + x[None, :] ** 2) / (4 * cfg["sigma_S"] ** 2)
                 - (x[:, None] - x[None, :]) ** 2 / (2 * cfg["sigma_mu"] ** 2))
    gt = torch.tensor(gax, dtype=torch.float64, device="cuda")
    m64 = torch.tensor(mask.astype(np.complex128), device="cuda")
    left = 0.0
    for a in range(N):
        # W0[a, b, c, d] = A conj(m[a, b]) g[a, c] g[b, d] m[c, d]
        blk = (cfg["A"] * torch.conj(m64[a])[:, None, None] * gt[a][None, :, None] * gt[:, None, :]) * m64[None]
        left += float(torch.sum(torch.conj(c.W[a].cdouble()) * blk).real)
    c.close()
    # right: Re <2 Y, W_B> from S and the P1 row, Y built from the same FP32 S and mu (R22)
    Sh = S.cpu().numpy().astype(np.float64)
    muh = mu.cpu().numpy().astype(np.complex128)
    rowh = row.cpu().numpy().astype(np.complex128)
    gSh = gS.cpu().numpy().astype(np.float64)
    gmuh = gmu.cpu().numpy().astype(np.complex128)
    sp = Sh[P1]
    ok = sp * Sh > 0
    D = np.sqrt(np.where(ok, sp * Sh, 1.0))
    r = np.where(ok, np.real(np.conj(gmuh) * muh), 0.0)
    dS = gSh - np.where(ok & (Sh > 0), r / (2 * np.where(Sh > 0, Sh, 1.0)), 0.0)
    dS[P1] -= r.sum() / (2 * sp)
    gw = np.where(ok, gmuh / D, 0.0)
    right = float(np.sum(dS * Sh) + np.real(np.sum(np.conj(gw) * rowh)))
    from gpu_cases import record
    e = abs(left - right) / abs(right)
    record("n256_adjoint_dot", left=left, right=right, rel=e)
    assert e < 1e-5, (left, right, e)


def test_n256_diagonal_far_field():
    """Delta-correlated source W0 = w d(xi1) delta(xi1 - xi2) generated in-kernel, far field z = 2 m:
    12 output rows (corners and edges included) against the oracle's collapsed row sum, and the
    whole S against its closed form S(X) = s w sum_xi d(xi) (the phases cancel on the diagonal)."""
    import torch
    import paper_2203_02734_gb300 as pw
    N, dxi, lam, z, w = 256, 20e-6, 633e-9, 2.0, 0.5
    d = (0.2 + WL.uniform01(31, N * N).reshape(N, N)).astype(np.float32)
    c = pw.CSD(N, dxi, lam)
    dd = torch.from_numpy(d).cuda()
    pw.pw_source_diagonal(c.h, dd.data_ptr(), w)
    c.propagate_farfield(z)
    S = c.spectral_density().cpu().numpy().astype(np.float64)
    rows = [(0, 0), (0, 255), (255, 0), (255, 255), (128, 128), (1, 64), (64, 200), (127, 129), (200, 37),
            (250, 3), (90, 140), (160, 160)]
    Wrows = [c.W[a, b].cpu().numpy().astype(np.complex128) for a, b in rows]
    pw.pw_csd_check(c.h)
    c.close()
    ref = O.propagate_rows_diagonal(d.astype(np.float64), w, N, dxi, lam, z, rows, farfield=True)
    errs = [np.linalg.norm(Wrows[r] - ref[r]) / np.linalg.norm(ref[r]) for r in range(len(rows))]
    assert max(errs) < 1e-5, errs
    S_ref = O.propagation_scale(dxi, lam, z) * w * d.astype(np.float64).sum()
    assert np.linalg.norm(S - S_ref) / (S_ref * N) < 1e-5
