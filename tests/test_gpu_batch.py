"""Batched runs on the GPU, in both execution modes (one persistent launch over all instances;
the instances one after the other on the single-instance kernels): parity with the FP64 oracle,
repeatability, CUDA-graph replay, the autotuner, and the bounded dependency wait of the
persistent launch (a stalled instance yields PW_ETIMEOUT while the others complete)."""
import numpy as np
import pytest

import oracle as O
import workloads as WL
from gpu_cases import oracle_run, rel, source_mask

pytestmark = pytest.mark.gpu

DXI, LAM = 20e-6, 633e-9
TOL = 1e-5


def _mask(N, seed):
    u = WL.uniform01(seed, 2 * N * N).reshape(2, N, N)
    return (0.6 + 0.4 * u[0]) * np.exp(2j * np.pi * u[1])


SPECS = [  # (N, z, farfield, lam, aperture, lens, with mask, full W)
    (16, 0.4, 0, 633e-9, 0.12e-3, 0.25, True, True),
    (32, 0.6, 1, 550e-9, 0.0, 0.0, False, False),
    (64, 0.5, 0, 700e-9, 0.5e-3, 0.0, True, True),
    (32, 1.5, 0, 600e-9, 0.3e-3, 0.4, False, True),
]


def _setup(torch, pw, stream=None, pool=2):
    insts, bufs, srcs = [], [], []
    for k, (N, z, ff, lam, ap, lf, use_mask, full) in enumerate(SPECS):
        m = WL.to_c64(_mask(N, 40 + k)) if use_mask else None
        mt = torch.from_numpy(m).cuda() if use_mask else None
        W = torch.empty((N,) * 4, dtype=torch.complex64, device="cuda") if full else None
        S = torch.empty((N, N), dtype=torch.float32, device="cuda")
        mu = torch.empty((N, N), dtype=torch.complex64, device="cuda")
        P1 = (N // 2 - 1, N // 2 + 1)
        bufs.append((mt, W, S, mu))
        insts.append(pw.pw_instance(N, DXI, lam, z, ff, 0.1e-3, 0.05e-3, 1.0 + 0.1 * k, ap, lf,
                                    mt.data_ptr() if use_mask else None, P1[0], P1[1],
                                    W.data_ptr() if full else None, S.data_ptr(), mu.data_ptr()))
        srcs.append(dict(N=N, z=z, ff=ff, lam=lam, ap=ap, lf=lf, mask=m, A=1.0 + 0.1 * k, P1=P1, full=full))
    nb = pw.pw_batch_workspace_bytes(insts, pool)
    ws = torch.full((nb,), 0xAB, dtype=torch.uint8, device="cuda")  # stale bytes must not matter
    s = stream.cuda_stream if stream is not None else torch.cuda.current_stream().cuda_stream
    b = pw.pw_batch_create(insts, pool, ws.data_ptr(), nb, s)
    return b, bufs, srcs, ws


def _oracle(src):
    N = src["N"]
    kind = "farfield" if src["ff"] else "fresnel"
    W, _ = oracle_run(N, DXI, src["lam"], [(kind, src["z"])], gsm=(0.1e-3, 0.05e-3, src["A"]),
                      aperture=src["ap"] or None, lens_f=src["lf"] or None, mask=src["mask"])
    return W


def _check(bufs, srcs):
    errs = []
    for (mt, W, S, mu), src in zip(bufs, srcs):
        ref = _oracle(src)
        Sref = np.real(O.spectral_density(ref))
        muref = O.degree_of_coherence(ref, *src["P1"])
        eS = rel(S.cpu().numpy(), Sref)
        sel = Sref >= 1e-4 * Sref.max()
        emu = rel(mu.cpu().numpy()[sel], muref[sel])
        eW = rel(W.cpu().numpy(), ref) if W is not None else 0.0
        errs.append((eW, eS, emu))
        assert eS < TOL and emu < TOL and eW < TOL, (src["N"], eW, eS, emu)
    return errs


@pytest.mark.parametrize("mode", ["persistent", "sequenced"])
def test_batch_matches_oracle_and_repeats(mode):
    import torch
    import paper_2203_02734_gb300 as pw
    b, bufs, srcs, ws = _setup(torch, pw)
    pw.pw_batch_set_mode(b, pw.PW_BATCH_PERSISTENT if mode == "persistent" else pw.PW_BATCH_SEQUENCED)
    pw.pw_batch_run(b)
    pw.pw_batch_check(b)
    _check(bufs, srcs)
    first = [S.clone() for (_, _, S, _) in bufs]
    pw.pw_batch_run(b)
    pw.pw_batch_check(b)
    for f, (_, _, S, _) in zip(first, bufs):
        assert torch.equal(f, S)
    pw.pw_batch_destroy(b)


def test_batch_graph_replay_and_autotune():
    import torch
    import paper_2203_02734_gb300 as pw
    s = torch.cuda.Stream()
    b, bufs, srcs, ws = _setup(torch, pw, stream=s)
    chunk = pw.pw_batch_autotune(b)
    assert chunk in (4, 8, 16, 32, 64) and pw.pw_batch_get_chunk(b) == chunk
    assert pw.pw_batch_get_mode(b) in (pw.PW_BATCH_PERSISTENT, pw.PW_BATCH_SEQUENCED)
    with torch.cuda.stream(s):
        pw.pw_batch_run(b)
    s.synchronize()
    for (_, _, S, _) in bufs:
        S.zero_()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        pw.pw_batch_run(b)
    g.replay()
    torch.cuda.synchronize()
    pw.pw_batch_check(b)
    _check(bufs, srcs)
    pw.pw_batch_destroy(b)


def test_batch_stalled_instance_times_out():
    """Failure detection without a device fault: instance 1's pass-A work is left out on the host,
    its pass-B work gives up after the bounded wait, the run reports PW_ETIMEOUT, and the other
    instances are still correct."""
    import torch
    import paper_2203_02734_gb300 as pw
    # a pool slot per instance: no other instance waits on the stalled one's buffer
    b, bufs, srcs, ws = _setup(torch, pw, pool=len(SPECS))
    pw.pw_batch_set_mode(b, pw.PW_BATCH_PERSISTENT)  # the bounded waits belong to the persistent launch
    pw.pw_batch_inject_stall(b, 1, 0.2)
    pw.pw_batch_run(b)
    with pytest.raises(pw.PwError, match="PW_ETIMEOUT"):
        pw.pw_batch_check(b)
    pw.pw_batch_check(b)  # cleared
    ok = [0, 2, 3]
    _check([bufs[i] for i in ok], [srcs[i] for i in ok])
    pw.pw_batch_destroy(b)


def test_batch_rejects_bad_instances():
    import torch
    import paper_2203_02734_gb300 as pw
    S = torch.empty((48, 48), dtype=torch.float32, device="cuda")
    inst = [pw.pw_instance(48, DXI, LAM, 0.5, 0, 1e-4, 5e-5, 1.0, 0.0, 0.0, None, 0, 0, None, S.data_ptr(), None)]
    ws = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    with pytest.raises(pw.PwError, match="PW_EUNSUPPORTED"):
        pw.pw_batch_create(inst, 1, ws.data_ptr(), ws.numel())
    S16 = torch.empty((16, 16), dtype=torch.float32, device="cuda")
    ok = [pw.pw_instance(16, DXI, LAM, 0.5, 0, 1e-4, 5e-5, 1.0, 0.0, 0.0, None, 0, 0, None, S16.data_ptr(), None)]
    nb = pw.pw_batch_workspace_bytes(ok, 1)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    b = pw.pw_batch_create(ok, 1, ws.data_ptr(), nb)
    assert pw.pw_batch_get_mode(b) == pw.PW_BATCH_PERSISTENT  # small instances: the default
    with pytest.raises(pw.PwError, match="PW_EINVAL"):
        pw.pw_batch_set_mode(b, 7)
    pw.pw_batch_destroy(b)


@pytest.mark.parametrize("mode", ["persistent", "sequenced"])
def test_batch_mixes_register_engine_n128(mode):
    """An N = 128 instance (register-resident engine: TMA-stored slices, gathered columns) in the
    same launch as an N = 64 one, run twice.  The N = 128 GSM source behind a thin lens is
    separable, so the oracle's per-axis quadrature gives its exact propagated CSDA."""
    import torch
    import paper_2203_02734_gb300 as pw
    N1, z1, lam1, lf1, A1 = 128, 0.5, 600e-9, 0.4, 1.2
    N2, z2, lam2 = 64, 0.7, 650e-9
    W1 = torch.empty((N1,) * 4, dtype=torch.complex64, device="cuda")
    S1 = torch.empty((N1, N1), dtype=torch.float32, device="cuda")
    mu1 = torch.empty((N1, N1), dtype=torch.complex64, device="cuda")
    m2 = WL.to_c64(_mask(N2, 77))
    m2t = torch.from_numpy(m2).cuda()
    S2 = torch.empty((N2, N2), dtype=torch.float32, device="cuda")
    mu2 = torch.empty((N2, N2), dtype=torch.complex64, device="cuda")
    P1 = (N1 // 2, N1 // 2 - 3)
    N3, z3, lam3, lf3 = 96, 0.8, 620e-9, 0.5  # register-resident N = 96 engine, S and mu only
    S3 = torch.empty((N3, N3), dtype=torch.float32, device="cuda")
    mu3 = torch.empty((N3, N3), dtype=torch.complex64, device="cuda")
    P3 = (47, 50)
    insts = [pw.pw_instance(N1, DXI, lam1, z1, 0, 0.1e-3, 0.05e-3, A1, 0.0, lf1, None, P1[0], P1[1],
                            W1.data_ptr(), S1.data_ptr(), mu1.data_ptr()),
             pw.pw_instance(N2, DXI, lam2, z2, 0, 0.1e-3, 0.05e-3, 1.0, 0.45e-3, 0.0, m2t.data_ptr(), 30, 33,
                            None, S2.data_ptr(), mu2.data_ptr()),
             pw.pw_instance(N3, DXI, lam3, z3, 0, 0.1e-3, 0.05e-3, 0.9, 0.0, lf3, None, P3[0], P3[1],
                            None, S3.data_ptr(), mu3.data_ptr())]
    nb = pw.pw_batch_workspace_bytes(insts, 2)
    ws = torch.full((nb,), 0xAB, dtype=torch.uint8, device="cuda")
    b = pw.pw_batch_create(insts, 2, ws.data_ptr(), nb, torch.cuda.current_stream().cuda_stream)
    assert pw.pw_batch_get_mode(b) == pw.PW_BATCH_SEQUENCED  # every N >= 64: the default
    pw.pw_batch_set_mode(b, pw.PW_BATCH_PERSISTENT if mode == "persistent" else pw.PW_BATCH_SEQUENCED)
    for rep in range(2):
        S1.zero_()
        pw.pw_batch_run(b)
        pw.pw_batch_check(b)
        torch.cuda.synchronize()
        ref = O.gsm_separable_quadrature(N1, DXI, lam1, z1, 0.1e-3, 0.05e-3, A1, lens_f=lf1)
        for (a, c) in [P1, (60, 70), (70, 58)]:
            assert rel(W1[a, c].cpu().numpy(), ref[a, c]) < TOL
        Sref = np.real(np.einsum("abab->ab", ref))
        assert rel(S1.cpu().numpy(), Sref) < TOL
        muref = O.degree_of_coherence(ref, *P1)
        sel = Sref >= 1e-4 * Sref.max()
        assert rel(mu1.cpu().numpy()[sel], muref[sel]) < TOL
        del ref
        ref2 = _oracle(dict(N=N2, z=z2, ff=0, lam=lam2, ap=0.45e-3, lf=0.0, mask=m2, A=1.0))
        S2ref = np.real(O.spectral_density(ref2))
        assert rel(S2.cpu().numpy(), S2ref) < TOL
        ref3 = O.gsm_separable_quadrature(N3, DXI, lam3, z3, 0.1e-3, 0.05e-3, 0.9, lens_f=lf3)
        S3ref = np.real(np.einsum("abab->ab", ref3))
        assert rel(S3.cpu().numpy(), S3ref) < TOL
        mu3ref = O.degree_of_coherence(ref3, *P3)
        sel = S3ref >= 1e-4 * S3ref.max()
        assert rel(mu3.cpu().numpy()[sel], mu3ref[sel]) < TOL
        del ref3
    pw.pw_batch_destroy(b)


def test_spectral_sum_on_common_grid():
    """Polychromatic intensity I = sum_i w_i S_i (Sec. 3.5) over wavelengths placed on one output
    grid (z_i = z0 lambda0 / lambda_i gives the same sampling lambda_i z_i / (N dxi))."""
    import torch
    import paper_2203_02734_gb300 as pw
    N, z0, lam0 = 32, 0.5, 600e-9
    lams = [550e-9, 600e-9, 650e-9, 700e-9]
    wts = [0.4, 1.0, 0.8, 0.3]
    Ss = [torch.empty((N, N), dtype=torch.float32, device="cuda") for _ in lams]
    insts = [pw.pw_instance(N, DXI, lam, z0 * lam0 / lam, 0, 0.1e-3, 0.05e-3, 1.0, 0.25e-3, 0.0, None, 16, 16,
                            None, S.data_ptr(), None) for lam, S in zip(lams, Ss)]
    nb = pw.pw_batch_workspace_bytes(insts, 2)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    b = pw.pw_batch_create(insts, 2, ws.data_ptr(), nb)
    I = torch.empty((N, N), dtype=torch.float32, device="cuda")
    pw.pw_batch_run(b)
    pw.pw_batch_spectral_sum(b, wts, I.data_ptr())
    pw.pw_batch_check(b)
    ref = np.zeros((N, N))
    for lam, w in zip(lams, wts):
        W, _ = oracle_run(N, DXI, lam, [("fresnel", z0 * lam0 / lam)], gsm=(0.1e-3, 0.05e-3, 1.0), aperture=0.25e-3)
        ref += w * np.real(O.spectral_density(W))
    assert rel(I.cpu().numpy(), ref) < TOL
    pw.pw_batch_destroy(b)
    # different output grids: rejected
    bad = [pw.pw_instance(N, DXI, lam, z0, 0, 0.1e-3, 0.05e-3, 1.0, 0.0, 0.0, None, 16, 16, None, S.data_ptr(), None)
           for lam, S in zip(lams[:2], Ss[:2])]
    nb = pw.pw_batch_workspace_bytes(bad, 1)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    b = pw.pw_batch_create(bad, 1, ws.data_ptr(), nb)
    with pytest.raises(pw.PwError, match="no common grid"):
        pw.pw_batch_spectral_sum(b, [1.0, 1.0], I.data_ptr())
    pw.pw_batch_destroy(b)


def test_batch_s_mu_only_pruned_pass():
    """Instances that keep no W take the pruned second pass (two dot products per column instead of
    the DFT over point 1): N = 128 and 96 (register-resident pass A; separable GSM behind a lens,
    exact by the per-axis quadrature), N = 64 with aperture and mask, N = 32 with aperture and mask
    in the far field, N = 16 in the far field, each against the FP64 oracle, sequenced mode, run
    twice.  Every size has its own grid of the S/mu pass (one wave of equal blocks)."""
    import torch
    import paper_2203_02734_gb300 as pw
    cases = [  # (N, z, farfield, lam, aperture, lens, with mask, P1)
        (128, 0.45, 0, 610e-9, 0.0, 0.35, False, (61, 66)),
        (64, 0.3, 0, 580e-9, 0.4e-3, 0.0, True, (30, 35)),
        (16, 0.7, 1, 633e-9, 0.0, 0.0, False, (7, 9)),
        (96, 0.5, 0, 600e-9, 0.0, 0.4, False, (47, 50)),
        (32, 0.6, 1, 620e-9, 0.25e-3, 0.0, True, (15, 17)),
    ]
    insts, outs, keep = [], [], []
    for k, (N, z, ff, lam, ap, lf, use_mask, P1) in enumerate(cases):
        m = WL.to_c64(_mask(N, 90 + k)) if use_mask else None
        mt = torch.from_numpy(m).cuda() if use_mask else None
        S = torch.empty((N, N), dtype=torch.float32, device="cuda")
        mu = torch.empty((N, N), dtype=torch.complex64, device="cuda")
        keep.append(mt)
        outs.append((S, mu, m))
        insts.append(pw.pw_instance(N, DXI, lam, z, ff, 0.1e-3, 0.05e-3, 1.0 + 0.1 * k, ap, lf,
                                    mt.data_ptr() if use_mask else None, P1[0], P1[1], None, S.data_ptr(),
                                    mu.data_ptr()))
    nb = pw.pw_batch_workspace_bytes(insts, 2)
    ws = torch.full((nb,), 0xAB, dtype=torch.uint8, device="cuda")
    b = pw.pw_batch_create(insts, 2, ws.data_ptr(), nb, torch.cuda.current_stream().cuda_stream)
    pw.pw_batch_set_mode(b, pw.PW_BATCH_SEQUENCED)
    for rep in range(2):
        for S, mu, _ in outs:
            S.zero_()
            mu.zero_()
        pw.pw_batch_run(b)
        pw.pw_batch_check(b)
        torch.cuda.synchronize()
        for k, ((N, z, ff, lam, ap, lf, use_mask, P1), (S, mu, m)) in enumerate(zip(cases, outs)):
            if N in (96, 128):
                ref = O.gsm_separable_quadrature(N, DXI, lam, z, 0.1e-3, 0.05e-3, 1.0 + 0.1 * k, lens_f=lf)
            else:
                ref = _oracle(dict(N=N, z=z, ff=ff, lam=lam, ap=ap, lf=lf, mask=m, A=1.0 + 0.1 * k))
            Sref = np.real(np.einsum("abab->ab", ref))
            assert rel(S.cpu().numpy(), Sref) < TOL, (N, rel(S.cpu().numpy(), Sref))
            muref = O.degree_of_coherence(ref, *P1)
            sel = Sref >= 1e-4 * Sref.max()
            assert rel(mu.cpu().numpy()[sel], muref[sel]) < TOL, (N, rel(mu.cpu().numpy()[sel], muref[sel]))
            del ref
    pw.pw_batch_destroy(b)
