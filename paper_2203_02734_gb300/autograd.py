"""torch.autograd bridge: S and mu(P1, .) at distance z of a source, with the hand-written adjoint
of include/pywolf_gb.h (pw_propagate_fresnel_adjoint / pw_propagate_farfield_adjoint) as the
backward.  Forward and backward both run in the library's kernels; torch supplies the buffers and
the loss arithmetic the caller writes on S and mu.

Two sources:
  GSMPropagation: the amplitude-masked GSM source W0 = A a(xi1) a(xi2) G(xi1, xi2; sigma_S, sigma_mu),
    differentiable in sigma_S, sigma_mu, A and the real N x N mask a (GSMIntensity: S only);
  CSDPropagation: an uploaded CSDA W0 (N^4 complex64 tensor), differentiable in W0 itself.
Complex gradients follow torch's convention, dL/dRe + i dL/dIm."""
import torch

from . import abi
from .csd import CSD


def _ptr(t):
    return 0 if t is None else t.data_ptr()


class _Model:
    """The handle, its two N^4 device buffers and the output buffers, reused by every call."""

    def __init__(self, N, dxi, lam, z, P1, farfield, device):
        self.N, self.dxi, self.lam, self.z, self.farfield = N, float(dxi), float(lam), float(z), bool(farfield)
        self.P1 = (N // 2, N // 2) if P1 is None else (int(P1[0]), int(P1[1]))
        self.dx = self.lam * self.z / (N * self.dxi)
        self.csd = CSD(N, self.dxi, self.lam, device=device)
        dev = self.csd.W.device
        self.S = torch.empty((N, N), dtype=torch.float32, device=dev)
        self.mu = torch.empty((N, N), dtype=torch.complex64, device=dev)
        self.g3 = torch.zeros(3, dtype=torch.float64, device=dev)
        self.gmask = torch.empty((N, N), dtype=torch.float32, device=dev)

    def propagate_and_read(self):
        h = self.csd.h
        (abi.pw_propagate_farfield if self.farfield else abi.pw_propagate_fresnel)(h, self.z)
        abi.pw_spectral_density(h, self.S.data_ptr())
        abi.pw_degree_of_coherence(h, self.P1[0], self.P1[1], self.mu.data_ptr())

    def adjoint(self, gS, gmu, S, mu, **kw):
        """One adjoint call from the output plane; gS / gmu are torch's upstream gradients or None."""
        h = self.csd.h
        adj = abi.pw_adjoint()
        keep = []
        if gS is not None:
            gS = gS.detach().to(torch.float32).contiguous()
            keep.append(gS)
            adj.dev_dS = gS.data_ptr()
        if gmu is not None:
            gmu = gmu.detach().to(torch.complex64).contiguous()
            keep.append(gmu)
            adj.dev_dmu = gmu.data_ptr()
            adj.dev_S, adj.dev_mu = S.data_ptr(), mu.data_ptr()
        adj.iP, adj.jP = self.P1
        for k, v in kw.items():
            setattr(adj, k, v)
        abi.pw_csd_reset(h, self.dx)  # the output plane's sampling
        (abi.pw_propagate_farfield_adjoint if self.farfield else abi.pw_propagate_fresnel_adjoint)(h, self.z, adj)
        return keep

    def close(self):
        self.csd.close()


class GSMPropagation:
    """(S, mu(P1, .)) at distance z (Fresnel, or far field) of W0 = A a(xi1) a(xi2) G(xi1, xi2;
    sigma_S, sigma_mu), differentiable in sigma_S, sigma_mu, A and the amplitude mask a (N x N,
    real).  One instance owns the two N^4 device buffers and the handle, reused by every call."""

    def __init__(self, N, dxi, lam, z, P1=None, farfield=False, device=None):
        self.m = _Model(N, dxi, lam, z, P1, farfield, device)
        self.mask_c = torch.zeros((N, N), dtype=torch.complex64, device=self.m.csd.W.device)

    def __call__(self, sigma_S, sigma_mu, A, amask):
        return _GSMFn.apply(sigma_S, sigma_mu, A, amask, self)

    def close(self):
        self.m.close()


class GSMIntensity(GSMPropagation):
    """S alone of GSMPropagation (a loss on S only)."""

    def __init__(self, N, dxi, lam, z, farfield=False, device=None):
        super().__init__(N, dxi, lam, z, P1=None, farfield=farfield, device=device)

    def __call__(self, sigma_S, sigma_mu, A, amask):
        return _GSMFn.apply(sigma_S, sigma_mu, A, amask, self)[0]


class _GSMFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, sigma_S, sigma_mu, A, amask, model):
        m = model.m
        h = m.csd.h
        am = amask.detach().to(torch.float32).contiguous()
        model.mask_c.real.copy_(am)  # the amplitude mask as a complex mask (argument marshalling)
        abi.pw_csd_reset(h, m.dxi)
        abi.pw_source_gsm(h, float(sigma_S), float(sigma_mu), float(A))
        abi.pw_source_mask(h, model.mask_c.data_ptr())
        m.propagate_and_read()
        S, mu = m.S.clone(), m.mu.clone()
        ctx.model = model
        ctx.params = (float(sigma_S), float(sigma_mu), float(A))
        ctx.like = [(x.device, x.dtype) if torch.is_tensor(x) else None for x in (sigma_S, sigma_mu, A)]
        ctx.save_for_backward(am, S, mu)
        ctx.set_materialize_grads(False)  # an unused output (mu of an S-only loss) gets no adjoint term
        return S, mu

    @staticmethod
    def backward(ctx, gS, gmu):
        m = ctx.model.m
        am, S, mu = ctx.saved_tensors
        if gS is None and gmu is None:
            return None, None, None, None, None
        sS, sM, A = ctx.params
        keep = m.adjoint(gS, gmu, S, mu, sigma_S_m=sS, sigma_mu_m=sM, amplitude=A, dev_amask=am.data_ptr(),
                         dev_grad3=m.g3.data_ptr(), dev_grad_amask=m.gmask.data_ptr())
        g = m.g3.clone()
        del keep
        out = [None if lk is None else g[k].to(device=lk[0], dtype=lk[1]) for k, lk in enumerate(ctx.like)]
        return out[0], out[1], out[2], m.gmask.clone().to(dtype=am.dtype), None


class CSDPropagation:
    """(S, mu(P1, .)) at distance z (Fresnel, or far field) of an uploaded CSDA W0 (N^4 complex64
    CUDA tensor), differentiable in W0.  hermitian: W0 is Hermitian (every CSD is, Sec. 3.3), which
    lets the forward store its output rows contiguously; the gradient is the one of a general
    complex W0 either way."""

    def __init__(self, N, dxi, lam, z, P1=None, farfield=False, hermitian=True, device=None):
        self.m = _Model(N, dxi, lam, z, P1, farfield, device)
        self.hermitian = bool(hermitian)

    def __call__(self, W0):
        return _CSDFn.apply(W0, self)

    def close(self):
        self.m.close()


class _CSDFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, W0, model):
        m = model.m
        h = m.csd.h
        W0c = W0.detach().to(torch.complex64).contiguous()
        abi.pw_csd_reset(h, m.dxi)
        abi.pw_source_array(h, W0c.data_ptr(), 1 if model.hermitian else 0)
        m.propagate_and_read()
        S, mu = m.S.clone(), m.mu.clone()
        ctx.model = model
        ctx.save_for_backward(S, mu)
        ctx.set_materialize_grads(False)
        return S, mu

    @staticmethod
    def backward(ctx, gS, gmu):
        m = ctx.model.m
        S, mu = ctx.saved_tensors
        if gS is None and gmu is None:
            return None, None
        keep = m.adjoint(gS, gmu, S, mu, grad_W0=1)
        g = m.csd.W.clone()
        del keep
        return g, None
