// grad.cuh -- parameter gradients of a loss through the propagation, from the adjoint.
//
// For W_B = P(W0) and a real loss L, the conjugate-Wirtinger gradient W0bar = dL/dW0* equals
// P^H(dL/dW_B*), and P^H of a Fresnel propagation over z from sampling d is the conjugate of a
// Fresnel propagation over the same z of the conjugated array, started from the output sampling
// dx = lambda z/(N d) and scaled by (d/dx)^4 (the factorisation P = s D_out F D_in with
// F^H = conj F).  The caller runs that forward propagation; its result R on the source grid gives
// conj(W0bar) = c R (c = (d/dx)^4, times q(xi1) q*(xi2) for a far-field forward P).  This kernel
// then forms, for the amplitude-masked GSM source W0 = A a(xi1) a(xi2) G(xi1, xi2) (Sec. 5.4),
//   dL/dtheta = 2 Re sum conj(W0bar) dW0/dtheta   (theta = sigma_S, sigma_mu, A, a(eta)),
// reading R once; W0 and dW0/dtheta are generated in registers.
#pragma once
#include "propagate.cuh"

namespace pw {

struct GradArgs {
  int N;
  double d;           // source sampling
  double sigma_S, sigma_mu, A;
  const float* amask; // N x N amplitude mask or nullptr (a = 1)
  const float2* R;    // N^4 result of the adjoint propagation
  double c;           // (d/dx)^4
  int farfield;
  double Kq;          // far field: q(xi) = exp(2 pi i Kq n^2) per axis, Kq = d^2/(2 lambda z)
  double* part;       // N^2 x 3 per-row partial sums (scratch)
  float* gtab;        // N x N GSM axis factor G(i, k) (scratch, filled by gsm_gradient_tables)
  float2* qtab;       // N far-field factors q(x_i) (scratch)
  double* g3;         // [dL/dsigma_S, dL/dsigma_mu, dL/dA]
  float* gmask;       // N x N dL/da or nullptr
};

// The GSM axis factor G(i, k) = exp(-(x_i^2 + x_k^2)/(4 sigma_S^2) - (x_i - x_k)^2/(2 sigma_mu^2))
// (the same table serves both axes: y_j = -x_j) and the far-field factors, in FP64, once.
__global__ void gsm_gradient_tables(GradArgs g) {
  const int N = g.N, M = N / 2;
  const double d = g.d;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < N * N; idx += gridDim.x * blockDim.x) {
    const int i = idx / N, k = idx - i * N;
    const double xi = (i - M) * d, xk = (k - M) * d;
    if (g.sigma_S > 0.0)
      g.gtab[idx] = (float)exp(-(xi * xi + xk * xk) / (4 * g.sigma_S * g.sigma_S) -
                               (xi - xk) * (xi - xk) / (2 * g.sigma_mu * g.sigma_mu));
    if (idx < N) {
      const double n2 = (double)(idx - M) * (idx - M);
      g.qtab[idx] = cis_turns(frac_turns(n2 * g.Kq));
    }
  }
}

// One CTA per row eta = (ea, eb) of R; R is Hermitian, so the column sums of the mask gradient
// equal the row sums and dL/da(eta) = 4 Re sum_xi2 conj(W0bar)(eta, xi2) A a(xi2) G(eta, xi2).
// The row is read as pairs of adjacent elements (16-byte loads, N even), two pairs in flight per
// thread, with the pair's (c, e) advanced incrementally; the row's three parameter sums go to
// g.part (reduced by gsm_gradient_reduce).  FF: far-field forward propagation.
template <bool FF>
__global__ void __launch_bounds__(256) gsm_gradient_kernel(GradArgs g) {
  extern __shared__ double gsm_sh[];
  const int N = g.N, M = N / 2;
  const int eta = blockIdx.x;
  const int ea = eta / N, eb = eta - ea * N;
  float* gx = reinterpret_cast<float*>(gsm_sh);  // G along the first axis for row ea
  float* gy = gx + N;                            // G along the second axis for row eb
  float2* qx = reinterpret_cast<float2*>(gy + N);  // far field: q(x_c) conj factors
  double* red = reinterpret_cast<double*>(qx + 2 * N);
  const double d = g.d;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    gx[i] = g.gtab[ea * N + i];  // G along the first axis for row ea
    gy[i] = g.gtab[eb * N + i];  // G along the second axis for row eb (y_j = -x_j)
    if (FF) qx[i] = g.qtab[i];
  }
  __syncthreads();
  // conj(W0bar)(eta, xi2) = c R q(eta) q*(xi2) in the far field (q of both axes)
  float2 qe = make_float2(1.f, 0.f);
  if (FF) qe = cmul(qx[ea], qx[eb]);
  const float* amask = g.amask;
  const float ae = amask ? amask[eta] : 1.f;
  const float d2 = (float)(d * d);
  const float r2e = (float)((ea - M) * (ea - M) + (M - eb) * (M - eb));  // in units of d^2
  // per-thread partial sums in FP32 (each thread adds N^2 / blockDim terms), reduced in FP64
  float sS = 0.f, sM = 0.f, sA = 0.f;
  const float4* Rrow = reinterpret_cast<const float4*>(g.R + (size_t)eta * N * N);
  const int NP = N * N / 2, step = blockDim.x;
  auto term = [&](float2 r, int c, int e, float ax) {
    if (FF) r = cmul(r, cmul(qe, cconj(cmul(qx[c], qx[e]))));
    const float tG = r.x * ax * gx[c] * gy[e];  // dW0/dtheta is real: only Re(conj(W0bar)) enters
    const float r2x = (float)((c - M) * (c - M) + (M - e) * (M - e));
    const float dx2 = (float)((ea - c) * (ea - c) + (eb - e) * (eb - e));
    sS = fmaf(tG, r2e + r2x, sS);
    sM = fmaf(tG, dx2, sM);
    sA += tG;
  };
  // element x = 2 p of the pair: (c, e) = (x / N, x mod N), e even (N even)
  const int dc = (2 * step) / N, de = (2 * step) - dc * N;
  int c = (2 * threadIdx.x) / N, e = 2 * threadIdx.x - c * N;
#pragma unroll 2
  for (int p = threadIdx.x; p < NP; p += step) {
    const float4 rr = __ldg(Rrow + p);
    const int x = 2 * p;
    float2 am = make_float2(1.f, 1.f);
    if (amask) am = make_float2(__ldg(amask + x), __ldg(amask + x + 1));  // 4-byte alignment only
    term(make_float2(rr.x, rr.y), c, e, am.x);
    term(make_float2(rr.z, rr.w), c, e + 1, am.y);
    e += de;
    c += dc;
    if (e >= N) {
      e -= N;
      ++c;
    }
  }
  // the mask-gradient sum is A * sA; the others scale with w0 = A a(eta) a(xi2) G
  const float sa = sA;
  sS *= ae * d2;
  sM *= ae * d2;
  sA *= ae;
  // block reduction of the four sums
  double v[4] = {(double)sS, (double)sM, (double)sA, (double)sa};
  for (int k = 0; k < 4; ++k) {
    double x = v[k];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0) red[k * 8 + (threadIdx.x >> 5)] = x;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double x = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) x += red[threadIdx.x * 8 + w];
    // sS, sM carry a(eta) a(xi2) G t (r^2 terms), sA carries a(eta) a(xi2) G t, sa carries a(xi2) G t
    if (threadIdx.x < 3) g.part[(size_t)eta * 3 + threadIdx.x] = x;
    if (threadIdx.x == 3 && g.gmask) g.gmask[eta] = (float)(4.0 * g.c * g.A * x);
  }
}

// g3 from the per-row partial sums: one CTA, FP64, a fixed summation order (deterministic).
__global__ void __launch_bounds__(256) gsm_gradient_reduce(GradArgs g) {
  __shared__ double red[3][8];
  const int rows = g.N * g.N;
  double v[3] = {0.0, 0.0, 0.0};
  for (int r = threadIdx.x; r < rows; r += blockDim.x)
    for (int k = 0; k < 3; ++k) v[k] += g.part[(size_t)r * 3 + k];
  for (int k = 0; k < 3; ++k) {
    double x = v[k];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0) red[k][threadIdx.x >> 5] = x;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double x = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) x += red[threadIdx.x][w];
    const double s3 = g.sigma_S * g.sigma_S * g.sigma_S, m3 = g.sigma_mu * g.sigma_mu * g.sigma_mu;
    const double scale = threadIdx.x == 0 ? g.A / s3 : (threadIdx.x == 1 ? 2.0 * g.A / m3 : 2.0);
    g.g3[threadIdx.x] = g.c * scale * x;
  }
}

// ---- the adjoint source of a loss on S and mu (reading R22), on the output plane -----------------
// Given the real gradients gS = dL/dS and gmu = dL/dRe mu + i dL/dIm mu of mu(P1, .), and S, mu of
// the output plane: with D(x) = sqrt(S(P1) S(x)), r(x) = Re(conj(gmu(x)) mu(x)) (0 where D = 0),
//   dL/dS(y) = gS(y) - r(y) / (2 S(y)) - [y = P1] sum_x r(x) / (2 S(P1)),
//   dL/dW_B* = (1/2) dL/dS(y) on the diagonal (y, y) and (1/2) gmu(x) / D(x) on the row (P1, x).
// The kernel writes the source of the adjoint propagation, the conjugate of that array: d(y) =
// (1/2) dL/dS(y) and cross(x) = conj((1/2) gmu(x) / D(x)).  One CTA (the sum over x is a block
// reduction in FP64, a fixed order).
struct AdjPrepArgs {
  int N, iP, jP;
  const float* gS;     // N x N or nullptr
  const float2* gmu;   // N x N or nullptr
  const float* S;      // N x N (with gmu)
  const float2* mu;    // N x N (with gmu)
  float* d;            // out: N x N
  float2* cross;       // out: N x N
};

__global__ void __launch_bounds__(1024) adjoint_prep_kernel(AdjPrepArgs a) {
  __shared__ double red[32];
  const int NN = a.N * a.N, xp = a.iP * a.N + a.jP;
  const float sp = a.gmu ? a.S[xp] : 0.f;
  double rs = 0.0;
  if (a.gmu) {
    for (int x = threadIdx.x; x < NN; x += blockDim.x) {
      const float sx = a.S[x];
      if (sp * sx > 0.f) {
        const float2 g = a.gmu[x], m = a.mu[x];
        rs += (double)(g.x * m.x + g.y * m.y);
      }
    }
    for (int o = 16; o > 0; o >>= 1) rs += __shfl_down_sync(0xffffffffu, rs, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = rs;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
      red[0] = t;
    }
    __syncthreads();
    rs = red[0];
  }
  for (int x = threadIdx.x; x < NN; x += blockDim.x) {
    float dS = a.gS ? a.gS[x] : 0.f;
    float2 c = make_float2(0.f, 0.f);
    if (a.gmu) {
      const float sx = a.S[x];
      if (sp * sx > 0.f) {
        const float2 g = a.gmu[x], m = a.mu[x];
        if (sx > 0.f) dS -= (g.x * m.x + g.y * m.y) / (2.f * sx);
        const float inv = rsqrtf(sp * sx);
        c = make_float2(0.5f * g.x * inv, -0.5f * g.y * inv);
      }
      if (x == xp && sp > 0.f) dS -= (float)(rs / (2.0 * (double)sp));
    }
    a.d[x] = 0.5f * dS;
    a.cross[x] = c;
  }
}

// dL/dRe W0 + i dL/dIm W0 = 2 W0bar = 2 c conj(R ff) in place over the N^4 array R that the
// adjoint propagation left in W (ff = q(x1) q*(x2) after a far-field forward propagation).
__global__ void w0_gradient_kernel(float2* R, int N, float twoc, const float2* __restrict__ qff) {
  const size_t NN = (size_t)N * N, total = NN * NN;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    float2 r = R[i];
    if (qff) {
      const size_t x1 = i / NN, x2 = i - x1 * NN;
      const int a = (int)(x1 / N), b = (int)(x1 % N), c = (int)(x2 / N), d = (int)(x2 % N);
      r = cmul(r, cmul(cmul(qff[a], qff[b]), cconj(cmul(qff[c], qff[d]))));
    }
    R[i] = make_float2(twoc * r.x, -twoc * r.y);
  }
}


// ---- pass A of an adjoint propagation written directly (N <= 128) ------------------------------
// The adjoint source (AdjSlice) of slice x1 = (a, b) is d(x1) at x2 = x1, plus, for the Hermitian
// part of a mu term, conj(r(x1)) / 2 at x2 = P1, plus the row w_r r(x2) in the slice x1 = P1.  The
// sign -1 2D DFT of pass A maps a point to a plane wave, so with s_ab = A conj F(a, b):
//   V(a, b; c', d') = s_ab [ d(x1) F(a, b) e^{-2 pi i (a c' + b d')/N}
//                            + col(x1) F(P1) e^{-2 pi i (iP c' + jP d')/N} ]
//                     + [x1 = P1] s_P1 w_r sum_{c,d} e^{-2 pi i (c c' + d d')/N} F(c, d) r(c, d).
// adj_row_kernel writes the last term (one 2D DFT, separable: N blocks over c', N threads over d)
// into the P1 slice's own places of V; adj_direct_kernel then writes every element of V in memory
// order (coalesced), adding to those.  Same values as the transform of the same source, in
// exact arithmetic; this replaces pass A's 2D DFT of an almost empty source by one V write.
template <int N>
__global__ void __launch_bounds__(N) adj_row_kernel(PassAArgs p, float2* __restrict__ V) {
  __shared__ float2 u[N];
  __shared__ float2 tw[N];
  const int cq = blockIdx.x, t = threadIdx.x, p1 = p.iP * N + p.jP;
  tw[t] = p.tw[t];
  __syncthreads();
  float2 acc = make_float2(0.f, 0.f);  // sum_c e^{-2 pi i c c' / N} F(c, d) r(c, d), d = t
  for (int c = 0; c < N; ++c)
    acc = cadd(acc, cmul(tw[(c * cq) % N], cmul(__ldg(p.F + c * N + t), __ldg(p.cross + c * N + t))));
  u[t] = acc;
  __syncthreads();
  float2 r = make_float2(0.f, 0.f);  // d' = t
  for (int d = 0; d < N; ++d) r = cadd(r, cmul(tw[(d * t) % N], u[d]));
  const float2 coef = cscale(cconj(__ldg(p.F + p1)), p.A * (p.herm ? 0.5f : 1.f));
  V[v_offset<N>(p1, cq, t)] = cmul(coef, r);
}

template <int N> __host__ __device__ constexpr int adj_nt() { return 4 * N < 512 ? 4 * N : 512; }

template <int N>
__global__ void __launch_bounds__(adj_nt<N>()) adj_direct_kernel(PassAArgs p, float2* __restrict__ V) {
  constexpr int G = vgroup<N>(), ROW = N * G, NT = adj_nt<N>(), SLOTS = ROW / NT, NG = N / G;
  static_assert(G == 4 && ROW % NT == 0, "rows of V split evenly over the block");
  __shared__ float2 tw[N];
  const int t = threadIdx.x;
  for (int i = t; i < N; i += NT) tw[i] = p.tw[i];
  __syncthreads();
  const int p1 = p.iP * N + p.jP;
  const bool rowterm = p.cross != nullptr;         // the P1 slice holds adj_row_kernel's term
  const bool colterm = p.cross != nullptr && p.herm;
  const float2 fp1 = __ldg(p.F + p1);
  // V rows (vrow(c'), d'/G, a) of N G values; block blockIdx.x takes a contiguous range of rows, so
  // that a runs fastest: b d' mod N is fixed for N rows and a c' mod N grows by c' per row.
  constexpr int ROWS = N * NG * N;
  const int per = (ROWS + gridDim.x - 1) / gridDim.x;
  const int r0 = blockIdx.x * per, r1 = min(ROWS, r0 + per);
  if (r0 >= r1) return;
  int a = r0 % N, dg = (r0 / N) % NG, cr = r0 / (N * NG);
  int cq = vrow_inv<N>(cr), ac = (a * cq) % N;
  int bdq[SLOTS], jdq[SLOTS];  // b d' mod N and jP d' mod N of the thread's values in the current (c', d'/G)
  auto set_d = [&]() {
#pragma unroll
    for (int s = 0; s < SLOTS; ++s) {
      const int k = t + NT * s, dq = G * dg + (k % G);
      bdq[s] = ((k / G) * dq) % N;
      jdq[s] = (p.jP * dq) % N;
    }
  };
  set_d();
  int pc = (p.iP * cq) % N;
  for (int rr = r0; rr < r1; ++rr) {
    float2* Vr = V + (size_t)rr * ROW;
#pragma unroll
    for (int s = 0; s < SLOTS; ++s) {
      const int k = t + NT * s, ab = a * N + k / G;
      const float2 fab = __ldg(p.F + ab);
      const float dd = p.diag ? __ldg(p.diag + ab) : 0.f;
      int i1 = ac + bdq[s];
      i1 -= i1 >= N ? N : 0;
      float2 v = cscale(tw[i1], p.A * dd * (fab.x * fab.x + fab.y * fab.y));
      if (colterm) {
        int i2 = pc + jdq[s];
        i2 -= i2 >= N ? N : 0;
        const float2 col = cscale(cconj(__ldg(p.cross + ab)), 0.5f * p.A);
        v = cadd(v, cmul(cmul(cconj(fab), col), cmul(fp1, tw[i2])));
      }
      if (rowterm && ab == p1) v = cadd(v, Vr[k]);
      Vr[k] = v;
    }
    // next row: a + 1, then d'/G + 1, then c'
    ac += cq;
    ac -= ac >= N ? N : 0;
    if (++a == N) {
      a = 0;
      ac = 0;
      if (++dg == NG) {
        dg = 0;
        ++cr;
        if (cr < N) {
          cq = vrow_inv<N>(cr);
          pc = (p.iP * cq) % N;
        }
      }
      set_d();
    }
  }
}

}  // namespace pw
