// dense.cuh -- the propagation as four dense axis contractions: zero padding with cropped output
// (Sec. 3.2: the FFT runs on a grid of size Nz > N and the result is cropped back to N x N), and
// grid sizes without an FFT plan.
//
// With the source at the centre of the padded grid and the output cropped to the centre, each
// axis of Eq. W_fresnel becomes the pruned centred DFT of size Nz restricted to N inputs and N
// outputs, a dense N x N matrix.  The propagators are separable per axis (|r|^2 = x^2 + y^2, and
// y(j)^2 = x(j)^2 on the centred index), so they fold into the same matrix:
//   E(k, n) = q(X_k) exp(-2 pi i (k - N/2)(n - N/2) / Nz) q(xi_n),
//   q(X_k) = exp(i pi X_k^2 / (lambda z)), X_k = (k - N/2) dx, dx = lambda z / (Nz dxi),
//   q(xi_n) = exp(i pi xi_n^2 / (lambda z)) (1 for the far field, Eq. W_farfield);
// and the propagated CSDA is
//   W_B(a', b', c', d') = s sum conj(E(a', a)) conj(E(b', b)) E(c', c) E(d', d) W0(a, b, c, d),
// point 1 taking the conjugate kernel (h* in Eq. W_general), s = dxi^4 / (lambda z)^2.  The
// phase of E is taken in FP64 with the integer product (k - N/2)(n - N/2) reduced mod Nz exactly.
//
// Passes (W0 built in place first; W and work alternate): contract d with E, then c with E, then
// b with conj(E), then a with s conj(E); the last pass also takes S = Re W_B(x, x).  Each pass is
// C[k][j] = sum_n A(k, n) B[n][j] over the N^3 columns j of the CSDA viewed along the contracted
// axis: B[n][j] sits at (j / L) L N + n L + (j mod L), L = the product of the axes after it.
#pragma once
#include <cstdint>

#include "propagate.cuh"

namespace pw {
namespace dense {

struct TabArgs {
  int N, Nz;
  double Kin;   // turns per n^2 of the input propagator (0 for the far field)
  double Kout;  // turns per k^2 of the output propagator
  float2* E;    // N x N, row k (output), column n (input)
};

// E(k, n) in FP64 turns: Kout (k-M)^2 - ((k-M)(n-M) mod Nz) / Nz + Kin (n-M)^2, M = N/2.
__global__ void tables_kernel(TabArgs t) {
  const int N = t.N, M = N / 2;
  const int NN = N * N;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < NN; idx += gridDim.x * blockDim.x) {
    const int k = idx / N, n = idx - k * N;
    const long long pk = k - M, pn = n - M;
    long long r = (pk * pn) % t.Nz;
    if (r < 0) r += t.Nz;
    const double turns =
        frac_turns((double)(pk * pk) * t.Kout) - (double)r / (double)t.Nz + frac_turns((double)(pn * pn) * t.Kin);
    t.E[idx] = cis_turns(turns);
  }
}

// W0 in place (W may alias the uploaded source): the GSM model, an uploaded CSDA or a diagonal
// source, times conj(m(a, b)) m(c, d) with m = M0 (mask x aperture x lens, 1 without masks).
struct SrcArgs {
  int N, mode;          // mode: SRC_GSM, SRC_ARRAY, SRC_DIAG
  const float* G;       // GSM axis factor (N x N)
  const float2* M0;     // source-plane mask (N x N)
  const float2* W0;     // uploaded CSDA (SRC_ARRAY)
  const float* diag;    // N x N diagonal (SRC_DIAG)
  float A;              // GSM amplitude or diagonal weight
  float2* W;            // output, N^4
};

__global__ void source_kernel(SrcArgs s) {
  const int N = s.N;
  const size_t NN = (size_t)N * N, total = NN * NN;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const size_t ab = idx / NN, cd = idx - ab * NN;
    const int a = (int)(ab / N), b = (int)(ab - (size_t)a * N), c = (int)(cd / N), d = (int)(cd - (size_t)c * N);
    const float2 m1 = cconj(s.M0[ab]), m2 = s.M0[cd];
    float2 v;
    if (s.mode == SRC_GSM) {
      v = cscale(cmul(m1, m2), s.A * s.G[a * N + c] * s.G[b * N + d]);
    } else if (s.mode == SRC_ARRAY) {
      v = cmul(cmul(m1, s.W0[idx]), m2);
    } else {
      v = (a == c && b == d) ? cscale(cmul(m1, m2), s.A * s.diag[ab]) : make_float2(0.f, 0.f);
    }
    s.W[idx] = v;
  }
}

// One axis contraction, C[k][j] = scale sum_n A(k, n) B[n][j], A = E or conj(E), in FP32.
// Tile 64 (k) x 64 (j) per CTA of 256 threads, 16 values of n per step through shared memory
// (two buffers: the next step's values are loaded into registers while the current step
// computes); thread (ty, tx) = (t / 16, t mod 16) accumulates k = k0 + 4 ty + i, j = j0 + 4 tx + jj
// (i, jj < 4), so that 16 threads store 64 consecutive columns of one output row.  The k tiles of
// one column tile are consecutive CTAs, so the column block they all read (N x 64) comes from L2
// after the first.  S_OUT (last pass, L = N^3): S(a', b') = Re C at k = a', j = (b', a', b').
struct AxisArgs {
  int N;
  long long L;      // elements after the contracted axis
  long long ncols;  // N^3
  const float2* E;
  float scale;
  const float2* in;
  float2* out;
  float* S;
  int stall;  // failure-detection test (0 = off): CTA 0 of the tensor-core kernel never copies operand chunk
              // `stall` (> 0), or never announces A tile -stall (< 0)
  // Tensor-core kernel, first contraction (L = 1) of a GSM source: gen != 0 builds the input
  // W0(a, b, c, d) = A conj(M0(a, b)) G(a, c) G(b, d) M0(c, d) in the converters instead of reading
  // `in` (source_kernel is then not run).
  int gen;
  const float* G;
  const float2* M0;
  float A;
};

constexpr int BM = 64, BN = 64, BK = 16, PITCH = 66, NT = 256;

__device__ __forceinline__ long long col_base(long long j, long long L, int N) {
  const long long p = j / L;
  return p * L * N + (j - p * L);
}

template <bool CONJ, bool S_OUT>
__global__ void __launch_bounds__(NT) axis_kernel(AxisArgs p) {
  __shared__ __align__(16) float2 As[2][BK][PITCH];
  __shared__ __align__(16) float2 Bs[2][BK][PITCH];
  const int t = threadIdx.x, ty = t >> 4, tx = t & 15;
  const int N = p.N;
  const long long L = p.L, ncols = p.ncols;
  const int ktiles = (N + BM - 1) / BM;
  const int k0 = (int)(blockIdx.x % ktiles) * BM;
  const long long j0 = (long long)(blockIdx.x / ktiles) * BN;
  // B loads: L > 1 -> column jl = t mod 64 fixed, rows kk = t / 64 + 4 i (contiguous columns);
  //          L = 1 -> row kk = t mod 16 fixed, columns jl = t / 16 + 16 i (contiguous rows).
  const bool rowwise = L == 1;
  long long bbase[4];
  int bk[4], bj[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    bk[i] = rowwise ? (t & 15) : (t >> 6) + 4 * i;
    bj[i] = rowwise ? (t >> 4) + 16 * i : (t & 63);
    const long long j = j0 + bj[i];
    bbase[i] = j < ncols ? col_base(j, L, N) : -1;
  }
  float2 ra[4], rb[4];
  auto load = [&](int n0) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {  // A: 64 x 16, n fastest
      const int e = t + NT * i, kk = e & 15, kl = e >> 4;
      const int k = k0 + kl, n = n0 + kk;
      ra[i] = (k < N && n < N) ? p.E[k * N + n] : make_float2(0.f, 0.f);
      if (CONJ) ra[i].y = -ra[i].y;
      const int nb = n0 + bk[i];
      rb[i] = (bbase[i] >= 0 && nb < N) ? p.in[bbase[i] + (long long)nb * L] : make_float2(0.f, 0.f);
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int e = t + NT * i;
      As[buf][e & 15][e >> 4] = ra[i];
      Bs[buf][bk[i]][bj[i]] = rb[i];
    }
  };
  float2 acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) acc[i][jj] = make_float2(0.f, 0.f);
  load(0);
  store(0);
  __syncthreads();
  for (int n0 = 0, buf = 0; n0 < N; n0 += BK, buf ^= 1) {
    const bool more = n0 + BK < N;
    if (more) load(n0 + BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      const float4 a01 = *reinterpret_cast<const float4*>(&As[buf][kk][4 * ty]);
      const float4 a23 = *reinterpret_cast<const float4*>(&As[buf][kk][4 * ty + 2]);
      const float4 b01 = *reinterpret_cast<const float4*>(&Bs[buf][kk][4 * tx]);
      const float4 b23 = *reinterpret_cast<const float4*>(&Bs[buf][kk][4 * tx + 2]);
      const float2 a[4] = {make_float2(a01.x, a01.y), make_float2(a01.z, a01.w), make_float2(a23.x, a23.y),
                           make_float2(a23.z, a23.w)};
      const float2 b[4] = {make_float2(b01.x, b01.y), make_float2(b01.z, b01.w), make_float2(b23.x, b23.y),
                           make_float2(b23.z, b23.w)};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
          acc[i][jj].x = fmaf(a[i].x, b[jj].x, fmaf(-a[i].y, b[jj].y, acc[i][jj].x));
          acc[i][jj].y = fmaf(a[i].x, b[jj].y, fmaf(a[i].y, b[jj].x, acc[i][jj].y));
        }
    }
    if (more) store(buf ^ 1);  // buffer buf ^ 1 was last read before the previous barrier
    __syncthreads();
  }
  const long long NN = (long long)N * N;
#pragma unroll
  for (int jj = 0; jj < 4; ++jj) {
    const long long j = j0 + 4 * tx + jj;
    if (j >= ncols) continue;
    const long long ob = col_base(j, L, N);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int k = k0 + 4 * ty + i;
      if (k >= N) continue;
      const float2 v = cscale(acc[i][jj], p.scale);
      p.out[ob + (long long)k * L] = v;
      if (S_OUT) {
        const int b = (int)(j / NN), c = (int)((j / N) % N), d = (int)(j % N);
        if (c == k && d == b) p.S[k * N + b] = v.x;
      }
    }
  }
}

}  // namespace dense
}  // namespace pw
