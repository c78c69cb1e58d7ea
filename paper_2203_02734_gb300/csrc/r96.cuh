// r96.cuh -- register-resident 2D DFT of a 96 x 96 slice for the two passes at N = 96.
//
// Per axis 96 = 8 x 3 x 4 along p (first slice index) and 3 x 8 x 4 along q (second), as three
// 2D Stockham stages (the convention of fft.cuh, one radix per axis per stage); 192 threads, 48
// points per thread in every stage:
//   stage 1: radices (8, 3), butterflies (jp < 12, jq < 32), two per thread (jp = warp + 6 i,
//            jq = lane); inputs (jp + 12 kp, jq + 32 kq); outputs (8 jp + kp, 3 jq + kq);
//   stage 2: radices (3, 8), NS = (8, 3), butterflies (jp < 32, jq < 12), two per thread
//            (jp = lane, jq = warp + 6 i); inputs (jp + 32 kp, jq + 12 kq); twiddles
//            w24^(kp (jp mod 8)) w24^(kq (jq mod 3)); outputs (24 (jp/8) + jp mod 8 + 8 kp,
//            24 (jq/3) + jq mod 3 + 3 kq);
//   stage 3: radices (4, 4), NS = (24, 24), butterflies (jp < 24, jq < 24), three per thread
//            (u = t + 192 i: jq = u mod 24, jp = u / 24); inputs (jp + 24 kp, jq + 24 kq);
//            twiddles w96^(kp jp) w96^(kq jq); outputs in natural order at the input positions
// (w_L = exp(SIGN 2 pi i / L)).  Points move between stages through one 96 x 97 shared buffer
// (odd pitch: the stage-2 reads, a lane per row, hit distinct banks).  The block is small (76 KB
// of shared memory, <= 170 registers per thread), so two CTAs share each SM and hide each other's
// memory latency; the corner-turn layout of V is the generic one (runs of 4 columns), so these
// passes pair with the generic engine's.
#pragma once
#include "propagate.cuh"
#include "r128.cuh"

namespace pw {
namespace r96 {

constexpr int N = 96;
constexpr int NT = 192;
constexpr int P = N + 1;  // exchange pitch

// v[kp][kq] *= (p twiddle of stage (RP, NSP) for jp) x (q twiddle of stage (RQ, NSQ) for jq)
template <int RP, int NSP, int RQ, int NSQ, int SIGN>
__device__ __forceinline__ void twiddle2d(float2 (&v)[RP][RQ], int jp, int jq, const float2* tw) {
  if constexpr (NSP > 1) {
    const int k = jp % NSP;
    constexpr int STEP = N / (NSP * RP);
#pragma unroll
    for (int r = 1; r < RP; ++r) {
      float2 w = tw[r * k * STEP];
      if (SIGN > 0) w.y = -w.y;
#pragma unroll
      for (int c = 0; c < RQ; ++c) v[r][c] = cmul(v[r][c], w);
    }
  }
  if constexpr (NSQ > 1) {
    const int k = jq % NSQ;
    constexpr int STEP = N / (NSQ * RQ);
#pragma unroll
    for (int r = 1; r < RQ; ++r) {
      float2 w = tw[r * k * STEP];
      if (SIGN > 0) w.y = -w.y;
#pragma unroll
      for (int c = 0; c < RP; ++c) v[c][r] = cmul(v[c][r], w);
    }
  }
}

// Stages 2 and 3 from the stage-1 inputs v (the thread's two (8, 3) blocks, before their DFT),
// through X.  On return w3[i][kp][kq] holds the transform at (jp3 + 24 kp, jq3 + 24 kq), with
// u = t + 192 i, jq3 = u mod 24, jp3 = u / 24.  Contract: X is free on entry; on return every
// thread has finished reading X (a block barrier has been passed).
template <int SIGN>
__device__ __forceinline__ void stages(float2 (&v)[2][8][3], float2 (&w3)[3][4][4], float2* X, const float2* tw) {
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    r128::dft2d<8, 3, SIGN>(v[i]);
    const int jp = warp + 6 * i, jq = lane;
#pragma unroll
    for (int kp = 0; kp < 8; ++kp)
#pragma unroll
      for (int kq = 0; kq < 3; ++kq) X[(8 * jp + kp) * P + 3 * jq + kq] = v[i][kp][kq];
  }
  __syncthreads();
  float2 u2[2][3][8];
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int jp = lane, jq = warp + 6 * i;
#pragma unroll
    for (int kp = 0; kp < 3; ++kp)
#pragma unroll
      for (int kq = 0; kq < 8; ++kq) u2[i][kp][kq] = X[(jp + 32 * kp) * P + jq + 12 * kq];
    twiddle2d<3, 8, 8, 3, SIGN>(u2[i], jp, jq, tw);
    r128::dft2d<3, 8, SIGN>(u2[i]);
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int jp = lane, jq = warp + 6 * i;
    const int p0 = 24 * (jp >> 3) + (jp & 7), q0 = 24 * (jq / 3) + jq % 3;
#pragma unroll
    for (int kp = 0; kp < 3; ++kp)
#pragma unroll
      for (int kq = 0; kq < 8; ++kq) X[(p0 + 8 * kp) * P + q0 + 3 * kq] = u2[i][kp][kq];
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const int u = t + NT * i, jq = u % 24, jp = u / 24;
#pragma unroll
    for (int kp = 0; kp < 4; ++kp)
#pragma unroll
      for (int kq = 0; kq < 4; ++kq) w3[i][kp][kq] = X[(jp + 24 * kp) * P + jq + 24 * kq];
    twiddle2d<4, 24, 4, 24, SIGN>(w3[i], jp, jq, tw);
    r128::dft2d<4, 4, SIGN>(w3[i]);
  }
  __syncthreads();
}

// Pass A at N = 96, persistent (two CTAs per SM).  Per point-1 pair (a, b): build W1(c, d) =
// s_ab F(c, d) G(a,c) G(b,d) (or W0 x factors, or the diagonal source) in registers at the
// thread's stage-1 input points, 2D DFT (sign -1), natural-order slice into shared memory, one TMA
// tensor store into the V layout.  F(c, d) = Ein(c) Ein(d) Y(c, d) m(c, d) from the per-axis
// factors, the aperture test and the optional mask.
template <int SRC, bool MASK>
__global__ void __launch_bounds__(NT, 2)
    pass_a_r96(const __grid_constant__ CUtensorMap vmap, PassAArgs p, const float2* __restrict__ Ein,
               const float2* __restrict__ mask, int ap_ithr) {
  constexpr bool ARRAY = SRC == SRC_ARRAY, DIAG = SRC == SRC_DIAG;
  extern __shared__ __align__(1024) float2 smem[];
  float2* X = smem;  // exchange buffer; the first N x N entries also stage the slice for TMA
  float2* tw = X + N * P;
  float2* ein = tw + N;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  for (int i = t; i < N; i += NT) {
    tw[i] = p.tw[i];
    ein[i] = Ein[i];
  }
  auto inside = [&](int i, int j) {
    const int ni = i - N / 2, nj = j - N / 2;
    return ap_ithr < 0 || ni * ni + nj * nj <= ap_ithr;
  };
  // aperture pattern of the thread's 48 points (c, d) = (warp + 6 i + 12 kp, lane + 32 kq)
  unsigned long long inmask = 0;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int kp = 0; kp < 8; ++kp)
#pragma unroll
      for (int kq = 0; kq < 3; ++kq)
        if (inside(warp + 6 * i + 12 * kp, lane + 32 * kq)) inmask |= 1ull << (i * 24 + kp * 3 + kq);
  __syncthreads();  // tw, ein
  // the GSM factors G(a, c), G(b, d) are read through L1 (no per-slice table, no barrier)
  const float* __restrict__ G = p.G;
  for (int ab = blockIdx.x; ab < N * N; ab += gridDim.x) {
    const int a = ab / N, b = ab - a * N;
    float2 fab = inside(a, b) ? cmul(ein[a], ein[b]) : make_float2(0.f, 0.f);
    if (MASK) fab = cmul(fab, __ldg(mask + a * N + b));
    float2 s_ab = cconj(fab);
    if (SRC == SRC_GSM || SRC == SRC_ADJ) s_ab = cscale(s_ab, p.A);
    if (DIAG) s_ab = cscale(s_ab, p.A * __ldg(p.diag + ab));
    const float2* W0 = ARRAY ? p.W0 + (size_t)ab * N * N : nullptr;
    AdjSlice adj{};
    if (SRC == SRC_ADJ) adj = adj_slice(p, ab, N);
    float2 ed[3];  // Ein(d) G(b, d)
#pragma unroll
    for (int kq = 0; kq < 3; ++kq) {
      const int d = lane + 32 * kq;
      ed[kq] = SRC == SRC_GSM ? cscale(ein[d], __ldg(G + b * N + d)) : ein[d];
    }
    float2 v[2][8][3];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int kp = 0; kp < 8; ++kp) {
        const int c = warp + 6 * i + 12 * kp;
        const float2 sc = SRC == SRC_GSM ? cmul(s_ab, cscale(ein[c], __ldg(G + a * N + c))) : cmul(s_ab, ein[c]);
#pragma unroll
        for (int kq = 0; kq < 3; ++kq) {
          const int d = lane + 32 * kq;
          float2 x = cmul(sc, ed[kq]);
          if (MASK) x = cmul(x, __ldg(mask + c * N + d));
          if (ARRAY) x = cmul(x, __ldg(W0 + c * N + d));
          if (SRC == SRC_ADJ) x = cmul(x, adj.at(p.cross, c * N + d));
          bool keep = (inmask >> (i * 24 + kp * 3 + kq)) & 1ull;
          if (DIAG) keep = keep && c == a && d == b;
          v[i][kp][kq] = keep ? x : make_float2(0.f, 0.f);
        }
      }
    if (t == 0) bulk_wait_read_all();  // the previous slice's TMA store has left X
    __syncthreads();
    float2 w3[3][4][4];
    stages<-1>(v, w3, X, tw);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const int u = t + NT * i, jq = u % 24, jp = u / 24;
#pragma unroll
      for (int kp = 0; kp < 4; ++kp)
#pragma unroll
        for (int kq = 0; kq < 4; ++kq) X[(jp + 24 * kp) * N + jq + 24 * kq] = w3[i][kp][kq];
    }
    fence_proxy_async_smem();
    __syncthreads();
    if (t == 0) {
      tma_store_5d(&vmap, X, 0, b, a, 0, 0);
      bulk_commit();
    }
  }
  if (t == 0) bulk_wait_all();
}

constexpr size_t pass_a_smem() { return (size_t)N * P * sizeof(float2) + 2 * N * sizeof(float2); }
constexpr size_t pass_b_smem() {
  return (size_t)N * P * sizeof(float2) + 2 * N * sizeof(float2) + 4 * 32 * sizeof(double);
}

// Pass B at N = 96, persistent (two CTAs per SM).  CTA blockIdx.x handles point-2 output pairs
// cd = blockIdx.x + k gridDim.x: every thread loads its 48 stage-1 inputs of the strided column
// V(., ., c', d') (8 bytes from each 32-byte run) straight into registers -- the other CTA of the
// SM computes meanwhile -- with the column group's block brought into L2 two columns ahead; the
// inverse-sign 2D DFT; the epilogue (scale, output propagators, S on the diagonal, with ROW the P1
// row) and, for WST = W_HERM, the conjugated column as the contiguous row W(c', d', ., .) from
// registers (W_NONE: no W store).
template <int WST, bool ROW = false>
__global__ void __launch_bounds__(NT, 2) pass_b_r96(PassBArgs p) {
  extern __shared__ __align__(1024) float2 smem[];
  float2* X = smem;
  float2* tw = X + N * P;
  float2* eo = tw + N;
  double* red = reinterpret_cast<double*>(eo + N);  // W_GRAD: block reduction
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  constexpr int g = vgroup<N>();
  constexpr size_t NN = (size_t)N * N;
  for (int i = t; i < N; i += NT) {
    tw[i] = p.tw[i];
    eo[i] = p.Eout[i];
  }
  auto prefetch = [&](int cdn) {
    if (t == 0 && cdn < N * N) {
      const int cn = cdn / N, dn = cdn % N;
      bulk_prefetch_l2(p.V + ((size_t)(vrow<N>(cn) * (N / g) + dn / g) * g + dn % g) * NN, (unsigned)(NN * sizeof(float2)));
    }
  };
  prefetch(blockIdx.x);
  prefetch(blockIdx.x + gridDim.x);
  __syncthreads();
  float2* rw = p.row;
  const int iP = p.iP, jP = p.jP;
  for (int cd = blockIdx.x; cd < N * N; cd += gridDim.x) {
    const int c = cd / N, d = cd - c * N;
    prefetch(cd + 2 * gridDim.x);
    const float2* Vg = p.V + v_offset<N>(0, c, d);
    float2 v[2][8][3];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int kp = 0; kp < 8; ++kp)
#pragma unroll
        for (int kq = 0; kq < 3; ++kq) {
          const int a = warp + 6 * i + 12 * kp, b = lane + 32 * kq;
          v[i][kp][kq] = __ldg(Vg + (size_t)(a * N + b) * g);
        }
    float2 w3[3][4][4];
    stages<+1>(v, w3, X, tw);
    const float2 ecd = cscale(cmul(eo[c], eo[d]), p.scale);
    float2* Wrow = p.W + (size_t)cd * NN;
    if constexpr (WST == W_GRAD) {
      GradSums gs;
      const float2 ecg = grad_col(p.gr, c, d, ecd);
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const int u = t + NT * i, jq = u % 24, jp = u / 24;
        GradAxis B[4];
#pragma unroll
        for (int kq = 0; kq < 4; ++kq) B[kq] = grad_axis(p.gr, N, jq + 24 * kq, d, cconj(eo[jq + 24 * kq]));
#pragma unroll
        for (int kp = 0; kp < 4; ++kp) {
          const int a = jp + 24 * kp;
          const GradAxis A = grad_axis(p.gr, N, a, c, cmul(cconj(eo[a]), ecg));
#pragma unroll
          for (int kq = 0; kq < 4; ++kq) gs.add(A, B[kq], grad_mask(p.gr, N, a, jq + 24 * kq), w3[i][kp][kq]);
        }
      }
      grad_reduce(p.gr, N, cd, gs, red);
    } else {
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const int u = t + NT * i, jq = u % 24, jp = u / 24;
#pragma unroll
        for (int kp = 0; kp < 4; ++kp) {
          const int a = jp + 24 * kp;
          const float2 ea = cmul(cconj(eo[a]), ecd);
#pragma unroll
          for (int kq = 0; kq < 4; ++kq) {
            const int b = jq + 24 * kq;
            const float2 w = cmul(cmul(ea, cconj(eo[b])), w3[i][kp][kq]);
            if (a == c && b == d) p.S[cd] = w.x;
            if (ROW && a == iP && b == jP) rw[cd] = w;
            if (WST == W_HERM) Wrow[a * N + b] = cconj(w);
          }
        }
      }
    }
  }
}

}  // namespace r96
}  // namespace pw
