// stream.cuh -- the N = 256 propagation as four streaming passes, one 1D DFT of 256 points per
// axis, instead of two passes with a 2D DFT per 512 KB slice spread over a cluster.  It needs no
// Hermitian source (it writes W in natural order), so it serves the sources the cluster engine
// cannot take; on the Hermitian phase-screen workload it is slower (76.7 ms per step against
// 58.4 ms: its tiles of 128-byte rows scattered along the strided axes do not stream near peak).
//
// With the factorisation of propagate.cuh, W_B = s conj(E(a')E(b')) E(c')E(d') DFT+_a DFT+_b DFT-_c
// DFT-_d [conj(F(a,b)) F(c,d) W0core]: the four 1D DFTs commute, and each is done by one pass over
// the array in its natural layout W[a][b][c][d]:
//   pass d: generate the source (GSM / uploaded / diagonal, times conj(F(a,b)) F(c,d)) for 16
//           consecutive rows (a, b, c), DFT- along d, store (8 B/point);
//   pass c, pass b: load tiles of 256 (along the axis) x 16 consecutive d (128-byte rows), DFT,
//           store in place (16 B/point each);
//   pass a: the same, times s conj(E(a')E(b')) E(c')E(d'), S = Re W_B on the diagonal, stored to W.
// Each pass moves more bytes than the two-pass design (56 B/point in all against 24) but needs no
// cluster exchange and no strided gather: every access is a 128-byte row (or a 2 KB row in pass d).
//
// DFT-256 of one line (16 threads j, line l): x[n], n = n1 + 16 n2.  Stage 1: thread n1 takes
// x[n1 + 16 n2] (n2 < 16), DFT-16 over n2, twiddle w256^(n1 k2), writes y[n1][k2] to position
// n1 + 16 k2 (the positions it read).  Stage 2: thread k2 takes positions n1 + 16 k2 (n1 < 16),
// DFT-16 over n1, and holds X[k2 + 16 k1] for k1 < 16 in natural order, stored straight to global.
// The tile sits in shared memory as [n][l] with a pitch of 17 complex per n (conflict-free for
// 16 consecutive lines and for 16 consecutive n).
#pragma once
#include <cstdint>

#include "propagate.cuh"

namespace pw {
namespace stream {

constexpr int N = 256, L = 16, P = L + 1, NT = 256;
constexpr size_t NN = (size_t)N * N, NNN = NN * N;

template <int SIGN> __device__ __forceinline__ float2 tw_of(const float2* tw, int m) {
  float2 w = tw[m & (N - 1)];
  if (SIGN > 0) w.y = -w.y;
  return w;
}

// Stage 1 in shared memory for the calling thread (line l, column n1); the caller syncs around it.
template <int SIGN>
__device__ __forceinline__ void stage1(float2* X, const float2* tw, int l, int n1) {
  float2 v[16];
#pragma unroll
  for (int n2 = 0; n2 < 16; ++n2) v[n2] = X[(n1 + 16 * n2) * P + l];
  Dft<16, SIGN>::run(v);
#pragma unroll
  for (int k2 = 1; k2 < 16; ++k2) v[k2] = cmul(v[k2], tw_of<SIGN>(tw, n1 * k2));
#pragma unroll
  for (int k2 = 0; k2 < 16; ++k2) X[(n1 + 16 * k2) * P + l] = v[k2];
}

// Stage 2 into registers: out[k1] = X[k2 + 16 k1] of line l.
template <int SIGN>
__device__ __forceinline__ void stage2(const float2* X, int l, int k2, float2 (&out)[16]) {
#pragma unroll
  for (int n1 = 0; n1 < 16; ++n1) out[n1] = X[(n1 + 16 * k2) * P + l];
  Dft<16, SIGN>::run(out);
}

struct GenArgs {
  int src;             // SRC_GSM, SRC_ARRAY, SRC_DIAG, SRC_ADJ
  const float2* F;     // N x N input factor (propagator, checkerboard, aperture, lens, mask)
  const float* G;      // GSM axis factor
  const float2* W0;    // uploaded CSDA (SRC_ARRAY)
  const float* diag;   // N x N diagonal (SRC_DIAG, SRC_ADJ)
  PassAArgs adj;       // SRC_ADJ: diag, cross, P1, herm (the other fields unused)
  float A;
  const float2* tw;    // exp(-2 pi i m / N)
  float2* out;         // N^4, natural layout
};

// Pass d: tile = 16 consecutive rows r = (a, b, c); grid-stride over N^3 / 16 tiles.
__global__ void __launch_bounds__(NT) gen_d_kernel(GenArgs g) {
  __shared__ float2 X[N * P];
  __shared__ float2 tw[N];
  const int t = threadIdx.x;
  tw[t] = g.tw[t];
  const int l = t & (L - 1), j = t >> 4;
  for (size_t tile = blockIdx.x; tile < NNN / L; tile += gridDim.x) {
    const size_t r0 = tile * L;
    const int ab = (int)(r0 / N), a = ab / N, b = ab % N, c0 = (int)(r0 % N);
    const float2 fab = cconj(g.F[ab]);
    AdjSlice adj{};
    if (g.src == SRC_ADJ) adj = adj_slice(g.adj, ab, N);
    __syncthreads();  // the previous tile's stage 2 has read X; tw is written
    // generate: thread t -> d = t, all 16 rows (c = c0 + l) of the tile
    const int d = t;
#pragma unroll 4
    for (int ll = 0; ll < L; ++ll) {
      const int c = c0 + ll;
      float2 v;
      const float2 f = cmul(fab, g.F[c * N + d]);
      if (g.src == SRC_GSM) {
        v = cscale(f, g.A * g.G[a * N + c] * g.G[b * N + d]);
      } else if (g.src == SRC_ARRAY) {
        v = cmul(f, g.W0[(r0 + ll) * N + d]);
      } else if (g.src == SRC_ADJ) {
        v = cmul(cscale(f, g.A), adj.at(g.adj.cross, c * N + d));
      } else {
        v = (a == c && b == d) ? cscale(f, g.A * g.diag[ab]) : make_float2(0.f, 0.f);
      }
      X[d * P + ll] = v;
    }
    __syncthreads();
    stage1<-1>(X, tw, l, j);
    __syncthreads();
    float2 o[16];
    stage2<-1>(X, l, j, o);
#pragma unroll
    for (int k1 = 0; k1 < 16; ++k1) g.out[(r0 + l) * N + j + 16 * k1] = o[k1];
  }
}

struct AxisArgs {
  int axis;          // 2 = c, 1 = b, 0 = a (the contracted index of W[a][b][c][d])
  float2* X;         // input (and output, in place, unless EPI)
  float2* out;       // EPI: the propagated CSDA
  const float2* tw;
  const float2* Eout;  // EPI: output factors
  float scale;         // EPI: s
  float* S;            // EPI: S (N x N)
};

// One 1D DFT pass along axis c, b or a over tiles of 256 x 16 consecutive d.  EPI: the last pass.
template <int SIGN, bool EPI>
__global__ void __launch_bounds__(NT) axis_kernel(AxisArgs p) {
  __shared__ float2 X[N * P];
  __shared__ float2 tw[N];
  const int t = threadIdx.x;
  tw[t] = p.tw[t];
  const int l = t & (L - 1), j = t >> 4;
  // strides of the contracted axis (sn) and of the two other non-d axes (su, sv)
  const size_t sa = NNN, sb = NN, sc = N;
  const size_t sn = p.axis == 2 ? sc : (p.axis == 1 ? sb : sa);
  const size_t su = p.axis == 0 ? sb : sa;
  const size_t sv = p.axis == 2 ? sb : sc;
  for (size_t tile = blockIdx.x; tile < NNN / L; tile += gridDim.x) {
    const size_t uv = tile / (N / L);
    const int db = (int)(tile % (N / L));
    const int u = (int)(uv / N), v = (int)(uv % N);
    const size_t base = u * su + v * sv + (size_t)db * L;
    __syncthreads();  // the previous tile's stage 2 has read X; tw is written
#pragma unroll 4
    for (int i = 0; i < L; ++i) {  // row n = j + 16 i: 16 threads per 128-byte row
      const int n = j + 16 * i;
      X[n * P + l] = p.X[base + n * sn + l];
    }
    __syncthreads();
    stage1<SIGN>(X, tw, l, j);
    __syncthreads();
    float2 o[16];
    stage2<SIGN>(X, l, j, o);
    if (!EPI) {
#pragma unroll
      for (int k1 = 0; k1 < 16; ++k1) p.X[base + (size_t)(j + 16 * k1) * sn + l] = o[k1];
    } else {
      // axis a: u = b', v = c', d' = 16 db + l, a' = j + 16 k1
      const int bq = u, cq = v, dq = db * L + l;
      const float2 e = cscale(cmul(cconj(p.Eout[bq]), cmul(p.Eout[cq], p.Eout[dq])), p.scale);
#pragma unroll
      for (int k1 = 0; k1 < 16; ++k1) {
        const int aq = j + 16 * k1;
        const float2 w = cmul(cmul(cconj(p.Eout[aq]), e), o[k1]);
        p.out[base + (size_t)aq * sn + l] = w;
        if (aq == cq && dq == bq) p.S[aq * N + bq] = w.x;
      }
    }
  }
}

}  // namespace stream
}  // namespace pw
