// r128.cuh -- register-resident 2D DFT of a 128 x 128 slice for the two passes at N = 128.
//
// The 2D transform runs as three 2D Stockham stages with radices (p, q) = (8, 4), (4, 8),
// (4, 4) (p = first slice index, q = second), 512 threads, 32 points per thread per stage:
//   stage 1: butterfly (jp < 16, jq < 32), inputs (jp + 16 rp, jq + 32 rq), no twiddles,
//            outputs (8 jp + rp, 4 jq + rq);
//   stage 2: butterfly (jp < 32, jq < 16), inputs (jp + 32 rp, jq + 16 rq), twiddles
//            w32^(rp (jp mod 8)) w32^(rq (jq mod 4)), outputs (32 (jp/8) + jp mod 8 + 8 rp,
//            32 (jq/4) + jq mod 4 + 4 rq);
//   stage 3: butterfly (jp < 32, jq < 32), inputs (jp + 32 rp, jq + 32 rq), twiddles
//            w128^(rp jp) w128^(rq jq), outputs in natural order at the input positions;
// (w_L = exp(SIGN 2 pi i / L)).  Points move between stages through one shared buffer whose
// q index is XOR-swizzled per exchange (sw1, sw2) so that every half-warp touches 16 distinct
// 8-byte bank pairs on both the write and the read side.
#pragma once
#include "cluster.cuh"
#include "propagate.cuh"

namespace pw {
namespace r128 {

constexpr int N = 128;
constexpr int NT = 512;

__device__ __forceinline__ int sw1(int q) { return q ^ ((q >> 4) & 3); }
__device__ __forceinline__ int sw2(int q) { return q ^ (((q >> 5) & 3) << 2); }

template <int SIGN> __device__ __forceinline__ float2 twid(const float2* tw, int m) {
  float2 w = tw[m];
  if (SIGN > 0) w.y = -w.y;
  return w;
}

template <int RP, int RQ, int SIGN> __device__ __forceinline__ void dft2d(float2 (&v)[RP][RQ]) {
#pragma unroll
  for (int rq = 0; rq < RQ; ++rq) {
    float2 c[RP];
#pragma unroll
    for (int rp = 0; rp < RP; ++rp) c[rp] = v[rp][rq];
    Dft<RP, SIGN>::run(c);
#pragma unroll
    for (int rp = 0; rp < RP; ++rp) v[rp][rq] = c[rp];
  }
#pragma unroll
  for (int rp = 0; rp < RP; ++rp) Dft<RQ, SIGN>::run(v[rp]);
}

// v[rp][rq] *= tw[mp * rp] (rp >= 1) and tw[mq * rq] (rq >= 1)
template <int RP, int RQ, int SIGN>
__device__ __forceinline__ void twiddle2d(float2 (&v)[RP][RQ], const float2* tw, int mp, int mq) {
#pragma unroll
  for (int rp = 1; rp < RP; ++rp) {
    const float2 w = twid<SIGN>(tw, mp * rp);
#pragma unroll
    for (int rq = 0; rq < RQ; ++rq) v[rp][rq] = cmul(v[rp][rq], w);
  }
#pragma unroll
  for (int rq = 1; rq < RQ; ++rq) {
    const float2 w = twid<SIGN>(tw, mq * rq);
#pragma unroll
    for (int rp = 0; rp < RP; ++rp) v[rp][rq] = cmul(v[rp][rq], w);
  }
}

// Stages 2 and 3 from stage-1 outputs v (already the thread's 8 x 4 block), through buf.
// On return w3[i][rp][rq] holds the transform at (jp3 + 32 rp, lane + 32 rq), jp3 = warp + 16 i.
// ROWS: the second exchange puts row p at buffer row vrow(p), so that the rows stage 3 of a warp
// reads (c' = warp + 16 i + 32 rp) are the eight buffer rows 8 warp .. 8 warp + 7.
// Contract: buf is free on entry (all threads passed a barrier after its last use).
template <int SIGN, bool ROWS = false>
__device__ __forceinline__ void stages_23(float2 (&v)[8][4], float2 (&w3)[2][4][4], float2* buf,
                                         const float2* tw) {
  auto row = [](int p) { return ROWS ? vrow<N>(p) : p; };
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
#pragma unroll
  for (int rp = 0; rp < 8; ++rp)
#pragma unroll
    for (int rq = 0; rq < 4; ++rq) buf[(8 * warp + rp) * N + sw1(4 * lane + rq)] = v[rp][rq];
  __syncthreads();
  const int jq2 = t & 15, jp2 = t >> 4;
  float2 u[4][8];
#pragma unroll
  for (int rp = 0; rp < 4; ++rp)
#pragma unroll
    for (int rq = 0; rq < 8; ++rq) u[rp][rq] = buf[(jp2 + 32 * rp) * N + sw1(jq2 + 16 * rq)];
  twiddle2d<4, 8, SIGN>(u, tw, 4 * (jp2 & 7), 4 * (jq2 & 3));
  dft2d<4, 8, SIGN>(u);
  __syncthreads();
#pragma unroll
  for (int rp = 0; rp < 4; ++rp)
#pragma unroll
    for (int rq = 0; rq < 8; ++rq)
      buf[row((jp2 >> 3) * 32 + (jp2 & 7) + 8 * rp) * N + sw2((jq2 >> 2) * 32 + (jq2 & 3) + 4 * rq)] = u[rp][rq];
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int jp3 = warp + 16 * i;
#pragma unroll
    for (int rp = 0; rp < 4; ++rp)
#pragma unroll
      for (int rq = 0; rq < 4; ++rq) w3[i][rp][rq] = buf[row(jp3 + 32 * rp) * N + sw2(lane + 32 * rq)];
    twiddle2d<4, 4, SIGN>(w3[i], tw, jp3, lane);
    dft2d<4, 4, SIGN>(w3[i]);
  }
}

// Pass A at N = 128, persistent.  Per point-1 pair (a, b): build W1(c, d) = s_ab F(c, d) G(a,c)
// G(b,d) (or W0 x factors) in registers, 2D DFT (sign -1) over (c, d), natural-order slice into
// shared memory, one TMA tensor store into the V layout.  F(c, d) = Ein(c) Ein(d) Y(c, d) m(c, d)
// from the per-axis factors, the aperture test and the optional mask; the GSM factors G(a, c),
// G(b, d) are read through L1.  Stage 3 reads and writes only its warp's eight buffer rows (the
// second exchange permutes rows by vrow), so the natural-order write after it needs only a warp
// barrier, and each warp leaves its rows by its own TMA store (8 rows of V, 256 runs of 32 bytes),
// which drains while the next slice is built.
template <int SRC, bool MASK>
__global__ void __launch_bounds__(NT, 1)
    pass_a_r128(const __grid_constant__ CUtensorMap vmap, PassAArgs p, const float2* __restrict__ Ein,
                const float2* __restrict__ mask, int ap_ithr) {
  constexpr bool ARRAY = SRC == SRC_ARRAY, DIAG = SRC == SRC_DIAG;
  extern __shared__ __align__(1024) float2 smem[];
  float2* buf = smem;
  float2* tw = buf + N * N;
  float2* ein = tw + N;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  for (int i = t; i < N; i += NT) {
    tw[i] = p.tw[i];
    ein[i] = Ein[i];
  }
  // aperture: integer r^2 <= ap_ithr = floor of the FP64 threshold (same decision, no FP64 work)
  auto inside = [&](int i, int j) {
    const int ni = i - N / 2, nj = j - N / 2;
    return ap_ithr < 0 || ni * ni + nj * nj <= ap_ithr;
  };
  // The thread's 32 points (c, d) = (warp + 16 rp, lane + 32 rq) are the same in every slice:
  // their aperture pattern is one 32-bit mask.
  unsigned inmask = 0;
#pragma unroll
  for (int rp = 0; rp < 8; ++rp)
#pragma unroll
    for (int rq = 0; rq < 4; ++rq)
      if (inside(warp + 16 * rp, lane + 32 * rq)) inmask |= 1u << (rp * 4 + rq);
  __syncthreads();  // tw, ein
  for (int ab = blockIdx.x; ab < N * N; ab += gridDim.x) {
    const int a = ab / N, b = ab - a * N;
    // s_ab = A conj(F(a, b)), F(i, j) = Ein(i) Ein(j) Y(i, j) m(i, j)
    float2 fab = inside(a, b) ? cmul(ein[a], ein[b]) : make_float2(0.f, 0.f);
    if (MASK) fab = cmul(fab, __ldg(mask + a * N + b));
    float2 s_ab = cconj(fab);
    if (SRC == SRC_GSM || SRC == SRC_ADJ) s_ab = cscale(s_ab, p.A);
    if (DIAG) s_ab = cscale(s_ab, p.A * __ldg(p.diag + ab));
    const float2* W0 = ARRAY ? p.W0 + (size_t)ab * N * N : nullptr;
    AdjSlice adj{};
    if (SRC == SRC_ADJ) adj = adj_slice(p, ab, N);
    float2 ed[4];  // Ein(d) G(b, d)
#pragma unroll
    for (int rq = 0; rq < 4; ++rq) {
      const int d = lane + 32 * rq;
      ed[rq] = SRC == SRC_GSM ? cscale(ein[d], __ldg(p.G + b * N + d)) : ein[d];
    }
    float2 v[8][4];
#pragma unroll
    for (int rp = 0; rp < 8; ++rp) {
      const int c = warp + 16 * rp;
      const float2 sc = SRC == SRC_GSM ? cmul(s_ab, cscale(ein[c], __ldg(p.G + a * N + c))) : cmul(s_ab, ein[c]);
#pragma unroll
      for (int rq = 0; rq < 4; ++rq) {
        const int d = lane + 32 * rq;
        float2 x = cmul(sc, ed[rq]);
        if (MASK) x = cmul(x, __ldg(mask + c * N + d));
        if (ARRAY) x = cmul(x, __ldg(W0 + c * N + d));
        if (SRC == SRC_ADJ) x = cmul(x, adj.at(p.cross, c * N + d));
        bool keep = (inmask >> (rp * 4 + rq)) & 1u;
        if (DIAG) keep = keep && c == a && d == b;
        v[rp][rq] = keep ? x : make_float2(0.f, 0.f);
      }
    }
    dft2d<8, 4, -1>(v);
    // Since the last block barrier of the previous slice each warp has touched only its own eight
    // buffer rows (stage 3, the write-back, its TMA store), and exchange 1 writes only those rows:
    // a warp barrier after the wait for the warp's own store is enough.
    if (lane == 0) bulk_wait_read_all();  // this warp's store of the previous slice has left its rows
    __syncwarp();
    float2 w3[2][4][4];
    stages_23<-1, true>(v, w3, buf, tw);
    __syncwarp();  // stage 3 read only the warp's own buffer rows 8 warp .. 8 warp + 7
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int rp = 0; rp < 4; ++rp)
#pragma unroll
        for (int rq = 0; rq < 4; ++rq) buf[(8 * warp + i + 2 * rp) * N + lane + 32 * rq] = w3[i][rp][rq];
    fence_proxy_async_smem();
    __syncwarp();
    if (lane == 0) {  // V rows vrow(c') = 8 warp + i + 2 rp of this slice
      tma_store_5d(&vmap, buf + 8 * warp * N, 0, b, a, 0, 8 * warp);
      bulk_commit();
    }
  }
  if (lane == 0) bulk_wait_all();
}

constexpr size_t pass_a_smem() { return (size_t)N * N * sizeof(float2) + 2 * N * sizeof(float2); }

}  // namespace r128
}  // namespace pw

namespace pw {
namespace r128 {

// Stages 2 and 3 through a half-size buffer (64 rows x 128): each exchange runs in two rounds.
// Round h moves the rows p with hsel(p) == h; hsel mixes a register bit and a thread bit of p on
// both sides, so every thread writes half and reads half of its points in each round, and at most
// 32 points per thread are live at any time.
//   exchange 1: hsel = (p & 1) ^ ((p >> 5) & 1), local row p >> 1, column sw1(q)
//   exchange 2: hsel = ((p >> 3) & 1) ^ ((p >> 5) & 1), local row (p & 7) | ((p >> 4) << 3), column sw2(q)
// The register index of each half is chosen with selects (no dynamic register indexing).
__device__ __forceinline__ float2 sel2(bool c, float2 a, float2 b) { return c ? a : b; }

template <int SIGN>
__device__ __forceinline__ void stages_23_half(float2 (&v)[8][4], float2 (&w3)[2][4][4], float2* xb,
                                              const float2* tw) {
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int jq2 = t & 15, jp2 = t >> 4;
  // ---- exchange 1 ----
  const bool wb = (warp >> 2) & 1;  // round 0 writes rp = 2k + wb
  float2 y[4][4];
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int rq = 0; rq < 4; ++rq) {
      xb[(4 * warp + k) * N + sw1(4 * lane + rq)] = sel2(wb, v[2 * k + 1][rq], v[2 * k][rq]);
      y[k][rq] = sel2(wb, v[2 * k][rq], v[2 * k + 1][rq]);
    }
  __syncthreads();
  const bool jb = jp2 & 1;  // round h reads rp = 2k + (h ^ jb)
  float2 z0[2][8], z1[2][8];
#pragma unroll
  for (int k = 0; k < 2; ++k)
#pragma unroll
    for (int rq = 0; rq < 8; ++rq)
      z0[k][rq] = xb[((jp2 >> 1) + 16 * (2 * k + (jb ? 1 : 0))) * N + sw1(jq2 + 16 * rq)];
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int rq = 0; rq < 4; ++rq) xb[(4 * warp + k) * N + sw1(4 * lane + rq)] = y[k][rq];
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 2; ++k)
#pragma unroll
    for (int rq = 0; rq < 8; ++rq)
      z1[k][rq] = xb[((jp2 >> 1) + 16 * (2 * k + (jb ? 0 : 1))) * N + sw1(jq2 + 16 * rq)];
  __syncthreads();
  float2 u[4][8];
#pragma unroll
  for (int k = 0; k < 2; ++k)
#pragma unroll
    for (int rq = 0; rq < 8; ++rq) {
      u[2 * k][rq] = sel2(jb, z1[k][rq], z0[k][rq]);
      u[2 * k + 1][rq] = sel2(jb, z0[k][rq], z1[k][rq]);
    }
  twiddle2d<4, 8, SIGN>(u, tw, 4 * (jp2 & 7), 4 * (jq2 & 3));
  dft2d<4, 8, SIGN>(u);
  // ---- exchange 2 ----
  const bool ub = (jp2 >> 3) & 1;  // round 0 writes rp = 2k + ub
  float2 y2[2][8];
#pragma unroll
  for (int k = 0; k < 2; ++k)
#pragma unroll
    for (int rq = 0; rq < 8; ++rq) {
      xb[((jp2 & 7) | (((jp2 >> 3) * 2 + k) << 3)) * N + sw2((jq2 >> 2) * 32 + (jq2 & 3) + 4 * rq)] =
          sel2(ub, u[2 * k + 1][rq], u[2 * k][rq]);
      y2[k][rq] = sel2(ub, u[2 * k][rq], u[2 * k + 1][rq]);
    }
  __syncthreads();
  const bool cb = (warp >> 3) & 1;  // round h reads rp = 2k + (h ^ cb)
  float2 q0[2][2][4], q1[2][2][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int k = 0; k < 2; ++k)
#pragma unroll
      for (int rq = 0; rq < 4; ++rq)
        q0[i][k][rq] = xb[((warp & 7) | ((i + 2 * (2 * k + (cb ? 1 : 0))) << 3)) * N + sw2(lane + 32 * rq)];
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 2; ++k)
#pragma unroll
    for (int rq = 0; rq < 8; ++rq)
      xb[((jp2 & 7) | (((jp2 >> 3) * 2 + k) << 3)) * N + sw2((jq2 >> 2) * 32 + (jq2 & 3) + 4 * rq)] = y2[k][rq];
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int k = 0; k < 2; ++k)
#pragma unroll
      for (int rq = 0; rq < 4; ++rq)
        q1[i][k][rq] = xb[((warp & 7) | ((i + 2 * (2 * k + (cb ? 0 : 1))) << 3)) * N + sw2(lane + 32 * rq)];
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 2; ++i) {
#pragma unroll
    for (int k = 0; k < 2; ++k)
#pragma unroll
      for (int rq = 0; rq < 4; ++rq) {
        w3[i][2 * k][rq] = sel2(cb, q1[i][k][rq], q0[i][k][rq]);
        w3[i][2 * k + 1][rq] = sel2(cb, q0[i][k][rq], q1[i][k][rq]);
      }
    twiddle2d<4, 4, SIGN>(w3[i], tw, warp + 16 * i, lane);
    dft2d<4, 4, SIGN>(w3[i]);
  }
}

constexpr size_t kStageBytes = (size_t)N * N * sizeof(float2);  // prefetched stage-1 inputs
constexpr size_t kXBytes = (size_t)N * N * sizeof(float2) / 2;     // half-size exchange buffer
constexpr size_t pass_b_smem() { return kStageBytes + kXBytes + 2 * N * sizeof(float2) + 4 * 32 * sizeof(double); }

// Pass B at N = 128, persistent.  CTA blockIdx.x handles point-2 output pairs cd = blockIdx.x +
// k gridDim.x.  Every thread gathers exactly the 32 points (a, b) = (warp + 16 rp, lane + 32 rq)
// of the strided column V(., ., c', d') that its stage-1 butterfly needs, one slice ahead, with
// 8-byte asynchronous copies into a staging tile it alone reads: the gather of slice k+1 is in
// flight while slice k is transformed, and no barrier guards the tile.  The inverse-sign 2D DFT
// runs in registers (stages_23_half through a 64 KB exchange buffer), and the epilogue (scale,
// output propagators, S on the diagonal, and with ROW the P1 row) writes, for WST = W_HERM, the
// conjugated column as the contiguous row W(c', d', ., .) straight from registers (Hermitian
// store); W_NONE stores no W.
template <int WST, bool ROW = false>
__global__ void __launch_bounds__(NT, 1) pass_b_r128(PassBArgs p) {
  extern __shared__ __align__(1024) float2 smem[];
  float2* stg = smem;
  float2* xb = stg + N * N;
  float2* tw = xb + N * N / 2;
  float2* eo = tw + N;
  double* red = reinterpret_cast<double*>(eo + N);  // W_GRAD: block reduction
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  constexpr int g = vgroup<N>();
  for (int i = t; i < N; i += NT) {
    tw[i] = p.tw[i];
    eo[i] = p.Eout[i];
  }
  auto gather = [&](int cdn) {
    const float2* Vg = p.V + v_offset<N>(0, cdn / N, cdn % N);
#pragma unroll
    for (int rp = 0; rp < 8; ++rp)
#pragma unroll
      for (int rq = 0; rq < 4; ++rq) {
        const int a = warp + 16 * rp, b = lane + 32 * rq;
        cp_async8(stg + a * N + b, Vg + (size_t)(a * N + b) * g);
      }
  };
  // The four columns d' = 4 (d'/4) + j of one (c', d'/4) share one 512 KB block of V; the CTA of
  // column j brings quarter j of the block of the column after next into L2, so that the gathers
  // (8 bytes from every 32-byte sector) hit L2 instead of waiting on DRAM.
  auto prefetch = [&](int cdn) {
    if (t == 0 && cdn < N * N) {
      const int cn = cdn / N, dn = cdn % N;
      bulk_prefetch_l2(p.V + ((size_t)(vrow<N>(cn) * (N / g) + dn / g) * g + dn % g) * N * N, (unsigned)(N * N * sizeof(float2)));
    }
  };
  prefetch(blockIdx.x + gridDim.x);
  if (blockIdx.x < N * N) gather(blockIdx.x);
  cp_async_commit();
  __syncthreads();  // tw, eo
  for (int cd = blockIdx.x; cd < N * N; cd += gridDim.x) {
    const int c = cd / N, d = cd - c * N;
    cp_async_wait_all();
    float2 v[8][4];
#pragma unroll
    for (int rp = 0; rp < 8; ++rp)
#pragma unroll
      for (int rq = 0; rq < 4; ++rq) v[rp][rq] = stg[(warp + 16 * rp) * N + lane + 32 * rq];
    dft2d<8, 4, +1>(v);  // consumes every staged value before the tile is refilled
    if (cd + (int)gridDim.x < N * N) gather(cd + gridDim.x);
    cp_async_commit();
    prefetch(cd + 2 * gridDim.x);
    float2 w3[2][4][4];
    stages_23_half<+1>(v, w3, xb, tw);
    const float2 ecd = cscale(cmul(eo[c], eo[d]), p.scale);
    float2* Wrow = p.W + (size_t)cd * N * N;
    float2* rw = p.row;
    const int iP = p.iP, jP = p.jP;
    if constexpr (WST == W_GRAD) {
      GradSums gs;
      const float2 ecg = grad_col(p.gr, c, d, ecd);
      GradAxis B[4];
#pragma unroll
      for (int rq = 0; rq < 4; ++rq) B[rq] = grad_axis(p.gr, N, lane + 32 * rq, d, cconj(eo[lane + 32 * rq]));
#pragma unroll
      for (int i = 0; i < 2; ++i) {
#pragma unroll
        for (int rp = 0; rp < 4; ++rp) {
          const int a = warp + 16 * i + 32 * rp;
          const GradAxis A = grad_axis(p.gr, N, a, c, cmul(cconj(eo[a]), ecg));
#pragma unroll
          for (int rq = 0; rq < 4; ++rq) gs.add(A, B[rq], grad_mask(p.gr, N, a, lane + 32 * rq), w3[i][rp][rq]);
        }
      }
      grad_reduce(p.gr, N, cd, gs, red);
    } else {
#pragma unroll
      for (int i = 0; i < 2; ++i) {
#pragma unroll
        for (int rp = 0; rp < 4; ++rp) {
          const int a = warp + 16 * i + 32 * rp;
          const float2 ea = cmul(cconj(eo[a]), ecd);
#pragma unroll
          for (int rq = 0; rq < 4; ++rq) {
            const int b = lane + 32 * rq;
            const float2 w = cmul(cmul(ea, cconj(eo[b])), w3[i][rp][rq]);
            if (a == c && b == d) p.S[cd] = w.x;
            if (ROW && a == iP && b == jP) rw[cd] = w;
            if (WST == W_HERM) Wrow[a * N + b] = cconj(w);
          }
        }
      }
    }
  }
  cp_async_wait_all();
}

}  // namespace r128
}  // namespace pw
