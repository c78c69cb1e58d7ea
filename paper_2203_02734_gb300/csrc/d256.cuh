// d256.cuh -- the two passes at N = 256, where one 256 x 256 complex64 slice (512 KB) exceeds
// what one SM holds: each slice is distributed over a cluster of 4 CTAs, CTA r owning the 64
// rows [64 r, 64 r + 64) of the slice (128 KB, 32 points per thread in registers).
//
// 2D DFT of a slice X(p, q) (p = first index, q = second):
//   q1: radix 16 along q on the CTA's rows (butterfly jq < 16, inputs q = jq + 16 rq), outputs to
//       the CTA's slab at [row][sw(16 jq + rq)], sw(q) = q ^ ((q >> 4) & 15);
//   q2: radix 16 along q (inputs jq + 16 rq, twiddles w256^(rq jq)), natural outputs stored at
//       [row][q' ^ (row & 15)] for the cross-CTA read;
//   p1: CTA r takes its 64 columns q' = 64 r + 2 lane + e (e = 0, 1): radix 16 along p with inputs
//       p = jp + 16 rp read as 16-byte pairs from CTA rp / 4 (distributed shared memory), outputs to
//       the slab at [16 jp + rp][q' - 64 r];
//   p2: radix 16 along p (inputs jp + 16 rp, twiddles w256^(rp jp)), natural outputs (p', q').
// Every exchange is bank-conflict free: the XOR swizzles give each half-warp 16 distinct 8-byte
// bank pairs, the 16-byte pair reads are contiguous per warp.
#pragma once
#include "cluster.cuh"
#include "propagate.cuh"

namespace pw {
namespace d256 {

constexpr int N = 256;
constexpr int CS = 4;      // CTAs per cluster (slice rows per CTA: N / CS = 64)
constexpr int RPC = N / CS;
constexpr int NT = 512;

__device__ __forceinline__ int swq(int q) { return q ^ ((q >> 4) & 15); }

template <int SIGN> __device__ __forceinline__ float2 twid(const float2* tw, int m) {
  float2 w = tw[m];
  if (SIGN > 0) w.y = -w.y;
  return w;
}

// q2 stage from the slab (in place) and the cross-CTA layout; v holds q1 outputs on entry.
template <int SIGN>
__device__ __forceinline__ void q_stage2(float2 (&v)[2][16], float2* slab, const float2* tw) {
  const int t = threadIdx.x, jq = t & 15, rg = t >> 4;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int row = rg + 32 * h;
#pragma unroll
    for (int r = 0; r < 16; ++r) slab[row * N + swq(16 * jq + r)] = v[h][r];
  }
  __syncthreads();
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int row = rg + 32 * h;
#pragma unroll
    for (int r = 0; r < 16; ++r) v[h][r] = slab[row * N + swq(jq + 16 * r)];
#pragma unroll
    for (int r = 1; r < 16; ++r) v[h][r] = cmul(v[h][r], twid<SIGN>(tw, r * jq));
    Dft<16, SIGN>::run(v[h]);
  }
  __syncthreads();
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int row = rg + 32 * h;
#pragma unroll
    for (int r = 0; r < 16; ++r) slab[row * N + ((jq + 16 * r) ^ (row & 15))] = v[h][r];
  }
}

// p1 + p2: on entry every slab of the cluster holds q2 outputs and a cluster barrier has been
// passed; on return u[e][r] holds the transform at (p' = jp + 16 r, q' = 64 rank + 2 lane + e),
// jp = warp.  Leaves the own slab free (after a block barrier) for the caller.
template <int SIGN>
__device__ __forceinline__ void p_stages(float2 (&u)[2][16], float2* slab, const float2* tw,
                                         const unsigned (&rslab)[CS], unsigned rank) {
  const int t = threadIdx.x, lane = t & 31, jp = t >> 5;
  const int p0 = RPC * (int)rank + 2 * lane;  // first of the two columns
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    const int row = jp + 16 * (r & 3);  // row of p = jp + 16 r in CTA r / 4; row & 15 == jp
    const unsigned addr = rslab[r >> 2] + (unsigned)((row * N + (p0 ^ (jp & ~1))) * 8);
    const float4 pr = ld_cluster4(addr);
    const float2 lo = make_float2(pr.x, pr.y), hi = make_float2(pr.z, pr.w);
    u[0][r] = (jp & 1) ? hi : lo;
    u[1][r] = (jp & 1) ? lo : hi;
  }
  cluster_sync();  // every CTA has read all slabs of the cluster
#pragma unroll
  for (int e = 0; e < 2; ++e) Dft<16, SIGN>::run(u[e]);
  float4* slab4 = reinterpret_cast<float4*>(slab);
#pragma unroll
  for (int r = 0; r < 16; ++r)
    slab4[((16 * jp + r) * RPC + 2 * lane) / 2] = make_float4(u[0][r].x, u[0][r].y, u[1][r].x, u[1][r].y);
  __syncthreads();
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    const float4 pr = slab4[((jp + 16 * r) * RPC + 2 * lane) / 2];
    u[0][r] = make_float2(pr.x, pr.y);
    u[1][r] = make_float2(pr.z, pr.w);
  }
  __syncthreads();
#pragma unroll
  for (int e = 0; e < 2; ++e) {
#pragma unroll
    for (int r = 1; r < 16; ++r) u[e][r] = cmul(u[e][r], twid<SIGN>(tw, r * jp));
    Dft<16, SIGN>::run(u[e]);
  }
}

// Pass A at N = 256, persistent over clusters: cluster k handles point-1 pairs ab = k,
// k + #clusters, ...  CTA r builds rows c in [64 r, 64 r + 64) of W1(c, d) (GSM x factors, or
// the uploaded W0 x factors), runs the 2D DFT (sign -1) with the rest of the cluster, and leaves
// its 256 x 64 output tile (all c', d' in [64 r, 64 r + 64)) by one TMA tensor store
// (box {2g floats, 1, 1, 64/g, 256}) into the V layout.
template <int SRC, bool MASK>
__global__ void __launch_bounds__(NT, 1)
    pass_a_d256(const __grid_constant__ CUtensorMap vmap, PassAArgs p, const float2* __restrict__ Ein,
                const float2* __restrict__ mask, int ap_ithr) {
  constexpr bool ARRAY = SRC == SRC_ARRAY, DIAG = SRC == SRC_DIAG;
  extern __shared__ __align__(1024) float2 smem[];
  float2* slab = smem;  // RPC x N
  float2* tw = slab + RPC * N;
  float2* ein = tw + N;
  float* gA = reinterpret_cast<float*>(ein + N);
  float* gB = gA + N;
  const int t = threadIdx.x, jq = t & 15, rg = t >> 4;
  const unsigned rank = cluster_rank();
  const int cluster = blockIdx.x / CS, nclusters = gridDim.x / CS;
  for (int i = t; i < N; i += NT) {
    tw[i] = p.tw[i];
    ein[i] = Ein[i];
  }
  unsigned rslab[CS];
#pragma unroll
  for (int q = 0; q < CS; ++q) rslab[q] = map_rank(slab, q);
  auto inside = [&](int i, int j) {
    const int ni = i - N / 2, nj = j - N / 2;
    return ap_ithr < 0 || ni * ni + nj * nj <= ap_ithr;
  };
  constexpr int g = vgroup<N>();
  for (int ab = cluster; ab < N * N; ab += nclusters) {
    const int a = ab / N, b = ab - a * N;
    if (SRC == SRC_GSM) {
      for (int i = t; i < N; i += NT) {
        gA[i] = p.G[a * N + i];
        gB[i] = p.G[b * N + i];
      }
    }
    __syncthreads();
    float2 fab = inside(a, b) ? cmul(ein[a], ein[b]) : make_float2(0.f, 0.f);
    if (MASK) fab = cmul(fab, __ldg(mask + a * N + b));
    float2 s_ab = cconj(fab);
    if (SRC == SRC_GSM) s_ab = cscale(s_ab, p.A);
    if (DIAG) s_ab = cscale(s_ab, p.A * __ldg(p.diag + ab));
    const float2* W0 = ARRAY ? p.W0 + (size_t)ab * N * N : nullptr;
    float2 v[2][16];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int c = RPC * (int)rank + rg + 32 * h;
      const float2 sc = SRC == SRC_GSM ? cmul(s_ab, cscale(ein[c], gA[c])) : cmul(s_ab, ein[c]);
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        const int d = jq + 16 * r;
        float2 x = cmul(sc, SRC == SRC_GSM ? cscale(ein[d], gB[d]) : ein[d]);
        if (MASK) x = cmul(x, __ldg(mask + c * N + d));
        if (ARRAY) x = cmul(x, __ldg(W0 + (size_t)c * N + d));
        bool keep = inside(c, d);
        if (DIAG) keep = keep && c == a && d == b;
        v[h][r] = keep ? x : make_float2(0.f, 0.f);
      }
      Dft<16, -1>::run(v[h]);
    }
    if (t == 0) bulk_wait_read_all();  // the previous tile has left the slab
    __syncthreads();
    q_stage2<-1>(v, slab, tw);
    cluster_sync();
    float2 u[2][16];
    p_stages<-1>(u, slab, tw, rslab, rank);
    float4* slab4 = reinterpret_cast<float4*>(slab);
#pragma unroll
    for (int r = 0; r < 16; ++r)
      slab4[((t >> 5) + 16 * r) * (RPC / 2) + (t & 31)] = make_float4(u[0][r].x, u[0][r].y, u[1][r].x, u[1][r].y);
    fence_proxy_async_smem();
    __syncthreads();
    if (t == 0) {
      tma_store_5d(&vmap, slab, 0, b, a, (int)rank * (RPC / g), 0);
      bulk_commit();
    }
  }
  if (t == 0) bulk_wait_all();
  cluster_sync();  // no CTA leaves while another may still read its slab
}

// Pass B at N = 256, persistent over clusters: cluster k handles point-2 output pairs cd = k,
// k + #clusters, ...  CTA r gathers rows a in [64 r, 64 r + 64) of the strided column
// V(., ., c', d'), runs the inverse-sign 2D DFT with the rest of the cluster, applies the epilogue
// (scale, output propagators, S on the diagonal) and writes its 64-column part of the contiguous
// row W(c', d', ., .) (Hermitian store) straight from registers.
__global__ void __launch_bounds__(NT, 1) pass_b_d256(PassBArgs p) {
  extern __shared__ __align__(1024) float2 smem[];
  float2* slab = smem;
  float2* tw = slab + RPC * N;
  float2* eo = tw + N;
  const int t = threadIdx.x, jq = t & 15, rg = t >> 4, lane = t & 31, jp = t >> 5;
  const unsigned rank = cluster_rank();
  const int cluster = blockIdx.x / CS, nclusters = gridDim.x / CS;
  constexpr int g = vgroup<N>();
  constexpr size_t NN = (size_t)N * N;
  for (int i = t; i < N; i += NT) {
    tw[i] = p.tw[i];
    eo[i] = p.Eout[i];
  }
  unsigned rslab[CS];
#pragma unroll
  for (int q = 0; q < CS; ++q) rslab[q] = map_rank(slab, q);
  __syncthreads();
  for (int cd = cluster; cd < N * N; cd += nclusters) {
    const int c = cd / N, d = cd - c * N;
    const float2* Vg = p.V + v_offset<N>(0, c, d);
    float2 v[2][16];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int a = RPC * (int)rank + rg + 32 * h;
#pragma unroll
      for (int r = 0; r < 16; ++r) v[h][r] = __ldg(Vg + (size_t)(a * N + jq + 16 * r) * g);
      Dft<16, +1>::run(v[h]);
    }
    __syncthreads();  // the previous slice's reads of the slab are done
    q_stage2<+1>(v, slab, tw);
    cluster_sync();
    float2 u[2][16];
    p_stages<+1>(u, slab, tw, rslab, rank);
    const float2 ecd = cscale(cmul(eo[c], eo[d]), p.scale);
    float2* Wrow = p.W + (size_t)cd * NN;
    const int b0 = RPC * (int)rank + 2 * lane;
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const int a = jp + 16 * r;
      const float2 ea = cmul(cconj(eo[a]), ecd);
      float2 w[2];
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        w[e] = cmul(cmul(ea, cconj(eo[b0 + e])), u[e][r]);
        if (a == c && b0 + e == d) p.S[cd] = w[e].x;
      }
      *reinterpret_cast<float4*>(Wrow + (size_t)a * N + b0) = make_float4(w[0].x, -w[0].y, w[1].x, -w[1].y);
    }
  }
  cluster_sync();  // no CTA leaves while another may still read its slab
}

constexpr size_t pass_a_smem() {
  return (size_t)RPC * N * sizeof(float2) + 2 * N * sizeof(float2) + 2 * N * sizeof(float);
}
constexpr size_t pass_b_smem() { return (size_t)RPC * N * sizeof(float2) + 2 * N * sizeof(float2); }

}  // namespace d256
}  // namespace pw
