// d256.cuh -- the two passes at N = 256, where one 256 x 256 complex64 slice (512 KB) exceeds
// what one SM holds: each slice is distributed over a cluster of CS CTAs (CS = 4 or 8), CTA r
// owning the RPC = 256 / CS rows [RPC r, RPC r + RPC) of the slice, with NT = 8 RPC threads and 32
// points per thread in registers (RPC x 256 x 8 bytes of shared memory: 128 KB for CS = 4, one
// CTA per SM; 64 KB for CS = 8, two CTAs per SM, so that one CTA's waits overlap the other's work).
//
// 2D DFT of a slice X(p, q) (p = first index, q = second), HALF = RPC / 2:
//   q1: radix 16 along q on the CTA's rows (butterfly jq < 16, rows rg + HALF h, inputs
//       q = jq + 16 rq), outputs to the CTA's slab at [row][sw(16 jq + rq)], sw(q) = q ^ ((q >> 4) & 15);
//   q2: radix 16 along q (inputs jq + 16 rq, twiddles w256^(rq jq)), natural outputs stored at
//       [row][q' ^ (row & 15)] for the cross-CTA read;
//   p1: CTA r takes its RPC columns q' = RPC r + 2 pair + e (e = 0, 1; thread t: jp = t / HALF,
//       pair = t mod HALF): radix 16 along p with inputs p = jp + 16 rp read as 16-byte pairs from
//       CTA 16 rp / RPC (distributed shared memory), outputs to the slab at [16 jp + rp][q' - RPC r];
//   p2: radix 16 along p (inputs jp + 16 rp, twiddles w256^(rp jp)), natural outputs (p', q').
// Every exchange is bank-conflict free: the XOR swizzles give each half-warp 16 distinct 8-byte
// bank pairs, the 16-byte pair reads are contiguous per half-warp.
#pragma once
#include "cluster.cuh"
#include "propagate.cuh"
#include "tc16.cuh"

namespace pw {
namespace d256 {

constexpr int N = 256;
template <int CS> struct Geo {
  static constexpr int RPC = N / CS;   // slice rows (and p-stage columns) per CTA
  static constexpr int NT = 8 * RPC;   // threads per CTA (32 points each)
  static constexpr int HALF = RPC / 2; // q-stage row groups; p-stage column pairs
  static constexpr int MINB = CS == 8 ? 2 : 1;  // CTAs per SM
};
// The cluster sizes the library launches, measured per pass: pass A gains from two CTAs per SM
// (one CTA's tile store and barriers overlap the other's DFT), pass B loses by it.
constexpr int CLUSTER_A = 8, CLUSTER_B = 4;

__device__ __forceinline__ int swq(int q) { return q ^ ((q >> 4) & 15); }

template <int SIGN> __device__ __forceinline__ float2 twid(const float2* tw, int m) {
  float2 w = tw[m];
  if (SIGN > 0) w.y = -w.y;
  return w;
}

// q2 stage from the slab (in place) and the cross-CTA layout; v holds q1 outputs on entry, for the
// slab rows rg + RS h (RS = threads / 16: the slab's rows of one slice, or of two stacked slices).
template <int RS, int SIGN>
__device__ __forceinline__ void q_stage2(float2 (&v)[2][16], float2* slab, const float2* tw) {
  const int t = threadIdx.x, jq = t & 15, rg = t >> 4;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int row = rg + RS * h;
#pragma unroll
    for (int r = 0; r < 16; ++r) slab[row * N + swq(16 * jq + r)] = v[h][r];
  }
  __syncthreads();
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int row = rg + RS * h;
#pragma unroll
    for (int r = 0; r < 16; ++r) v[h][r] = slab[row * N + swq(jq + 16 * r)];
#pragma unroll
    for (int r = 1; r < 16; ++r) v[h][r] = cmul(v[h][r], twid<SIGN>(tw, r * jq));
    Dft<16, SIGN>::run(v[h]);
  }
  __syncthreads();
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int row = rg + RS * h;
#pragma unroll
    for (int r = 0; r < 16; ++r) slab[row * N + ((jq + 16 * r) ^ (row & 15))] = v[h][r];
  }
}

// p1 + p2 of one slice: on entry the slice's slab (RPC x N at `slab`, the same offset in every CTA)
// of every CTA of the cluster holds q2 outputs and a cluster barrier has been passed; on return
// u[e][r] holds the transform at (p' = jp + 16 r, q' = RPC rank + 2 pair + e), jp = tl / HALF,
// pair = tl mod HALF, tl = the thread's index among the slice's 8 RPC threads.  Leaves the own
// slab free (after a block barrier) for the caller.
template <int CS, int SIGN>
__device__ __forceinline__ void p_stages(float2 (&u)[2][16], float2* slab, const float2* tw, unsigned rank, int tl) {
  constexpr int RPC = Geo<CS>::RPC, HALF = Geo<CS>::HALF, RG = RPC / 16;
  const int jp = tl / HALF, pair = tl % HALF;
  const int p0 = RPC * (int)rank + 2 * pair;  // first of the two columns
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    const int row = jp + 16 * (r % RG);  // row of p = jp + 16 r in CTA 16 r / RPC; row & 15 == jp
    const float4 pr = ld_cluster4(map_rank(slab + row * N + (p0 ^ (jp & ~1)), r / RG));
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
    slab4[((16 * jp + r) * RPC + 2 * pair) / 2] = make_float4(u[0][r].x, u[0][r].y, u[1][r].x, u[1][r].y);
  __syncthreads();
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    const float4 pr = slab4[((jp + 16 * r) * RPC + 2 * pair) / 2];
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
// k + #clusters, ...  CTA r builds rows c in [RPC r, RPC r + RPC) of W1(c, d) (GSM x factors, or
// the uploaded W0 x factors), runs the 2D DFT (sign -1) with the rest of the cluster, and leaves
// its 256 x RPC output tile (all c', d' in [RPC r, RPC r + RPC)) by one TMA tensor store
// (box {2g floats, 1, 1, RPC/g, 256}) into the V layout.
// TC: the first radix-16 stage (q1) runs on the tensor cores with split-BF16x3 operands
// (tc16.cuh) instead of the FP32 codelet: per half h of the thread's rows, the 256 vectors
// (row rg + HALF h, jq) of the CTA go through shared memory as two 128-row tiles, tensor memory
// holds D (columns 64 h + 32 tile), and thread t reads back its own vector t.  The stage lives in
// the slab while it is free (A 48 KB, then B 6 KB and the mbarrier, rebuilt every slice), so the
// kernel needs no more shared memory than the FP32 one: at 6 KB more, the occupancy calculator
// fits one CTA per SM instead of two (15 clusters of 8 instead of 36, measured).
// A bounded wait that gives up sets *err and leaves the stage's outputs zero.
template <int CS, int SRC, bool MASK, bool TC = false>
__global__ void __launch_bounds__(Geo<CS>::NT, Geo<CS>::MINB)
    pass_a_d256(const __grid_constant__ CUtensorMap vmap, PassAArgs p, const float2* __restrict__ Ein,
                const float2* __restrict__ mask, int ap_ithr, int* err) {
  constexpr bool ARRAY = SRC == SRC_ARRAY, DIAG = SRC == SRC_DIAG;
  constexpr int RPC = Geo<CS>::RPC, NT = Geo<CS>::NT, HALF = Geo<CS>::HALF;
  static_assert(!TC || NT == 256, "the tensor-core stage maps thread t to vector t of two 128-row tiles");
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
  unsigned char* Ast = reinterpret_cast<unsigned char*>(slab);  // A: 2 tiles x 3 splits = 48 KB
  unsigned char* Bm = Ast + 6 * tc16::A_SPLIT_BYTES;                  // B: 6 KB
  uint64_t* mbar = reinterpret_cast<uint64_t*>(Bm + tc16::B_BYTES);
  uint32_t tmem = 0;
  bool tc_ok = true;
  if constexpr (TC) {
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);  // read once, before the slab is used
    if (t < 32) tc16::tmem_alloc(tslot, 128);
    tc16::fence_before_sync();
    __syncthreads();
    tc16::fence_after_sync();
    tmem = *tslot;
  }
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
    if (SRC == SRC_GSM || SRC == SRC_ADJ) s_ab = cscale(s_ab, p.A);
    if (DIAG) s_ab = cscale(s_ab, p.A * __ldg(p.diag + ab));
    const float2* W0 = ARRAY ? p.W0 + (size_t)ab * N * N : nullptr;
    AdjSlice adj{};
    if (SRC == SRC_ADJ) adj = adj_slice(p, ab, N);
    float2 v[2][16];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int c = RPC * (int)rank + rg + HALF * h;
      const float2 sc = SRC == SRC_GSM ? cmul(s_ab, cscale(ein[c], gA[c])) : cmul(s_ab, ein[c]);
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        const int d = jq + 16 * r;
        float2 x = cmul(sc, SRC == SRC_GSM ? cscale(ein[d], gB[d]) : ein[d]);
        if (MASK) x = cmul(x, __ldg(mask + c * N + d));
        if (ARRAY) x = cmul(x, __ldg(W0 + (size_t)c * N + d));
        if (SRC == SRC_ADJ) x = cmul(x, adj.at(p.cross, c * N + d));
        bool keep = inside(c, d);
        if (DIAG) keep = keep && c == a && d == b;
        v[h][r] = keep ? x : make_float2(0.f, 0.f);
      }
      if (!TC) Dft<16, -1>::run(v[h]);
    }
    if (t == 0) bulk_wait_read_all();  // the previous tile has left the slab
    __syncthreads();
    if constexpr (TC) {
      tc16::fence_after_sync();
      const int w = t >> 5;
      tc16::build_b<-1>(Bm, tw, t, NT);
      if (t == 0) tc16::mbar_init(mbar);  // phase 0 for h = 0, phase 1 for h = 1
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        tc16::stage_row(Ast, 2, t >> 7, t & 127, v[h]);
        fence_proxy_async_smem();
        __syncthreads();
        tc16::fence_after_sync();
        // One thread issues and waits; the others sleep at the block barrier that shares its result.
        int okv = 1;
        if (t == 0) {
          okv = tc_ok;
          if (okv) {
            tc16::issue<2>(tmem, 64 * h, Ast, Bm, mbar);
            okv = tc16::mbar_wait(mbar, (uint32_t)h);
            if (!okv) atomicExch(err, 1);
          }
          if (h == 1) tc16::mbar_inval(mbar);  // the slab is reused after this stage
        }
        const bool ok = __syncthreads_and(okv) != 0;
        tc_ok = ok;
        tc16::fence_after_sync();
        if (ok) {
          tc16::load_row(v[h], tmem + ((uint32_t)(32 * (w & 3)) << 16) + 64 * h + 32 * (w >> 2));
        } else {
#pragma unroll
          for (int r = 0; r < 16; ++r) v[h][r] = make_float2(0.f, 0.f);
        }
      }
      tc16::fence_before_sync();
      // The slab is free again: each thread passed the wait, so the MMAs have read their operands.
    }
    q_stage2<HALF, -1>(v, slab, tw);
    cluster_sync();
    float2 u[2][16];
    p_stages<CS, -1>(u, slab, tw, rank, t);
    float4* slab4 = reinterpret_cast<float4*>(slab);
#pragma unroll
    for (int r = 0; r < 16; ++r)
      slab4[(t / HALF + 16 * r) * HALF + t % HALF] = make_float4(u[0][r].x, u[0][r].y, u[1][r].x, u[1][r].y);
    fence_proxy_async_smem();
    __syncthreads();
    if (t == 0) {
      tma_store_5d(&vmap, slab, 0, b, a, (int)rank * (RPC / g), 0);
      bulk_commit();
    }
  }
  if (t == 0) bulk_wait_all();
  if constexpr (TC) tc16::fence_before_sync();
  cluster_sync();  // no CTA leaves while another may still read its slab
  if constexpr (TC) {
    tc16::fence_after_sync();
    if (t < 32) tc16::tmem_dealloc(tmem, 128);
  }
}

// Pass B at N = 256, persistent over clusters: cluster k handles point-2 output pairs cd = k,
// k + #clusters, ...  CTA r gathers rows a in [RPC r, RPC r + RPC) of the strided column
// V(., ., c', d'), runs the inverse-sign 2D DFT with the rest of the cluster, applies the epilogue
// (scale, output propagators, S on the diagonal) and writes its RPC-column part of the contiguous
// row W(c', d', ., .) (Hermitian store) straight from registers.
template <int CS>
__global__ void __launch_bounds__(Geo<CS>::NT, Geo<CS>::MINB) pass_b_d256(PassBArgs p) {
  constexpr int RPC = Geo<CS>::RPC, NT = Geo<CS>::NT, HALF = Geo<CS>::HALF;
  extern __shared__ __align__(1024) float2 smem[];
  float2* slab = smem;
  float2* tw = slab + RPC * N;
  float2* eo = tw + N;
  const int t = threadIdx.x, jq = t & 15, rg = t >> 4, pair = t % HALF, jp = t / HALF;
  const unsigned rank = cluster_rank();
  const int cluster = blockIdx.x / CS, nclusters = gridDim.x / CS;
  constexpr int g = vgroup<N>();
  constexpr size_t NN = (size_t)N * N;
  for (int i = t; i < N; i += NT) {
    tw[i] = p.tw[i];
    eo[i] = p.Eout[i];
  }
  __syncthreads();
  for (int cd = cluster; cd < N * N; cd += nclusters) {
    const int c = cd / N, d = cd - c * N;
    const float2* Vg = p.V + v_offset<N>(0, c, d);
    float2 v[2][16];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int a = RPC * (int)rank + rg + HALF * h;
#pragma unroll
      for (int r = 0; r < 16; ++r) v[h][r] = __ldg(Vg + (size_t)(a * N + jq + 16 * r) * g);
      Dft<16, +1>::run(v[h]);
    }
    __syncthreads();  // the previous slice's reads of the slab are done
    q_stage2<HALF, +1>(v, slab, tw);
    cluster_sync();
    float2 u[2][16];
    p_stages<CS, +1>(u, slab, tw, rank, t);
    const float2 ecd = cscale(cmul(eo[c], eo[d]), p.scale);
    float2* Wrow = p.W + (size_t)cd * NN;
    const int b0 = RPC * (int)rank + 2 * pair;
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

template <int CS> constexpr size_t pass_a_smem() {
  return (size_t)Geo<CS>::RPC * N * sizeof(float2) + 2 * N * sizeof(float2) + 2 * N * sizeof(float);
}
// The tensor-core stage's operands and mbarrier fit in the slab's free tail.
static_assert(6 * tc16::A_SPLIT_BYTES + tc16::B_BYTES + 16 <= Geo<8>::RPC * N * sizeof(float2), "slab too small");
template <int CS> constexpr size_t pass_b_smem() {
  return (size_t)Geo<CS>::RPC * N * sizeof(float2) + 2 * N * sizeof(float2);
}

}  // namespace d256
}  // namespace pw
