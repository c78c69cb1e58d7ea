// t256.cuh -- the propagation at N = 256 as three streaming passes over independent tiles.
//
// One 256 x 256 slice (512 KB) does not fit one SM, and spreading it over a cluster makes every
// point cross the SM-to-SM network, which on this GPU moves about 4 TB/s in all (less than HBM).
// Here the exchange goes through HBM instead, in three passes of 8 + 16 + 16 bytes per point,
// each on tiles that one CTA owns.  With the factorisation of propagate.cuh and the point-2 row
// index split as c = r + 4 m (r < 4, m < 64), k_c = k_l + 64 k_h:
//   e^{-2 pi i c k_c / 256} = e^{-2 pi i r k_h / 4} e^{-2 pi i r k_l / 256} e^{-2 pi i m k_l / 64},
// so the point-2 transform is a DFT-64 over m and a DFT-256 over d for each r (pass 1), then a
// twiddle e^{-2 pi i r k_l / 256} and a DFT-4 over r (pass 2).  With d' = 8 g + j (j < 8) the
// intermediate array lives in the work buffer as
//   Y[a][b][kperm(k_l)][g][r][j]  (after pass 1)  and  Y[a][b'][kperm(k_l)][g][k_h][j]  (after pass 2),
// so that the 4 x 8 values one pass-2 line group needs are one 256-byte run (kperm: below).
//   pass 1, tile (a, b, r): the source rows c = r + 4 m of slice (a, b) are generated in registers
//     (W1(c, d) = conj F(a, b) F(c, d) x source), transformed over (m, d) as a 64 x 256 2D DFT in
//     registers through one shared buffer, and stored to Y by TMA (64-byte pieces of the 256-byte
//     runs; the four r tiles of a slice run side by side and fill each run together).
//   pass 2, tile (a, k_l, g): the 256 runs Y[a][.][k_l][g] (all b, r, j) arrive by one TMA tensor
//     load; twiddle e^{-2 pi i r k_l / 256}, DFT-4 over r (-> k_h), DFT-256 over b (sign +1);
//     stored back to the same runs (the tile reads and writes one set of addresses).
//   pass 3, tile (b', c' = k_l + 64 k_h, 32 consecutive d'): the 256 x 32 block arrives by one TMA
//     tensor load (four 64-byte pieces per a); DFT-256 over a (sign +1), output propagators,
//     scale and S; stored to W[a][b'][c'][d'] in 256-byte runs.  The four k_h tiles of a run group
//     are consecutive, so the pieces of each 256-byte run are read at about the same time.
// Passes 2 and 3 run two CTAs per SM, so that one CTA's tile load overlaps the other's DFT.  None
// of the passes needs a Hermitian source.
#pragma once
#include <cuda.h>
#include <cstdint>

#include "propagate.cuh"
#include "r128.cuh"
#include "tc16.cuh"

namespace pw {
namespace t256 {

constexpr int N = 256;
constexpr int NT1 = 512;  // pass 1: 32 points per thread of a 64 x 256 tile
constexpr int NT2 = 256;  // passes 2 and 3: 32 points per thread of an 8192-point tile

// ---- TMA tensor loads into shared memory, completing on an mbarrier ----
__device__ __forceinline__ void mbar_expect(uint64_t* mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void tma_load_5d(void* smem, const void* tmap, uint64_t* mbar, int c0, int c1, int c2,
                                            int c3, int c4) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5, %6, %7}], "
      "[%2];" ::"r"(smem_u32(smem)),
      "l"(tmap), "r"(smem_u32(mbar)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4)
      : "memory");
}
template <int SIGN> __device__ __forceinline__ float2 twid(const float2* tw, int m) {
  float2 w = tw[m & (N - 1)];
  if (SIGN > 0) w.y = -w.y;
  return w;
}

// ---------------------------------------------------------------------------------------------
// Pass 1.  Tile (a, b, r): T(m, d) = W1(a, b, r + 4 m, d), m < 64, d < 256, 512 threads (warp w,
// lane l).  The 2D DFT (sign -1) over (m, d) runs as three 2D Stockham stages (p = m, q = d):
//   stage 1: radices (4, 8), butterfly (jp = w, jq = l), inputs (w + 16 rp, l + 32 rq), the
//            thread's own generated points; outputs (4 jp + rp, 8 jq + rq);
//   stage 2: radices (4, 8), NS = (4, 8), butterfly (w, l), inputs (w + 16 rp, l + 32 rq),
//            twiddles w16^(rp (jp mod 4)) w64^(rq (jq mod 8)); outputs (16 (jp / 4) + jp mod 4 +
//            4 rp, 64 (jq / 8) + jq mod 8 + 8 rq);
//   stage 3: radices (4, 4), NS = (16, 64), butterflies (w, l + 32 h), h < 2, inputs
//            (jp + 16 rp, jq + 64 rq), twiddles w64^(rp jp) w256^(rq jq); outputs in natural order
//            (k_l, d') at the input positions;
// (w_L = e^{-2 pi i / L}).  The two exchanges go through one 128 KB buffer whose column index is
// XOR-swizzled per exchange so that every access of a warp touches each 8-byte bank pair twice:
//   exchange 1: q ^ ((q >> 4) & 7);  exchange 2: q ^ (((q >> 6) & 3) << 3);
// exchange 2 also permutes the rows (logical row p at buffer row kperm(p)), so that the rows of a
// stage-3 warp are adjacent.  Stage 3 writes its outputs back over its own rows in natural order and
// each warp leaves its four rows by one TMA tensor store into Y[a][b][kperm(k_l)][d' / 8][r][d' mod 8];
// the next tile's first exchange waits (per warp, before the block barrier) until those stores have
// read the buffer.  The twiddle e^{-2 pi i r k_l / 256} is applied by pass 2, which has issue slots
// to spare.
// Pass 1's codelets with each complex add / subtract as one packed FP32x2 instruction (the same
// rounding as two FP32 adds, so the same results as Dft<R, S>): fewer issued instructions where
// pass 1 is bound by its arithmetic.  Passes 2 and 3 keep Dft (packed adds slowed pass 2).
__device__ __forceinline__ unsigned long long pk2(float2 a) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
  return r;
}
__device__ __forceinline__ float2 up2(unsigned long long r) {
  float2 d;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(d.x), "=f"(d.y) : "l"(r));
  return d;
}
__device__ __forceinline__ float2 padd(float2 a, float2 b) {
  unsigned long long d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk2(a)), "l"(pk2(b)));
  return up2(d);
}
__device__ __forceinline__ float2 psub(float2 a, float2 b) {
  unsigned long long d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk2(a)), "l"(pk2(b)));
  return up2(d);
}
template <int R, int S> struct PDft;
template <int S> struct PDft<4, S> {
  __device__ __forceinline__ static void run(float2* v) {
    const float2 t0 = padd(v[0], v[2]), t1 = psub(v[0], v[2]);
    const float2 t2 = padd(v[1], v[3]), t3 = mul_si<S>(psub(v[1], v[3]));
    v[0] = padd(t0, t2);
    v[2] = psub(t0, t2);
    v[1] = padd(t1, t3);
    v[3] = psub(t1, t3);
  }
};
template <int S> struct PDft<8, S> {
  __device__ __forceinline__ static void run(float2* v) {
    float2 e[4] = {v[0], v[2], v[4], v[6]};
    float2 o[4] = {v[1], v[3], v[5], v[7]};
    PDft<4, S>::run(e);
    PDft<4, S>::run(o);
    o[1] = mul_cs<S>(o[1], kR2, kR2);
    o[2] = mul_si<S>(o[2]);
    o[3] = mul_cs<S>(o[3], -kR2, kR2);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      v[k] = padd(e[k], o[k]);
      v[k + 4] = psub(e[k], o[k]);
    }
  }
};
template <int RP, int RQ, int S> __device__ __forceinline__ void pdft2d(float2 (&v)[RP][RQ]) {
#pragma unroll
  for (int rq = 0; rq < RQ; ++rq) {
    float2 c[RP];
#pragma unroll
    for (int rp = 0; rp < RP; ++rp) c[rp] = v[rp][rq];
    PDft<RP, S>::run(c);
#pragma unroll
    for (int rp = 0; rp < RP; ++rp) v[rp][rq] = c[rp];
  }
#pragma unroll
  for (int rp = 0; rp < RP; ++rp) PDft<RQ, S>::run(v[rp]);
}

// Position of k_l along the k_l index of Y: the four rows k_l = w + 16 i that stage 3 of warp w
// owns are adjacent (4 w + i), so that one TMA store moves them.
__device__ __forceinline__ int kperm(int kl) { return 4 * (kl & 15) + (kl >> 4); }
__device__ __forceinline__ int xs1(int q) { return q ^ ((q >> 4) & 7); }
__device__ __forceinline__ int xs2(int q) { return q ^ (((q >> 6) & 3) << 3); }

constexpr size_t pass1_smem() { return (size_t)64 * N * sizeof(float2) + N * sizeof(float2); }

template <int SRC>
__global__ void __launch_bounds__(NT1, 1) pass1_kernel(const __grid_constant__ CUtensorMap smap, PassAArgs p) {
  constexpr bool ARRAY = SRC == SRC_ARRAY, DIAG = SRC == SRC_DIAG;
  extern __shared__ __align__(1024) float2 smem[];
  float2* buf = smem;  // 64 x 256
  float2* tw = buf + 64 * N;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  for (int i = t; i < N; i += NT1) tw[i] = p.tw[i];
  const float2* __restrict__ F = p.F;
  const float* __restrict__ G = p.G;
  for (int tile = blockIdx.x; tile < N * N * 4; tile += gridDim.x) {
    const int ab = tile >> 2, r = tile & 3;
    const int a = ab / N, b = ab - a * N;
    float2 s_ab = cconj(__ldg(F + ab));
    if (SRC == SRC_GSM || SRC == SRC_ADJ) s_ab = cscale(s_ab, p.A);
    if (DIAG) s_ab = cscale(s_ab, p.A * __ldg(p.diag + ab));
    const float2* W0 = ARRAY ? p.W0 + (size_t)ab * N * N : nullptr;
    AdjSlice adj{};
    if (SRC == SRC_ADJ) adj = adj_slice(p, ab, N);
    // stage 1 inputs: m = w + 16 rp (c = r + 4 m), d = l + 32 rq
    float gb[8];
    if (SRC == SRC_GSM) {
#pragma unroll
      for (int rq = 0; rq < 8; ++rq) gb[rq] = __ldg(G + b * N + lane + 32 * rq);
    }
    float2 v[4][8];
#pragma unroll
    for (int rp = 0; rp < 4; ++rp) {
      const int c = r + 4 * (w + 16 * rp);
      const float ga = SRC == SRC_GSM ? __ldg(G + a * N + c) : 1.f;
#pragma unroll
      for (int rq = 0; rq < 8; ++rq) {
        const int d = lane + 32 * rq;
        float2 x = cmul(s_ab, __ldg(F + c * N + d));
        if (SRC == SRC_GSM) x = cscale(x, ga * gb[rq]);
        if (ARRAY) x = cmul(x, __ldg(W0 + c * N + d));
        if (DIAG) x = (c == a && d == b) ? x : make_float2(0.f, 0.f);
        if (SRC == SRC_ADJ) x = cmul(x, adj.at(p.cross, c * N + d));
        v[rp][rq] = x;
      }
    }
#pragma unroll
    for (int rp = 0; rp < 4; ++rp) PDft<8, -1>::run(v[rp]);  // rows first: the first rows' DFTs overlap later loads
#pragma unroll
    for (int rq = 0; rq < 8; ++rq) {
      float2 cc[4];
#pragma unroll
      for (int rp = 0; rp < 4; ++rp) cc[rp] = v[rp][rq];
      PDft<4, -1>::run(cc);
#pragma unroll
      for (int rp = 0; rp < 4; ++rp) v[rp][rq] = cc[rp];
    }
    // Since the last block barrier of the previous tile each warp has touched only its own four
    // buffer rows (stage 3, the write-back, its TMA store), and exchange 1 writes only those rows;
    // tw is first read after the next block barrier.  A warp barrier after the wait for the warp's
    // own store is enough.
    if (lane == 0) bulk_wait_read_all();  // this warp's row stores of the previous tile have left its rows
    __syncwarp();
#pragma unroll
    for (int rp = 0; rp < 4; ++rp)
#pragma unroll
      for (int rq = 0; rq < 8; ++rq) buf[(4 * w + rp) * N + xs1(8 * lane + rq)] = v[rp][rq];
    __syncthreads();
#pragma unroll
    for (int rp = 0; rp < 4; ++rp)
#pragma unroll
      for (int rq = 0; rq < 8; ++rq) v[rp][rq] = buf[(w + 16 * rp) * N + xs1(lane + 32 * rq)];
    r128::twiddle2d<4, 8, -1>(v, tw, 16 * (w & 3), 4 * (lane & 7));
    pdft2d<4, 8, -1>(v);
    __syncthreads();
#pragma unroll
    for (int rp = 0; rp < 4; ++rp)
#pragma unroll
      for (int rq = 0; rq < 8; ++rq)
        buf[(4 * ((w & 3) + 4 * rp) + (w >> 2)) * N + xs2(64 * (lane >> 3) + (lane & 7) + 8 * rq)] = v[rp][rq];
    __syncthreads();
    // stage 3 on the warp's own rows k_l = w + 16 rp (buffer rows 4 w + rp): read both halves,
    // transform, write the outputs back in natural order, then one TMA store of the four rows
    // (4 x 32 pieces of 64 bytes into Y), which drains while the next tile's stage 1 runs
    float2 u[2][4][4];
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int rp = 0; rp < 4; ++rp)
#pragma unroll
        for (int rq = 0; rq < 4; ++rq) u[h][rp][rq] = buf[(4 * w + rp) * N + xs2(lane + 32 * h + 64 * rq)];
    __syncwarp();
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int jq = lane + 32 * h;
      r128::twiddle2d<4, 4, -1>(u[h], tw, 4 * w, jq);
      pdft2d<4, 4, -1>(u[h]);
#pragma unroll
      for (int rp = 0; rp < 4; ++rp)
#pragma unroll
        for (int rq = 0; rq < 4; ++rq) buf[(4 * w + rp) * N + jq + 64 * rq] = u[h][rp][rq];
    }
    fence_proxy_async_smem();
    __syncwarp();
    if (lane == 0) {
      tma_store_5d(&smap, buf + 4 * w * N, 0, r, 0, 4 * w, ab);  // rows k_l' = 4 w + rp (k_l = w + 16 rp)
      bulk_commit();
    }
  }
  if (lane == 0) bulk_wait_all();
}

// Bounded wait on the tile load of a pass-2/3 CTA; every thread learns the outcome.  A wait that
// gives up sets *err; the caller leaves its loop (after which no load of its own is in flight
// that it has not waited for, up to the bound).
__device__ __forceinline__ bool tile_arrived(uint64_t* mbar, uint32_t parity, int* err) {
  int ok = 1;
  if (threadIdx.x == 0) {
    ok = tc16::mbar_wait(mbar, parity) ? 1 : 0;
    if (!ok) atomicExch(err, 1);
  }
  return __syncthreads_and(ok) != 0;
}

// ---------------------------------------------------------------------------------------------
// Pass 2.  Tile (a, k_l, g): X[b][r][j] = Y[a][b][kperm(k_l)][g][r][j] (b < 256, r < 4, j < 8),
// 64 KB by one TMA load (tensor map: Y as floats {64, 32, 64, 256, 256}, box {64, 1, 1, 256, 1}).
//   phase 1: twiddle e^{-2 pi i r k_l / 256} and DFT-4 over r (sign -1) for each (b, j), in place
//            (r -> k_h);
//   phase 2: DFT-256 over b (sign +1), first radix-16 stage: line L = (k_h, j) = lane, butterflies
//            n1 = w and w + 8, inputs b = n1 + 16 n2, twiddle w256^(n1 k2), in place;
//   phase 3: second stage: butterflies k2 = w, w + 8, inputs n1 + 16 k2, outputs b' = k2 + 16 k1.
// Outputs go back to the runs they came from, Y[a][b'][kperm(k_l)][g][k_h][j] (line L = 8 k_h + j = lane:
// one 256-byte run per warp store).  The next tile's load is issued once every thread has read the
// buffer.
constexpr size_t pass2_smem() { return (size_t)N * 4 * 8 * sizeof(float2) + N * sizeof(float2) + 64; }

__global__ void __launch_bounds__(NT2, 2) pass2_kernel(const __grid_constant__ CUtensorMap ymap, const float2* tw_g,
                                                     float2* __restrict__ Y, int* err) {
  extern __shared__ __align__(1024) float2 smem[];
  float2* X = smem;  // [256][4][8]
  float2* tw = X + N * 32;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(tw + N);
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  for (int i = t; i < N; i += NT2) tw[i] = tw_g[i];
  constexpr int NTILES = N * 64 * 32;
  auto issue = [&](int tile) {
    const int db = tile & 31, kl = (tile >> 5) & 63, a = tile >> 11;
    fence_proxy_async_smem();
    mbar_expect(mbar, (uint32_t)(N * 32 * sizeof(float2)));
    tma_load_5d(X, &ymap, mbar, 0, db, kperm(kl), 0, a);
  };
  bool pending = false;  // thread 0: a load was issued and not yet seen complete
  if (t == 0) {
    tc16::mbar_init(mbar);
    if ((int)blockIdx.x < NTILES) {
      issue(blockIdx.x);
      pending = true;
    }
  }
  __syncthreads();
  uint32_t parity = 0;
  for (int tile = blockIdx.x; tile < NTILES; tile += gridDim.x, parity ^= 1u) {
    const int db = tile & 31, kl = (tile >> 5) & 63, a = tile >> 11;
    if (!tile_arrived(mbar, parity, err)) break;
    pending = false;
    // phase 1: (b, j) pairs u = t + 256 i, b = u >> 3, j = u & 7: twiddle e^{-2 pi i r k_l / 256}, DFT-4
    const float2 tr1 = twid<-1>(tw, kl), tr2 = twid<-1>(tw, 2 * kl), tr3 = twid<-1>(tw, 3 * kl);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int u = t + NT2 * i, bb = u >> 3, j = u & 7;
      float2 x[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) x[r] = X[bb * 32 + r * 8 + j];
      x[1] = cmul(x[1], tr1);
      x[2] = cmul(x[2], tr2);
      x[3] = cmul(x[3], tr3);
      Dft<4, -1>::run(x);
#pragma unroll
      for (int r = 0; r < 4; ++r) X[bb * 32 + r * 8 + j] = x[r];
    }
    __syncthreads();
    // phase 2: lines L = lane, n1 = w, w + 8
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int n1 = w + 8 * e;
      float2 x[16];
#pragma unroll
      for (int n2 = 0; n2 < 16; ++n2) x[n2] = X[(n1 + 16 * n2) * 32 + lane];
      Dft<16, +1>::run(x);
#pragma unroll
      for (int k2 = 1; k2 < 16; ++k2) x[k2] = cmul(x[k2], twid<+1>(tw, n1 * k2));
#pragma unroll
      for (int k2 = 0; k2 < 16; ++k2) X[(n1 + 16 * k2) * 32 + lane] = x[k2];
    }
    __syncthreads();
    float2 y[2][16];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int k2 = w + 8 * e;
#pragma unroll
      for (int n1 = 0; n1 < 16; ++n1) y[e][n1] = X[(n1 + 16 * k2) * 32 + lane];
      Dft<16, +1>::run(y[e]);
    }
    __syncthreads();  // every thread has read X: the next tile may land there
    if (t == 0 && tile + (int)gridDim.x < NTILES) {
      issue(tile + gridDim.x);
      pending = true;
    }
    float2* Ya = Y + (size_t)a * N * N * N + kperm(kl) * 1024 + db * 32 + lane;
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int k2 = w + 8 * e;
#pragma unroll
      for (int k1 = 0; k1 < 16; ++k1) Ya[(size_t)(k2 + 16 * k1) * N * N] = y[e][k1];
    }
  }
  if (t == 0 && pending) tc16::mbar_wait(mbar, parity);  // a load left in flight by a failed wait
  __syncthreads();
}

// ---------------------------------------------------------------------------------------------
// Pass 3.  Tile (k_h, q, k_l, b'), k_h fastest: c' = k_l + 64 k_h, d' = 32 q + j,
// X[a][j] = Y[a][b'][kperm(k_l)][4 q + j / 8][k_h][j mod 8] (a < 256, j < 32), 64 KB by one TMA load
// (tensor map: Y as floats {64, 32, 64, 256, 256}, box {16, 4, 1, 1, 256}).  DFT-256 over a (sign
// +1) as two radix-16 stages (line j = lane; butterflies 2 w, 2 w + 1), then the epilogue
// W_B = s conj(E(a') E(b')) E(c') E(d') X and S on the diagonal, stored to W[a'][b'][c'][d'].
constexpr size_t pass3_smem() { return (size_t)N * 32 * sizeof(float2) + 2 * N * sizeof(float2) + 64; }

__global__ void __launch_bounds__(NT2, 2) pass3_kernel(const __grid_constant__ CUtensorMap y3map, PassBArgs p,
                                                     int* err) {
  extern __shared__ __align__(1024) float2 smem[];
  float2* X = smem;  // [256][32]
  float2* tw = X + N * 32;
  float2* eo = tw + N;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(eo + N);
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  for (int i = t; i < N; i += NT2) {
    tw[i] = p.tw[i];
    eo[i] = p.Eout[i];
  }
  constexpr int NTILES = N * N * 8;
  auto issue = [&](int tile) {
    const int kh = tile & 3, q = (tile >> 2) & 7, kl = (tile >> 5) & 63, bq = tile >> 11;
    fence_proxy_async_smem();
    mbar_expect(mbar, (uint32_t)(N * 32 * sizeof(float2)));
    tma_load_5d(X, &y3map, mbar, 16 * kh, 4 * q, kperm(kl), bq, 0);
  };
  bool pending = false;  // thread 0: a load was issued and not yet seen complete
  if (t == 0) {
    tc16::mbar_init(mbar);
    if ((int)blockIdx.x < NTILES) {
      issue(blockIdx.x);
      pending = true;
    }
  }
  __syncthreads();
  uint32_t parity = 0;
  for (int tile = blockIdx.x; tile < NTILES; tile += gridDim.x, parity ^= 1u) {
    const int q = (tile >> 2) & 7, bq = tile >> 11, cq = ((tile >> 5) & 63) + 64 * (tile & 3);
    if (!tile_arrived(mbar, parity, err)) break;
    pending = false;
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int n1 = 2 * w + e;
      float2 x[16];
#pragma unroll
      for (int n2 = 0; n2 < 16; ++n2) x[n2] = X[(n1 + 16 * n2) * 32 + lane];
      Dft<16, +1>::run(x);
#pragma unroll
      for (int k2 = 1; k2 < 16; ++k2) x[k2] = cmul(x[k2], twid<+1>(tw, n1 * k2));
#pragma unroll
      for (int k2 = 0; k2 < 16; ++k2) X[(n1 + 16 * k2) * 32 + lane] = x[k2];
    }
    __syncthreads();
    float2 y[2][16];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int k2 = 2 * w + e;
#pragma unroll
      for (int n1 = 0; n1 < 16; ++n1) y[e][n1] = X[(n1 + 16 * k2) * 32 + lane];
      Dft<16, +1>::run(y[e]);
    }
    __syncthreads();  // every thread has read X: the next tile may land there
    if (t == 0 && tile + (int)gridDim.x < NTILES) {
      issue(tile + gridDim.x);
      pending = true;
    }
    const int dq = 32 * q + lane;
    const float2 e_bcd = cscale(cmul(cconj(eo[bq]), cmul(eo[cq], eo[dq])), p.scale);
    float2* Wt = p.W + ((size_t)bq * N + cq) * N + dq;
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int k2 = 2 * w + e;
#pragma unroll
      for (int k1 = 0; k1 < 16; ++k1) {
        const int aq = k2 + 16 * k1;
        const float2 v = cmul(cmul(cconj(eo[aq]), e_bcd), y[e][k1]);
        Wt[(size_t)aq * N * N * N] = v;
        if (aq == cq && dq == bq) p.S[cq * N + bq] = v.x;
      }
    }
  }
  if (t == 0 && pending) tc16::mbar_wait(mbar, parity);  // a load left in flight by a failed wait
  __syncthreads();
}

}  // namespace t256
}  // namespace pw
