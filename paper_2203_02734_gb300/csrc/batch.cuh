// batch.cuh -- many propagations (frequencies of a polychromatic spectrum, distances, grid sizes)
// in one persistent launch.
//
// The launch walks a host-built list of work items (instance, pass, slices first + k stride,
// k < count); CTAs claim items in list order through one atomic counter.  The J items of one pass
// are strided (item j takes slices j, j + J, ...), so the CTAs that claim consecutive items work
// on neighbouring slices at the same time: in pass B the g columns that share each 32-byte run of
// V are gathered together, while the run is in L2.  A pass-B item of instance i first waits until
// all pass-A slices of i are done; a pass-A item of instance i whose half-transformed buffer slot
// is shared with instance i - P (P = pool depth) first waits until pass B of i - P is done.
// Because items are claimed in list order and every awaited item precedes its waiter in the
// list, a waiting CTA always waits on items already claimed by running CTAs: no deadlock.  Each
// wait is bounded (about a second of clock64 cycles); when it gives up it sets the error flag,
// the item is skipped, and the host reads PW_ETIMEOUT.
//
// Per instance the passes are those of the single-instance path: pass A builds the GSM x masks x
// input propagators slice, runs the direct 2D DFT and stores it into the instance's V slot in the
// tiled corner-turn layout; pass B gathers a column, runs the inverse-sign 2D DFT, applies the
// scale and output propagators and keeps S (diagonal) and the mu numerator W(P1, x) (the element
// of the column at P1) -- and the whole propagated CSDA (Hermitian row store) when the instance
// asks for it.  N = 128 runs on the register-resident engine (r128.cuh); the other sizes on the
// generic shared-memory Stockham engine.
#pragma once
#include "propagate.cuh"
#include "r128.cuh"

namespace pw {
namespace batch {

constexpr int NT = 512;  // threads per block; every grid size's plan runs on all of them

struct Inst {
  int N;
  int iP, jP;
  int slices;  // N * N
  float A;
  float scale;
  const float2* F;  // N x N input factors (propagators, lens, aperture, mask, checkerboard)
  const float* G;   // N x N GSM axis factor
  const float2* tw;
  const float2* Eout;
  float2* V;        // this instance's slot of the half-transformed pool
  float2* W;        // full output (row-major CSDA) or nullptr
  float* S;         // N x N
  float2* row;      // N x N: W(P1, x)
  const void* vmap; // N = 128: tensor map (global memory) of this instance's V slot
  const float2* Ein;   // N per-axis input factors (-1)^i exp(2 pi i Kin n_i^2)
  const float2* mask;  // user mask (N x N) or nullptr
  int ap_ithr;         // aperture: n_i^2 + n_j^2 <= ap_ithr (integer floor of the FP64 bound), < 0 = none
};

struct Item {
  int inst;
  int pass;  // 0 = A, 1 = B
  int first, count, stride;
};

struct Args {
  const Inst* inst;
  const Item* items;
  int nitems;
  int pool;
  int* next;    // item counter
  int* doneA;   // per instance: pass-A slices done
  int* doneB;   // per instance: pass-B slices done
  int* err;     // set when a bounded wait gives up
  long long wait_cycles;
};

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Thread 0 waits until *p >= target, at most `cycles` clock cycles; returns false on timeout.
__device__ __forceinline__ bool wait_ge(const int* p, int target, long long cycles) {
  const long long t0 = clock64();
  while (ld_acquire(p) < target) {
    if (clock64() - t0 > cycles) return false;
    __nanosleep(256);
  }
  return true;
}

// Stages I..IEND-1 along AXIS (0: element (line, pos) at line*P + pos; 1: at pos*P + line), each
// from src into dst (two shared buffers, swapped after every stage).
template <int N, int SIGN, int AXIS, int I, int IEND>
__device__ __forceinline__ void stages_pp(float2*& src, float2*& dst, const float2* tw) {
  if constexpr (I < IEND) {
    constexpr int P = pitch<N>();
    const float2* s = src;
    float2* d = dst;
    auto ld = [s](int line, int pos) { return AXIS == 0 ? s[line * P + pos] : s[pos * P + line]; };
    auto st = [d](int line, int pos, float2 v) {
      if (AXIS == 0) d[line * P + pos] = v; else d[pos * P + line] = v;
    };
    fft_stage_stream<N, StageInfo<N, I>::R, StageInfo<N, I>::NS, SIGN, false, NT>(tw, ld, st);
    __syncthreads();
    float2* x = src;
    src = dst;
    dst = x;
    stages_pp<N, SIGN, AXIS, I + 1, IEND>(src, dst, tw);
  }
}

// Generic engine (N <= 96): every stage out of place between two shared buffers, one butterfly
// per thread at a time, so the 512-thread block stays within its register budget.
template <int N>
__device__ __forceinline__ void slice_a(const Inst& in, int ab, float2* smem) {
  constexpr int P = pitch<N>(), S = Plan<N>::stages;
  float2* buf0 = smem;
  float2* buf1 = buf0 + N * P;
  float2* tw = buf1 + N * P;
  float* gA = reinterpret_cast<float*>(tw + N);
  float* gB = gA + N;
  const int a = ab / N, b = ab - a * N;
  for (int i = threadIdx.x; i < N; i += NT) {
    tw[i] = in.tw[i];
    gA[i] = in.G[a * N + i];
    gB[i] = in.G[b * N + i];
  }
  __syncthreads();
  const float2 s_ab = cscale(cconj(__ldg(in.F + ab)), in.A);
  const float2* F = in.F;
  auto gen = [&](int d, int c) -> float2 { return cscale(cmul(s_ab, __ldg(F + c * N + d)), gA[c] * gB[d]); };
  auto st1 = [buf0](int d, int c, float2 v) { buf0[c * P + d] = v; };
  fft_stage_stream<N, StageInfo<N, 0>::R, 1, -1, false, NT>(tw, gen, st1);
  __syncthreads();
  float2* src = buf0;
  float2* dst = buf1;
  stages_pp<N, -1, 1, 1, S>(src, dst, tw);
  stages_pp<N, -1, 0, 0, S - 1>(src, dst, tw);
  float2* V = in.V;
  const float2* last = src;
  auto ld0 = [last](int c, int d) { return last[c * P + d]; };
  auto out = [V, ab](int c, int d, float2 v) { V[v_offset<N>(ab, c, d)] = v; };
  fft_stage_stream<N, StageInfo<N, S - 1>::R, StageInfo<N, S - 1>::NS, -1, true, NT>(tw, ld0, out);
  __syncthreads();  // the shared buffers are reused by the next slice
}

template <int N>
__device__ __forceinline__ void slice_b(const Inst& in, int cd, float2* smem) {
  constexpr int P = pitch<N>(), S = Plan<N>::stages;
  constexpr size_t NN = (size_t)N * N;
  float2* buf0 = smem;
  float2* buf1 = buf0 + N * P;
  float2* tw = buf1 + N * P;
  float2* eo = tw + N;
  for (int i = threadIdx.x; i < N; i += NT) {
    tw[i] = in.tw[i];
    eo[i] = in.Eout[i];
  }
  __syncthreads();
  const int c = cd / N, d = cd - c * N;
  const float2* Vg = in.V + v_offset<N>(0, c, d);
  // V is written by other CTAs of this launch: read it through L2 (never the read-only path)
  auto gather = [Vg](int b, int a) { return __ldcg(Vg + (size_t)(a * N + b) * vgroup<N>()); };
  auto st1 = [buf0](int b, int a, float2 v) { buf0[a * P + b] = v; };
  fft_stage_stream<N, StageInfo<N, 0>::R, 1, +1, false, NT>(tw, gather, st1);
  __syncthreads();
  float2* src = buf0;
  float2* dst = buf1;
  stages_pp<N, +1, 1, 1, S>(src, dst, tw);
  stages_pp<N, +1, 0, 0, S - 1>(src, dst, tw);
  const float2 ecd = cscale(cmul(eo[c], eo[d]), in.scale);
  const int iP = in.iP, jP = in.jP;
  float2* W = in.W;
  float* Sd = in.S;
  float2* rw = in.row;
  const float2* last = src;
  auto ld0 = [last](int a, int b) { return last[a * P + b]; };
  auto epi = [=](int a, int b, float2 y) {
    const float2 w = cmul(cmul(cconj(cmul(eo[a], eo[b])), ecd), y);
    if (a == c && b == d) Sd[cd] = w.x;
    if (a == iP && b == jP) rw[cd] = w;
    if (W) W[(size_t)cd * NN + a * N + b] = cconj(w);
  };
  fft_stage_stream<N, StageInfo<N, S - 1>::R, StageInfo<N, S - 1>::NS, +1, true, NT>(tw, ld0, epi);
  __syncthreads();
}

template <int N>
__device__ __noinline__ void run_item(const Inst& in, const Item& it, float2* smem) {
  for (int k = 0, s = it.first; k < it.count; ++k, s += it.stride) {
    if (it.pass == 0) slice_a<N>(in, s, smem);
    else slice_b<N>(in, s, smem);
  }
}

// ---- N = 128 on the register-resident engine ----

// Pass-A slices first + k stride (k < count): source in registers from the per-axis factors (as the single-instance
// pass A), 2D DFT (sign -1) in registers through the shared buffer, natural-order slice left by
// one TMA tensor store per slice.  Before the item is counted as done, thread 0 waits for its
// stores and orders them before its release (async proxy -> generic proxy), because pass-B items
// of this launch read V with ordinary loads.
template <bool MASK>
__device__ __noinline__ void item_a_r128(const Inst& in, int first, int count, int stride, float2* smem) {
  using r128::N;
  float2* buf = smem;
  float2* tw = buf + N * N;
  float2* ein = tw + N;
  float* gA = reinterpret_cast<float*>(ein + N);
  float* gB = gA + N;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  // the descriptor lives in memory (reference argument): keep its fields in registers
  const float* G = in.G;
  const float2* mask = in.mask;
  const void* vmap = in.vmap;
  const float A = in.A;
  for (int i = t; i < N; i += NT) {
    tw[i] = in.tw[i];
    ein[i] = in.Ein[i];
  }
  const int ap_ithr = in.ap_ithr;
  auto inside = [&](int i, int j) {
    const int ni = i - N / 2, nj = j - N / 2;
    return ap_ithr < 0 || ni * ni + nj * nj <= ap_ithr;
  };
  unsigned inmask = 0;  // aperture pattern of the thread's 32 points (the same in every slice)
#pragma unroll
  for (int rp = 0; rp < 8; ++rp)
#pragma unroll
    for (int rq = 0; rq < 4; ++rq)
      if (inside(warp + 16 * rp, lane + 32 * rq)) inmask |= 1u << (rp * 4 + rq);
  for (int k = 0, ab = first; k < count; ++k, ab += stride) {
    const int a = ab / N, b = ab - a * N;
    for (int i = t; i < N; i += NT) {
      gA[i] = G[a * N + i];
      gB[i] = G[b * N + i];
    }
    __syncthreads();
    float2 fab = inside(a, b) ? cmul(ein[a], ein[b]) : make_float2(0.f, 0.f);
    if (MASK) fab = cmul(fab, __ldg(mask + a * N + b));
    const float2 s_ab = cscale(cconj(fab), A);
    float2 ed[4];  // Ein(d) G(b, d)
#pragma unroll
    for (int rq = 0; rq < 4; ++rq) ed[rq] = cscale(ein[lane + 32 * rq], gB[lane + 32 * rq]);
    float2 v[8][4];
#pragma unroll
    for (int rp = 0; rp < 8; ++rp) {
      const int c = warp + 16 * rp;
      const float2 sc = cmul(s_ab, cscale(ein[c], gA[c]));
#pragma unroll
      for (int rq = 0; rq < 4; ++rq) {
        float2 x = cmul(sc, ed[rq]);
        if (MASK) x = cmul(x, __ldg(mask + c * N + lane + 32 * rq));
        v[rp][rq] = (inmask >> (rp * 4 + rq)) & 1u ? x : make_float2(0.f, 0.f);
      }
    }
    r128::dft2d<8, 4, -1>(v);
    if (t == 0) bulk_wait_read_all();  // the previous slice's store has left buf
    __syncthreads();
    float2 w3[2][4][4];
    r128::stages_23<-1>(v, w3, buf, tw);
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int rp = 0; rp < 4; ++rp)
#pragma unroll
        for (int rq = 0; rq < 4; ++rq)
          buf[vrow<N>(warp + 16 * i + 32 * rp) * N + lane + 32 * rq] = w3[i][rp][rq];
    fence_proxy_async_smem();
    __syncthreads();
    if (t == 0) {  // the tensor map's box is 8 rows of V (rows in vrow order)
#pragma unroll 1
      for (int r8 = 0; r8 < N; r8 += 8) tma_store_5d(vmap, buf + r8 * N, 0, b, a, 0, r8);
      bulk_commit();
    }
  }
  if (t == 0) {
    bulk_wait_all();
    fence_proxy_async_global();
  }
  __syncthreads();
}

// Pass-B columns first + k stride (k < count): 8-byte asynchronous gather of the next column
// while the current one is transformed (each thread refills only the staging slots it alone
// reads), the inverse-sign 2D DFT in registers, and the epilogue from registers.  The CTAs of
// the neighbouring items gather the other columns of the same runs at about the same time; each
// CTA brings the group block of its column after next into L2.
template <bool STORE_W>
__device__ __noinline__ void item_b_r128(const Inst& in, int first, int count, int stride, float2* smem) {
  using r128::N;
  constexpr int g = vgroup<N>();
  constexpr size_t NN = (size_t)N * N;
  float2* stg = smem;
  float2* xb = stg + N * N;
  float2* tw = xb + N * N / 2;
  float2* eo = tw + N;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  // the descriptor lives in memory (reference argument): keep its fields in registers
  const float2* V = in.V;
  float2* W = STORE_W ? in.W : nullptr;
  float* Sd = in.S;
  float2* rw = in.row;
  const float scale = in.scale;
  for (int i = t; i < N; i += NT) {
    tw[i] = in.tw[i];
    eo[i] = in.Eout[i];
  }
  auto gather = [&](int cdn) {
    const float2* Vg = V + v_offset<N>(0, cdn / N, cdn % N);
#pragma unroll
    for (int rp = 0; rp < 8; ++rp)
#pragma unroll
      for (int rq = 0; rq < 4; ++rq) {
        const int a = warp + 16 * rp, b = lane + 32 * rq;
        cp_async8(stg + a * N + b, Vg + (size_t)(a * N + b) * g);
      }
  };
  const int last = first + (count - 1) * stride;
  // the whole g-column block of column cdn: the CTAs of the other columns of the group claim their
  // items at other times, so the block is not split between them (a second request hits in L2)
  auto prefetch = [&](int cdn) {
    if (t == 0 && cdn <= last) {
      const int cn = cdn / N, dn = cdn % N;
      const float2* blk = V + (size_t)(vrow<N>(cn) * (N / g) + dn / g) * g * NN;
#pragma unroll
      for (int j = 0; j < g; ++j) bulk_prefetch_l2(blk + (size_t)j * NN, (unsigned)(NN * sizeof(float2)));
    }
  };
  prefetch(first + stride);
  gather(first);
  cp_async_commit();
  __syncthreads();  // tw, eo
  const int iP = in.iP, jP = in.jP;
  for (int k = 0, cd = first; k < count; ++k, cd += stride) {
    const int c = cd / N, d = cd - c * N;
    cp_async_wait_all();
    float2 v[8][4];
#pragma unroll
    for (int rp = 0; rp < 8; ++rp)
#pragma unroll
      for (int rq = 0; rq < 4; ++rq) v[rp][rq] = stg[(warp + 16 * rp) * N + lane + 32 * rq];
    r128::dft2d<8, 4, +1>(v);  // consumes every staged value before the tile is refilled
    if (k + 1 < count) gather(cd + stride);
    cp_async_commit();
    prefetch(cd + 2 * stride);
    float2 w3[2][4][4];
    r128::stages_23_half<+1>(v, w3, xb, tw);
    const float2 ecd = cscale(cmul(eo[c], eo[d]), scale);
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
          if (a == c && b == d) Sd[cd] = w.x;
          if (a == iP && b == jP) rw[cd] = w;
          if (STORE_W) W[(size_t)cd * NN + a * N + b] = cconj(w);
        }
      }
    }
  }
  cp_async_wait_all();
  __syncthreads();  // shared buffers are reused by the next item
}

__global__ void __launch_bounds__(NT, 1) batch_kernel(Args g) {
  // 1024-byte alignment: the N = 128 pass-A items leave slices by TMA from the start of this buffer
  extern __shared__ __align__(1024) float2 smem[];
  __shared__ int s_item, s_ok;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(g.next, 1);
    __syncthreads();
    const int k = s_item;
    if (k >= g.nitems) break;
    const Item it = g.items[k];
    const Inst in = g.inst[it.inst];
    if (threadIdx.x == 0) {
      bool ok = true;
      if (it.pass == 1) ok = wait_ge(g.doneA + it.inst, in.slices, g.wait_cycles);
      else if (it.inst >= g.pool)
        ok = wait_ge(g.doneB + it.inst - g.pool, g.inst[it.inst - g.pool].slices, g.wait_cycles);
      if (!ok) atomicOr(g.err, 1);
      s_ok = ok;
    }
    __syncthreads();
    if (s_ok) {
      switch (in.N) {
        case 16: run_item<16>(in, it, smem); break;
        case 32: run_item<32>(in, it, smem); break;
        case 64: run_item<64>(in, it, smem); break;
        case 96: run_item<96>(in, it, smem); break;
        case 128:
          if (it.pass == 1) {
            if (in.W) item_b_r128<true>(in, it.first, it.count, it.stride, smem);
            else item_b_r128<false>(in, it.first, it.count, it.stride, smem);
          }
          else if (in.mask) item_a_r128<true>(in, it.first, it.count, it.stride, smem);
          else item_a_r128<false>(in, it.first, it.count, it.stride, smem);
          break;
        default: break;
      }
    }
    __threadfence();  // this item's stores are visible before its completion is counted
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd((it.pass == 0 ? g.doneA : g.doneB) + it.inst, it.count);
  }
}

// The FP64 tables of every instance (blockIdx.y = instance), as tables_kernel does for one.
__global__ void batch_tables_kernel(const TableArgs* targs) {
  const TableArgs t = targs[blockIdx.y];
  const int N = t.N, M = N / 2, NN = N * N;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < NN; idx += gridDim.x * blockDim.x) {
    const int i = idx / N, j = idx - i * N;
    const double ni = (double)(i - M), nj = (double)(j - M);
    const double n2i = ni * ni, n2j = nj * nj;
    const bool inside = t.ap_thr < 0.0 || (n2i + n2j) <= t.ap_thr;
    float2 m = t.mask ? t.mask[idx] : make_float2(1.f, 0.f);
    if (!inside) m = make_float2(0.f, 0.f);
    const double turns = frac_turns(n2i * t.Kin) + frac_turns(n2j * t.Kin) + 0.5 * ((i + j) & 1);
    t.F[idx] = cmul(cis_turns(turns), m);
    const double dij = (double)(i - j);
    t.G[idx] = (float)exp(-(n2i + n2j) * t.gs - dij * dij * t.gm);
    if (idx < N) {
      const double nk = (double)(idx - M);
      t.tw[idx] = cis_turns(-(double)idx / (double)N);
      t.Eout[idx] = cis_turns(frac_turns(nk * nk * t.Kout) + 0.5 * (idx & 1));
      if (t.Ein) t.Ein[idx] = cis_turns(frac_turns(nk * nk * t.Kin) + 0.5 * (idx & 1));
    }
  }
}

// I(x) = sum_i w_i S_i(x) over the instances (common grid), accumulated in FP64.
__global__ void batch_sum_kernel(const Inst* inst, const double* w, int n, float* I, int NN) {
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < NN; x += gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int i = 0; i < n; ++i) acc += w[i] * (double)inst[i].S[x];
    I[x] = (float)acc;
  }
}

// mu(P1, x) = row(x) / sqrt(S(P1) S(x)) for every instance (blockIdx.y = instance).
__global__ void batch_mu_kernel(const Inst* inst, float2* const* mu_out) {
  const Inst in = inst[blockIdx.y];
  float2* mu = mu_out[blockIdx.y];
  if (!mu) return;
  const int NN = in.N * in.N;
  const float sp = in.S[in.iP * in.N + in.jP];
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < NN; x += gridDim.x * blockDim.x) {
    const float den = sp * in.S[x];
    mu[x] = den > 0.f ? cscale(in.row[x], rsqrtf(den)) : make_float2(0.f, 0.f);
  }
}

constexpr size_t cmax(size_t a, size_t b) { return a > b ? a : b; }
constexpr size_t smem_bytes() {
  return cmax((size_t)2 * 96 * pitch<96>() * sizeof(float2) + 2 * 96 * sizeof(float2) + 2 * 96 * sizeof(float),
              cmax(r128::pass_a_smem(), r128::pass_b_smem()));
}

}  // namespace batch
}  // namespace pw
