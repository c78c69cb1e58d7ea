// batch.cuh -- many propagations (frequencies of a polychromatic spectrum, distances, grid sizes)
// in one persistent launch.
//
// The launch walks a host-built list of work items (instance, pass, slices [s0, s1)); CTAs claim
// items in list order through one atomic counter.  A pass-B item of instance i first waits until
// all pass-A slices of i are done; a pass-A item of instance i whose half-transformed buffer slot
// is shared with instance i - P (P = pool depth) first waits until pass B of i - P is done.
// Because items are claimed in list order and every awaited item precedes its waiter in the
// list, a waiting CTA always waits on items already claimed by running CTAs: no deadlock.  Each
// wait is bounded (about a second of clock64 cycles); when it gives up it sets the error flag,
// the item is skipped, and the host reads PW_ETIMEOUT.
//
// Per instance the passes are those of the single-instance path (generic shared-memory Stockham
// engine): pass A builds the GSM x masks x input propagators slice in shared memory, runs the
// direct 2D DFT and stores it into the instance's V slot in the tiled corner-turn layout; pass B
// gathers a column, runs the inverse-sign 2D DFT, applies the scale and output propagators and
// keeps S (diagonal) and the mu numerator W(P1, x) (the element of the column at P1) -- and the
// whole propagated CSDA (Hermitian row store) when the instance asks for it.
#pragma once
#include "propagate.cuh"

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
};

struct Item {
  int inst;
  int pass;  // 0 = A, 1 = B
  int s0, s1;
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

template <int N>
__device__ __forceinline__ void slice_a(const Inst& in, int ab, float2* smem) {
  constexpr int P = pitch<N>(), S = Plan<N>::stages;
  float2* buf = smem;
  float2* tw = buf + N * P;
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
  auto st1 = [buf](int d, int c, float2 v) { buf[c * P + d] = v; };
  fft_stage<N, StageInfo<N, 0>::R, 1, -1, false, NT>(tw, gen, NoMid{}, st1);
  __syncthreads();
  smem_stages<N, -1, 1, 1, S, NT>(buf, tw);
  smem_stages<N, -1, 0, 0, S - 1, NT>(buf, tw);
  float2* V = in.V;
  auto ld0 = [buf](int c, int d) { return buf[c * P + d]; };
  auto out = [V, ab](int c, int d, float2 v) { V[v_offset<N>(ab, c, d)] = v; };
  fft_stage<N, StageInfo<N, S - 1>::R, StageInfo<N, S - 1>::NS, -1, true, NT>(tw, ld0, NoMid{}, out);
  __syncthreads();  // the shared buffer is reused by the next item
}

template <int N>
__device__ __forceinline__ void slice_b(const Inst& in, int cd, float2* smem) {
  constexpr int P = pitch<N>(), S = Plan<N>::stages;
  constexpr size_t NN = (size_t)N * N;
  float2* buf = smem;
  float2* tw = buf + N * P;
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
  auto st1 = [buf](int b, int a, float2 v) { buf[a * P + b] = v; };
  fft_stage<N, StageInfo<N, 0>::R, 1, +1, false, NT>(tw, gather, NoMid{}, st1);
  __syncthreads();
  smem_stages<N, +1, 1, 1, S, NT>(buf, tw);
  smem_stages<N, +1, 0, 0, S - 1, NT>(buf, tw);
  const float2 ecd = cscale(cmul(eo[c], eo[d]), in.scale);
  const int iP = in.iP, jP = in.jP;
  float2* W = in.W;
  float* Sd = in.S;
  float2* rw = in.row;
  auto ld0 = [buf](int a, int b) { return buf[a * P + b]; };
  auto epi = [=](int a, int b, float2 y) {
    const float2 w = cmul(cmul(cconj(cmul(eo[a], eo[b])), ecd), y);
    if (a == c && b == d) Sd[cd] = w.x;
    if (a == iP && b == jP) rw[cd] = w;
    if (W) W[(size_t)cd * NN + a * N + b] = cconj(w);
  };
  fft_stage<N, StageInfo<N, S - 1>::R, StageInfo<N, S - 1>::NS, +1, true, NT>(tw, ld0, NoMid{}, epi);
  __syncthreads();
}

template <int N>
__device__ __noinline__ void run_item(const Inst& in, const Item& it, float2* smem) {
  for (int s = it.s0; s < it.s1; ++s) {
    if (it.pass == 0) slice_a<N>(in, s, smem);
    else slice_b<N>(in, s, smem);
  }
}

__global__ void __launch_bounds__(NT, 1) batch_kernel(Args g) {
  extern __shared__ __align__(16) float2 smem[];
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
        case 128: run_item<128>(in, it, smem); break;
        default: break;
      }
    }
    __threadfence();  // this item's stores are visible before its completion is counted
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd((it.pass == 0 ? g.doneA : g.doneB) + it.inst, it.s1 - it.s0);
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
    }
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

constexpr size_t smem_bytes() {
  return (size_t)128 * pitch<128>() * sizeof(float2) + 2 * 128 * sizeof(float2) + 2 * 128 * sizeof(float);
}

}  // namespace batch
}  // namespace pw
