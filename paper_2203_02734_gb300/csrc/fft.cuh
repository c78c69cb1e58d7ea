// fft.cuh -- FP32 complex DFT codelets and one Stockham autosort stage for the 2D DFTs of
// the two propagation passes (Algorithm 2: N^2 direct 2D DFTs over one point pair, N^2
// inverse-sign 2D DFTs over the other).
//
// Stage convention (mixed radix, autosort, Govindaraju et al. 2008 formulation): a length-N
// transform is a sequence of radix-R stages; with NS = product of the radices already done,
// butterfly j (0 <= j < N/R) of a line reads positions j + r*N/R (r < R), multiplies input r
// by w^(r*(j mod NS)) with w = exp(SIGN 2 pi i / (NS R)), runs a length-R DFT and writes
// output r to position (j/NS)*NS*R + (j mod NS) + r*NS.  After the last stage the line holds
// sum_n x[n] exp(SIGN 2 pi i n k / N) in natural order.
#pragma once
#include <cuda_runtime.h>

namespace pw {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// a * (S i), S = +-1
template <int S> __device__ __forceinline__ float2 mul_si(float2 a) {
  return S > 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}
// a * (c + S i s)
template <int S> __device__ __forceinline__ float2 mul_cs(float2 a, float c, float s) {
  return S > 0 ? make_float2(fmaf(a.x, c, -a.y * s), fmaf(a.y, c, a.x * s))
               : make_float2(fmaf(a.x, c, a.y * s), fmaf(a.y, c, -a.x * s));
}

// cos(pi/4), cos(pi/8), sin(pi/8), sqrt(3)/2
constexpr float kR2 = 0.70710678118654752440f;
constexpr float kC8 = 0.92387953251128675613f;
constexpr float kS8 = 0.38268343236508977173f;
constexpr float kH3 = 0.86602540378443864676f;

// In-place length-R DFT with kernel exp(S 2 pi i n k / R), natural order in and out.
template <int R, int S> struct Dft;

template <int S> struct Dft<2, S> {
  __device__ __forceinline__ static void run(float2* v) {
    float2 t = v[0];
    v[0] = cadd(t, v[1]);
    v[1] = csub(t, v[1]);
  }
};

template <int S> struct Dft<3, S> {
  __device__ __forceinline__ static void run(float2* v) {
    float2 t = cadd(v[1], v[2]);
    float2 u = cscale(mul_si<S>(csub(v[1], v[2])), kH3);
    float2 m = make_float2(fmaf(-0.5f, t.x, v[0].x), fmaf(-0.5f, t.y, v[0].y));
    v[0] = cadd(v[0], t);
    v[1] = cadd(m, u);
    v[2] = csub(m, u);
  }
};

template <int S> struct Dft<4, S> {
  __device__ __forceinline__ static void run(float2* v) {
    float2 t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
    float2 t2 = cadd(v[1], v[3]), t3 = mul_si<S>(csub(v[1], v[3]));
    v[0] = cadd(t0, t2);
    v[2] = csub(t0, t2);
    v[1] = cadd(t1, t3);
    v[3] = csub(t1, t3);
  }
};

template <int S> struct Dft<8, S> {
  __device__ __forceinline__ static void run(float2* v) {
    float2 e[4] = {v[0], v[2], v[4], v[6]};
    float2 o[4] = {v[1], v[3], v[5], v[7]};
    Dft<4, S>::run(e);
    Dft<4, S>::run(o);
    o[1] = mul_cs<S>(o[1], kR2, kR2);
    o[2] = mul_si<S>(o[2]);
    o[3] = mul_cs<S>(o[3], -kR2, kR2);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      v[k] = cadd(e[k], o[k]);
      v[k + 4] = csub(e[k], o[k]);
    }
  }
};

template <int S> struct Dft<16, S> {
  __device__ __forceinline__ static void run(float2* v) {
    float2 e[8], o[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      e[k] = v[2 * k];
      o[k] = v[2 * k + 1];
    }
    Dft<8, S>::run(e);
    Dft<8, S>::run(o);
    o[1] = mul_cs<S>(o[1], kC8, kS8);
    o[2] = mul_cs<S>(o[2], kR2, kR2);
    o[3] = mul_cs<S>(o[3], kS8, kC8);
    o[4] = mul_si<S>(o[4]);
    o[5] = mul_cs<S>(o[5], -kS8, kC8);
    o[6] = mul_cs<S>(o[6], -kR2, kR2);
    o[7] = mul_cs<S>(o[7], -kC8, kS8);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      v[k] = cadd(e[k], o[k]);
      v[k + 8] = csub(e[k], o[k]);
    }
  }
};

// Inter-stage twiddles: input r of butterfly j times w^(r k), k = j mod NS,
// w = exp(SIGN 2 pi i/(NS R)) = tw[N/(NS R)] (tw[m] = exp(-2 pi i m/N), conjugated for SIGN > 0).
template <int N, int R, int NS, int SIGN>
__device__ __forceinline__ void twiddle(float2* v, int j, const float2* tw) {
  if constexpr (NS > 1) {
    const int k = j % NS;
    constexpr int STEP = N / (NS * R);
#pragma unroll
    for (int r = 1; r < R; ++r) {
      float2 w = tw[r * k * STEP];
      if (SIGN > 0) w.y = -w.y;
      v[r] = cmul(v[r], w);
    }
  }
}

// One stage over all N lines of an N x N slice, run by NT threads.
//   JFAST = false: butterfly u -> line = u % N, j = u / N (lanes walk across lines)
//   JFAST = true : butterfly u -> j = u % (N/R), line = u / (N/R) (lanes walk along a line)
//   load(line, pos) -> float2, store(line, pos, float2); mid() runs between all loads and all
//   stores (a barrier for an in-place stage on shared memory, or nothing).  Threads with index
//   >= NT (a block larger than the plan) take part in mid() only.
template <int N, int R, int NS, int SIGN, bool JFAST, int NT, class Load, class Mid, class Store>
__device__ __forceinline__ void fft_stage(const float2* tw, Load load, Mid mid, Store store) {
  static_assert(N % R == 0, "radix must divide N");
  constexpr int NJ = N / R;
  constexpr int NB = N * NJ;
  constexpr int PER = (NB + NT - 1) / NT;
  float2 v[PER][R];
#pragma unroll
  for (int it = 0; it < PER; ++it) {
    const int u = threadIdx.x + it * NT;
    if (NB % NT == 0 || u < NB) {
      const int line = JFAST ? u / NJ : u % N;
      const int j = JFAST ? u % NJ : u / N;
#pragma unroll
      for (int r = 0; r < R; ++r) v[it][r] = load(line, j + r * NJ);
      twiddle<N, R, NS, SIGN>(v[it], j, tw);
      Dft<R, SIGN>::run(v[it]);
    }
  }
  mid();
#pragma unroll
  for (int it = 0; it < PER; ++it) {
    const int u = threadIdx.x + it * NT;
    if (NB % NT == 0 || u < NB) {
      const int line = JFAST ? u / NJ : u % N;
      const int j = JFAST ? u % NJ : u / N;
      const int base = (j / NS) * NS * R + (j % NS);
#pragma unroll
      for (int r = 0; r < R; ++r) store(line, base + r * NS, v[it][r]);
    }
  }
}

// The same stage out of place, one butterfly at a time: load(line, pos) must not read what
// store(line, pos, v) writes.  Only the R values of the current butterfly are live, so a block
// larger than its register budget allows for fft_stage still runs without spills.
template <int N, int R, int NS, int SIGN, bool JFAST, int NT, class Load, class Store>
__device__ __forceinline__ void fft_stage_stream(const float2* tw, Load load, Store store) {
  static_assert(N % R == 0, "radix must divide N");
  constexpr int NJ = N / R;
  constexpr int NB = N * NJ;
#pragma unroll 2
  for (int u = threadIdx.x; u < NB; u += NT) {
    const int line = JFAST ? u / NJ : u % N;
    const int j = JFAST ? u % NJ : u / N;
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = load(line, j + r * NJ);
    twiddle<N, R, NS, SIGN>(v, j, tw);
    Dft<R, SIGN>::run(v);
    const int base = (j / NS) * NS * R + (j % NS);
#pragma unroll
    for (int r = 0; r < R; ++r) store(line, base + r * NS, v[r]);
  }
}

struct SyncMid {
  __device__ __forceinline__ void operator()() const { __syncthreads(); }
};
struct NoMid {
  __device__ __forceinline__ void operator()() const {}
};

// Compile-time radix plans per axis length and thread count per CTA.
template <int N> struct Plan;
#define PW_PLAN(NN, NTT, ...)                                   \
  template <> struct Plan<NN> {                                 \
    static constexpr int NT = NTT;                              \
    static constexpr int radix[] = {__VA_ARGS__};               \
    static constexpr int stages = sizeof(radix) / sizeof(int);  \
  };
PW_PLAN(2, 32, 2)
PW_PLAN(4, 32, 4)
PW_PLAN(6, 32, 3, 2)
PW_PLAN(8, 32, 8)
PW_PLAN(12, 64, 4, 3)
PW_PLAN(16, 64, 16)
PW_PLAN(24, 96, 8, 3)
PW_PLAN(32, 128, 8, 4)
PW_PLAN(48, 192, 16, 3)
PW_PLAN(64, 256, 8, 8)
PW_PLAN(96, 384, 8, 4, 3)
PW_PLAN(128, 512, 16, 8)
#undef PW_PLAN

template <int N, int I> struct StageInfo {
  static constexpr int R = Plan<N>::radix[I];
  static constexpr int NS = StageInfo<N, I - 1>::NS * StageInfo<N, I - 1>::R;
};
template <int N> struct StageInfo<N, 0> {
  static constexpr int R = Plan<N>::radix[0];
  static constexpr int NS = 1;
};

}  // namespace pw
