// propagate.cuh -- the two fused passes of one propagation, the FP64 table kernel and the
// S / mu kernel.
//
// With index centring (x(i) = (i - N/2) d, and the same for the flipped second axis), the
// discretised Eq. W_fresnel factorises exactly as
//   W_B(a',b',c',d') = s conj(E(a') E(b')) E(c') E(d')
//                        sum_{a,b} e^{+2 pi i (a a' + b b')/N}  sum_{c,d} e^{-2 pi i (c c' + d d')/N}
//                        conj(F(a,b)) F(c,d) W0core(a,b,c,d)
// where F(i,j) = (-1)^(i+j) exp(2 pi i (tau_i + tau_j)) Y(i,j) m(i,j) folds the input
// propagator q(xi) (Algorithm 3), a thin lens q*(f, xi), the aperture Y and a mask m, and
// E(i) = (-1)^i exp(2 pi i tau'_i) is the output propagator on the new grid; the
// checkerboards carry the centring and s = d^4/(lambda z)^2.  (a,b) is point 1, (c,d) point 2.
//
// Pass A (one CTA per point-1 pair (a,b), contiguous slice): generate conj(F(a,b)) F(c,d)
//   A G(a,c) G(b,d) (GSM) or read the uploaded W0 slice, run the direct 2D DFT over (c,d)
//   in shared memory, store the slice of V once.
// Pass B (one CTA per point-2 output pair (c',d'), strided slice): gather V(., ., c', d'),
//   run the inverse-sign 2D DFT over (a,b), apply s and the output propagators, write S on
//   the diagonal and store.  Because a CSD is Hermitian (Sec. 3.3), the column
//   W_B(., ., c', d') is stored conjugated as the contiguous row W_B(c', d', ., .); the
//   general (non-Hermitian) variant stores the column in place.
//
// Layout of V (the corner turn between the passes): V[c'][d'/g][a][b][d' mod g], g = vgroup_of(N).
// Pass A writes each (c', d'/g) run of g outputs as one piece (a 32-byte sector for g = 4); the g
// columns of one group sit in one contiguous N^2 g-element block, and consecutive (a, b) of one
// column are g elements apart.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "cluster.cuh"
#include "fft.cuh"

namespace pw {

__device__ __forceinline__ double frac_turns(double t) { return t - rint(t); }

// exp(2 pi i t) from turns t, reduced to [-1/2, 1/2] in FP64 before sincospi.
__device__ __forceinline__ float2 cis_turns(double t) {
  double s, c;
  sincospi(2.0 * frac_turns(t), &s, &c);
  return make_float2((float)c, (float)s);
}

struct TableArgs {
  int N;
  double Kin;     // turns per n^2 of the point-2 input factor (propagator and lens)
  double K0;      // turns per n^2 of the lens alone (source-plane view, no propagator)
  double Kout;    // turns per n^2 of the output propagator
  double gs, gm;  // GSM: d^2/(4 sigma_S^2) and d^2/(2 sigma_mu^2)
  double ap_thr;  // aperture: n_i^2 + n_j^2 <= ap_thr (pixels^2), < 0 = none
  const float2* mask;  // user mask (N x N) or nullptr
  float2* F;      // N x N input factor
  float2* M0;     // N x N source-plane mask Y * lens * m (or nullptr)
  float* G;       // N x N GSM axis factor (or nullptr)
  float2* tw;     // N twiddles exp(-2 pi i m / N)
  float2* Eout;   // N output factors
  float2* Ein;    // N per-axis input factors (-1)^i exp(2 pi i Kin n_i^2), or nullptr
};

static __global__ void tables_kernel(TableArgs t) {
  const int N = t.N, M = N / 2;
  const int NN = N * N;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < NN; idx += gridDim.x * blockDim.x) {
    const int i = idx / N, j = idx - i * N;
    const double ni = (double)(i - M), nj = (double)(j - M);
    const double n2i = ni * ni, n2j = nj * nj;
    const bool inside = t.ap_thr < 0.0 || (n2i + n2j) <= t.ap_thr;
    float2 m = t.mask ? t.mask[idx] : make_float2(1.f, 0.f);
    if (!inside) m = make_float2(0.f, 0.f);
    const double turns = frac_turns(n2i * t.Kin) + frac_turns(n2j * t.Kin) + 0.5 * ((i + j) & 1);
    t.F[idx] = cmul(cis_turns(turns), m);
    if (t.M0) t.M0[idx] = cmul(cis_turns(frac_turns(n2i * t.K0) + frac_turns(n2j * t.K0)), m);
    if (t.G) {
      const double dij = (double)(i - j);
      t.G[idx] = (float)exp(-(n2i + n2j) * t.gs - dij * dij * t.gm);
    }
    if (idx < N) {
      const double nk = (double)(idx - M);
      t.tw[idx] = cis_turns(-(double)idx / (double)N);
      t.Eout[idx] = cis_turns(frac_turns(nk * nk * t.Kout) + 0.5 * (idx & 1));
      if (t.Ein) t.Ein[idx] = cis_turns(frac_turns(nk * nk * t.Kin) + 0.5 * (idx & 1));
    }
  }
}

// Source of pass A: the GSM model, an uploaded CSDA, a diagonal (delta-correlated, incoherent)
// source W0 = w d(xi1) delta(xi1 - xi2) with d real, or the adjoint source of a loss on S and mu
// (SRC_ADJ): the diagonal d plus the row of the coherence point P1,
//   Y(x1, x2) = d(x1) delta(x1 - x2) + delta(x1 - P1) r(x2),
// completed to its Hermitian part (r halved on the row, conj(r)/2 on the column of P1) when the
// propagated array must be Hermitian.
enum SrcMode { SRC_GSM = 0, SRC_ARRAY = 1, SRC_DIAG = 2, SRC_ADJ = 3 };

struct PassAArgs {
  const float2* F;
  const float* G;
  const float2* tw;
  const float2* W0;   // uploaded source (SRC_ARRAY) or nullptr
  const float* diag;  // N x N diagonal (SRC_DIAG, SRC_ADJ) or nullptr
  float A;            // GSM amplitude, or the weight w of the diagonal / adjoint source
  const float2* cross;  // SRC_ADJ: N x N row r of P1, or nullptr
  int iP, jP;           // SRC_ADJ: P1
  int herm;             // SRC_ADJ: nonzero = Hermitian part (row and column of P1, halved)
};

// The adjoint source of one slice x1 = ab, evaluated at x2 = cd (SRC_ADJ).
struct AdjSlice {
  int ab, p1;
  float dg;      // d(x1), or 0
  float2 col;    // conj(r(x1)) / 2 (Hermitian part), or 0
  bool row;      // x1 == P1: the slice holds the row r
  float wr;      // weight of the row: 1/2 (Hermitian part) or 1
  __device__ __forceinline__ float2 at(const float2* __restrict__ cross, int cd) const {
    float2 v = make_float2(cd == ab ? dg : 0.f, 0.f);
    if (cd == p1) v = cadd(v, col);
    if (row) v = cadd(v, cscale(__ldg(cross + cd), wr));
    return v;
  }
};

__device__ __forceinline__ AdjSlice adj_slice(const PassAArgs& p, int ab, int N) {
  AdjSlice s;
  s.ab = ab;
  s.p1 = p.iP * N + p.jP;
  s.dg = p.diag ? __ldg(p.diag + ab) : 0.f;
  s.row = p.cross != nullptr && ab == s.p1;
  s.wr = p.herm ? 0.5f : 1.f;
  s.col = (p.cross != nullptr && p.herm) ? cscale(cconj(__ldg(p.cross + ab)), 0.5f) : make_float2(0.f, 0.f);
  return s;
}

template <int N> __host__ __device__ constexpr int pitch() { return N + 1; }
// Width g of the d' runs of the V layout: 4 (one 32-byte sector per run; 2 when 4 does not
// divide N).  Narrower 16-byte runs halve pass B's gather traffic but make pass A's TMA store
// issue twice as many half-sector writes, which costs more than it saves (measured at N = 128).
// g = 4 makes each run one 32-byte sector.  N = 256 uses g = 8: its pass A leaves each 128 KB
// output tile by TMA between two uses of the same shared buffer, and the store of 64-byte runs
// drains in half the time (pass B's 8-byte gathers cost about the same either way).
__host__ __device__ constexpr int vgroup_of(int n) { return n == 256 ? 8 : n % 4 == 0 ? 4 : 2; }
template <int N> __host__ __device__ constexpr int vgroup() { return vgroup_of(N); }
// Row of c' along V's c' index.  At N = 128 the eight rows c' = w + 16 i that one pass-A warp
// finishes are adjacent (8 w + i), so that the warp leaves them by one TMA store; other N keep c'.
template <int N> __host__ __device__ constexpr int vrow(int c) { return N == 128 ? 8 * (c & 15) + (c >> 4) : c; }
template <int N> __host__ __device__ constexpr int vrow_inv(int r) { return N == 128 ? 16 * (r & 7) + (r >> 3) : r; }
// offset of V(a, b, c', d') in the V layout
template <int N>
__device__ __forceinline__ size_t v_offset(int ab, int c, int d) {
  constexpr int g = vgroup<N>();
  return (((size_t)(vrow<N>(c) * (N / g) + d / g) * (N * N) + ab) * g) + (d % g);
}

template <int N> __host__ __device__ constexpr size_t pass_a_smem() {
  return (size_t)N * pitch<N>() * sizeof(float2) + N * sizeof(float2) + 2 * N * sizeof(float);
}
template <int N> __host__ __device__ constexpr size_t pass_b_smem() {
  return (size_t)N * pitch<N>() * sizeof(float2) + 2 * N * sizeof(float2) + 4 * 32 * sizeof(double);
}

// ---- bulk asynchronous copies (TMA) issued by one thread, tracked as bulk groups ----
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// Orders this thread's completed async-proxy writes to global memory (bulk / tensor stores)
// before its later generic-proxy operations (a release that publishes them).
__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// wait until every committed bulk copy of this thread has finished reading shared memory
__device__ __forceinline__ void bulk_wait_read_all() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
// wait until every committed bulk copy of this thread is complete
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// tiled 5D tensor store from shared memory (box and layout fixed by the tensor map)
__device__ __forceinline__ void tma_store_5d(const void* tmap, const void* smem, int c0, int c1, int c2,
                                             int c3, int c4) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile(
      "cp.async.bulk.tensor.5d.global.shared::cta.tile.bulk_group [%0, {%2, %3, %4, %5, %6}], [%1];" ::"l"(tmap),
      "r"(s), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4)
      : "memory");
}
// contiguous bulk store of `bytes` (multiple of 16, both addresses 16-byte aligned)
__device__ __forceinline__ void bulk_store(void* gdst, const void* smem, unsigned bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gdst), "r"(s), "r"(bytes)
               : "memory");
}

// Barrier that first lets thread 0 wait for its earlier bulk stores to finish reading shared
// memory: used before a slice's first write into the buffer the previous slice is leaving by TMA.
struct SmemFreeMid {
  __device__ __forceinline__ void operator()() const {
    if (threadIdx.x == 0) bulk_wait_read_all();
    __syncthreads();
  }
};

// In-place shared-memory stages I..IEND-1 along AXIS (0: along the second index, element
// (line, pos) at line*P + pos; 1: along the first index, element (pos, line) at pos*P + line).
template <int N, int SIGN, int AXIS, int I, int IEND, int NT = Plan<N>::NT>
__device__ __forceinline__ void smem_stages(float2* buf, const float2* tw) {
  if constexpr (I < IEND) {
    constexpr int P = pitch<N>();
    constexpr int R = StageInfo<N, I>::R, NS = StageInfo<N, I>::NS;
    auto ld = [buf](int line, int pos) { return AXIS == 0 ? buf[line * P + pos] : buf[pos * P + line]; };
    auto st = [buf](int line, int pos, float2 v) {
      if (AXIS == 0) buf[line * P + pos] = v; else buf[pos * P + line] = v;
    };
    fft_stage<N, R, NS, SIGN, false, NT>(tw, ld, SyncMid{}, st);
    __syncthreads();
    smem_stages<N, SIGN, AXIS, I + 1, IEND, NT>(buf, tw);
  }
}

// Pass A, persistent: CTA blockIdx.x handles point-1 pairs ab = blockIdx.x + k gridDim.x.
// Per slice: generate + DFT along c (lanes along d), DFT along d, write the natural-order slice
// into shared memory and leave it by one TMA tensor store into the V layout (the 5D box
// {2g floats, 1, 1, N/g, N} over (d' mod g, b, a, d'/g, c')).
template <int N, int SRC>
__global__ void __launch_bounds__(Plan<N>::NT, 1) pass_a_kernel(const __grid_constant__ CUtensorMap vmap, PassAArgs p) {
  constexpr bool ARRAY = SRC == SRC_ARRAY, DIAG = SRC == SRC_DIAG;
  constexpr int NT = Plan<N>::NT, P = pitch<N>(), S = Plan<N>::stages;
  extern __shared__ __align__(1024) float2 smem[];
  float2* buf = smem;
  float2* tw = buf + N * P;
  float* gA = reinterpret_cast<float*>(tw + N);
  float* gB = gA + N;
  for (int i = threadIdx.x; i < N; i += NT) tw[i] = p.tw[i];
  const float2* F = p.F;
  for (int ab = blockIdx.x; ab < N * N; ab += gridDim.x) {
    const int a = ab / N, b = ab - a * N;
    if (SRC == SRC_GSM) {
      for (int i = threadIdx.x; i < N; i += NT) {
        gA[i] = p.G[a * N + i];
        gB[i] = p.G[b * N + i];
      }
    }
    __syncthreads();
    float2 s_ab = cconj(__ldg(F + ab));
    if (SRC == SRC_GSM || SRC == SRC_ADJ) s_ab = cscale(s_ab, p.A);
    if (DIAG) s_ab = cscale(s_ab, p.A * __ldg(p.diag + ab));
    const float2* W0 = ARRAY ? p.W0 + (size_t)ab * N * N : nullptr;
    AdjSlice adj{};
    if (SRC == SRC_ADJ) adj = adj_slice(p, ab, N);
    auto gen = [&](int d, int c) -> float2 {
      const float2 f = __ldg(F + c * N + d);
      if (ARRAY) return cmul(cmul(s_ab, __ldg(W0 + c * N + d)), f);
      if (DIAG) return (c * N + d == ab) ? cmul(s_ab, f) : make_float2(0.f, 0.f);
      if (SRC == SRC_ADJ) return cmul(cmul(s_ab, f), adj.at(p.cross, c * N + d));
      return cscale(cmul(s_ab, f), gA[c] * gB[d]);
    };
    auto st1 = [buf](int d, int c, float2 v) { buf[c * P + d] = v; };
    fft_stage<N, StageInfo<N, 0>::R, 1, -1, false, NT>(tw, gen, SmemFreeMid{}, st1);
    __syncthreads();
    smem_stages<N, -1, 1, 1, S>(buf, tw);
    smem_stages<N, -1, 0, 0, S - 1>(buf, tw);
    auto ld0 = [buf](int c, int d) { return buf[c * P + d]; };
    auto nat = [buf](int c, int d, float2 v) { buf[c * N + d] = v; };
    fft_stage<N, StageInfo<N, S - 1>::R, StageInfo<N, S - 1>::NS, -1, true, NT>(tw, ld0, SyncMid{}, nat);
    fence_proxy_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
      tma_store_5d(&vmap, buf, 0, b, a, 0, 0);
      bulk_commit();
    }
  }
  if (threadIdx.x == 0) bulk_wait_all();
}

// Parameter gradients of the amplitude-masked GSM source W0 = A a(x1) a(x2) G(x1, x2) reduced in
// the epilogue of the adjoint propagation's second pass (W_GRAD): the array R it computes gives
// conj(W0bar) = c R ff (ff = q(x1) q*(x2) after a far-field forward propagation, else 1), and per
// output column x2 the kernel adds, over x1, t = Re(R ff) G(x1, x2) a(x1):
//   part[x2][0] = a(x2) d^2 sum t (r^2(x1) + r^2(x2)),  part[x2][1] = a(x2) d^2 sum t |x1 - x2|^2,
//   part[x2][2] = a(x2) sum t  (r^2 and |x1 - x2|^2 in pixels^2),  gmask[x2] = gscale sum t,
// the same per-point sums the standalone gradient kernel forms row by row (R and G symmetric).
struct GradEpi {
  const float* gtab;   // N x N GSM axis factor G(i, k), the same table for both axes
  const float* amask;  // N x N amplitude mask, or nullptr (a = 1)
  const float2* qff;   // far field: q(x_i) per axis (N entries), or nullptr
  double* part;        // N^2 x 3 per-column sums
  float* gmask;        // N^2 mask gradient (4 c A sum t), or nullptr
  float gscale;        // 4 c A
  float d2;            // d^2 of the source grid
};

struct PassBArgs {
  const float2* V;
  const float2* tw;
  const float2* Eout;
  float2* W;
  float* S;
  float scale;
  float2* row;   // optional: row[x] = W(P1, x) (the mu numerator), P1 = (iP, jP); nullptr = none
  int iP, jP;
  GradEpi gr;    // W_GRAD only
};

// What pass B stores of the propagated CSDA: nothing (S and the optional row only), the
// conjugated column as the contiguous row (Hermitian CSDA), every element at its own place, or
// (W_GRAD) nothing but the GSM parameter-gradient sums of the adjoint.
enum WStore { W_NONE = 0, W_HERM = 1, W_GENERAL = 2, W_GRAD = 3 };

// W_GRAD epilogue for one column x2 = (c, d).  With R = Re(W_B conj-factors) the per-point terms
//   t = R G(a, c) G(b, d) m(a, b),  sum t r^2,  sum t |x1 - x2|^2,  sum t
// are separable in a and b: r^2 = (a-M)^2 + (b-M)^2 + (c-M)^2 + (d-M)^2 and |x1 - x2|^2 =
// (a-c)^2 + (b-d)^2, so each point-1 index carries its own G factor, squares and output factor
// (GradAxis), set up once per row / column of the thread; the column's (c-M)^2 + (d-M)^2 enters
// in grad_reduce.  In the far field W_B is also multiplied by q(a) q(b) conj(q(c) q(d)), folded
// into the same factors (grad_col for the column part).
struct GradAxis {
  float g, r, dd;  // G(a, c), (a - M)^2, (a - c)^2
  float2 e;        // output factor of this index (times q(a) in the far field)
};
__device__ __forceinline__ GradAxis grad_axis(const GradEpi& g, int N, int a, int c, float2 e) {
  GradAxis x;
  x.g = __ldg(g.gtab + a * N + c);
  const float m = (float)(a - N / 2), dd = (float)(a - c);
  x.r = m * m;
  x.dd = dd * dd;
  x.e = g.qff ? cmul(e, __ldg(g.qff + a)) : e;
  return x;
}
// the column factor s E(c) E(d) (times conj(q(c) q(d)) in the far field)
__device__ __forceinline__ float2 grad_col(const GradEpi& g, int c, int d, float2 ecd) {
  return g.qff ? cmul(ecd, cconj(cmul(__ldg(g.qff + c), __ldg(g.qff + d)))) : ecd;
}
struct GradSums {
  float sS = 0.f, sM = 0.f, sA = 0.f;  // sS without the column's (c-M)^2 + (d-M)^2 (grad_reduce)
  // transform value y at x1 = (a, b) (axis factors A of a, B of b; m = mask value m(a, b))
  __device__ __forceinline__ void add(const GradAxis& A, const GradAxis& B, float m, float2 y) {
    const float2 e = cmul(A.e, B.e);
    const float t = (e.x * y.x - e.y * y.y) * (A.g * B.g) * m;
    sS = fmaf(t, A.r + B.r, sS);
    sM = fmaf(t, A.dd + B.dd, sM);
    sA += t;
  }
};
__device__ __forceinline__ float grad_mask(const GradEpi& g, int N, int a, int b) {
  return g.amask ? __ldg(g.amask + a * N + b) : 1.f;
}

// Block reduction of the W_GRAD sums of column cd (red: 4 x 32 doubles of shared memory); writes
// part[cd] and gmask[cd].  Every thread of the block must call it.
__device__ __forceinline__ void grad_reduce(const GradEpi& g, int N, int cd, const GradSums& s, double* red) {
  const float a2 = g.amask ? __ldg(g.amask + cd) : 1.f;
  const int c = cd / N, d = cd - c * N;
  const float rc = (float)((c - N / 2) * (c - N / 2) + (d - N / 2) * (d - N / 2));
  const float sS = fmaf(rc, s.sA, s.sS);
  double v[4] = {(double)sS * a2 * g.d2, (double)s.sM * a2 * g.d2, (double)s.sA * a2, (double)s.sA};
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    double x = v[k];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) red[k * 32 + warp] = x;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double x = 0.0;
    for (int w = 0; w < nw; ++w) x += red[threadIdx.x * 32 + w];
    if (threadIdx.x < 3) g.part[(size_t)cd * 3 + threadIdx.x] = x;
    else if (g.gmask) g.gmask[cd] = (float)(g.gscale * x);
  }
  __syncthreads();
}

// Pass B, persistent: CTA blockIdx.x handles point-2 output pairs cd = blockIdx.x + k gridDim.x.
// Per slice: gather V(., ., c', d') + DFT along a (lanes along b), DFT along b with the
// epilogue (scale, output propagators, S on the diagonal, and with ROW the P1 row).  WST = W_HERM:
// the conjugated column is the contiguous row W(c', d', ., .), written to shared memory and left
// by one bulk store; W_GENERAL: strided stores; W_NONE: no store of W.
template <int N, int WST, bool ROW = false>
__global__ void __launch_bounds__(Plan<N>::NT, 1) pass_b_kernel(PassBArgs p) {
  constexpr int NT = Plan<N>::NT, P = pitch<N>(), S = Plan<N>::stages;
  constexpr size_t NN = (size_t)N * N;
  extern __shared__ __align__(1024) float2 smem[];
  float2* buf = smem;
  float2* tw = buf + N * P;
  float2* eo = tw + N;
  double* red = reinterpret_cast<double*>(eo + N);  // W_GRAD: block reduction
  for (int i = threadIdx.x; i < N; i += NT) {
    tw[i] = p.tw[i];
    eo[i] = p.Eout[i];
  }
  // The g columns of one (c', d'/g) share one block of V; the CTA of column j brings part j of the
  // block of its column after next into L2, so that the gathers (8 bytes from every 32-byte run)
  // hit L2 instead of waiting on DRAM (V is larger than L2 from N = 32 on).
  constexpr int g = vgroup<N>();
  auto prefetch = [&](int cdn) {
    if (N >= 32 && threadIdx.x == 0 && cdn < N * N) {
      const int cn = cdn / N, dn = cdn % N;
      bulk_prefetch_l2(p.V + ((size_t)(vrow<N>(cn) * (N / g) + dn / g) * g + dn % g) * NN, (unsigned)(NN * sizeof(float2)));
    }
  };
  prefetch(blockIdx.x);
  prefetch(blockIdx.x + gridDim.x);
  __syncthreads();
  for (int cd = blockIdx.x; cd < N * N; cd += gridDim.x) {
    prefetch(cd + 2 * gridDim.x);
    const int c = cd / N, d = cd - c * N;
    const float2* Vg = p.V + v_offset<N>(0, c, d);
    auto gather = [Vg](int b, int a) { return __ldg(Vg + (size_t)(a * N + b) * vgroup<N>()); };
    auto st1 = [buf](int b, int a, float2 v) { buf[a * P + b] = v; };
    fft_stage<N, StageInfo<N, 0>::R, 1, +1, false, NT>(tw, gather, SmemFreeMid{}, st1);
    __syncthreads();
    smem_stages<N, +1, 1, 1, S>(buf, tw);
    smem_stages<N, +1, 0, 0, S - 1>(buf, tw);
    const float2 ecd = cscale(cmul(eo[c], eo[d]), p.scale);
    float* Sd = p.S;
    auto ld0 = [buf](int a, int b) { return buf[a * P + b]; };
    float2* rw = p.row;
    const int iP = p.iP, jP = p.jP;
    if constexpr (WST == W_HERM) {
      auto epi = [=](int a, int b, float2 y) {
        const float2 w = cmul(cmul(cconj(cmul(eo[a], eo[b])), ecd), y);
        if (a == c && b == d) Sd[cd] = w.x;
        if (ROW && a == iP && b == jP) rw[cd] = w;
        buf[a * N + b] = cconj(w);
      };
      fft_stage<N, StageInfo<N, S - 1>::R, StageInfo<N, S - 1>::NS, +1, true, NT>(tw, ld0, SyncMid{}, epi);
      fence_proxy_async_smem();
      __syncthreads();
      if (threadIdx.x == 0) {
        bulk_store(p.W + (size_t)cd * NN, buf, (unsigned)(NN * sizeof(float2)));
        bulk_commit();
      }
    } else if constexpr (WST == W_GRAD) {
      GradSums gs;
      const GradEpi& ge = p.gr;
      const float2 ecg = grad_col(ge, c, d, ecd);
      auto epi = [&](int a, int b, float2 y) {
        gs.add(grad_axis(ge, N, a, c, cmul(cconj(eo[a]), ecg)), grad_axis(ge, N, b, d, cconj(eo[b])),
               grad_mask(ge, N, a, b), y);
      };
      fft_stage<N, StageInfo<N, S - 1>::R, StageInfo<N, S - 1>::NS, +1, true, NT>(tw, ld0, NoMid{}, epi);
      grad_reduce(ge, N, cd, gs, red);
    } else {
      float2* W = p.W;
      auto epi = [=](int a, int b, float2 y) {
        const float2 w = cmul(cmul(cconj(cmul(eo[a], eo[b])), ecd), y);
        if (a == c && b == d) Sd[cd] = w.x;
        if (ROW && a == iP && b == jP) rw[cd] = w;
        if (WST == W_GENERAL) W[(size_t)(a * N + b) * NN + cd] = w;
      };
      fft_stage<N, StageInfo<N, S - 1>::R, StageInfo<N, S - 1>::NS, +1, true, NT>(tw, ld0, NoMid{}, epi);
    }
  }
  if (threadIdx.x == 0) bulk_wait_all();
}

// S and mu of the current plane (Eq. defS / Algorithm 4, Eq. defMu / Algorithm coherence),
// including masks recorded for this plane (W+ = conj(M0(x1)) W M0(x2)).
struct SMuArgs {
  int N;
  int mode;            // 0: GSM model, 1: CSDA in Wsrc (S from its diagonal), 2: CSDA + S in Sprop,
                       // 3: diagonal source A d(x)
  const float* G;
  float A;
  const float2* M0;    // nullptr = no mask
  const float2* Wsrc;
  const float* Sprop;
  const float* diag;
  int iP, jP;
  float* S_out;        // nullptr = skip
  float2* mu_out;      // nullptr = skip
};

__device__ __forceinline__ float smu_S(const SMuArgs& a, int x) {
  const int N = a.N, i = x / N, j = x - i * N;
  float s;
  if (a.mode == 0) s = a.A * a.G[i * N + i] * a.G[j * N + j];
  else if (a.mode == 3) s = a.A * a.diag[x];
  else if (a.mode == 2) s = a.Sprop[x];
  else s = a.Wsrc[(size_t)x * N * N + x].x;
  if (a.M0) {
    const float2 m = a.M0[x];
    s *= m.x * m.x + m.y * m.y;
  }
  return s;
}

static __global__ void s_mu_kernel(SMuArgs a) {
  const int N = a.N, NN = N * N;
  const int xp = a.iP * N + a.jP;
  const float sp = smu_S(a, xp);
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < NN; x += gridDim.x * blockDim.x) {
    const float sx = smu_S(a, x);
    if (a.S_out) a.S_out[x] = sx;
    if (a.mu_out) {
      const int i = x / N, j = x - i * N;
      float2 w;
      if (a.mode == 0) {
        w = make_float2(a.A * a.G[a.iP * N + i] * a.G[a.jP * N + j], 0.f);
      } else if (a.mode == 3) {
        w = make_float2(x == xp ? a.A * a.diag[x] : 0.f, 0.f);
      } else {
        w = a.Wsrc[(size_t)xp * NN + x];
      }
      if (a.M0) w = cmul(cmul(cconj(a.M0[xp]), a.M0[x]), w);
      const float den = sp * sx;
      a.mu_out[x] = den > 0.f ? cscale(w, rsqrtf(den)) : make_float2(0.f, 0.f);
    }
  }
}

// S and the P1 row of one propagation from V alone, for callers that keep no W (the batch).  Of
// the sign-+1 2D DFT over x1 = (a, b) that pass B runs on column x2 = (c, d), only two outputs are
// used: (a', b') = (c, d) for S and (a', b') = P1 for the mu numerator.  Each is one dot product
//   X(a', b') = sum_{a,b} e^{+2 pi i (a a' + b b') / N} V(a, b; c, d)
// with a separable phase, so V is streamed in its own layout V[c][d/4][a][b][d mod 4]: one block of
// 4 N^2 contiguous values per (c, d/4) (row vrow(c)), four columns, no gather.  The block has one thread per value
// of an a-row (4 N, at most 512; SMU_SLOTS rows' worth otherwise): thread t owns the (b, j) pairs
// k = t + SMU_NT s (j = d mod 4 = t mod 4), sums over a with e^{+2 pi i a c / N} and
// e^{+2 pi i a iP / N}, then applies the b phase, and the block reduces over b.  The epilogue is
// pass B's: W(a', b'; c, d) = s conj(E(a') E(b')) E(c) E(d) X(a', b').
template <int N> __host__ __device__ constexpr int smu_nt() { return 4 * N < 512 ? 4 * N : 512; }

template <int N>
__global__ void __launch_bounds__(smu_nt<N>(), 2048 / smu_nt<N>()) smu_from_v_kernel(PassBArgs p) {
  constexpr int G = 4, ROW = N * G, NT = smu_nt<N>(), SLOTS = ROW / NT, NW = NT / 32, NG = N * N / G;
  static_assert(ROW % NT == 0 && NT % 32 == 0, "a-rows split evenly over the block");
  __shared__ float2 phc[N], php[N];
  __shared__ float2 red[NW][4][2];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5, j = t & 3;
  const bool row = p.row != nullptr;
  for (int q = blockIdx.x; q < NG; q += gridDim.x) {
    const int cr = q / (N / G), dg = q - cr * (N / G), c = vrow_inv<N>(cr);  // block q holds V row cr
    __syncthreads();  // the previous group's tables and partial sums are consumed
    for (int a = t; a < N; a += NT) {
      phc[a] = cconj(__ldg(p.tw + (a * c) % N));
      php[a] = cconj(__ldg(p.tw + (a * p.iP) % N));
    }
    __syncthreads();
    const float2* __restrict__ Vq = p.V + (size_t)q * N * ROW;
    float2 ad[SLOTS], ap[SLOTS];
#pragma unroll
    for (int s = 0; s < SLOTS; ++s) ad[s] = ap[s] = make_float2(0.f, 0.f);
#pragma unroll 8
    for (int a = 0; a < N; ++a) {
      const float2 pc = phc[a], pp = php[a];
#pragma unroll
      for (int s = 0; s < SLOTS; ++s) {
        const float2 v = __ldg(Vq + a * ROW + t + NT * s);
        ad[s] = cadd(ad[s], cmul(pc, v));
        ap[s] = cadd(ap[s], cmul(pp, v));
      }
    }
    float2 sd = make_float2(0.f, 0.f), sp = make_float2(0.f, 0.f);
    const int d = G * dg + j;
#pragma unroll
    for (int s = 0; s < SLOTS; ++s) {
      const int b = (t + NT * s) >> 2;
      sd = cadd(sd, cmul(cconj(__ldg(p.tw + (b * d) % N)), ad[s]));
      sp = cadd(sp, cmul(cconj(__ldg(p.tw + (b * p.jP) % N)), ap[s]));
    }
#pragma unroll
    for (int o = 4; o < 32; o <<= 1) {
      sd.x += __shfl_xor_sync(0xffffffffu, sd.x, o);
      sd.y += __shfl_xor_sync(0xffffffffu, sd.y, o);
      sp.x += __shfl_xor_sync(0xffffffffu, sp.x, o);
      sp.y += __shfl_xor_sync(0xffffffffu, sp.y, o);
    }
    if (lane < 4) {
      red[warp][lane][0] = sd;
      red[warp][lane][1] = sp;
    }
    __syncthreads();
    if (t < 4) {
      float2 xd = make_float2(0.f, 0.f), xp = make_float2(0.f, 0.f);
#pragma unroll
      for (int w = 0; w < NW; ++w) {
        xd = cadd(xd, red[w][t][0]);
        xp = cadd(xp, red[w][t][1]);
      }
      const int dd = G * dg + t, cd = c * N + dd;
      const float2 ecd = cscale(cmul(__ldg(p.Eout + c), __ldg(p.Eout + dd)), p.scale);
      const float2 wd = cmul(cmul(cmul(cconj(__ldg(p.Eout + c)), ecd), cconj(__ldg(p.Eout + dd))), xd);
      p.S[cd] = wd.x;
      if (row) p.row[cd] = cmul(cmul(cmul(cconj(__ldg(p.Eout + p.iP)), ecd), cconj(__ldg(p.Eout + p.jP))), xp);
    }
  }
}

}  // namespace pw
