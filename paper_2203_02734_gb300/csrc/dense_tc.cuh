// dense_tc.cuh -- the dense axis contraction of dense.cuh on the tensor cores (tcgen05.mma,
// kind::f16, BF16 operands split in three, FP32 accumulators in tensor memory), N <= 256.
//
// C[k][j] = scale sum_n A(k, n) B[n][j] as a real GEMM D = X Q^T per tile of 128 columns j:
//   X (128 x 2Np): row = column j, (Re B[n][j], Im B[n][j]) at 2n, 2n + 1 (zero for n >= N);
//   Q (2Np x 2Np): Q(2k, 2n) = Re A, Q(2k, 2n+1) = -Im A, Q(2k+1, 2n) = Im A, Q(2k+1, 2n+1) = Re A;
//   D (128 x 2Np FP32, tensor memory lanes x columns): (Re C[k][j], Im C[k][j]) at 2k, 2k + 1;
// Np = N rounded up to 16.  Both operands are split in three BF16 parts and D accumulates the six
// products of tc16.cuh.  K runs in chunks of 16 complex inputs (32 reals, two MMA K-steps); the
// 2 Np output reals go through one MMA where 2 Np <= 256 (the MMA's N limit), else through two
// halves of Np, so a chunk is 6 x 2 = 12 or 6 x 2 x 2 = 24 MMAs.
//
// Q is split once per propagation by qsplit_kernel into a global buffer laid out chunk by chunk
// in the canonical K-major layout (no swizzle): per chunk, split s and K-step ks, core matrices
// [kb < 2][row group < 2Np / 8] of 8 rows x 16 bytes, so one chunk is 384 Np contiguous bytes and
// arrives by bulk copies into one of two chunk buffers.  The A tile (24 KB) of a chunk is built by
// the 256 converter threads (thread t: column t mod 128, K-step t / 128), in one of ABUF tiles
// (two where they fit, Np <= 224, so that the split of chunk c + 1 overlaps the MMAs of chunk c).
//
// Roles: eight warps split the operand chunks into A tiles and read the result back; one warp
// copies B and issues the MMAs (see axis_tc_kernel for the mbarrier hand-offs).
#pragma once
#include <cuda_bf16.h>
#include <cstdint>

#include "dense.cuh"
#include "tc16.cuh"

namespace pw {
namespace dense_tc {

constexpr int NT = 288;  // 8 converter warps + 1 issuer warp
constexpr int MAX_N = 256;

__host__ __device__ constexpr int npad(int N) { return (N + 15) / 16 * 16; }
__host__ __device__ constexpr size_t chunk_bytes(int N) { return (size_t)384 * npad(N); }
__host__ __device__ constexpr int nchunks(int N) { return npad(N) / 16; }
constexpr uint32_t A_BYTES = 3 * 2 * 4096;  // 3 splits x 2 K-steps x (128 rows x 16 bf16)
__host__ __device__ constexpr size_t smem_bytes(int N, int abuf) { return abuf * A_BYTES + 2 * chunk_bytes(N) + 128; }
constexpr size_t SMEM_MAX = 232448;  // per-CTA dynamic shared memory limit
__host__ __device__ constexpr int a_buffers(int N) { return smem_bytes(N, 2) <= SMEM_MAX ? 2 : 1; }
// Tensor-memory columns to allocate: a power of two >= 32 holding D's 2 Np columns.
__host__ __device__ constexpr uint32_t tmem_cols(int N) {
  return 2 * npad(N) <= 32 ? 32 : 2 * npad(N) <= 64 ? 64 : 2 * npad(N) <= 128 ? 128 : 2 * npad(N) <= 256 ? 256 : 512;
}

// Instruction descriptor: D FP32, A and B BF16, K-major, M = 128, N = n (a multiple of 16 <= 256).
__host__ __device__ constexpr uint32_t idesc(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((128u >> 4) << 24);
}

// Split Q for chunk c: element (row r < 2Np, K index kk < 32 of the chunk) of split s goes to
// chunk c, block (s, ks = kk / 16), core matrix (kb = (kk mod 16) / 8, row group r / 8).
struct QArgs {
  int N;
  const float2* E;  // N x N, row k, column n
  int conj;         // A = conj(E)
  __nv_bfloat16* Q; // nchunks x chunk_bytes
};

__global__ void qsplit_kernel(QArgs a) {
  const int N = a.N, Np = npad(N), R = 2 * Np;
  const int total = nchunks(N) * R * 32;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    const int c = idx / (R * 32), rem = idx - c * R * 32, r = rem / 32, kk = rem - r * 32;
    const int k = r >> 1, cp = r & 1, n = c * 16 + (kk >> 1), cc = kk & 1;
    float v = 0.f;
    if (k < N && n < N) {
      float2 e = a.E[k * N + n];
      if (a.conj) e.y = -e.y;
      v = cp == 0 ? (cc == 0 ? e.x : -e.y) : (cc == 0 ? e.y : e.x);
    }
    const __nv_bfloat16 s1 = __float2bfloat16_rn(v);
    const float r1 = v - __bfloat162float(s1);
    const __nv_bfloat16 s2 = __float2bfloat16_rn(r1);
    const __nv_bfloat16 s3 = __float2bfloat16_rn(r1 - __bfloat162float(s2));
    const int ks = kk >> 4, kb = (kk >> 3) & 1, e8 = kk & 7;
    const size_t block = (size_t)64 * Np;  // bytes of one (split, K-step) block
    const size_t off = (size_t)c * chunk_bytes(N) + (size_t)ks * block +
                       (size_t)((kb * (R / 8) + (r >> 3)) * 128 + (r & 7) * 16 + e8 * 2);
    unsigned char* base = reinterpret_cast<unsigned char*>(a.Q);
    *reinterpret_cast<__nv_bfloat16*>(base + off) = s1;
    *reinterpret_cast<__nv_bfloat16*>(base + off + 2 * block) = s2;
    *reinterpret_cast<__nv_bfloat16*>(base + off + 4 * block) = s3;
  }
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(mbar))
               : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mma_np(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile("{.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
               "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;}" ::"r"(d),
               "l"(a), "l"(b), "r"(id), "r"(acc));
}

__device__ __forceinline__ void tmem_ld16(float (&r)[16], uint32_t taddr) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=f"(r[0]), "=f"(r[1]), "=f"(r[2]), "=f"(r[3]), "=f"(r[4]), "=f"(r[5]), "=f"(r[6]), "=f"(r[7]), "=f"(r[8]),
        "=f"(r[9]), "=f"(r[10]), "=f"(r[11]), "=f"(r[12]), "=f"(r[13]), "=f"(r[14]), "=f"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// One tile of 128 columns j per CTA (grid = ceil(N^3 / 128)), NT = 288 threads: warps 0-7 split
// the operand (thread t < 256: column t mod 128, K-step t / 128) and read the result back, warp 8
// (one lane) copies B and issues the MMAs.  No block-wide barrier inside the chunk loop: the roles
// hand off through mbarriers -- afull[b] (8 warp arrivals: A tile b is written), bfull[b] (bytes
// of B buffer b have landed), mdone[b] (tcgen05.commit: the MMAs of the last chunk with parity b
// have completed, so its A tile and B buffer are free).  A tile c mod ABUF holds chunk c, its
// (c / ABUF)-th fill; no barrier can run two phases ahead of a wait on it (each next fill depends
// on the completion being waited for).  Every wait is bounded; a wait that gives up sets the
// shared abort flag and *err, after which no role waits again, and the tile's outputs are not
// written.
template <bool S_OUT, int ABUF>
__global__ void __launch_bounds__(NT, 1) axis_tc_kernel(dense::AxisArgs p, const unsigned char* __restrict__ Q,
                                                         int* err) {
  extern __shared__ __align__(1024) unsigned char sm[];
  const int N = p.N, Np = npad(N), nch = nchunks(N);
  const uint32_t cb = (uint32_t)chunk_bytes(N);
  unsigned char* As0 = sm;
  unsigned char* Bs0 = sm + ABUF * A_BYTES;
  uint64_t* bfull = reinterpret_cast<uint64_t*>(sm + ABUF * A_BYTES + 2 * cb);  // [2]
  uint64_t* mdone = bfull + 2;                                                 // [2]
  uint64_t* afull = bfull + 4;                                                 // [2]
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bfull + 6);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
  volatile int* committed = abort_flag + 1;  // the last chunk whose MMAs the issuer committed
  // Issuer lane only: chunks whose B copies were started (bit c) and whose bfull wait completed
  // (bit c); on an abort, copies still in flight are drained before the CTA exits.
  uint32_t b_issued = 0, b_landed = 0;
  const int t = threadIdx.x, w = t >> 5, m = t & 127, ks = (t >> 7) & 1;
  const long long L = p.L, ncols = p.ncols;
  const long long j = (long long)blockIdx.x * 128 + m;
  const long long jb = (t < 256 && j < ncols) ? dense::col_base(j, L, N) : -1;
  // gen (L = 1, column j = (a N + b) N + c): W0(a, b, c, n) = [A conj M0(a, b) G(a, c)] M0(c, n) G(b, n)
  float2 gcol = make_float2(0.f, 0.f);
  const float2* gm = nullptr;
  const float* gg = nullptr;
  if (p.gen && jb >= 0) {
    const int c = (int)(j % N), b = (int)((j / N) % N), a = (int)(j / ((long long)N * N));
    gcol = cscale(cconj(__ldg(p.M0 + a * N + b)), p.A * __ldg(p.G + a * N + c));
    gm = p.M0 + c * N;
    gg = p.G + b * N;
  }

  if (w == 0) tc16::tmem_alloc(tslot, tmem_cols(N));
  if (t == 0) {
    for (int b = 0; b < 2; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bfull[b])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mdone[b])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 8;" ::"r"(smem_u32(&afull[b])));
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *abort_flag = 0;
    *committed = -1;
  }
  tc16::fence_before_sync();
  __syncthreads();
  tc16::fence_after_sync();
  const uint32_t tmem = *tslot;
  auto fail_now = [&]() {
    *abort_flag = 1;
    atomicExch(err, 1);
  };
  // bounded wait that also gives up at once when another role has aborted
  auto wait = [&](uint64_t* bar, uint32_t parity) -> bool {
    if (*abort_flag) return false;
    if (tc16::mbar_wait(bar, parity)) return true;
    fail_now();
    return false;
  };

  if (w == 8) {
    // ---- the issuer: B copies and MMAs, one lane
    if ((t & 31) == 0) {
      // 2 Np output reals in one MMA where they fit its N (<= 256), else two halves of Np
      const int halves = 2 * Np <= 256 ? 1 : 2;
      const int nh = 2 * Np / halves;
      const uint32_t id = idesc(nh);
      auto load_chunk = [&](int c) {
        if (p.stall > 0 && c == p.stall && blockIdx.x == 0) return;  // injected: this phase never completes
        b_issued |= 1u << c;
        unsigned char* dst = Bs0 + (c & 1) * cb;
        const unsigned char* src = Q + (size_t)c * cb;
        mbar_expect_tx(&bfull[c & 1], cb);
        const uint32_t piece = cb / 4;  // 96 Np bytes, a multiple of 16
        for (int q = 0; q < 4; ++q) bulk_g2s(dst + q * piece, src + (size_t)q * piece, piece, &bfull[c & 1]);
      };
      load_chunk(0);
      if (nch > 1) load_chunk(1);
      constexpr int ti[6] = {0, 0, 1, 0, 1, 2}, tj[6] = {0, 1, 0, 2, 1, 0};
      const uint32_t blk = (uint32_t)(64 * Np);
      for (int c = 0; c < nch; ++c) {
        if (!wait(&afull[c % ABUF], (uint32_t)((c / ABUF) & 1))) break;
        if (!wait(&bfull[c & 1], (uint32_t)((c >> 1) & 1))) break;
        b_landed |= 1u << c;
        tc16::fence_after_sync();
        const uint64_t a0 = tc16::sdesc(smem_u32(As0 + (c % ABUF) * A_BYTES), 2048, 128);
        const uint64_t b0 = tc16::sdesc(smem_u32(Bs0 + (c & 1) * cb), (uint32_t)(32 * Np), 128);
#pragma unroll
        for (int q = 0; q < 6; ++q)
#pragma unroll
          for (int s2 = 0; s2 < 2; ++s2)
#pragma unroll
            for (int h = 0; h < halves; ++h) {
              const uint64_t ad = a0 + (uint64_t)((ti[q] * 8192 + s2 * 4096) >> 4);
              const uint64_t bd = b0 + (uint64_t)(((tj[q] * 2 + s2) * blk + h * (nh / 8) * 128) >> 4);
              mma_np(tmem + (uint32_t)(h * nh), ad, bd, id, (c | q | s2) ? 1u : 0u);
            }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&mdone[c & 1]))
                     : "memory");
        *committed = c;
        // B buffer (c + 1) & 1 last held chunk c - 1: refill it once those MMAs are done
        if (c >= 1 && c + 1 < nch) {
          if (!wait(&mdone[(c - 1) & 1], (uint32_t)(((c - 1) >> 1) & 1))) break;
          load_chunk(c + 1);
        }
      }
    }
  } else {
    // ---- the converters: split the operand chunk by chunk, then read the result back
    for (int c = 0; c < nch; ++c) {
      float2 x[8];  // the thread's 8 inputs n = 16 c + 8 ks + i of column j
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int n = 16 * c + 8 * ks + i;
        x[i] = (jb >= 0 && n < N) ? (gm ? cscale(cmul(gcol, __ldg(gm + n)), __ldg(gg + n)) : p.in[jb + (long long)n * L])
                                  : make_float2(0.f, 0.f);
      }
      if (c >= ABUF) {  // A tile c mod ABUF last held chunk c - ABUF
        const int pc = c - ABUF;
        bool ok = true;
        if ((t & 31) == 0) ok = wait(&mdone[pc & 1], (uint32_t)((pc >> 1) & 1));
        ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
        if (!ok) break;
      }
      unsigned char* As = As0 + (c % ABUF) * A_BYTES;
#pragma unroll
      for (int kb = 0; kb < 2; ++kb) {
        uint32_t wv[3][4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float2 v = x[4 * kb + q];
          const __nv_bfloat162 h1 = __floats2bfloat162_rn(v.x, v.y);
          const float rx = v.x - __low2float(h1), ry = v.y - __high2float(h1);
          const __nv_bfloat162 h2 = __floats2bfloat162_rn(rx, ry);
          const __nv_bfloat162 h3 = __floats2bfloat162_rn(rx - __low2float(h2), ry - __high2float(h2));
          wv[0][q] = tc16::bf2_bits(h1);
          wv[1][q] = tc16::bf2_bits(h2);
          wv[2][q] = tc16::bf2_bits(h3);
        }
#pragma unroll
        for (int sp = 0; sp < 3; ++sp)
          *reinterpret_cast<uint4*>(As + sp * 8192 + ks * 4096 + (kb * 16 + (m >> 3)) * 128 + (m & 7) * 16) =
              make_uint4(wv[sp][0], wv[sp][1], wv[sp][2], wv[sp][3]);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      // injected (p.stall < 0): CTA 0 never announces A tile -p.stall, so the issuer's wait gives up
      // while the B copy of that chunk may still be in flight
      const bool skip = p.stall < 0 && c == -p.stall && blockIdx.x == 0;
      if ((t & 31) == 0 && !skip)
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&afull[c % ABUF])) : "memory");
    }
    // the last chunk's MMAs complete after all earlier ones
    bool ok = true;
    if ((t & 31) == 0) ok = wait(&mdone[(nch - 1) & 1], (uint32_t)(((nch - 1) >> 1) & 1));
    ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
    tc16::fence_after_sync();
    if (ok && !*abort_flag) {
      // warp w reads lanes 32 (w mod 4) .. + 31 (columns j) of output half w / 4
      const int h = w >> 2;
      const long long NN = (long long)N * N;
      for (int q = 0; q < Np / 16; ++q) {  // 16 columns (8 complex outputs) per load, Np per half
        float r[16];
        tmem_ld16(r, tmem + ((uint32_t)(32 * (w & 3)) << 16) + (uint32_t)(h * Np + 16 * q));
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int k = (h * Np + 16 * q) / 2 + i;
          if (jb >= 0 && k < N) {
            const float2 v = make_float2(r[2 * i] * p.scale, r[2 * i + 1] * p.scale);
            p.out[jb + (long long)k * L] = v;
            if (S_OUT) {
              const int b = (int)(j / NN), cc = (int)((j / N) % N), d = (int)(j % N);
              if (cc == k && d == b) p.S[k * N + b] = v.x;
            }
          }
        }
      }
    }
  }
  tc16::fence_before_sync();
  __syncthreads();
  if (w == 8 && (t & 31) == 0 && *abort_flag) {
    // no MMA may still write tensor memory when it is freed: the last commit covers all (bounded)
    if (*committed >= 0) {
      const int lc = *committed;
      tc16::mbar_wait(&mdone[lc & 1], (uint32_t)((lc >> 1) & 1));
    }
    // no bulk copy may still write shared memory when the CTA exits: wait (bounded) for every B
    // copy that was started and not yet seen complete; at most one is outstanding per buffer
    for (int c = 0; c < nch; ++c)
      if ((b_issued >> c) & 1u && !((b_landed >> c) & 1u)) tc16::mbar_wait(&bfull[c & 1], (uint32_t)((c >> 1) & 1));
  }
  __syncthreads();
  tc16::fence_after_sync();
  if (w == 0) tc16::tmem_dealloc(tmem, tmem_cols(N));
}

}  // namespace dense_tc
}  // namespace pw
