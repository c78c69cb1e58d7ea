// tc16.cuh -- a radix-16 DFT stage on the fifth-generation tensor cores (tcgen05.mma, kind::f16,
// BF16 operands, FP32 accumulators in tensor memory), with split-BF16x3 operands for FP32-level
// accuracy.  Used by the N = 256 pass A as its first stage when a handle asks for it.
//
// One stage transforms a batch of length-16 complex vectors X (one vector per row) by the
// 16 x 16 DFT matrix F(n', j) = exp(SIGN 2 pi i n' j / 16) as a real GEMM, D = A B^T:
//   A (vectors x 32): row m = (Re X0, Im X0, Re X1, Im X1, ..., Im X15)  (k = 2 j + c);
//   B (32 x 32): row n = 2 n' + c' holds Re Y(n') (c' = 0) or Im Y(n') (c' = 1) as a function of
//     k:  B(2n', 2j) = Re F, B(2n', 2j+1) = -Im F, B(2n'+1, 2j) = Im F, B(2n'+1, 2j+1) = Re F;
//   D (vectors x 32 FP32, in tensor memory): row m = (Re Y0, Im Y0, ..., Im Y15).
// Each FP32 operand x is split into three BF16 parts x = x1 + x2 + x3 (x1 = bf16(x),
// x2 = bf16(x - x1), x3 = bf16(x - x1 - x2)), and D accumulates the six products Ai Bj with
// i + j <= 4 (1-based): A1B1 + A1B2 + A2B1 + A1B3 + A2B2 + A3B1.  The dropped terms are below
// 2^-24 relative; the FP32 accumulation rounds like the CUDA-core codelet.
//
// Shared-memory operands use the canonical K-major layout without swizzle: 8-row x 16-byte core
// matrices of 128 contiguous bytes, core matrices adjacent in K 2048 bytes apart (A tile of 128
// rows) or 512 bytes apart (B, 32 rows), adjacent in M/N 128 bytes apart.  One MMA instruction
// covers M = 128, N = 32, K = 16, so one tile of 128 vectors takes 6 products x 2 K-steps = 12
// instructions.  Tensor memory holds a tile's D in 32 columns x 128 lanes; warp w may read lanes
// 32 (w mod 4) .. 32 (w mod 4) + 31, so thread t of a 256-thread CTA owns vector t (tile t / 128,
// lane t mod 128).
#pragma once
#include <cuda_bf16.h>
#include <cstdint>
#include "cluster.cuh"

namespace pw {
namespace tc16 {

constexpr uint32_t A_SPLIT_BYTES = 128 * 32 * 2;  // one split of one 128-vector tile
constexpr uint32_t B_SPLIT_BYTES = 32 * 32 * 2;
constexpr uint32_t B_BYTES = 3 * B_SPLIT_BYTES;

// Instruction descriptor of kind::f16: D FP32 (bits 4-5 = 1), A and B BF16 (bits 7-9, 10-12 = 1),
// both K-major (bits 15, 16 = 0), N >> 3 in bits 17-22, M >> 4 in bits 24-28.
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);

// Shared-memory matrix descriptor: start address >> 4 (bits 0-13), leading-dimension (K) byte
// offset >> 4 (bits 16-29), stride-dimension (M/N) byte offset >> 4 (bits 32-45), descriptor
// version 1 (bits 46-47), base offset 0, no swizzle (bits 61-63 = 0).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
         (1ull << 46);
}

// Byte offset of the 16-byte chunk (row m, k-block kb = k / 8) in a 128-row tile, and in B.
__device__ __forceinline__ uint32_t a_chunk(int m, int kb) { return (uint32_t)((kb * 16 + (m >> 3)) * 128 + (m & 7) * 16); }
__device__ __forceinline__ uint32_t b_off(int n, int k) {
  return (uint32_t)(((k >> 3) * 4 + (n >> 3)) * 128 + (n & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {  // one whole warp
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {  // one whole warp
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}
__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint64_t* mbar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)));
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Before the mbarrier's memory is used for anything else.
__device__ __forceinline__ void mbar_inval(uint64_t* mbar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(mbar)) : "memory");
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait for the completion of phase `parity`: gives up (false) after about a second of
// wall-clock time (or 2^24 polls), so that a phase that never completes ends the kernel with an
// error flag instead of a hang.
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity) {
  uint32_t done = 0;
  const uint64_t t0 = global_ns();
  for (int it = 0; it < (1 << 24) && !done; ++it) {
    asm volatile("{.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;}"
                 : "=r"(done)
                 : "r"(smem_u32(mbar)), "r"(parity)
                 : "memory");
    if (!done && (it & 255) == 255 && global_ns() - t0 > 1000000000ull) break;
  }
  return done != 0;
}

// B of the sign-SIGN DFT-16, split in three, from tw[m] = exp(-2 pi i m / 256) (FP64-derived).
template <int SIGN>
__device__ __forceinline__ void build_b(unsigned char* B, const float2* __restrict__ tw, int t, int nthreads) {
  for (int e = t; e < 32 * 32; e += nthreads) {
    const int n = e >> 5, k = e & 31, np = n >> 1, j = k >> 1;
    float2 f = tw[16 * ((np * j) & 15)];
    if (SIGN > 0) f.y = -f.y;
    const float v = (n & 1) == 0 ? ((k & 1) == 0 ? f.x : -f.y) : ((k & 1) == 0 ? f.y : f.x);
    const __nv_bfloat16 s1 = __float2bfloat16_rn(v);
    const float r1 = v - __bfloat162float(s1);
    const __nv_bfloat16 s2 = __float2bfloat16_rn(r1);
    const __nv_bfloat16 s3 = __float2bfloat16_rn(r1 - __bfloat162float(s2));
    *reinterpret_cast<__nv_bfloat16*>(B + b_off(n, k)) = s1;
    *reinterpret_cast<__nv_bfloat16*>(B + B_SPLIT_BYTES + b_off(n, k)) = s2;
    *reinterpret_cast<__nv_bfloat16*>(B + 2 * B_SPLIT_BYTES + b_off(n, k)) = s3;
  }
}

__device__ __forceinline__ uint32_t bf2_bits(__nv_bfloat162 h) { return *reinterpret_cast<uint32_t*>(&h); }

// Split the vector x (16 complex) into three BF16 parts and store them as row m of tile `tile`
// of the A staging area (split i of tile T at A + (i * ntiles + T) * A_SPLIT_BYTES).
__device__ __forceinline__ void stage_row(unsigned char* A, int ntiles, int tile, int m, const float2 (&x)[16]) {
#pragma unroll
  for (int kb = 0; kb < 4; ++kb) {
    uint32_t w[3][4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float2 v = x[4 * kb + q];
      const __nv_bfloat162 h1 = __floats2bfloat162_rn(v.x, v.y);
      const float rx = v.x - __low2float(h1), ry = v.y - __high2float(h1);
      const __nv_bfloat162 h2 = __floats2bfloat162_rn(rx, ry);
      const __nv_bfloat162 h3 = __floats2bfloat162_rn(rx - __low2float(h2), ry - __high2float(h2));
      w[0][q] = bf2_bits(h1);
      w[1][q] = bf2_bits(h2);
      w[2][q] = bf2_bits(h3);
    }
#pragma unroll
    for (int i = 0; i < 3; ++i)
      *reinterpret_cast<uint4*>(A + (i * ntiles + tile) * A_SPLIT_BYTES + a_chunk(m, kb)) =
          make_uint4(w[i][0], w[i][1], w[i][2], w[i][3]);
  }
}

__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile("{.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
               "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;}" ::"r"(d),
               "l"(a), "l"(b), "r"(IDESC), "r"(acc));
}

// One thread: the 12 MMAs of each of the ntiles tiles (D of tile T at tensor-memory column
// dcol + 32 T), then one commit that arrives on mbar when they have completed.
template <int NTILES>
__device__ __forceinline__ void issue(uint32_t tmem, uint32_t dcol, const unsigned char* A, const unsigned char* B,
                                      uint64_t* mbar) {
  constexpr int ti[6] = {0, 0, 1, 0, 1, 2}, tj[6] = {0, 1, 0, 2, 1, 0};
  // The address field is the low 14 bits (16-byte units): operands at fixed offsets from one base
  // descriptor differ only by offset / 16 (no carry out of the field for a 256 KB window).
  const uint64_t a0 = sdesc(smem_u32(A), 2048, 128), b0 = sdesc(smem_u32(B), 512, 128);
  // Tiles innermost: consecutive MMAs go to independent accumulators.
#pragma unroll
  for (int q = 0; q < 6; ++q)
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int T = 0; T < NTILES; ++T)
        mma(tmem + dcol + 32 * T, a0 + (((ti[q] * NTILES + T) * A_SPLIT_BYTES + 2 * s * 2048) >> 4),
            b0 + ((tj[q] * B_SPLIT_BYTES + 2 * s * 512) >> 4), (q | s) ? 1u : 0u);
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar))
               : "memory");
}

// The calling warp's 32 lanes of one tile: 32 FP32 columns from tensor-memory address taddr.
__device__ __forceinline__ void load_row(float2 (&y)[16], uint32_t taddr) {
  float r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=f"(r[0]), "=f"(r[1]), "=f"(r[2]), "=f"(r[3]), "=f"(r[4]), "=f"(r[5]), "=f"(r[6]), "=f"(r[7]), "=f"(r[8]),
        "=f"(r[9]), "=f"(r[10]), "=f"(r[11]), "=f"(r[12]), "=f"(r[13]), "=f"(r[14]), "=f"(r[15]), "=f"(r[16]),
        "=f"(r[17]), "=f"(r[18]), "=f"(r[19]), "=f"(r[20]), "=f"(r[21]), "=f"(r[22]), "=f"(r[23]), "=f"(r[24]),
        "=f"(r[25]), "=f"(r[26]), "=f"(r[27]), "=f"(r[28]), "=f"(r[29]), "=f"(r[30]), "=f"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) y[i] = make_float2(r[2 * i], r[2 * i + 1]);
}

}  // namespace tc16
}  // namespace pw
