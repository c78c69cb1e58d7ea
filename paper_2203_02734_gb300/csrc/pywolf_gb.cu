// pywolf_gb.cu -- C ABI of include/pywolf_gb.h: handle state, argument checks, FP64 table
// set-up and the launch sequence of one propagation (tables -> pass A -> pass B).
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/pywolf_gb.h"
#include "propagate.cuh"
#include "d256.cuh"
#include "dense.cuh"
#include "dense_tc.cuh"
#include "t256.cuh"
#include "grad.cuh"
#include "r128.cuh"
#include "r96.cuh"

namespace {

thread_local std::string g_err;

pw_status fail(pw_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

pw_status cuda_fail(cudaError_t e, const char* what) {
  cudaGetLastError();  // clear a sticky launch error so the next call starts clean
  return fail(PW_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

// Device pointers are dereferenced as 16-byte bulk / tensor copies (the CSDA buffers), 8-byte
// complex values (masks, uploaded arrays, mu) or floats (S, diagonals).
bool aligned(const void* p, size_t a) { return reinterpret_cast<uintptr_t>(p) % a == 0; }

// SRC_ADJOINT: the adjoint source of a loss on S and mu, set only inside the adjoint calls.
enum SourceKind { SRC_NONE = 0, SRC_GSM = 1, SRC_ARRAY = 2, SRC_PROPAGATED = 3, SRC_DIAGONAL = 4, SRC_ADJOINT = 5 };

}  // namespace

namespace pwi {
// Sets the thread's message returned by pw_last_error() (used by other translation units).
void set_last_error(const char* msg) { g_err = msg; }
pw_status encode_vmap(CUtensorMap* map, void* work, int N);
cudaError_t launch_batch_instance(int N, const CUtensorMap& vmap, const pw::PassAArgs& a, const pw::PassBArgs& b,
                                  const float2* Ein, const float2* mask, int ap_ithr, cudaStream_t s);
}  // namespace pwi

struct pw_csd {
  int N;
  double d;       // sampling of the current plane
  double lambda;
  pw_c32* W;
  pw_c32* work;
  cudaStream_t stream;
  // source of the current plane
  SourceKind kind;
  double sigma_S, sigma_mu, A;
  const pw_c32* W0;
  const float* diag;  // diagonal source values (SRC_DIAGONAL)
  int hermitian;
  // masks of the current plane
  double aperture;  // <= 0: none
  double lens_f;    // 0: none
  const pw_c32* mask;
  // small device tables (one allocation)
  void* tables;
  float2* F;
  float2* M0;
  float* G;
  float2* tw;
  float2* Eout;
  float2* Ein;    // per-axis input factors
  float* S;       // S of the last propagated plane (pass-B epilogue)
  int* err;       // device flag: a bounded wait in a kernel gave up
  // adjoint scratch (O(N^2)): the adjoint source (diagonal, P1 row), per-column gradient sums, the
  // GSM factor and far-field factors of the source grid, and a spare gradient triple
  float* adj_d;
  float2* adj_c;
  double* gpart;
  float* gtab;
  float2* qtab;
  double* g3tmp;
  // the adjoint source of the next propagation (kind == SRC_ADJOINT)
  int adj_herm;     // Hermitian part (row and column of P1) or the general array (row only)
  int adj_mu;       // the source has a P1 row (a mu term)
  int adj_iP, adj_jP;
  const pw::GradEpi* adj_grad;  // non-null: reduce the GSM parameter gradients in pass B (W_GRAD)
  CUtensorMap vmap;  // TMA map of the work buffer in the V layout
  CUtensorMap ymap;  // N = 256: the second pass's tiles of the work buffer
  CUtensorMap y3map;  // N = 256: the third pass's tiles of the work buffer
  CUtensorMap y1map;  // N = 256: the first pass's stores (four rows per warp) into the work buffer
  int dft_mode;      // PW_DFT_AUTO, PW_DFT_FP32 or PW_DFT_TC_BF16X3
  int Nz;            // zero padding: transform size (0 = none); the dense path runs when set
  void* qbuf;        // split DFT matrices of the tensor-core dense path (allocated on first use)
  int stall;         // failure-detection test: chunk whose copy CTA 0 leaves out, next dense TC run only
  // optional per-pass timing: 4 events per recorded propagation (before the first pass, after it,
  // after the last, and between the second and third passes of the N = 256 engine)
  std::vector<cudaEvent_t> events;
  std::vector<char> three;  // per recorded propagation: the middle event was recorded
  int timed;
};

namespace {

bool supported(int N) {
  switch (N) {
    case 2: case 4: case 6: case 8: case 12: case 16: case 24: case 32: case 48: case 64:
    case 96: case 128: case 256:
      return true;
    default:
      return false;
  }
}

size_t table_bytes(int N) {
  const size_t NN = (size_t)N * N;
  const size_t base = NN * sizeof(float2) * 2 + NN * sizeof(float) * 2 + (size_t)N * sizeof(float2) * 3 + 1024 + 256;
  const size_t adj = NN * (sizeof(float) + sizeof(float2) + 3 * sizeof(double) + sizeof(float)) +
                     (size_t)N * sizeof(float2) + 3 * sizeof(double) + 6 * 256;
  return base + adj;
}

int num_sms() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

// Persistent grid: as many CTAs as fit on the device at once, at most one per slice.
template <class K>
cudaError_t persistent_grid(K kernel, int threads, size_t smem, int slices, int* grid) {
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  const long g = (long)per_sm * num_sms();
  *grid = (int)(g < slices ? g : slices);
  return cudaSuccess;
}

template <int N, int SRC>
cudaError_t launch_a(const CUtensorMap& vmap, const pw::PassAArgs& a, cudaStream_t s) {
  constexpr size_t smem = pw::pass_a_smem<N>();
  static int grid = 0;
  if (grid == 0) {
    cudaError_t e = cudaFuncSetAttribute(pw::pass_a_kernel<N, SRC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = persistent_grid(pw::pass_a_kernel<N, SRC>, pw::Plan<N>::NT, smem, N * N, &grid);
    if (e != cudaSuccess) return e;
  }
  pw::pass_a_kernel<N, SRC><<<grid, pw::Plan<N>::NT, smem, s>>>(vmap, a);
  return cudaGetLastError();
}

// N = 128: register-resident pass A (r128.cuh).
struct R128Extra {
  const float2* Ein;
  const float2* mask;
  int ap_ithr;
  int* err;
  int dft_tc;  // N = 256: first stage of the first pass on the tensor cores
};

template <int SRC, bool MASK>
cudaError_t launch_a_r128(const CUtensorMap& vmap, const pw::PassAArgs& a, const R128Extra& x, cudaStream_t s) {
  constexpr size_t smem = pw::r128::pass_a_smem();
  static int grid = 0;
  if (grid == 0) {
    cudaError_t e = cudaFuncSetAttribute(pw::r128::pass_a_r128<SRC, MASK>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = persistent_grid(pw::r128::pass_a_r128<SRC, MASK>, pw::r128::NT, smem, 128 * 128, &grid);
    if (e != cudaSuccess) return e;
  }
  pw::r128::pass_a_r128<SRC, MASK><<<grid, pw::r128::NT, smem, s>>>(vmap, a, x.Ein, x.mask, x.ap_ithr);
  return cudaGetLastError();
}

// N = 128, Hermitian store or none: register-resident pass B with prefetched gather (r128.cuh).
template <int WST, bool ROW = false>
cudaError_t launch_b_r128(const pw::PassBArgs& b, cudaStream_t s) {
  constexpr size_t smem = pw::r128::pass_b_smem();
  static int grid = 0;
  if (grid == 0) {
    cudaError_t e = cudaFuncSetAttribute(pw::r128::pass_b_r128<WST, ROW>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = persistent_grid(pw::r128::pass_b_r128<WST, ROW>, pw::r128::NT, smem, 128 * 128, &grid);
    if (e != cudaSuccess) return e;
  }
  pw::r128::pass_b_r128<WST, ROW><<<grid, pw::r128::NT, smem, s>>>(b);
  return cudaGetLastError();
}

// N = 96: register-resident passes (r96.cuh), two CTAs per SM.
template <int SRC, bool MASK>
cudaError_t launch_a_r96(const CUtensorMap& vmap, const pw::PassAArgs& a, const R128Extra& x, cudaStream_t s) {
  constexpr size_t smem = pw::r96::pass_a_smem();
  static int grid = 0;
  if (grid == 0) {
    cudaError_t e = cudaFuncSetAttribute(pw::r96::pass_a_r96<SRC, MASK>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = persistent_grid(pw::r96::pass_a_r96<SRC, MASK>, pw::r96::NT, smem, 96 * 96, &grid);
    if (e != cudaSuccess) return e;
  }
  pw::r96::pass_a_r96<SRC, MASK><<<grid, pw::r96::NT, smem, s>>>(vmap, a, x.Ein, x.mask, x.ap_ithr);
  return cudaGetLastError();
}

template <int WST, bool ROW = false>
cudaError_t launch_b_r96(const pw::PassBArgs& b, cudaStream_t s) {
  constexpr size_t smem = pw::r96::pass_b_smem();
  static int grid = 0;
  if (grid == 0) {
    cudaError_t e = cudaFuncSetAttribute(pw::r96::pass_b_r96<WST, ROW>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = persistent_grid(pw::r96::pass_b_r96<WST, ROW>, pw::r96::NT, smem, 96 * 96, &grid);
    if (e != cudaSuccess) return e;
  }
  pw::r96::pass_b_r96<WST, ROW><<<grid, pw::r96::NT, smem, s>>>(b);
  return cudaGetLastError();
}

// Number of CTAs of the largest grid of `cs`-CTA clusters of `kernel` that can be co-resident.
template <class K>
cudaError_t cluster_capacity(K kernel, int cs, int threads, size_t smem, int* grid) {
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cfg.gridDim = dim3(cs * num_sms());
  int nclusters = 0;
  e = cudaOccupancyMaxActiveClusters(&nclusters, kernel, &cfg);
  if (e != cudaSuccess) return e;
  if (nclusters < 1) return cudaErrorInvalidConfiguration;
  *grid = nclusters * cs;
  return cudaSuccess;
}

// Persistent launch of a kernel compiled for clusters of `cs` CTAs: as many clusters as can be
// co-resident (queried once per kernel, unless *grid is already set).
template <class K, class... Args>
cudaError_t launch_clusters(K kernel, int cs, int threads, size_t smem, int* grid, cudaStream_t s, Args... args) {
  if (*grid == 0) {
    cudaError_t e = cluster_capacity(kernel, cs, threads, smem, grid);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cfg.gridDim = dim3(*grid);
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

template <int SRC, bool MASK, bool TC = false>
cudaError_t launch_a_d256(const CUtensorMap& vmap, const pw::PassAArgs& a, const R128Extra& x, cudaStream_t s) {
  static int grid = 0;
  constexpr int CS = pw::d256::CLUSTER_A;
  if (TC && grid == 0) {
    // The occupancy calculator fits one CTA per SM for a kernel that uses tensor memory (15
    // clusters of 8 instead of 36, measured). This one allocates 128 of an SM's 512 columns and
    // has the registers, threads and shared memory of its FP32 twin, which caps residency at two
    // CTAs per SM, so it takes the twin's grid (two per SM co-resident, measured: 53.8 -> 32.3 ms).
    cudaError_t e = cudaFuncSetAttribute(pw::d256::pass_a_d256<CS, SRC, MASK, TC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pw::d256::pass_a_smem<CS>());
    if (e != cudaSuccess) return e;
    e = cluster_capacity(pw::d256::pass_a_d256<CS, SRC, MASK, false>, CS, pw::d256::Geo<CS>::NT,
                         pw::d256::pass_a_smem<CS>(), &grid);
    if (e != cudaSuccess) return e;
  }
  return launch_clusters(pw::d256::pass_a_d256<CS, SRC, MASK, TC>, CS, pw::d256::Geo<CS>::NT,
                         pw::d256::pass_a_smem<CS>(), &grid, s, vmap, a, x.Ein, x.mask, x.ap_ithr, x.err);
}

cudaError_t launch_b_d256(const pw::PassBArgs& b, cudaStream_t s) {
  static int grid = 0;
  constexpr int CS = pw::d256::CLUSTER_B;
  return launch_clusters(pw::d256::pass_b_d256<CS>, CS, pw::d256::Geo<CS>::NT, pw::d256::pass_b_smem<CS>(), &grid,
                         s, b);
}

template <int N, int WST, bool ROW = false>
cudaError_t launch_b(const pw::PassBArgs& b, cudaStream_t s) {
  constexpr size_t smem = pw::pass_b_smem<N>();
  static int grid = 0;
  if (grid == 0) {
    cudaError_t e = cudaFuncSetAttribute(pw::pass_b_kernel<N, WST, ROW>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = persistent_grid(pw::pass_b_kernel<N, WST, ROW>, pw::Plan<N>::NT, smem, N * N, &grid);
    if (e != cudaSuccess) return e;
  }
  pw::pass_b_kernel<N, WST, ROW><<<grid, pw::Plan<N>::NT, smem, s>>>(b);
  return cudaGetLastError();
}

// ev: nullptr or three events recorded before pass A, between the passes and after pass B.
// Pass A of the source mode `src` (pw::SrcMode) on the engine for N.
template <int N, int SRC>
cudaError_t launch_a_mode(const CUtensorMap& vmap, const pw::PassAArgs& a, const R128Extra& x, cudaStream_t s) {
  if constexpr (N == 128) {
    return x.mask ? launch_a_r128<SRC, true>(vmap, a, x, s) : launch_a_r128<SRC, false>(vmap, a, x, s);
  } else if constexpr (N == 96) {
    return x.mask ? launch_a_r96<SRC, true>(vmap, a, x, s) : launch_a_r96<SRC, false>(vmap, a, x, s);
  } else if constexpr (N == 256) {
    if (x.dft_tc) {
      if constexpr (SRC == pw::SRC_GSM)
        return x.mask ? launch_a_d256<SRC, true, true>(vmap, a, x, s) : launch_a_d256<SRC, false, true>(vmap, a, x, s);
      else
        return cudaErrorNotSupported;
    }
    return x.mask ? launch_a_d256<SRC, true>(vmap, a, x, s) : launch_a_d256<SRC, false>(vmap, a, x, s);
  } else {
    return launch_a<N, SRC>(vmap, a, s);
  }
}

// Pass A of a source with at most one or two points per slice: the adjoint source (SRC_ADJ) and
// the delta-correlated source (SRC_DIAG, the adjoint form's diagonal term with the source's d and
// weight).  At N <= 128 (V layout with runs of 4) V is written directly (grad.cuh: adj_row_kernel
// for the P1 row of a mu term, then adj_direct_kernel); elsewhere the engine's pass A.
template <int N, int SRC>
cudaError_t launch_a_sparse(const CUtensorMap& vmap, const pw::PassAArgs& a, const pw::PassBArgs& b,
                            const R128Extra& x, cudaStream_t s) {
  if constexpr (N >= 16 && N <= 128 && pw::vgroup<N>() == 4) {
    if (SRC == pw::SRC_DIAG && a.cross) return cudaErrorInvalidValue;  // a diagonal source has no row
    float2* V = const_cast<float2*>(b.V);
    if (a.cross) {
      pw::adj_row_kernel<N><<<N, N, 0, s>>>(a, V);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
    constexpr int nt = pw::adj_nt<N>(), rows = N * (N / 4) * N;
    pw::adj_direct_kernel<N><<<std::min(rows, num_sms() * (2048 / nt)), nt, 0, s>>>(a, V);
    return cudaGetLastError();
  } else {
    return launch_a_mode<N, SRC>(vmap, a, x, s);
  }
}

// ev: nullptr or three events recorded before pass A, between the passes and after pass B.
// grad: pass B reduces the GSM parameter gradients of an adjoint propagation (W_GRAD) instead of
// storing W.
template <int N>
cudaError_t launch_passes(int src, bool herm, bool grad, const CUtensorMap& vmap, const pw::PassAArgs& a,
                          const pw::PassBArgs& b, const R128Extra& x, cudaStream_t s, cudaEvent_t* ev) {
  cudaError_t e;
  if (ev && (e = cudaEventRecord(ev[0], s)) != cudaSuccess) return e;
  if (src == pw::SRC_GSM) e = launch_a_mode<N, pw::SRC_GSM>(vmap, a, x, s);
  else if (src == pw::SRC_DIAG) e = launch_a_sparse<N, pw::SRC_DIAG>(vmap, a, b, x, s);
  else if (src == pw::SRC_ADJ) e = launch_a_sparse<N, pw::SRC_ADJ>(vmap, a, b, x, s);
  else e = launch_a_mode<N, pw::SRC_ARRAY>(vmap, a, x, s);
  if (e != cudaSuccess) return e;
  if (ev && (e = cudaEventRecord(ev[1], s)) != cudaSuccess) return e;
  if (grad) {
    if constexpr (N == 128) e = launch_b_r128<pw::W_GRAD>(b, s);
    else if constexpr (N == 96) e = launch_b_r96<pw::W_GRAD>(b, s);
    else if constexpr (N == 256) e = cudaErrorNotSupported;
    else e = launch_b<N, pw::W_GRAD>(b, s);
  } else if constexpr (N == 128) {
    e = herm ? launch_b_r128<pw::W_HERM>(b, s) : launch_b<N, pw::W_GENERAL>(b, s);
  } else if constexpr (N == 96) {
    e = herm ? launch_b_r96<pw::W_HERM>(b, s) : launch_b<N, pw::W_GENERAL>(b, s);
  } else if constexpr (N == 256) {
    e = herm ? launch_b_d256(b, s) : cudaErrorNotSupported;
  } else {
    e = herm ? launch_b<N, pw::W_HERM>(b, s) : launch_b<N, pw::W_GENERAL>(b, s);
  }
  if (e != cudaSuccess) return e;
  if (ev && (e = cudaEventRecord(ev[2], s)) != cudaSuccess) return e;
  return cudaSuccess;
}

cudaError_t dispatch(int N, int src, bool herm, bool grad, const CUtensorMap& vmap, const pw::PassAArgs& a,
                     const pw::PassBArgs& b, const R128Extra& x, cudaStream_t s, cudaEvent_t* ev) {
  switch (N) {
#define PW_CASE(NN) \
  case NN:          \
    return launch_passes<NN>(src, herm, grad, vmap, a, b, x, s, ev);
    PW_CASE(2) PW_CASE(4) PW_CASE(6) PW_CASE(8) PW_CASE(12) PW_CASE(16) PW_CASE(24)
    PW_CASE(32) PW_CASE(48) PW_CASE(64) PW_CASE(96) PW_CASE(128) PW_CASE(256)
#undef PW_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link against libcuda).
PFN_cuTensorMapEncodeTiled_v12000 encode_tiled() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// N = 256 (three-pass engine): Y[a][b][k_l'][d' / 8][r][d' mod 8] in the work buffer as floats
// {64, 32, 64, N, N} (the innermost 64 floats are one 256-byte run of 4 r x 8 d'), with the second
// pass's box {64, 1, 1, N, 1} (one run for every b) and the third pass's box {16, 4, 1, 1, N} (the
// 64-byte pieces of one k_h in four consecutive runs, for every a); the first pass stores through
// the same array as floats {16, 4, 32, 64, N^2} with box {16, 1, 32, 4, 1} (four k_l' rows of
// one r: 128 pieces of 64 bytes).
pw_status make_t256_maps(pw_csd* h) {
  auto enc = encode_tiled();
  if (!enc) return fail(PW_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
  constexpr cuuint64_t N = 256, run = 64 * sizeof(float);
  cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  const cuuint64_t dims[5] = {64, 32, 64, N, N};
  const cuuint64_t strides[4] = {run, run * 32, run * 32 * 64, run * 32 * 64 * N};
  const cuuint32_t box2[5] = {64, 1, 1, (cuuint32_t)N, 1}, box3[5] = {16, 4, 1, 1, (cuuint32_t)N};
  CUresult r = enc(&h->ymap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5, h->work, dims, strides, box2, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(PW_ECUDA, "cuTensorMapEncodeTiled (second-pass tiles) failed (CUresult %d)", (int)r);
  r = enc(&h->y3map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5, h->work, dims, strides, box3, estr,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(PW_ECUDA, "cuTensorMapEncodeTiled (third-pass tiles) failed (CUresult %d)", (int)r);
  {
    const cuuint64_t d1[5] = {16, 4, 32, 64, N * N};
    const cuuint64_t s1[4] = {64, 256, 256 * 32, 256 * 32 * 64};
    const cuuint32_t b1[5] = {16, 1, 32, 4, 1};
    r = enc(&h->y1map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5, h->work, d1, s1, b1, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(PW_ECUDA, "cuTensorMapEncodeTiled (first-pass rows) failed (CUresult %d)", (int)r);
  }
  return PW_OK;
}

pw_status make_vmap(pw_csd* h) {
  pw_status st = pwi::encode_vmap(&h->vmap, h->work, h->N);
  if (st == PW_OK && h->N == 256) st = make_t256_maps(h);
  return st;
}

// Fill F, M0, G, tw, Eout for a propagation over z (z <= 0: source-plane view only).
pw_status build_tables(pw_csd* h, double z, bool farfield) {
  const int N = h->N;
  const double d = h->d, lam = h->lambda;
  pw::TableArgs t{};
  t.N = N;
  const double invf = h->lens_f != 0.0 ? 1.0 / h->lens_f : 0.0;
  const double base = d * d / (2.0 * lam);
  t.K0 = -base * invf;
  if (z > 0.0) {
    t.Kin = farfield ? -base * invf : base * (1.0 / z - invf);
    const double dx = lam * z / (N * d);
    t.Kout = dx * dx / (2.0 * lam * z);
  }
  if (h->kind == SRC_GSM) {
    t.gs = d * d / (4.0 * h->sigma_S * h->sigma_S);
    t.gm = d * d / (2.0 * h->sigma_mu * h->sigma_mu);
    t.G = h->G;
  }
  if (h->aperture > 0.0) {
    const double rp = h->aperture / d;
    t.ap_thr = rp * rp;
  } else {
    t.ap_thr = -1.0;
  }
  t.mask = reinterpret_cast<const float2*>(h->mask);
  t.F = h->F;
  t.M0 = h->M0;
  t.tw = h->tw;
  t.Eout = h->Eout;
  t.Ein = h->Ein;
  const int NN = N * N;
  const int threads = 256;
  const int blocks = (NN + threads - 1) / threads;
  pw::tables_kernel<<<blocks, threads, 0, h->stream>>>(t);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "table kernel launch");
  return PW_OK;
}

bool has_masks(const pw_csd* h) { return h->aperture > 0.0 || h->lens_f != 0.0 || h->mask != nullptr; }

// Zero padding (Nz > N) or a grid size without an FFT plan: four dense axis contractions
// (dense.cuh).  W0 is built in W (for a GSM source on the tensor cores, inside the first
// contraction instead), then d (W -> work), c (work -> W), b (W -> work) and a (work -> W, with the
// scale and S).  Events as for the FFT passes: the first two contractions count as the first pass.
pw_status propagate_dense(pw_csd* h, double z, bool farfield, bool herm) {
  const int N = h->N, Nz = h->Nz > 0 ? h->Nz : N;
  pw_status st = build_tables(h, z, farfield);  // G and M0 (the FFT factors are not used here)
  if (st != PW_OK) return st;
  const double d = h->d, lz = h->lambda * z, dx = lz / (Nz * d);
  cudaEvent_t* ev = nullptr;
  if (!h->events.empty() && (size_t)(4 * (h->timed + 1)) <= h->events.size()) ev = &h->events[4 * h->timed++];
  cudaError_t e = cudaSuccess;
  if (ev && (e = cudaEventRecord(ev[0], h->stream)) != cudaSuccess) return cuda_fail(e, "event record");
  pw::dense::TabArgs t{};
  t.N = N;
  t.Nz = Nz;
  t.Kin = farfield ? 0.0 : d * d / (2.0 * lz);
  t.Kout = dx * dx / (2.0 * lz);
  t.E = h->F;  // the FFT input factor's storage (N x N complex) holds E on this path
  const int NN = N * N;
  pw::dense::tables_kernel<<<(NN + 255) / 256, 256, 0, h->stream>>>(t);
  pw::dense::SrcArgs sa{};
  sa.N = N;
  sa.mode = h->kind == SRC_GSM ? pw::SRC_GSM : (h->kind == SRC_DIAGONAL ? pw::SRC_DIAG : pw::SRC_ARRAY);
  sa.G = h->G;
  sa.M0 = h->M0;
  sa.W0 = reinterpret_cast<const float2*>(h->kind == SRC_PROPAGATED ? h->W : h->W0);
  sa.diag = h->diag;
  sa.A = (float)h->A;
  sa.W = reinterpret_cast<float2*>(h->W);
  const bool tc = h->dft_mode != PW_DFT_FP32 && N <= pw::dense_tc::MAX_N;
  const bool gen = tc && sa.mode == pw::SRC_GSM;  // the first tensor-core contraction builds W0 itself
  if (!gen) pw::dense::source_kernel<<<num_sms() * 8, 256, 0, h->stream>>>(sa);
  pw::dense::AxisArgs ax{};
  ax.G = h->G;
  ax.M0 = h->M0;
  ax.A = (float)h->A;
  ax.N = N;
  ax.ncols = (long long)N * N * N;
  ax.E = h->F;
  ax.S = h->S;
  const dim3 grid((unsigned)(((ax.ncols + pw::dense::BN - 1) / pw::dense::BN) * ((N + pw::dense::BM - 1) / pw::dense::BM)));
  float2* Wf = reinterpret_cast<float2*>(h->W);
  float2* Xf = reinterpret_cast<float2*>(h->work);
  const long long L[4] = {1, N, (long long)N * N, (long long)N * N * N};
  if (tc) {  // the split matrices of E (point 2) and conj(E) (point 1), then four tensor-core passes
    const size_t qb = (size_t)pw::dense_tc::nchunks(N) * pw::dense_tc::chunk_bytes(N);
    if (!h->qbuf && (e = cudaMalloc(&h->qbuf, 2 * qb)) != cudaSuccess) return cuda_fail(e, "cudaMalloc of the split DFT matrices");
    const int abuf = pw::dense_tc::a_buffers(N);
    const size_t smem = pw::dense_tc::smem_bytes(N, abuf);
    static size_t smem_set = 0;
    if (smem > smem_set) {
      if ((e = cudaFuncSetAttribute(pw::dense_tc::axis_tc_kernel<false, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem)) != cudaSuccess ||
          (e = cudaFuncSetAttribute(pw::dense_tc::axis_tc_kernel<true, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem)) != cudaSuccess ||
          (e = cudaFuncSetAttribute(pw::dense_tc::axis_tc_kernel<false, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem)) != cudaSuccess ||
          (e = cudaFuncSetAttribute(pw::dense_tc::axis_tc_kernel<true, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem)) != cudaSuccess)
        return cuda_fail(e, "shared memory of the tensor-core contraction");
      smem_set = smem;
    }
    unsigned char* q = reinterpret_cast<unsigned char*>(h->qbuf);
    for (int cj = 0; cj < 2; ++cj) {
      pw::dense_tc::QArgs qa{N, h->F, cj, reinterpret_cast<__nv_bfloat16*>(q + cj * qb)};
      pw::dense_tc::qsplit_kernel<<<num_sms() * 4, 256, 0, h->stream>>>(qa);
    }
    const dim3 tgrid((unsigned)((ax.ncols + 127) / 128));
    ax.stall = h->stall;  // first contraction only, then cleared
    h->stall = 0;
    for (int pass = 0; pass < 4; ++pass) {
      ax.L = L[pass];
      ax.in = pass % 2 == 0 ? Wf : Xf;
      ax.out = pass % 2 == 0 ? Xf : Wf;
      ax.scale = pass == 3 ? (float)((d * d / lz) * (d * d / lz)) : 1.0f;
      const unsigned char* qm = q + (pass < 2 ? 0 : qb);
      if (pass > 0) ax.stall = 0;
      ax.gen = gen && pass == 0 ? 1 : 0;
      if (abuf == 2) {
        if (pass < 3)
          pw::dense_tc::axis_tc_kernel<false, 2><<<tgrid, pw::dense_tc::NT, smem, h->stream>>>(ax, qm, h->err);
        else
          pw::dense_tc::axis_tc_kernel<true, 2><<<tgrid, pw::dense_tc::NT, smem, h->stream>>>(ax, qm, h->err);
      } else {
        if (pass < 3)
          pw::dense_tc::axis_tc_kernel<false, 1><<<tgrid, pw::dense_tc::NT, smem, h->stream>>>(ax, qm, h->err);
        else
          pw::dense_tc::axis_tc_kernel<true, 1><<<tgrid, pw::dense_tc::NT, smem, h->stream>>>(ax, qm, h->err);
      }
      if (pass == 1 && ev && (e = cudaEventRecord(ev[1], h->stream)) != cudaSuccess) return cuda_fail(e, "event record");
    }
  }
  for (int pass = 0; pass < 4 && !tc; ++pass) {
    ax.L = L[pass];
    ax.in = pass % 2 == 0 ? Wf : Xf;
    ax.out = pass % 2 == 0 ? Xf : Wf;
    ax.scale = pass == 3 ? (float)((d * d / lz) * (d * d / lz)) : 1.0f;
    if (pass < 2)
      pw::dense::axis_kernel<false, false><<<grid, pw::dense::NT, 0, h->stream>>>(ax);
    else if (pass == 2)
      pw::dense::axis_kernel<true, false><<<grid, pw::dense::NT, 0, h->stream>>>(ax);
    else
      pw::dense::axis_kernel<true, true><<<grid, pw::dense::NT, 0, h->stream>>>(ax);
    if (pass == 1 && ev && (e = cudaEventRecord(ev[1], h->stream)) != cudaSuccess) return cuda_fail(e, "event record");
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "dense propagation launch");
  if (ev && (e = cudaEventRecord(ev[2], h->stream)) != cudaSuccess) return cuda_fail(e, "event record");
  h->d = dx;
  h->kind = SRC_PROPAGATED;
  h->hermitian = herm ? 1 : 0;
  h->W0 = nullptr;
  h->diag = nullptr;
  h->aperture = 0.0;
  h->lens_f = 0.0;
  h->mask = nullptr;
  return PW_OK;
}

// N = 256, three streaming passes (t256.cuh): the source with the point-2 DFT over (m, d) into the
// work buffer, the radix-4 over r and the DFT over b in place there, the DFT over a with the output
// factors and S from the work buffer into W.  Any source (Hermitian or not; an uploaded W0 may be W
// itself, since the first pass writes only the work buffer).  Events: the first pass, then the
// second and third apart.
pw_status propagate_t256(pw_csd* h, double z, bool herm) {
  namespace T = pw::t256;
  const int src = h->kind == SRC_GSM ? pw::SRC_GSM
                  : h->kind == SRC_DIAGONAL ? pw::SRC_DIAG
                  : h->kind == SRC_ADJOINT ? pw::SRC_ADJ : pw::SRC_ARRAY;
  pw::PassAArgs a{};
  a.F = h->F;
  a.G = h->G;
  a.tw = h->tw;
  a.W0 = src == pw::SRC_ARRAY ? reinterpret_cast<const float2*>(h->kind == SRC_PROPAGATED ? h->W : h->W0) : nullptr;
  a.diag = h->diag;
  a.A = (float)h->A;
  if (src == pw::SRC_ADJ) {
    a.diag = h->adj_d;
    a.cross = h->adj_mu ? h->adj_c : nullptr;
    a.iP = h->adj_iP;
    a.jP = h->adj_jP;
    a.herm = h->adj_herm;
    a.A = 1.0f;
  }
  pw::PassBArgs b{};
  b.tw = h->tw;
  b.Eout = h->Eout;
  b.W = reinterpret_cast<float2*>(h->W);
  b.S = h->S;
  const double lz = h->lambda * z;
  b.scale = (float)((h->d * h->d / lz) * (h->d * h->d / lz));
  static int g2 = 0, g3 = 0;
  cudaError_t e = cudaSuccess;
  // one 512-thread CTA per SM; the shared-memory limit is raised once per source mode
  auto kernel1 = [&](auto k, bool& ready) -> cudaError_t {
    if (!ready) {
      cudaError_t r = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)T::pass1_smem());
      if (r != cudaSuccess) return r;
      ready = true;
    }
    k<<<num_sms(), T::NT1, T::pass1_smem(), h->stream>>>(h->y1map, a);
    return cudaGetLastError();
  };
  static bool ready1[4] = {false, false, false, false};
  if (g2 == 0) {
    if ((e = cudaFuncSetAttribute(T::pass2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)T::pass2_smem())) != cudaSuccess ||
        (e = cudaFuncSetAttribute(T::pass3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)T::pass3_smem())) != cudaSuccess ||
        (e = persistent_grid(T::pass2_kernel, T::NT2, T::pass2_smem(), 1 << 30, &g2)) != cudaSuccess ||
        (e = persistent_grid(T::pass3_kernel, T::NT2, T::pass3_smem(), 1 << 30, &g3)) != cudaSuccess)
      return cuda_fail(e, "set-up of the N = 256 passes");
  }
  cudaEvent_t* ev = nullptr;
  if (!h->events.empty() && (size_t)(4 * (h->timed + 1)) <= h->events.size()) {
    h->three[h->timed] = 1;
    ev = &h->events[4 * h->timed++];
  }
  if (ev && (e = cudaEventRecord(ev[0], h->stream)) != cudaSuccess) return cuda_fail(e, "event record");
  switch (src) {
    case pw::SRC_GSM: e = kernel1(T::pass1_kernel<pw::SRC_GSM>, ready1[pw::SRC_GSM]); break;
    case pw::SRC_DIAG: e = kernel1(T::pass1_kernel<pw::SRC_DIAG>, ready1[pw::SRC_DIAG]); break;
    case pw::SRC_ADJ: e = kernel1(T::pass1_kernel<pw::SRC_ADJ>, ready1[pw::SRC_ADJ]); break;
    default: e = kernel1(T::pass1_kernel<pw::SRC_ARRAY>, ready1[pw::SRC_ARRAY]); break;
  }
  if (e != cudaSuccess) return cuda_fail(e, "first-pass launch (N = 256)");
  if (ev && (e = cudaEventRecord(ev[1], h->stream)) != cudaSuccess) return cuda_fail(e, "event record");
  T::pass2_kernel<<<g2, T::NT2, T::pass2_smem(), h->stream>>>(h->ymap, h->tw, reinterpret_cast<float2*>(h->work), h->err);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "second-pass launch (N = 256)");
  if (ev && (e = cudaEventRecord(ev[3], h->stream)) != cudaSuccess) return cuda_fail(e, "event record");
  T::pass3_kernel<<<g3, T::NT2, T::pass3_smem(), h->stream>>>(h->y3map, b, h->err);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "third-pass launch (N = 256)");
  if (ev && (e = cudaEventRecord(ev[2], h->stream)) != cudaSuccess) return cuda_fail(e, "event record");
  h->d = lz / (h->N * h->d);
  h->kind = SRC_PROPAGATED;
  h->hermitian = herm ? 1 : 0;
  h->W0 = nullptr;
  h->diag = nullptr;
  h->aperture = 0.0;
  h->lens_f = 0.0;
  h->mask = nullptr;
  return PW_OK;
}

pw_status propagate(pw_csd* h, double z, bool farfield) {
  if (!h) return fail(PW_EINVAL, "null handle");
  if (!finite_pos(z)) return fail(PW_EINVAL, "propagation distance must be finite and > 0 (got %g)", z);
  if (h->kind == SRC_NONE) return fail(PW_ESTATE, "no source set for the current plane");
  const bool herm = h->kind == SRC_GSM || h->kind == SRC_DIAGONAL || (h->kind == SRC_ADJOINT ? h->adj_herm != 0 : h->hermitian != 0);
  if (h->kind == SRC_ADJOINT && (h->Nz > 0 || !supported(h->N)))
    return fail(PW_EUNSUPPORTED, "the adjoint propagation needs an unpadded grid with an FFT plan");
  if (h->Nz > 0 || !supported(h->N)) return propagate_dense(h, z, farfield, herm);
  if (h->dft_mode == PW_DFT_TC_BF16X3 && h->kind != SRC_GSM)
    return fail(PW_EUNSUPPORTED, "the tensor-core first stage is built for Gaussian Schell-model sources only");
  pw_status st = build_tables(h, z, farfield);
  if (st != PW_OK) return st;
  // N = 256: the three streaming passes (t256.cuh), any source; the cluster engine (d256.cuh) runs
  // only the comparison mode with the tensor-core first stage
  if (h->N == 256 && h->dft_mode != PW_DFT_TC_BF16X3) return propagate_t256(h, z, herm);
  const int src = h->kind == SRC_GSM ? pw::SRC_GSM
                  : h->kind == SRC_DIAGONAL ? pw::SRC_DIAG
                  : h->kind == SRC_ADJOINT ? pw::SRC_ADJ : pw::SRC_ARRAY;
  pw::PassAArgs a{};
  a.F = h->F;
  a.G = h->G;
  a.tw = h->tw;
  a.W0 = src == pw::SRC_ARRAY ? reinterpret_cast<const float2*>(h->kind == SRC_PROPAGATED ? h->W : h->W0) : nullptr;
  a.diag = h->diag;
  a.A = (float)h->A;
  if (src == pw::SRC_ADJ) {
    a.diag = h->adj_d;
    a.cross = h->adj_mu ? h->adj_c : nullptr;
    a.iP = h->adj_iP;
    a.jP = h->adj_jP;
    a.herm = h->adj_herm;
    a.A = 1.0f;
  }
  pw::PassBArgs b{};
  b.V = reinterpret_cast<const float2*>(h->work);
  b.tw = h->tw;
  b.Eout = h->Eout;
  b.W = reinterpret_cast<float2*>(h->W);
  b.S = h->S;
  const double lz = h->lambda * z;
  b.scale = (float)((h->d * h->d / lz) * (h->d * h->d / lz));
  cudaEvent_t* ev = nullptr;
  if (!h->events.empty() && (size_t)(4 * (h->timed + 1)) <= h->events.size()) ev = &h->events[4 * h->timed++];
  R128Extra x{};
  x.Ein = h->Ein;
  x.mask = reinterpret_cast<const float2*>(h->mask);
  x.ap_ithr = -1;
  x.err = h->err;
  x.dft_tc = h->dft_mode == PW_DFT_TC_BF16X3;
  if (h->aperture > 0.0) {
    const double rp = h->aperture / h->d;
    const double thr = rp * rp;  // the FP64 threshold of the table kernel; r^2 is an integer
    x.ap_ithr = thr >= 2147483647.0 ? 2147483647 : (int)std::floor(thr);
  }
  const bool grad = src == pw::SRC_ADJ && h->adj_grad != nullptr;
  if (grad) b.gr = *h->adj_grad;
  cudaError_t e = dispatch(h->N, src, herm, grad, h->vmap, a, b, x, h->stream, ev);
  if (e != cudaSuccess) return cuda_fail(e, "propagation kernel launch");
  // The output plane becomes the current plane; its CSDA is in W, its masks are unset.
  h->d = lz / (h->N * h->d);
  h->kind = SRC_PROPAGATED;
  h->hermitian = herm ? 1 : 0;
  h->W0 = nullptr;
  h->diag = nullptr;
  h->aperture = 0.0;
  h->lens_f = 0.0;
  h->mask = nullptr;
  return PW_OK;
}

pw_status s_mu(pw_csd* h, int iP, int jP, float* S, pw_c32* mu) {
  if (h->kind == SRC_NONE) return fail(PW_ESTATE, "no source set for the current plane");
  // A propagated plane without masks needs no tables: S comes from the pass-B epilogue.
  if (h->kind != SRC_PROPAGATED || has_masks(h)) {
    pw_status st = build_tables(h, 0.0, false);
    if (st != PW_OK) return st;
  }
  pw::SMuArgs a{};
  a.N = h->N;
  a.mode = h->kind == SRC_GSM ? 0 : (h->kind == SRC_ARRAY ? 1 : (h->kind == SRC_DIAGONAL ? 3 : 2));
  a.diag = h->diag;
  a.G = h->G;
  a.A = (float)h->A;
  a.M0 = has_masks(h) ? h->M0 : nullptr;
  a.Wsrc = reinterpret_cast<const float2*>(h->kind == SRC_ARRAY ? h->W0 : h->W);
  a.Sprop = h->S;
  a.iP = iP;
  a.jP = jP;
  a.S_out = S;
  a.mu_out = reinterpret_cast<float2*>(mu);
  const int NN = h->N * h->N;
  pw::s_mu_kernel<<<(NN + 255) / 256, 256, 0, h->stream>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "S/mu kernel launch");
  return PW_OK;
}

}  // namespace

namespace pwi {
// 5D map of a work buffer in the V layout, as 32-bit floats: dims (innermost first)
// (2g floats of one d' run, b, a, d'/g, c'); box = one whole slice {2g, 1, 1, N/g, N}
// (N = 256: each CTA of a cluster stores a tile of N / CLUSTER_A columns, d256.cuh).
pw_status encode_vmap(CUtensorMap* map, void* work, int N) {
  const int g = pw::vgroup_of(N);
  auto enc = encode_tiled();
  if (!enc) return fail(PW_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
  const cuuint64_t run = (cuuint64_t)2 * g * sizeof(float);
  cuuint64_t dims[5] = {(cuuint64_t)2 * g, (cuuint64_t)N, (cuuint64_t)N, (cuuint64_t)(N / g), (cuuint64_t)N};
  cuuint64_t strides[4] = {run, run * N, run * N * N, run * N * N * (N / g)};
  // N = 256 (cluster engine): each CTA stores N / CLUSTER_A columns of the slice; N = 128: each
  // warp stores its eight rows; otherwise the whole slice in one box
  const int cols = N == 256 ? N / pw::d256::CLUSTER_A : N;
  const int rows = N == 128 ? 8 : N;
  cuuint32_t box[5] = {(cuuint32_t)(2 * g), 1, 1, (cuuint32_t)(cols / g), (cuuint32_t)rows};
  cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5, work, dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(PW_ECUDA, "cuTensorMapEncodeTiled failed (CUresult %d)", (int)r);
  return PW_OK;
}

// The S / P1-row pass of an instance without W: one wave of resident blocks, each taking the same
// number of column groups (blocks left for a second wave, or a last round of a few blocks, stream V
// at a fraction of the bandwidth).  The grid is cached per N.
template <int NN>
cudaError_t launch_smu(const pw::PassBArgs& b, cudaStream_t s) {
  static int grid = 0;
  if (grid == 0) {
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pw::smu_from_v_kernel<NN>, pw::smu_nt<NN>(), 0);
    if (e != cudaSuccess) return e;
    const int groups = NN * NN / 4, resident = std::max(1, per_sm) * num_sms();
    const int rounds = (groups + resident - 1) / resident;
    grid = (groups + rounds - 1) / rounds;
  }
  pw::smu_from_v_kernel<NN><<<grid, pw::smu_nt<NN>(), 0, s>>>(b);
  return cudaGetLastError();
}

// One propagation of a batched GSM instance on the single-instance kernels, from the instance's
// tables: pass A, then pass B with S, the P1 row and, if b.W is set, the Hermitian W store.
cudaError_t launch_batch_instance(int N, const CUtensorMap& vmap, const pw::PassAArgs& a, const pw::PassBArgs& b,
                                  const float2* Ein, const float2* mask, int ap_ithr, cudaStream_t s) {
  R128Extra x{};
  x.Ein = Ein;
  x.mask = mask;
  x.ap_ithr = ap_ithr;
  cudaError_t e;
  // Without W (S and the P1 row only) the second pass is smu_from_v_kernel: two dot products per
  // column instead of the full DFT over point 1, reading V in its own layout.
  switch (N) {
#define PW_BCASE(NN)                                                                                        \
  case NN:                                                                                                  \
    if ((e = launch_a_mode<NN, pw::SRC_GSM>(vmap, a, x, s)) != cudaSuccess) return e;                       \
    if (!b.W) return launch_smu<NN>(b, s);                                                                  \
    if constexpr (NN == 128) return launch_b_r128<pw::W_HERM, true>(b, s);                                 \
    else if constexpr (NN == 96) return launch_b_r96<pw::W_HERM, true>(b, s);                              \
    else return launch_b<NN, pw::W_HERM, true>(b, s);
    PW_BCASE(16) PW_BCASE(32) PW_BCASE(64) PW_BCASE(96) PW_BCASE(128)
#undef PW_BCASE
    default:
      return cudaErrorInvalidValue;
  }
}
}  // namespace pwi

extern "C" {

const char* pw_last_error(void) { return g_err.c_str(); }

const char* pw_status_string(pw_status s) {
  switch (s) {
    case PW_OK: return "PW_OK";
    case PW_EINVAL: return "PW_EINVAL";
    case PW_ESIZE: return "PW_ESIZE";
    case PW_ECUDA: return "PW_ECUDA";
    case PW_ETIMEOUT: return "PW_ETIMEOUT";
    case PW_ESTATE: return "PW_ESTATE";
    case PW_EUNSUPPORTED: return "PW_EUNSUPPORTED";
  }
  return "PW_UNKNOWN";
}

int pw_supported_n(int N) { return supported(N) ? 1 : 0; }

size_t pw_csda_bytes(int N) {
  if (N <= 0) return 0;
  const size_t n = (size_t)N;
  return n * n * n * n * sizeof(pw_c32);
}

pw_status pw_csd_create(pw_csd** out, int N, double dxi_m, double lambda_m, pw_c32* dev_W,
                        size_t W_bytes, pw_c32* dev_work, size_t work_bytes, void* stream) {
  g_err.clear();
  if (!out) return fail(PW_EINVAL, "out is null");
  *out = nullptr;
  if (N < 2 || (N & 1)) return fail(PW_EINVAL, "N must be even and >= 2 (got %d)", N);
  if (!finite_pos(dxi_m)) return fail(PW_EINVAL, "sampling must be finite and > 0 (got %g)", dxi_m);
  if (!finite_pos(lambda_m)) return fail(PW_EINVAL, "wavelength must be finite and > 0 (got %g)", lambda_m);
  if (N > PW_MAX_N) return fail(PW_EUNSUPPORTED, "no propagation plan for N = %d (at most %d)", N, PW_MAX_N);
  if (!dev_W || !dev_work) return fail(PW_EINVAL, "dev_W and dev_work must be non-null");
  const size_t need = pw_csda_bytes(N);
  if (W_bytes < need || work_bytes < need)
    return fail(PW_ESIZE, "buffers need %zu bytes each (got W %zu, work %zu)", need, W_bytes, work_bytes);
  {
    const char* a0 = reinterpret_cast<const char*>(dev_W);
    const char* b0 = reinterpret_cast<const char*>(dev_work);
    if (a0 < b0 + need && b0 < a0 + need) return fail(PW_EINVAL, "dev_W and dev_work overlap");
  }
  if (!aligned(dev_W, 16) || !aligned(dev_work, 16)) return fail(PW_EINVAL, "dev_W and dev_work must be 16-byte aligned");
  pw_csd* h = new pw_csd{};
  h->N = N;
  h->d = dxi_m;
  h->lambda = lambda_m;
  h->W = dev_W;
  h->work = dev_work;
  h->stream = reinterpret_cast<cudaStream_t>(stream);
  h->kind = SRC_NONE;
  h->A = 1.0;
  cudaError_t e = cudaMalloc(&h->tables, table_bytes(N));
  if (e != cudaSuccess) {
    delete h;
    return cuda_fail(e, "cudaMalloc of the handle tables");
  }
  const size_t NN = (size_t)N * N;
  char* p = reinterpret_cast<char*>(h->tables);
  h->F = reinterpret_cast<float2*>(p);
  p += NN * sizeof(float2);
  h->M0 = reinterpret_cast<float2*>(p);
  p += NN * sizeof(float2);
  h->G = reinterpret_cast<float*>(p);
  p += NN * sizeof(float);
  h->S = reinterpret_cast<float*>(p);
  p += NN * sizeof(float);
  h->tw = reinterpret_cast<float2*>(p);
  p += N * sizeof(float2);
  h->Eout = reinterpret_cast<float2*>(p);
  p += N * sizeof(float2);
  h->Ein = reinterpret_cast<float2*>(p);
  p += N * sizeof(float2);
  h->err = reinterpret_cast<int*>(p);
  p += 256;
  auto carve = [&](size_t bytes) {
    char* q = p;
    p += (bytes + 255) / 256 * 256;
    return q;
  };
  h->adj_d = reinterpret_cast<float*>(carve(NN * sizeof(float)));
  h->adj_c = reinterpret_cast<float2*>(carve(NN * sizeof(float2)));
  h->gpart = reinterpret_cast<double*>(carve(NN * 3 * sizeof(double)));
  h->gtab = reinterpret_cast<float*>(carve(NN * sizeof(float)));
  h->qtab = reinterpret_cast<float2*>(carve((size_t)N * sizeof(float2)));
  h->g3tmp = reinterpret_cast<double*>(carve(3 * sizeof(double)));
  e = cudaMemsetAsync(h->err, 0, sizeof(int), h->stream);
  if (e != cudaSuccess) {
    cudaFree(h->tables);
    delete h;
    return cuda_fail(e, "clearing the error flag");
  }
  pw_status st = supported(N) ? make_vmap(h) : PW_OK;  // the dense path needs no tensor map
  if (st != PW_OK) {
    cudaFree(h->tables);
    delete h;
    return st;
  }
  *out = h;
  return PW_OK;
}

static void free_events(pw_csd* h) {
  for (cudaEvent_t e : h->events) cudaEventDestroy(e);
  h->events.clear();
  h->three.clear();
  h->timed = 0;
}

pw_status pw_csd_destroy(pw_csd* h) {
  g_err.clear();
  if (!h) return PW_OK;
  cudaError_t e1 = cudaStreamSynchronize(h->stream);
  free_events(h);
  cudaError_t e2 = cudaFree(h->tables);
  if (h->qbuf) cudaFree(h->qbuf);
  delete h;
  if (e1 != cudaSuccess) return cuda_fail(e1, "stream synchronize in destroy");
  if (e2 != cudaSuccess) return cuda_fail(e2, "cudaFree of the handle tables");
  return PW_OK;
}

pw_status pw_csd_set_stream(pw_csd* h, void* stream) {
  g_err.clear();
  if (!h) return fail(PW_EINVAL, "null handle");
  h->stream = reinterpret_cast<cudaStream_t>(stream);
  return PW_OK;
}

pw_status pw_csd_reset(pw_csd* h, double dxi_m) {
  g_err.clear();
  if (!h) return fail(PW_EINVAL, "null handle");
  if (!finite_pos(dxi_m)) return fail(PW_EINVAL, "sampling must be finite and > 0 (got %g)", dxi_m);
  h->d = dxi_m;
  h->kind = SRC_NONE;
  h->W0 = nullptr;
  h->A = 1.0;
  h->aperture = 0.0;
  h->lens_f = 0.0;
  h->mask = nullptr;
  return PW_OK;
}

pw_status pw_csd_check(pw_csd* h) {
  g_err.clear();
  if (!h) return fail(PW_EINVAL, "null handle");
  int flag = 0;
  cudaError_t e = cudaMemcpyAsync(&flag, h->err, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "reading the error flag");
  if (flag) {
    e = cudaMemsetAsync(h->err, 0, sizeof(int), h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "clearing the error flag");
    return fail(PW_ETIMEOUT, "a bounded device-side wait gave up; the last result is invalid");
  }
  return PW_OK;
}

pw_status pw_csd_enable_timing(pw_csd* h, int max_props) {
  g_err.clear();
  if (!h) return fail(PW_EINVAL, "null handle");
  if (max_props < 0) return fail(PW_EINVAL, "max_props must be >= 0");
  free_events(h);
  h->events.resize((size_t)4 * max_props);
  h->three.assign((size_t)max_props, 0);
  for (size_t i = 0; i < h->events.size(); ++i) {
    cudaError_t e = cudaEventCreate(&h->events[i]);
    if (e != cudaSuccess) {
      h->events.resize(i);
      free_events(h);
      return cuda_fail(e, "cudaEventCreate");
    }
  }
  return PW_OK;
}

pw_status pw_csd_pass_times3(pw_csd* h, double* ms_first, double* ms_second, double* ms_third, int* count) {
  g_err.clear();
  if (!h || !ms_first || !ms_second || !ms_third || !count) return fail(PW_EINVAL, "null argument");
  double sa = 0.0, sb = 0.0, sc = 0.0;
  for (int k = 0; k < h->timed; ++k) {
    cudaEvent_t* ev = &h->events[4 * k];
    float t1 = 0.f, t2 = 0.f, t3 = 0.f;
    cudaError_t e = cudaEventSynchronize(ev[2]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t1, ev[0], ev[1]);
    if (e == cudaSuccess) {
      if (h->three[k]) {
        e = cudaEventElapsedTime(&t2, ev[1], ev[3]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t3, ev[3], ev[2]);
      } else {
        e = cudaEventElapsedTime(&t2, ev[1], ev[2]);
      }
    }
    if (e != cudaSuccess) return cuda_fail(e, "pass timing events");
    sa += t1;
    sb += t2;
    sc += t3;
  }
  *ms_first = sa;
  *ms_second = sb;
  *ms_third = sc;
  *count = h->timed;
  h->timed = 0;
  return PW_OK;
}

pw_status pw_csd_pass_times(pw_csd* h, double* ms_first, double* ms_second, int* count) {
  double m3 = 0.0;
  pw_status st = pw_csd_pass_times3(h, ms_first, ms_second, &m3, count);
  if (st == PW_OK) *ms_second += m3;
  return st;
}

pw_status pw_csd_set_padding(pw_csd* h, int Nz) {
  g_err.clear();
  if (!h) return fail(PW_EINVAL, "null handle");
  if (Nz != 0 && (Nz < h->N || (Nz - h->N) % 2 != 0 || Nz > (1 << 20)))
    return fail(PW_EINVAL, "padded size must be 0 or N <= Nz <= 2^20 with Nz - N even (N = %d, Nz = %d)", h->N, Nz);
  h->Nz = Nz == h->N ? 0 : Nz;
  return PW_OK;
}

pw_status pw_csd_get_padding(const pw_csd* h, int* Nz) {
  g_err.clear();
  if (!h || !Nz) return fail(PW_EINVAL, "null argument");
  *Nz = h->Nz > 0 ? h->Nz : h->N;
  return PW_OK;
}

pw_status pw_csd_inject_stall(pw_csd* h, int chunk) {
  g_err.clear();
  if (!h) return fail(PW_EINVAL, "null handle");
  h->stall = chunk;
  return PW_OK;
}

pw_status pw_csd_set_dft_mode(pw_csd* h, int mode) {
  g_err.clear();
  if (!h) return fail(PW_EINVAL, "null handle");
  if (mode != PW_DFT_AUTO && mode != PW_DFT_FP32 && mode != PW_DFT_TC_BF16X3)
    return fail(PW_EINVAL, "unknown DFT mode %d", mode);
  if (mode == PW_DFT_TC_BF16X3 && h->N > pw::dense_tc::MAX_N)
    return fail(PW_EUNSUPPORTED, "the tensor-core paths exist for N <= %d (N = %d)", pw::dense_tc::MAX_N, h->N);
  h->dft_mode = mode;
  return PW_OK;
}

pw_status pw_csd_get_dft_mode(const pw_csd* h, int* mode) {
  g_err.clear();
  if (!h || !mode) return fail(PW_EINVAL, "null argument");
  *mode = h->dft_mode;
  return PW_OK;
}

pw_status pw_source_gsm(pw_csd* h, double sigma_S_m, double sigma_mu_m, double amplitude) {
  g_err.clear();
  if (!h) return fail(PW_EINVAL, "null handle");
  if (!finite_pos(sigma_S_m) || !finite_pos(sigma_mu_m))
    return fail(PW_EINVAL, "sigma_S and sigma_mu must be finite and > 0 (got %g, %g)", sigma_S_m, sigma_mu_m);
  if (!std::isfinite(amplitude)) return fail(PW_EINVAL, "amplitude must be finite");
  h->kind = SRC_GSM;
  h->sigma_S = sigma_S_m;
  h->sigma_mu = sigma_mu_m;
  h->A = amplitude;
  h->W0 = nullptr;
  return PW_OK;
}

pw_status pw_source_aperture(pw_csd* h, double radius_m) {
  g_err.clear();
  if (!h) return fail(PW_EINVAL, "null handle");
  if (!std::isfinite(radius_m)) return fail(PW_EINVAL, "aperture radius must be finite");
  h->aperture = radius_m > 0.0 ? radius_m : 0.0;
  return PW_OK;
}

pw_status pw_source_lens(pw_csd* h, double focal_m) {
  g_err.clear();
  if (!h) return fail(PW_EINVAL, "null handle");
  if (!std::isfinite(focal_m)) return fail(PW_EINVAL, "focal length must be finite");
  h->lens_f = focal_m;
  return PW_OK;
}

pw_status pw_source_mask(pw_csd* h, const pw_c32* dev_mask) {
  g_err.clear();
  if (!h) return fail(PW_EINVAL, "null handle");
  if (dev_mask && !aligned(dev_mask, 8)) return fail(PW_EINVAL, "dev_mask must be 8-byte aligned");
  h->mask = dev_mask;
  return PW_OK;
}

pw_status pw_source_array(pw_csd* h, const pw_c32* dev_W0, int hermitian) {
  g_err.clear();
  if (!h) return fail(PW_EINVAL, "null handle");
  if (!dev_W0) return fail(PW_EINVAL, "dev_W0 is null");
  if (!aligned(dev_W0, 8)) return fail(PW_EINVAL, "dev_W0 must be 8-byte aligned");
  {
    const size_t need = pw_csda_bytes(h->N);
    const char* a0 = reinterpret_cast<const char*>(dev_W0);
    const char* b0 = reinterpret_cast<const char*>(h->work);
    if (a0 < b0 + need && b0 < a0 + need) return fail(PW_EINVAL, "dev_W0 overlaps the work buffer");
  }
  h->kind = SRC_ARRAY;
  h->W0 = dev_W0;
  h->hermitian = hermitian ? 1 : 0;
  h->A = 1.0;
  return PW_OK;
}

pw_status pw_source_diagonal(pw_csd* h, const float* dev_d, double weight) {
  g_err.clear();
  if (!h) return fail(PW_EINVAL, "null handle");
  if (!dev_d) return fail(PW_EINVAL, "dev_d is null");
  if (!aligned(dev_d, 4)) return fail(PW_EINVAL, "dev_d must be 4-byte aligned");
  if (!std::isfinite(weight)) return fail(PW_EINVAL, "weight must be finite");
  h->kind = SRC_DIAGONAL;
  h->diag = dev_d;
  h->W0 = nullptr;
  h->A = weight;
  return PW_OK;
}

pw_status pw_gsm_gradient(pw_csd* h, double sigma_S_m, double sigma_mu_m, double amplitude, const float* dev_amask,
                          double lambda_m, double z_m, int farfield, double* dev_grad3, float* dev_grad_mask) {
  g_err.clear();
  if (!h || !dev_grad3) return fail(PW_EINVAL, "null argument");
  if (!finite_pos(sigma_S_m) || !finite_pos(sigma_mu_m) || !finite_pos(lambda_m) || !finite_pos(z_m))
    return fail(PW_EINVAL, "lengths must be finite and > 0");
  if (!std::isfinite(amplitude)) return fail(PW_EINVAL, "amplitude must be finite");
  if (h->kind != SRC_PROPAGATED) return fail(PW_ESTATE, "no propagated CSDA (run the adjoint propagation first)");
  if (h->Nz > 0 || !supported(h->N))
    return fail(PW_EUNSUPPORTED, "the GSM gradient needs an unpadded grid with an FFT plan");
  const int N = h->N;
  const double d = h->d;                    // the source plane of the forward propagation
  const double dx = lambda_m * z_m / (N * d);  // its output plane
  pw::GradArgs g{};
  g.N = N;
  g.d = d;
  g.sigma_S = sigma_S_m;
  g.sigma_mu = sigma_mu_m;
  g.A = amplitude;
  g.amask = dev_amask;
  g.R = reinterpret_cast<const float2*>(h->W);
  g.c = std::pow(d / dx, 4);
  g.farfield = farfield ? 1 : 0;
  g.Kq = d * d / (2.0 * lambda_m * z_m);
  g.g3 = dev_grad3;
  g.gmask = dev_grad_mask;
  // the work buffer is scratch between propagations: partial sums, then the FP64-built tables
  g.part = reinterpret_cast<double*>(h->work);
  g.gtab = reinterpret_cast<float*>(g.part + (size_t)N * N * 3);
  g.qtab = reinterpret_cast<float2*>(g.gtab + (size_t)N * N + (N & 1));
  pw::gsm_gradient_tables<<<(N * N + 255) / 256, 256, 0, h->stream>>>(g);
  cudaError_t e0 = cudaGetLastError();
  if (e0 != cudaSuccess) return cuda_fail(e0, "gradient table launch");
  const size_t sh = 2 * N * sizeof(float) + 2 * N * sizeof(float2) + 32 * sizeof(double) + 64;
  if (g.farfield) pw::gsm_gradient_kernel<true><<<N * N, 256, sh, h->stream>>>(g);
  else pw::gsm_gradient_kernel<false><<<N * N, 256, sh, h->stream>>>(g);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "gradient kernel launch");
  pw::gsm_gradient_reduce<<<1, 256, 0, h->stream>>>(g);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "gradient reduction launch");
  return PW_OK;
}

}  // extern "C"

namespace {

// The adjoint of one propagation (Fresnel or far field over z) for a loss on S and mu of its
// output plane; the handle's current plane is that output plane.  See pw_propagate_fresnel_adjoint.
pw_status adjoint(pw_csd* h, double z, bool farfield, const pw_adjoint* a) {
  if (!h || !a) return fail(PW_EINVAL, "null argument");
  if (!finite_pos(z)) return fail(PW_EINVAL, "propagation distance must be finite and > 0 (got %g)", z);
  if (h->Nz > 0 || !supported(h->N))
    return fail(PW_EUNSUPPORTED, "the adjoint propagation needs an unpadded grid with an FFT plan");
  const int N = h->N;
  const bool has_mu = a->dev_dmu != nullptr;
  if (!a->dev_dS && !has_mu) return fail(PW_EINVAL, "no upstream gradient (dev_dS and dev_dmu are both null)");
  if (has_mu) {
    if (!a->dev_S || !a->dev_mu) return fail(PW_EINVAL, "dev_dmu needs the output plane's dev_S and dev_mu");
    if (a->iP < 0 || a->jP < 0 || a->iP >= N || a->jP >= N)
      return fail(PW_EINVAL, "P1 = (%d, %d) outside the %d x %d grid", a->iP, a->jP, N, N);
  }
  const bool params = a->dev_grad3 != nullptr || a->dev_grad_amask != nullptr;
  if (!params && !a->grad_W0) return fail(PW_EINVAL, "no gradient requested");
  if (params && (!finite_pos(a->sigma_S_m) || !finite_pos(a->sigma_mu_m) || !std::isfinite(a->amplitude)))
    return fail(PW_EINVAL, "the GSM parameters must be finite (sigma_S, sigma_mu > 0)");
  if ((a->dev_dS && !aligned(a->dev_dS, 4)) || (a->dev_S && !aligned(a->dev_S, 4)) ||
      (a->dev_amask && !aligned(a->dev_amask, 4)) || (a->dev_grad_amask && !aligned(a->dev_grad_amask, 4)) ||
      (a->dev_dmu && !aligned(a->dev_dmu, 8)) || (a->dev_mu && !aligned(a->dev_mu, 8)) ||
      (a->dev_grad3 && !aligned(a->dev_grad3, 8)))
    return fail(PW_EINVAL, "misaligned device pointer");
  const double dx = h->d, lam = h->lambda, d = lam * z / (N * dx);
  const double c = std::pow(d / dx, 4);
  cudaStream_t st = h->stream;

  // the (conjugated) adjoint source on the output plane
  pw::AdjPrepArgs pa{};
  pa.N = N;
  pa.iP = a->iP;
  pa.jP = a->jP;
  pa.gS = a->dev_dS;
  pa.gmu = reinterpret_cast<const float2*>(a->dev_dmu);
  pa.S = a->dev_S;
  pa.mu = reinterpret_cast<const float2*>(a->dev_mu);
  pa.d = h->adj_d;
  pa.cross = h->adj_c;
  pw::adjoint_prep_kernel<<<1, 1024, 0, st>>>(pa);
  // the GSM factor (parameter gradients) and the far-field factors of the source grid
  pw::GradArgs g{};
  g.N = N;
  g.d = d;
  g.sigma_S = params ? a->sigma_S_m : 0.0;
  g.sigma_mu = params ? a->sigma_mu_m : 0.0;
  g.A = a->amplitude;
  g.amask = a->dev_amask;
  g.R = reinterpret_cast<const float2*>(h->W);
  g.c = c;
  g.farfield = farfield ? 1 : 0;
  g.Kq = d * d / (2.0 * lam * z);
  g.part = h->gpart;
  g.gtab = h->gtab;
  g.qtab = h->qtab;
  g.g3 = a->dev_grad3 ? a->dev_grad3 : h->g3tmp;
  g.gmask = a->dev_grad_amask;
  pw::gsm_gradient_tables<<<(N * N + 255) / 256, 256, 0, st>>>(g);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "adjoint set-up launch");

  // one adjoint propagation: a Fresnel propagation over z from the output sampling dx of the
  // conjugated source (back onto the source grid d)
  auto run = [&](bool herm, const pw::GradEpi* epi) -> pw_status {
    h->d = dx;
    h->kind = SRC_ADJOINT;
    h->adj_herm = herm ? 1 : 0;
    h->adj_mu = has_mu ? 1 : 0;
    h->adj_iP = a->iP;
    h->adj_jP = a->jP;
    h->adj_grad = epi;
    pw_status r = propagate(h, z, false);
    h->adj_grad = nullptr;
    return r;
  };
  bool R_herm_in_W = false;
  pw_status r = PW_OK;
  if (params) {
    // the Hermitian part of the source suffices: dW0/dtheta is Hermitian
    if (N != 256) {
      pw::GradEpi ge{};
      ge.gtab = h->gtab;
      ge.amask = a->dev_amask;
      ge.qff = farfield ? h->qtab : nullptr;
      ge.part = h->gpart;
      ge.gmask = a->dev_grad_amask;
      ge.gscale = (float)(4.0 * c * a->amplitude);
      ge.d2 = (float)(d * d);
      r = run(true, &ge);
    } else {
      r = run(true, nullptr);  // R stored in W, then the standalone gradient kernel
      if (r == PW_OK) {
        const size_t sh = 2 * N * sizeof(float) + 2 * N * sizeof(float2) + 32 * sizeof(double) + 64;
        if (farfield) pw::gsm_gradient_kernel<true><<<N * N, 256, sh, st>>>(g);
        else pw::gsm_gradient_kernel<false><<<N * N, 256, sh, st>>>(g);
        R_herm_in_W = true;
      }
    }
    if (r == PW_OK) pw::gsm_gradient_reduce<<<1, 256, 0, st>>>(g);
  }
  if (r == PW_OK && a->grad_W0) {
    // a general complex W0: the whole adjoint (the P1 row without its mirrored column)
    if (!(R_herm_in_W && !has_mu)) r = run(!has_mu, nullptr);
    if (r == PW_OK) {
      const int blocks = num_sms() * 8;
      pw::w0_gradient_kernel<<<blocks, 256, 0, st>>>(reinterpret_cast<float2*>(h->W), N, (float)(2.0 * c),
                                                     farfield ? h->qtab : nullptr);
    }
  }
  if (r == PW_OK && (e = cudaGetLastError()) != cudaSuccess) r = cuda_fail(e, "adjoint kernel launch");
  // the handle is at the source plane, with no source recorded
  h->d = d;
  h->kind = SRC_NONE;
  h->W0 = nullptr;
  h->diag = nullptr;
  return r;
}

}  // namespace

extern "C" {

pw_status pw_propagate_fresnel_adjoint(pw_csd* h, double z_m, const pw_adjoint* a) {
  g_err.clear();
  return adjoint(h, z_m, false, a);
}

pw_status pw_propagate_farfield_adjoint(pw_csd* h, double z_m, const pw_adjoint* a) {
  g_err.clear();
  return adjoint(h, z_m, true, a);
}

pw_status pw_propagate_fresnel(pw_csd* h, double z_m) {
  g_err.clear();
  return propagate(h, z_m, false);
}

pw_status pw_propagate_farfield(pw_csd* h, double z_m) {
  g_err.clear();
  return propagate(h, z_m, true);
}

pw_status pw_get_sampling(const pw_csd* h, double* d_m) {
  g_err.clear();
  if (!h || !d_m) return fail(PW_EINVAL, "null argument");
  *d_m = h->d;
  return PW_OK;
}

pw_status pw_spectral_density(pw_csd* h, float* dev_S) {
  g_err.clear();
  if (!h || !dev_S) return fail(PW_EINVAL, "null argument");
  if (!aligned(dev_S, 4)) return fail(PW_EINVAL, "dev_S must be 4-byte aligned");
  return s_mu(h, 0, 0, dev_S, nullptr);
}

pw_status pw_degree_of_coherence(pw_csd* h, int iP, int jP, pw_c32* dev_mu) {
  g_err.clear();
  if (!h || !dev_mu) return fail(PW_EINVAL, "null argument");
  if (!aligned(dev_mu, 8)) return fail(PW_EINVAL, "dev_mu must be 8-byte aligned");
  if (iP < 0 || jP < 0 || iP >= h->N || jP >= h->N)
    return fail(PW_EINVAL, "P1 = (%d, %d) outside the %d x %d grid", iP, jP, h->N, h->N);
  return s_mu(h, iP, jP, nullptr, dev_mu);
}

}  // extern "C"
