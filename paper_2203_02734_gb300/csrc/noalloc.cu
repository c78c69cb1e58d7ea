// noalloc.cu -- an allocation-free variant of one Fresnel propagation of a GSM source, for
// callers that cannot allocate device memory: applications whose framework reserves all
// device memory in its own pool and forbids libraries to call the CUDA allocator, and
// latency-critical loops that cannot afford the implicit device synchronisation of
// cudaMalloc / cudaFree.  The half-transformed CSDA and the small tables live in one
// file-scope device array of fixed size instead of handle memory and a work buffer.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <cmath>
#include <cstdarg>
#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <mutex>

#include "../../include/pywolf_gb.h"
#include "propagate.cuh"

namespace pwi {
void set_last_error(const char* msg);  // pywolf_gb.cu: message returned by pw_last_error()
}

namespace {

constexpr int kMaxN = 32;
constexpr size_t kMaxNN = (size_t)kMaxN * kMaxN;
// Scratch layout (bytes): V (N^4 complex64) | F (N^2 complex64) | G (N^2 float) | twiddles (N
// complex64) | output propagators (N complex64); sized for N = kMaxN, 256-byte aligned parts.
constexpr size_t kVBytes = kMaxNN * kMaxNN * sizeof(float2);
constexpr size_t kFBytes = kMaxNN * sizeof(float2);
constexpr size_t kGBytes = kMaxNN * sizeof(float);
constexpr size_t kTwBytes = 256;  // >= kMaxN * sizeof(float2)
constexpr size_t kScratchBytes = kVBytes + kFBytes + kGBytes + 2 * kTwBytes;

// Shared by every call on a device and kept until process exit; each call overwrites every byte
// it later reads, so nothing has to start at zero.  Calls whose work overlaps on the GPU race
// on this array.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_dev[kMaxDevices];  // device address of g_scratch, per device (set-up once)

pw_status fail(pw_status s, const char* fmt, ...) {
  char msg[256];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(msg, sizeof msg, fmt, ap);
  va_end(ap);
  pwi::set_last_error(msg);
  return s;
}

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

// Device address of g_scratch on the current device (looked up once per device).
pw_status scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(PW_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(PW_EUNSUPPORTED, "device ordinal %d beyond %d", dev, kMaxDevices);
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_dev[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(PW_ECUDA, "cudaGetSymbolAddress of the static scratch: %s", cudaGetErrorString(e));
    }
    g_scratch_dev[dev] = p;
  }
  *out = g_scratch_dev[dev];
  return PW_OK;
}

// Persistent grids of the two passes for N on the current device: occupancy queried on the
// first call per (device, N) and kept, so later calls issue no attribute or occupancy queries.
template <int N>
pw_status pass_grids(int* ga, int* gb) {
  static int grid_a[kMaxDevices], grid_b[kMaxDevices];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(PW_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(PW_EUNSUPPORTED, "device ordinal %d beyond %d", dev, kMaxDevices);
  std::lock_guard<std::mutex> lock(g_mu);
  if (grid_a[dev] == 0) {
    int sms = 0, per_a = 0, per_b = 0;
    const int NN = N * N;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
        (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_a, pw::pass_a_kernel<N, pw::SRC_GSM>,
                                                           pw::Plan<N>::NT, pw::pass_a_smem<N>())) != cudaSuccess ||
        (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_b, pw::pass_b_kernel<N, pw::W_HERM>,
                                                           pw::Plan<N>::NT, pw::pass_b_smem<N>())) != cudaSuccess) {
      cudaGetLastError();
      return fail(PW_ECUDA, "occupancy of the propagation passes: %s", cudaGetErrorString(e));
    }
    grid_a[dev] = (int)std::min<long>((long)std::max(per_a, 1) * std::max(sms, 1), NN);
    grid_b[dev] = (int)std::min<long>((long)std::max(per_b, 1) * std::max(sms, 1), NN);
  }
  *ga = grid_a[dev];
  *gb = grid_b[dev];
  return PW_OK;
}

template <int N>
pw_status run(const CUtensorMap& vmap, const pw::TableArgs& t, const pw::PassAArgs& a, const pw::PassBArgs& b,
              cudaStream_t s) {
  int ga = 0, gb = 0;
  pw_status st = pass_grids<N>(&ga, &gb);
  if (st != PW_OK) return st;
  const int NN = N * N;
  pw::tables_kernel<<<(NN + 255) / 256, 256, 0, s>>>(t);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) {
    pw::pass_a_kernel<N, pw::SRC_GSM><<<ga, pw::Plan<N>::NT, pw::pass_a_smem<N>(), s>>>(vmap, a);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    pw::pass_b_kernel<N, pw::W_HERM><<<gb, pw::Plan<N>::NT, pw::pass_b_smem<N>(), s>>>(b);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(PW_ECUDA, "kernel launch: %s", cudaGetErrorString(e));
  }
  return PW_OK;
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
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

}  // namespace

extern "C" pw_status pw_propagate_gsm_fresnel_noalloc(int N, double dxi_m, double lambda_m, double z_m,
                                                      double sigma_S_m, double sigma_mu_m, double amplitude,
                                                      double aperture_m, double lens_f_m,
                                                      const pw_c32* dev_mask, pw_c32* dev_W_out,
                                                      size_t W_bytes, float* dev_S_out, void* stream) {
  pwi::set_last_error("");
  if (N < 2 || (N & 1)) return fail(PW_EINVAL, "N must be even and >= 2 (got %d)", N);
  if (N > kMaxN)
    return fail(PW_EINVAL, "N = %d exceeds the maximum N = %d of the static scratch (%zu bytes)", N, kMaxN,
                kScratchBytes);
  if (!pw_supported_n(N)) return fail(PW_EUNSUPPORTED, "no propagation plan for N = %d", N);
  if (!finite_pos(dxi_m) || !finite_pos(lambda_m) || !finite_pos(z_m) || !finite_pos(sigma_S_m) ||
      !finite_pos(sigma_mu_m))
    return fail(PW_EINVAL, "lengths must be finite and > 0");
  if (!std::isfinite(amplitude) || !std::isfinite(aperture_m) || !std::isfinite(lens_f_m))
    return fail(PW_EINVAL, "amplitude, aperture and focal length must be finite");
  if (!dev_W_out || !dev_S_out) return fail(PW_EINVAL, "dev_W_out and dev_S_out must be non-null");
  if (W_bytes < pw_csda_bytes(N)) return fail(PW_ESIZE, "dev_W_out needs %zu bytes (got %zu)", pw_csda_bytes(N), W_bytes);
  // Pass B leaves W by bulk copies (16-byte aligned global addresses), S is written as floats and
  // the mask is read as 8-byte complex values: misaligned pointers are refused before any launch.
  if (reinterpret_cast<uintptr_t>(dev_W_out) % 16 != 0)
    return fail(PW_EINVAL, "dev_W_out must be 16-byte aligned");
  if (reinterpret_cast<uintptr_t>(dev_S_out) % 4 != 0) return fail(PW_EINVAL, "dev_S_out must be 4-byte aligned");
  if (dev_mask && reinterpret_cast<uintptr_t>(dev_mask) % 8 != 0)
    return fail(PW_EINVAL, "dev_mask must be 8-byte aligned");

  void* base = nullptr;
  pw_status st = scratch_address(&base);
  if (st != PW_OK) return st;
  char* p = reinterpret_cast<char*>(base);
  float2* V = reinterpret_cast<float2*>(p);
  float2* F = reinterpret_cast<float2*>(p + kVBytes);
  float* G = reinterpret_cast<float*>(p + kVBytes + kFBytes);
  float2* tw = reinterpret_cast<float2*>(p + kVBytes + kFBytes + kGBytes);
  float2* Eout = reinterpret_cast<float2*>(p + kVBytes + kFBytes + kGBytes + kTwBytes);

  // Same tables as the handle path (FP64 phases reduced mod 1 turn).
  const double d = dxi_m, lam = lambda_m;
  const double invf = lens_f_m != 0.0 ? 1.0 / lens_f_m : 0.0;
  pw::TableArgs t{};
  t.N = N;
  t.Kin = d * d / (2.0 * lam) * (1.0 / z_m - invf);
  t.K0 = 0.0;
  const double dx = lam * z_m / (N * d);
  t.Kout = dx * dx / (2.0 * lam * z_m);
  t.gs = d * d / (4.0 * sigma_S_m * sigma_S_m);
  t.gm = d * d / (2.0 * sigma_mu_m * sigma_mu_m);
  if (aperture_m > 0.0) {
    const double rp = aperture_m / d;
    t.ap_thr = rp * rp;
  } else {
    t.ap_thr = -1.0;
  }
  t.mask = reinterpret_cast<const float2*>(dev_mask);
  t.F = F;
  t.M0 = nullptr;
  t.G = G;
  t.tw = tw;
  t.Eout = Eout;

  // TMA map of V in the tiled layout (host-side descriptor, no allocation).
  auto enc = encode_fn();
  if (!enc) return fail(PW_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
  CUtensorMap vmap;
  const int g = pw::vgroup_of(N);
  const cuuint64_t run_b = (cuuint64_t)2 * g * sizeof(float);
  cuuint64_t dims[5] = {(cuuint64_t)2 * g, (cuuint64_t)N, (cuuint64_t)N, (cuuint64_t)(N / g), (cuuint64_t)N};
  cuuint64_t strides[4] = {run_b, run_b * N, run_b * N * N, run_b * N * N * (N / g)};
  cuuint32_t box[5] = {(cuuint32_t)(2 * g), 1, 1, (cuuint32_t)(N / g), (cuuint32_t)N};
  cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  CUresult r = enc(&vmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5, V, dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(PW_ECUDA, "cuTensorMapEncodeTiled failed (CUresult %d)", (int)r);

  pw::PassAArgs a{};
  a.F = F;
  a.G = G;
  a.tw = tw;
  a.W0 = nullptr;
  a.A = (float)amplitude;
  pw::PassBArgs b{};
  b.V = V;
  b.tw = tw;
  b.Eout = Eout;
  b.W = reinterpret_cast<float2*>(dev_W_out);
  b.S = dev_S_out;
  const double lz = lam * z_m;
  b.scale = (float)((d * d / lz) * (d * d / lz));

  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  switch (N) {
    case 2: return run<2>(vmap, t, a, b, s);
    case 4: return run<4>(vmap, t, a, b, s);
    case 6: return run<6>(vmap, t, a, b, s);
    case 8: return run<8>(vmap, t, a, b, s);
    case 12: return run<12>(vmap, t, a, b, s);
    case 16: return run<16>(vmap, t, a, b, s);
    case 24: return run<24>(vmap, t, a, b, s);
    case 32: return run<32>(vmap, t, a, b, s);
    default: break;
  }
  return fail(PW_EUNSUPPORTED, "no propagation plan for N = %d", N);
}
