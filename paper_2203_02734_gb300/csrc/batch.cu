// batch.cu -- C ABI of the batched run (pw_batch_*): instance descriptors, workspace layout,
// item list, launch sequence (counter reset, FP64 tables, one persistent launch, mu) and the
// chunk-size autotuner.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <vector>

#include "../../include/pywolf_gb.h"
#include "batch.cuh"

namespace pwi {  // pywolf_gb.cu
void set_last_error(const char* msg);
pw_status encode_vmap(CUtensorMap* map, void* work, int N);
cudaError_t launch_batch_instance(int N, const CUtensorMap& vmap, const pw::PassAArgs& a, const pw::PassBArgs& b,
                                  const float2* Ein, const float2* mask, int ap_ithr, cudaStream_t s);
}

namespace {

pw_status fail(pw_status s, const char* fmt, ...) {
  char msg[320];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(msg, sizeof msg, fmt, ap);
  va_end(ap);
  pwi::set_last_error(msg);
  return s;
}

pw_status cuda_fail(cudaError_t e, const char* what) {
  cudaGetLastError();
  return fail(PW_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

bool batch_n(int N) { return N == 16 || N == 32 || N == 64 || N == 96 || N == 128; }

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Workspace layout (offsets from the base, each part 256-byte aligned).
struct Layout {
  size_t inst, targs, mu, items, counters, tmaps, wts, tables, pool, total;
  int max_items;
  size_t slot_bytes;
};

constexpr int kMinChunk = 4;

Layout layout(const pw_instance* in, int n, int pool) {
  Layout L{};
  size_t off = 0;
  L.inst = off;
  off = align256(off + sizeof(pw::batch::Inst) * n);
  L.targs = off;
  off = align256(off + sizeof(pw::TableArgs) * n);
  L.mu = off;
  off = align256(off + sizeof(float2*) * n);
  long items = 0;
  int maxN = 0;
  for (int i = 0; i < n; ++i) {
    const long s = (long)in[i].N * in[i].N;
    items += 2 * ((s + kMinChunk - 1) / kMinChunk);
    if (in[i].N > maxN) maxN = in[i].N;
  }
  L.max_items = (int)items;
  L.items = off;
  off = align256(off + sizeof(pw::batch::Item) * items);
  L.counters = off;
  off = align256(off + sizeof(int) * (2 * (size_t)n + 2));
  L.tmaps = off;  // one tensor map per pool slot (N = 128 instances store V by TMA)
  off = align256(off + sizeof(CUtensorMap) * pool);
  L.wts = off;    // per-instance weights of pw_batch_spectral_sum
  off = align256(off + sizeof(double) * n);
  L.tables = off;
  for (int i = 0; i < n; ++i) {
    const size_t N = in[i].N, NN = N * N;
    off = align256(off + NN * sizeof(float2));  // F
    off = align256(off + NN * sizeof(float));   // G
    off = align256(off + N * sizeof(float2));   // twiddles
    off = align256(off + N * sizeof(float2));   // output propagators
    off = align256(off + N * sizeof(float2));   // per-axis input factors
    off = align256(off + NN * sizeof(float2));  // W(P1, .)
  }
  L.pool = off;
  L.slot_bytes = align256((size_t)maxN * maxN * maxN * maxN * sizeof(float2));
  off += L.slot_bytes * pool;
  L.total = off;
  return L;
}

}  // namespace

struct pw_batch {
  int n, pool, chunk;
  int mode;  // PW_BATCH_PERSISTENT or PW_BATCH_SEQUENCED
  std::vector<CUtensorMap> vmaps;  // per instance: its V slot in the layout of its N
  char* base;
  Layout L;
  cudaStream_t stream;
  std::vector<pw::batch::Inst> inst;
  std::vector<int> stalled;  // instances whose pass-A items are left out (failure-detection test)
  std::vector<double> dx_out;  // output sampling of every instance (lambda z / (N dxi))
  int nitems;
  long long wait_cycles;
};

namespace {

pw_status build_items(pw_batch* b) {
  std::vector<pw::batch::Item> items;
  // One pass = J = ceil(S / chunk) items.  N = 128 (register-resident engine, whose pass B
  // gathers 8 bytes from every 32-byte run of V): strided items, item j takes slices j, j + J,
  // j + 2 J, ..., so that neighbouring CTAs gather the columns of one run together.  Other sizes:
  // contiguous ranges of chunk slices (measured slightly faster there).
  auto add = [&](int i, int pass) {
    if (pass == 0 && b->stalled[i]) return;
    const int S = b->inst[i].slices;
    const int J = (S + b->chunk - 1) / b->chunk;
    for (int j = 0; j < J; ++j) {
      if (b->inst[i].N == 128) items.push_back({i, pass, j, (S - j + J - 1) / J, J});
      else items.push_back({i, pass, j * b->chunk, j + 1 < J ? b->chunk : S - j * b->chunk, 1});
    }
  };
  // Lookahead of L instances: A(0) .. A(L-1), then B(i), A(i + L) for i = 0, 1, ...  B(i) waits
  // for A(i), listed L phases earlier; A(i + L) reuses the slot of instance i + L - pool and waits
  // for its pass B, listed pool - L phases earlier.  L = pool - 2 (at least 1) leaves two phases
  // between every wait and the items it waits on, and every awaited item precedes its waiter.
  const int L = b->pool >= 3 ? b->pool - 2 : 1;
  for (int i = 0; i < L && i < b->n; ++i) add(i, 0);
  for (int i = 0; i < b->n; ++i) {
    add(i, 1);
    if (i + L < b->n) add(i + L, 0);
  }
  if ((int)items.size() > b->L.max_items) return fail(PW_EINVAL, "item list exceeds the workspace");
  b->nitems = (int)items.size();
  cudaError_t e = cudaMemcpyAsync(b->base + b->L.items, items.data(), items.size() * sizeof(pw::batch::Item),
                                  cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return cuda_fail(e, "uploading the item list");
  return PW_OK;
}

int num_sms() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

}  // namespace

extern "C" {

size_t pw_batch_workspace_bytes(const pw_instance* inst, int n, int pool) {
  if (!inst || n <= 0 || pool <= 0) return 0;
  return layout(inst, n, pool).total;
}

pw_status pw_batch_create(pw_batch** out, const pw_instance* in, int n, int pool, void* dev_ws, size_t ws_bytes,
                          void* stream) {
  pwi::set_last_error("");
  if (!out) return fail(PW_EINVAL, "out is null");
  *out = nullptr;
  if (!in || n <= 0) return fail(PW_EINVAL, "need at least one instance");
  if (pool <= 0) return fail(PW_EINVAL, "pool depth must be >= 1");
  if (!dev_ws) return fail(PW_EINVAL, "workspace is null");
  for (int i = 0; i < n; ++i) {
    const pw_instance& q = in[i];
    if (!batch_n(q.N)) return fail(PW_EUNSUPPORTED, "instance %d: N = %d (batched runs take N in {16, 32, 64, 96, 128})", i, q.N);
    if (!finite_pos(q.dxi_m) || !finite_pos(q.lambda_m) || !finite_pos(q.z_m) || !finite_pos(q.sigma_S_m) ||
        !finite_pos(q.sigma_mu_m))
      return fail(PW_EINVAL, "instance %d: lengths must be finite and > 0", i);
    if (!std::isfinite(q.amplitude) || !std::isfinite(q.aperture_m) || !std::isfinite(q.lens_f_m))
      return fail(PW_EINVAL, "instance %d: amplitude, aperture and focal length must be finite", i);
    if (q.iP < 0 || q.jP < 0 || q.iP >= q.N || q.jP >= q.N) return fail(PW_EINVAL, "instance %d: P1 outside the grid", i);
    if (!q.dev_S) return fail(PW_EINVAL, "instance %d: dev_S is required", i);
  }
  const Layout L = layout(in, n, pool);
  if (ws_bytes < L.total) return fail(PW_ESIZE, "workspace needs %zu bytes (got %zu)", L.total, ws_bytes);
  pw_batch* b = new pw_batch{};
  b->n = n;
  b->pool = pool;
  b->chunk = 8;
  b->base = reinterpret_cast<char*>(dev_ws);
  b->L = L;
  b->stream = reinterpret_cast<cudaStream_t>(stream);
  b->stalled.assign(n, 0);
  b->wait_cycles = 2000000000LL;  // ~1 s at 2 GHz
  // sequenced launches fill the GPU with one instance at a time from N = 64 on; smaller instances
  // are too small for that and share the persistent launch
  bool all_large = true;
  for (int i = 0; i < n; ++i) all_large = all_large && in[i].N >= 64;
  b->mode = all_large ? PW_BATCH_SEQUENCED : PW_BATCH_PERSISTENT;
  b->vmaps.resize(n);
  for (int i = 0; i < n; ++i) {
    pw_status st = pwi::encode_vmap(&b->vmaps[i], b->base + L.pool + L.slot_bytes * (i % pool), in[i].N);
    if (st != PW_OK) {
      delete b;
      return st;
    }
  }
  std::vector<pw::TableArgs> targs(n);
  std::vector<float2*> mus(n);
  b->inst.resize(n);
  size_t off = L.tables;
  for (int i = 0; i < n; ++i) {
    const pw_instance& q = in[i];
    const int N = q.N;
    const size_t NN = (size_t)N * N;
    pw::batch::Inst& d = b->inst[i];
    d.N = N;
    d.iP = q.iP;
    d.jP = q.jP;
    d.slices = (int)NN;
    d.A = (float)q.amplitude;
    const double lz = q.lambda_m * q.z_m;
    d.scale = (float)((q.dxi_m * q.dxi_m / lz) * (q.dxi_m * q.dxi_m / lz));
    float2* F = reinterpret_cast<float2*>(b->base + off);
    off = align256(off + NN * sizeof(float2));
    float* G = reinterpret_cast<float*>(b->base + off);
    off = align256(off + NN * sizeof(float));
    float2* tw = reinterpret_cast<float2*>(b->base + off);
    off = align256(off + N * sizeof(float2));
    float2* Eo = reinterpret_cast<float2*>(b->base + off);
    off = align256(off + N * sizeof(float2));
    float2* Ei = reinterpret_cast<float2*>(b->base + off);
    off = align256(off + N * sizeof(float2));
    d.row = reinterpret_cast<float2*>(b->base + off);
    off = align256(off + NN * sizeof(float2));
    d.F = F;
    d.G = G;
    d.tw = tw;
    d.Eout = Eo;
    d.Ein = Ei;
    d.mask = reinterpret_cast<const float2*>(q.dev_mask);
    d.V = reinterpret_cast<float2*>(b->base + L.pool + L.slot_bytes * (i % pool));
    d.vmap = N == 128 ? b->base + L.tmaps + sizeof(CUtensorMap) * (i % pool) : nullptr;
    d.W = reinterpret_cast<float2*>(q.dev_W);
    d.S = q.dev_S;
    mus[i] = reinterpret_cast<float2*>(q.dev_mu);
    // FP64 tables: same quantities as the single-instance path (propagator phases in turns)
    pw::TableArgs& t = targs[i];
    t = pw::TableArgs{};
    t.N = N;
    const double invf = q.lens_f_m != 0.0 ? 1.0 / q.lens_f_m : 0.0;
    const double base = q.dxi_m * q.dxi_m / (2.0 * q.lambda_m);
    t.Kin = q.farfield ? -base * invf : base * (1.0 / q.z_m - invf);
    const double dx = lz / (N * q.dxi_m);
    t.Kout = dx * dx / (2.0 * lz);
    b->dx_out.push_back(dx);
    t.gs = q.dxi_m * q.dxi_m / (4.0 * q.sigma_S_m * q.sigma_S_m);
    t.gm = q.dxi_m * q.dxi_m / (2.0 * q.sigma_mu_m * q.sigma_mu_m);
    if (q.aperture_m > 0.0) {
      const double rp = q.aperture_m / q.dxi_m;
      t.ap_thr = rp * rp;  // r^2 is an integer: the integer floor gives the same decision
      d.ap_ithr = t.ap_thr >= 2147483647.0 ? 2147483647 : (int)std::floor(t.ap_thr);
    } else {
      t.ap_thr = -1.0;
      d.ap_ithr = -1;
    }
    t.mask = reinterpret_cast<const float2*>(q.dev_mask);
    t.F = F;
    t.G = G;
    t.tw = tw;
    t.Eout = Eo;
    t.Ein = Ei;
  }
  bool any128 = false;
  for (int i = 0; i < n; ++i) any128 = any128 || in[i].N == 128;
  std::vector<CUtensorMap> maps(pool);
  if (any128) {
    for (int k = 0; k < pool; ++k) {
      pw_status st = pwi::encode_vmap(&maps[k], b->base + L.pool + L.slot_bytes * k, 128);
      if (st != PW_OK) {
        delete b;
        return st;
      }
    }
  }
  cudaError_t e = cudaMemcpyAsync(b->base + L.inst, b->inst.data(), sizeof(pw::batch::Inst) * n,
                                  cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess && any128)
    e = cudaMemcpyAsync(b->base + L.tmaps, maps.data(), sizeof(CUtensorMap) * pool, cudaMemcpyHostToDevice,
                        b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->base + L.targs, targs.data(), sizeof(pw::TableArgs) * n, cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->base + L.mu, mus.data(), sizeof(float2*) * n, cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess)  // counters and the error flag start at zero (the workspace may hold old data)
    e = cudaMemsetAsync(b->base + L.counters, 0, sizeof(int) * (2 * (size_t)n + 2), b->stream);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(pw::batch::batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)pw::batch::smem_bytes());
  if (e != cudaSuccess) {
    delete b;
    return cuda_fail(e, "batch set-up");
  }
  pw_status st = build_items(b);
  if (st != PW_OK) {
    delete b;
    return st;
  }
  *out = b;
  return PW_OK;
}

pw_status pw_batch_run(pw_batch* b) {
  pwi::set_last_error("");
  if (!b) return fail(PW_EINVAL, "null batch");
  int* cnt = reinterpret_cast<int*>(b->base + b->L.counters);
  cudaError_t e;
  if (b->mode == PW_BATCH_PERSISTENT) {
    e = cudaMemsetAsync(cnt, 0, sizeof(int) * (2 * (size_t)b->n + 1), b->stream);
    if (e != cudaSuccess) return cuda_fail(e, "resetting the batch counters");
  }
  int maxNN = 0;
  for (const auto& d : b->inst) maxNN = d.slices > maxNN ? d.slices : maxNN;
  dim3 tg((maxNN + 255) / 256, b->n);
  pw::batch::batch_tables_kernel<<<tg, 256, 0, b->stream>>>(reinterpret_cast<const pw::TableArgs*>(b->base + b->L.targs));
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "batch tables launch");
  if (b->mode == PW_BATCH_SEQUENCED) {
    // one instance after the other on the single-instance kernels (stream order reuses the slots)
    for (int i = 0; i < b->n; ++i) {
      const pw::batch::Inst& d = b->inst[i];
      pw::PassAArgs a{};
      a.F = d.F;
      a.G = d.G;
      a.tw = d.tw;
      a.A = d.A;
      pw::PassBArgs pb{};
      pb.V = d.V;
      pb.tw = d.tw;
      pb.Eout = d.Eout;
      pb.W = d.W;
      pb.S = d.S;
      pb.scale = d.scale;
      pb.row = d.row;
      pb.iP = d.iP;
      pb.jP = d.jP;
      e = pwi::launch_batch_instance(d.N, b->vmaps[i], a, pb, d.Ein, d.mask, d.ap_ithr, b->stream);
      if (e != cudaSuccess) return cuda_fail(e, "batch instance launch");
    }
    dim3 mg((maxNN + 255) / 256, b->n);
    pw::batch::batch_mu_kernel<<<mg, 256, 0, b->stream>>>(reinterpret_cast<const pw::batch::Inst*>(b->base + b->L.inst),
                                                          reinterpret_cast<float2* const*>(b->base + b->L.mu));
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "batch mu launch");
    return PW_OK;
  }
  pw::batch::Args g{};
  g.inst = reinterpret_cast<const pw::batch::Inst*>(b->base + b->L.inst);
  g.items = reinterpret_cast<const pw::batch::Item*>(b->base + b->L.items);
  g.nitems = b->nitems;
  g.pool = b->pool;
  g.next = cnt + 2 * b->n;
  g.doneA = cnt;
  g.doneB = cnt + b->n;
  g.err = cnt + 2 * b->n + 1;
  g.wait_cycles = b->wait_cycles;
  pw::batch::batch_kernel<<<num_sms(), pw::batch::NT, pw::batch::smem_bytes(), b->stream>>>(g);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "batch kernel launch");
  dim3 mg((maxNN + 255) / 256, b->n);
  pw::batch::batch_mu_kernel<<<mg, 256, 0, b->stream>>>(g.inst, reinterpret_cast<float2* const*>(b->base + b->L.mu));
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "batch mu launch");
  return PW_OK;
}

pw_status pw_batch_check(pw_batch* b) {
  pwi::set_last_error("");
  if (!b) return fail(PW_EINVAL, "null batch");
  int flag = 0;
  int* err = reinterpret_cast<int*>(b->base + b->L.counters) + 2 * b->n + 1;
  cudaError_t e = cudaMemcpyAsync(&flag, err, sizeof(int), cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return cuda_fail(e, "reading the batch error flag");
  if (flag) {
    e = cudaMemsetAsync(err, 0, sizeof(int), b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda_fail(e, "clearing the batch error flag");
    return fail(PW_ETIMEOUT, "a bounded wait of the batched launch gave up; some outputs are invalid");
  }
  return PW_OK;
}

pw_status pw_batch_set_chunk(pw_batch* b, int chunk) {
  pwi::set_last_error("");
  if (!b) return fail(PW_EINVAL, "null batch");
  if (chunk < kMinChunk) return fail(PW_EINVAL, "chunk must be >= %d", kMinChunk);
  b->chunk = chunk;
  return build_items(b);
}

pw_status pw_batch_spectral_sum(pw_batch* b, const double* weights, float* dev_I) {
  pwi::set_last_error("");
  if (!b || !weights || !dev_I) return fail(PW_EINVAL, "null argument");
  const int N = b->inst[0].N;
  for (int i = 0; i < b->n; ++i) {
    if (b->inst[i].N != N) return fail(PW_EINVAL, "instance %d: N = %d differs from instance 0 (N = %d)", i, b->inst[i].N, N);
    if (std::fabs(b->dx_out[i] / b->dx_out[0] - 1.0) > 1e-9)
      return fail(PW_EINVAL, "instance %d: output sampling %.9g m differs from instance 0 (%.9g m): no common grid",
                  i, b->dx_out[i], b->dx_out[0]);
    if (!std::isfinite(weights[i])) return fail(PW_EINVAL, "weight %d is not finite", i);
  }
  double* w = reinterpret_cast<double*>(b->base + b->L.wts);
  cudaError_t e = cudaMemcpyAsync(w, weights, sizeof(double) * b->n, cudaMemcpyHostToDevice, b->stream);
  if (e != cudaSuccess) return cuda_fail(e, "uploading the weights");
  const int NN = N * N;
  pw::batch::batch_sum_kernel<<<(NN + 255) / 256, 256, 0, b->stream>>>(
      reinterpret_cast<const pw::batch::Inst*>(b->base + b->L.inst), w, b->n, dev_I, NN);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "spectral sum launch");
  return PW_OK;
}

pw_status pw_batch_set_mode(pw_batch* b, int mode) {
  pwi::set_last_error("");
  if (!b) return fail(PW_EINVAL, "null batch");
  if (mode != PW_BATCH_PERSISTENT && mode != PW_BATCH_SEQUENCED) return fail(PW_EINVAL, "unknown batch mode %d", mode);
  b->mode = mode;
  return PW_OK;
}

pw_status pw_batch_get_mode(const pw_batch* b, int* mode) {
  pwi::set_last_error("");
  if (!b || !mode) return fail(PW_EINVAL, "null argument");
  *mode = b->mode;
  return PW_OK;
}

pw_status pw_batch_get_chunk(const pw_batch* b, int* chunk) {
  pwi::set_last_error("");
  if (!b || !chunk) return fail(PW_EINVAL, "null argument");
  *chunk = b->chunk;
  return PW_OK;
}

pw_status pw_batch_autotune(pw_batch* b, int* chunk_out) {
  pwi::set_last_error("");
  if (!b) return fail(PW_EINVAL, "null batch");
  // candidates: the sequenced launches, and the persistent launch at each chunk size
  const int cand[][2] = {{PW_BATCH_SEQUENCED, 0},   {PW_BATCH_PERSISTENT, 4},  {PW_BATCH_PERSISTENT, 8},
                         {PW_BATCH_PERSISTENT, 16}, {PW_BATCH_PERSISTENT, 32}, {PW_BATCH_PERSISTENT, 64}};
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return cuda_fail(cudaGetLastError(), "autotune events");
  float best = 1e30f;
  int best_m = b->mode, best_c = b->chunk;
  pw_status st = PW_OK;
  for (const auto& mc : cand) {
    b->mode = mc[0];
    if (mc[0] == PW_BATCH_PERSISTENT && (st = pw_batch_set_chunk(b, mc[1])) != PW_OK) break;
    if ((st = pw_batch_run(b)) != PW_OK) break;  // warm-up
    cudaEventRecord(e0, b->stream);
    if ((st = pw_batch_run(b)) != PW_OK) break;
    cudaEventRecord(e1, b->stream);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) {
      best = ms;
      best_m = mc[0];
      best_c = mc[0] == PW_BATCH_PERSISTENT ? mc[1] : best_c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != PW_OK) return st;
  if ((st = pw_batch_check(b)) != PW_OK) return st;
  b->mode = best_m;
  if (chunk_out) *chunk_out = best_c;
  return pw_batch_set_chunk(b, best_c);
}

pw_status pw_batch_inject_stall(pw_batch* b, int instance, double wait_s) {
  pwi::set_last_error("");
  if (!b) return fail(PW_EINVAL, "null batch");
  if (instance < 0 || instance >= b->n) return fail(PW_EINVAL, "instance out of range");
  if (!(wait_s > 0.0) || !std::isfinite(wait_s)) return fail(PW_EINVAL, "wait must be finite and > 0");
  b->stalled[instance] = 1;
  b->wait_cycles = (long long)(wait_s * 2.0e9);
  return build_items(b);
}

pw_status pw_batch_destroy(pw_batch* b) {
  pwi::set_last_error("");
  if (!b) return PW_OK;
  cudaError_t e = cudaStreamSynchronize(b->stream);
  delete b;
  if (e != cudaSuccess) return cuda_fail(e, "stream synchronize in batch destroy");
  return PW_OK;
}

}  // extern "C"
