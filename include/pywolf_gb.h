/*
 * pywolf_gb.h -- C ABI of the GB300 (sm_103a) library for the propagation of the 4D
 * cross-spectral density (CSD) W(x1, y1, x2, y2; omega) of a planar, partially coherent
 * source (PyWolf, arXiv 2203.02734).
 *
 * Data model (Sec. 3.1, Eqs. point, n12; the block layout of Sec. 3.1):
 *   A CSD array (CSDA) is an N x N x N x N row-major array of complex64 (pw_c32),
 *   element W[i1][j1][i2][j2] at offset ((i1*N + j1)*N + i2)*N + j2, sampling
 *   W(xi1, xi2) with xi(i) = (i - N/2) d and eta(j) = (N/2 - j) d, where d is the
 *   sampling of the current plane.  N must be even (N/2 is an index, Sec. 3.1).
 *
 * Pipeline (Algorithm 1): create a handle on caller-owned device buffers, describe the
 *   source (GSM model, aperture, thin lens, arbitrary mask, or an uploaded CSDA), then
 *   propagate (Fresnel, Eq. W_fresnel; or far field, Eq. W_farfield).  The source is
 *   generated inside the propagation (it is never materialised on its own).  After a
 *   propagation, the handle's current plane is the output plane; its CSDA is in dev_W and
 *   its sampling is lambda z / (N d) (Eq. spatial_resolution).  S (Eq. defS, Algorithm 4)
 *   and mu (Eq. defMu, Algorithm coherence) can be read for the current plane.
 *
 * Conventions fixed here (readings of the paper):
 *   - point 1 carries the conjugated kernel (Eq. W_general), so its DFT has sign +1 and the
 *     point-2 DFT sign -1 (Algorithm 2 applies the direct FFT to the point-2 slices);
 *   - scale s = d^4 / (lambda z)^2 (Eq. C with Lambda = 1/(i lambda)) for both regimes;
 *   - the circular aperture is inclusive, decided as integer r^2 <= (a/d)^2 in FP64.
 *
 * Ownership: every large buffer (the N^4 CSDA dev_W and the N^4 work buffer dev_work)
 *   belongs to the caller and must stay valid until pw_csd_destroy.  The library allocates
 *   only small O(N^2) tables (chirps, twiddles, GSM factors, S) per handle.
 * Streams: all device work is enqueued on the handle's stream and is asynchronous; results
 *   in device memory are valid once that stream has been synchronised.
 * Alignment: dev_W and dev_work 16-byte aligned (bulk and tensor copies); complex64 arrays
 *   (masks, uploaded CSDAs, mu) 8-byte aligned; float arrays 4-byte aligned.  A misaligned
 *   pointer returns PW_EINVAL before any device work.
 * Errors: no call aborts, traps or prints.  Each returns a pw_status; the message of the
 *   last failure on the calling thread is returned by pw_last_error().  Invalid arguments
 *   are rejected on the host before any device work is enqueued.
 */
#ifndef PYWOLF_GB_H
#define PYWOLF_GB_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pw_csd pw_csd; /* opaque handle */

typedef enum pw_status {
  PW_OK = 0,
  PW_EINVAL = 1,      /* invalid argument (odd N, non-finite or non-positive length, ...) */
  PW_ESIZE = 2,       /* a caller buffer is smaller than required */
  PW_ECUDA = 3,       /* a CUDA runtime call or kernel launch failed */
  PW_ETIMEOUT = 4,    /* a bounded device-side wait gave up */
  PW_ESTATE = 5,      /* call not valid in the handle's current state */
  PW_EUNSUPPORTED = 6 /* valid request that this build has no kernel plan for (e.g. this N) */
} pw_status;

typedef struct pw_c32 { float re, im; } pw_c32; /* layout-compatible with complex64 */

/* Human-readable text of the last failure on the calling thread ("" if none).  The
 * pointer stays valid until the next pw_* call on this thread. */
const char* pw_last_error(void);

/* Name of a status code ("PW_OK", ...). */
const char* pw_status_string(pw_status s);

/* 1 if this build has an FFT propagation plan for grid size N, else 0.  Other even N up to
 * PW_MAX_N propagate on the dense path (see pw_csd_set_padding). */
int pw_supported_n(int N);
enum { PW_MAX_N = 512 };

/* Bytes required for each of dev_W and dev_work: N^4 * sizeof(pw_c32). */
size_t pw_csda_bytes(int N);

/* Create a handle for an N x N x N x N CSDA on the current CUDA device.
 *   N         even, 2 <= N <= PW_MAX_N (FFT plans where pw_supported_n(N), else the dense path)
 *   dxi_m     sampling d of the source plane in metres (finite, > 0)           (Eq. point)
 *   lambda_m  wavelength in metres (finite, > 0); omega = 2 pi c / lambda     (Eq. q_factor)
 *   dev_W     device buffer of >= pw_csda_bytes(N) bytes: holds an uploaded source CSDA
 *             (pw_source_array may point here) and receives every propagated CSDA
 *   dev_work  device buffer of >= pw_csda_bytes(N) bytes, scratch for the half-transformed
 *             CSDA between the two passes; must not overlap dev_W
 *   stream    cudaStream_t to enqueue on (NULL = legacy default stream)
 * Returns PW_EINVAL / PW_ESIZE / PW_EUNSUPPORTED for bad arguments, PW_ECUDA if the small
 * per-handle tables cannot be allocated.  *out is NULL on failure. */
pw_status pw_csd_create(pw_csd** out, int N, double dxi_m, double lambda_m,
                        pw_c32* dev_W, size_t W_bytes, pw_c32* dev_work, size_t work_bytes,
                        void* stream);

/* Release the handle and its small tables (synchronises the handle's stream first).
 * Does not free dev_W / dev_work.  NULL is accepted. */
pw_status pw_csd_destroy(pw_csd* h);

/* Change the stream used by later calls. */
pw_status pw_csd_set_stream(pw_csd* h, void* stream);

/* Synchronise the handle's stream and report whether a bounded device-side wait gave up in
 * any kernel since the last check (PW_ETIMEOUT: the results of that work are invalid); clears
 * the condition.  PW_OK otherwise. */
pw_status pw_csd_check(pw_csd* h);

/* Start over at a source plane with sampling dxi_m (finite, > 0): forgets the current
 * plane's CSDA, source and masks (Algorithm 1 from its first line), keeps the buffers and
 * tables.  No device work. */
pw_status pw_csd_reset(pw_csd* h, double dxi_m);

/* Gaussian Schell-model source (Sec. 5.4, with the minus signs the printed exponents lost):
 *   W0 = A exp(-(|xi1|^2 + |xi2|^2) / (4 sigma_S^2)) exp(-|xi1 - xi2|^2 / (2 sigma_mu^2)).
 * sigma_S_m, sigma_mu_m finite > 0; amplitude finite.  Recorded only; generated inside the
 * next propagation.  Replaces any previous source of the current plane. */
pw_status pw_source_gsm(pw_csd* h, double sigma_S_m, double sigma_mu_m, double amplitude);

/* Circular aperture Y(xi) = 1 for |xi| <= a (appendix, Eq. circle), applied as
 * Y(xi1) W Y(xi2) at the current plane before the next propagation.  radius_m <= 0
 * removes it.  Must be finite. */
pw_status pw_source_aperture(pw_csd* h, double radius_m);

/* Thin lens T(xi) = q*(f, xi) (Sec. 2.2), applied as T*(xi1) W T(xi2) at the current plane
 * before the next propagation.  focal_m == 0 removes it; otherwise finite, non-zero
 * (negative = diverging lens). */
pw_status pw_source_lens(pw_csd* h, double focal_m);

/* Arbitrary complex mask m (N x N, row-major over (i, j), device memory) applied as
 * m*(xi1) W m(xi2) at the current plane before the next propagation (pupil, phase screen,
 * amplitude mask; Sec. 2.2 and Sec. 5.3).  The pointer is read during the next
 * propagation, not copied: keep it valid until then.  NULL removes it. */
pw_status pw_source_mask(pw_csd* h, const pw_c32* dev_mask);

/* Use an uploaded CSDA as the source of the current plane (Sec. 3.2: a CSDA exported by a
 * previous run or built by the user).  dev_W0 (N^4 complex64, device) may be dev_W itself.
 * hermitian != 0 declares W0(xi2, xi1) = conj W0(xi1, xi2) (true of every CSD, Sec. 3.3), which
 * lets the second pass store its output rows contiguously; hermitian == 0 selects the
 * general (strided-store) second pass for N <= 128.  The three-pass engine at N = 256 and the
 * dense path never use Hermiticity and need no declaration.  Read during the next propagation. */
pw_status pw_source_array(pw_csd* h, const pw_c32* dev_W0, int hermitian);

/* Delta-correlated (spatially incoherent) source W0 = weight d(xi1) delta(xi1 - xi2) with real
 * d (N x N, device), the incoherent sources of Sec. 5.2 / 5.3 (delta-correlated CSD).  Recorded;
 * generated inside the next propagation.  Also the adjoint source of an S-loss: if W_B = P(W0)
 * and L depends on S_B = Re diag W_B, dL/dW_B* is this diagonal with d = dL/dS_B, weight = 1/2. */
pw_status pw_source_diagonal(pw_csd* h, const float* dev_d, double weight);

/* Parameter gradients from the adjoint (the paper has no counterpart; backward of a loss on S or
 * on W through the propagation).  With W_B = P(W0) for the amplitude-masked GSM source
 * W0 = A a(xi1) a(xi2) G (Sec. 5.4; a real N x N, dev_amask NULL for a = 1) propagated over z_m
 * (farfield selects Eq. W_farfield), the adjoint P^H(Y) equals (d/dx)^4 conj(P'(conj Y)), where P'
 * is the Fresnel propagation over the same z_m from the output sampling dx back onto the source
 * grid d (times q(xi1) q*(xi2) in the far field).  Usage: on a handle whose current plane has
 * sampling dx, set the conjugate of dL/dW_B* as its source (pw_source_diagonal for an S-loss),
 * pw_propagate_fresnel(z_m), then call this: it reads the propagated CSDA (on grid d) and writes
 * dev_grad3 = [dL/dsigma_S, dL/dsigma_mu, dL/dA] (3 doubles, device) and, if non-NULL,
 * dev_grad_mask = dL/da (N x N float32, device); W0bar is never stored.  Asynchronous. */
pw_status pw_gsm_gradient(pw_csd* h, double sigma_S_m, double sigma_mu_m, double amplitude,
                          const float* dev_amask, double lambda_m, double z_m, int farfield,
                          double* dev_grad3, float* dev_grad_mask);

/* The adjoint of one propagation for a real loss L on S and mu of its output plane (the paper has
 * no adjoint; it is the transpose of the linear map of Eq. W_fresnel / Eq. W_farfield, reading R17).
 * Upstream gradients follow the real convention g = dL/dRe + i dL/dIm (torch's for complex
 * tensors).  With S(x) = Re W_B(x, x) (Algorithm 4) and mu(x) = W_B(P1, x) / sqrt(S(P1) S(x))
 * (Algorithm coherence, 0 where S(P1) S(x) <= 0), dL/dW_B* is (1/2) dL/dS on the diagonal plus
 * (1/2) gmu / sqrt(S(P1) S(x)) on the row of P1, dL/dS taking the mu term through S (reading R22);
 * the call builds that source in-kernel, propagates it back (P^H, Fresnel over z from the output
 * sampling dx onto the source grid d = lambda z / (N dx)) and forms the requested gradients:
 *   dev_grad3 / dev_grad_amask: dL/d(sigma_S, sigma_mu, A) and dL/da of the amplitude-masked GSM
 *     source W0 = A a(xi1) a(xi2) G (Sec. 5.4) that the forward propagation started from, reduced
 *     in the epilogue of the adjoint's second pass (W0bar is never stored; at N = 256 it goes
 *     through dev_W and one gradient kernel);
 *   grad_W0: dL/dRe W0 + i dL/dIm W0 for W0 taken as a general complex N^4 array, written into
 *     dev_W (a second, non-Hermitian adjoint propagation when both kinds are asked with a mu term).
 * The handle's current sampling must be the forward's output sampling dx (true right after the
 * forward propagation, or after pw_csd_reset(h, dx)); the current plane's contents are not used.
 * dev_work is used as scratch; dev_W is overwritten (the gradient with grad_W0, else unspecified).
 * On return the handle is at the source plane (sampling d) with no source recorded.  Asynchronous
 * on the handle's stream.
 * Errors: PW_EINVAL for a null or misaligned pointer, a P1 outside the grid, dev_dmu without
 * dev_S / dev_mu, no upstream gradient or no output, invalid GSM parameters with dev_grad3 /
 * dev_grad_amask; PW_EUNSUPPORTED on a zero-padded grid or one without an FFT plan. */
typedef struct pw_adjoint {
  const float* dev_dS;     /* N x N dL/dS of the output plane (float32, device), or NULL */
  const pw_c32* dev_dmu;   /* N x N dL/dRe mu + i dL/dIm mu of mu(P1, .) (device), or NULL */
  int iP, jP;              /* P1 of mu */
  const float* dev_S;      /* N x N S of the output plane (device), needed with dev_dmu */
  const pw_c32* dev_mu;    /* N x N mu(P1, .) of the output plane (device), needed with dev_dmu */
  double sigma_S_m, sigma_mu_m, amplitude;  /* the forward's GSM source, for dev_grad3 / dev_grad_amask */
  const float* dev_amask;  /* N x N real amplitude mask a of that source (device), or NULL for a = 1 */
  double* dev_grad3;       /* out: [dL/dsigma_S, dL/dsigma_mu, dL/dA] (3 doubles, device), or NULL */
  float* dev_grad_amask;   /* out: N x N dL/da (float32, device), or NULL */
  int grad_W0;             /* nonzero: write dL/dRe W0 + i dL/dIm W0 (N^4 complex64) into dev_W */
} pw_adjoint;
pw_status pw_propagate_fresnel_adjoint(pw_csd* h, double z_m, const pw_adjoint* a);
pw_status pw_propagate_farfield_adjoint(pw_csd* h, double z_m, const pw_adjoint* a);

/* Fresnel propagation over distance z_m > 0 (Eq. W_fresnel; Algorithm 2 without the
 * far-field switch).  Result: dev_W holds W at the new plane, sampling lambda z/(N d);
 * S of the new plane is computed on the way.  Returns PW_ESTATE if no source was set. */
pw_status pw_propagate_fresnel(pw_csd* h, double z_m);

/* Far-field propagation over z_m > 0 (Eq. W_farfield: input propagators set to 1, output
 * propagators and sampling as for Fresnel). */
pw_status pw_propagate_farfield(pw_csd* h, double z_m);

/* Sampling d of the current plane in metres. */
pw_status pw_get_sampling(const pw_csd* h, double* d_m);

/* Spectral density S[i][j] = Re W[i][j][i][j] of the current plane (Eq. defS, Algorithm 4)
 * into dev_S (N x N float32, device). */
pw_status pw_spectral_density(pw_csd* h, float* dev_S);

/* Spectral degree of coherence mu(P1, x) = W(P1, x) / sqrt(S(P1) S(x)) of the current plane
 * (Eq. defMu, Algorithm coherence) for P1 = (iP, jP), 0 <= iP, jP < N, into dev_mu (N x N
 * complex64, device); mu := 0 where S(P1) S(x) <= 0. */
pw_status pw_degree_of_coherence(pw_csd* h, int iP, int jP, pw_c32* dev_mu);

/* Zero padding with cropped output (Sec. 3.2: "if we use zero padding to perform the FFT, we must
 * consider the total size N_z in the term N ... even if we crop the matrix to its original size"):
 * later propagations evaluate the transform of size Nz of the source placed at the centre of an
 * Nz x Nz grid, at the central N x N output samples, with output sampling
 * dx = lambda z / (Nz dxi) instead of lambda z / (N dxi).
 *   Nz = 0 or Nz = N: no padding (the default).
 *   Nz > N with Nz - N even: padding.
 * A padded propagation (and any propagation at an N without an FFT plan) runs as four dense axis
 * contractions in FP32: the pruned DFT of size Nz with the propagators folded in, one N x N
 * complex matrix per axis (O(N) work per point instead of O(log N)).  It accepts every source
 * (GSM, uploaded CSDA, diagonal, propagated plane, with masks), produces the same outputs
 * (W, S, mu); its arithmetic follows pw_csd_set_dft_mode.
 * Returns PW_EINVAL for Nz < N (other than 0), odd Nz - N or Nz > 1 << 20; kept across
 * pw_csd_reset. */
pw_status pw_csd_set_padding(pw_csd* h, int Nz);
pw_status pw_csd_get_padding(const pw_csd* h, int* Nz);

/* Arithmetic of the DFT work that has a tensor-core form:
 *   - the first radix-16 stage of the first pass at N = 256 (FFT path, GSM sources; all other
 *     stages and FFT grid sizes always run FP32 codelets on the CUDA cores), and
 *   - the four dense axis contractions of the padded / no-FFT-plan path (N <= 256).
 *   PW_DFT_AUTO (default): the faster of the two per path, as measured on GB300: FP32 codelets on
 *     the FFT paths, the tensor cores for the dense contractions (N <= 256; FP32 above).
 *   PW_DFT_FP32: FP32 on the CUDA cores everywhere (codelets with FP64-derived twiddles, dense FP32
 *     complex products).
 *   PW_DFT_TC_BF16X3: the products as GEMMs on the tensor cores (tcgen05, BF16 operands,
 *     FP32 accumulation in tensor memory), each FP32 operand split into three BF16 parts and six
 *     partial products kept (relative error ~5e-7 per stage).
 * Returns PW_EINVAL for an unknown mode, PW_EUNSUPPORTED for PW_DFT_TC_BF16X3 at N > 256.  On the
 * FFT path at N = 256 a later propagation of a source other than the Gaussian Schell model
 * returns PW_EUNSUPPORTED while the tensor-core mode is set; at other FFT grid sizes the mode has
 * no effect.  A bounded device wait of a tensor-core kernel that gives up is reported by
 * pw_csd_check (PW_ETIMEOUT). */
enum { PW_DFT_AUTO = 0, PW_DFT_FP32 = 1, PW_DFT_TC_BF16X3 = 2 };

/* Failure-detection test hook (no counterpart in the paper): in the next dense propagation on the
 * tensor cores, CTA 0 of the first contraction never starts the copy of operand chunk `chunk`
 * (chunk >= 1), or its splitting warps never announce the A tile of chunk -chunk (chunk <= -1;
 * the copy of that chunk's B operand is then already in flight).  The bounded wait gives up after
 * about a second; the kernel waits (bounded) for its committed MMAs and its started copies, frees
 * its tensor memory and returns; that propagation's results are invalid, and pw_csd_check reports
 * PW_ETIMEOUT.  0 turns it off; it applies to one propagation.  No GPU fault is involved. */
pw_status pw_csd_inject_stall(pw_csd* h, int chunk);
pw_status pw_csd_set_dft_mode(pw_csd* h, int mode);
pw_status pw_csd_get_dft_mode(const pw_csd* h, int* mode);

/* Per-pass timing (measurement aid, no counterpart in the paper).  pw_csd_enable_timing
 * creates CUDA events for up to max_props propagations (0 disables and frees them); each
 * later propagation records events on the handle's stream around its first pass (source +
 * point-2 DFT) and second pass (point-1 DFT + output chirp + S).  pw_csd_pass_times waits
 * for the recorded events, returns the summed milliseconds of each pass and how many
 * propagations were recorded, and restarts the count.  Propagations beyond max_props are
 * not recorded. */
pw_status pw_csd_enable_timing(pw_csd* h, int max_props);
pw_status pw_csd_pass_times(pw_csd* h, double* ms_first, double* ms_second, int* count);
/* The same with the engine's passes apart: at N = 256 (three streaming passes) ms_first is the
 * first pass, ms_second and ms_third the second and third; elsewhere ms_third is 0. */
pw_status pw_csd_pass_times3(pw_csd* h, double* ms_first, double* ms_second, double* ms_third, int* count);

/* ---- Batched runs: many instances in one persistent launch --------------------------------
 * For the polychromatic case of Sec. 6 (future work in the paper: many frequencies of a
 * spectrum), several distances and uneven grid sizes.  Each instance is one propagation of a
 * GSM source (Sec. 5.4) times an optional aperture, thin lens and mask from its source plane;
 * it yields S (Eq. defS) and mu(P1, .) (Eq. defMu) of its output plane, and the whole propagated
 * CSDA when dev_W is given.  Two execution modes (pw_batch_set_mode, chosen by pw_batch_autotune):
 *   PW_BATCH_PERSISTENT: all instances in one persistent launch that walks a work list of
 *     (instance, pass, slice chunk) items; pass-B work of an instance starts after its pass-A
 *     work (bounded waits, see pw_batch_check);
 *   PW_BATCH_SEQUENCED: the instances one after the other on the single-instance kernels (each
 *     fills the GPU): pass A, then pass B with S, the mu numerator and W when dev_W is given;
 *     without dev_W the second pass computes only the two outputs per column that S and the mu
 *     numerator use (dot products over the point-1 pair, Eq. W_fresnel's point-1 sum at X1 = X2
 *     and at X1 = P1), reading the half-transformed CSDA in its own layout.
 * The default is SEQUENCED when every instance has N >= 64, else PERSISTENT.  In both modes the
 * half-transformed CSDAs share a pool of `pool` buffers of the largest N (instance i uses slot
 * i mod pool).  pw_batch_run enqueues only device work (no allocation, no synchronisation), so
 * the caller may capture it in a CUDA graph and replay it. */
typedef struct pw_instance {
  int N;                 /* grid size: 16, 32, 64, 96 or 128 */
  double dxi_m, lambda_m, z_m;
  int farfield;          /* 0: Fresnel (Eq. W_fresnel), 1: far field (Eq. W_farfield) */
  double sigma_S_m, sigma_mu_m, amplitude;  /* GSM source; amplitude may carry a spectral weight */
  double aperture_m;     /* <= 0: none */
  double lens_f_m;       /* 0: none */
  const pw_c32* dev_mask;/* N x N device mask or NULL */
  int iP, jP;            /* P1 of mu */
  pw_c32* dev_W;         /* N^4 device output or NULL (S and mu only) */
  float* dev_S;          /* N x N device output (required) */
  pw_c32* dev_mu;        /* N x N device output or NULL */
} pw_instance;

typedef struct pw_batch pw_batch; /* opaque */

enum { PW_BATCH_PERSISTENT = 0, PW_BATCH_SEQUENCED = 1 };

/* Bytes of device workspace pw_batch_create needs for these instances and this pool depth
 * (tables, work list, counters and `pool` half-transformed buffers of the largest N). */
size_t pw_batch_workspace_bytes(const pw_instance* inst, int n, int pool);

/* Validate the instances (N in {16, 32, 64, 96, 128}, finite positive lengths, P1 inside the
 * grid, dev_S given), lay out the caller-owned workspace (>= pw_batch_workspace_bytes) and upload
 * the descriptors and the work list (synchronises `stream`).  The output pointers are kept. */
pw_status pw_batch_create(pw_batch** out, const pw_instance* inst, int n, int pool, void* dev_workspace,
                          size_t workspace_bytes, void* stream);

/* Enqueue one batched run on the batch's stream: FP64 tables of every instance, then (persistent
 * mode) counter reset + the persistent launch or (sequenced mode) two pass launches per
 * instance, then mu.  Asynchronous; no allocation; capturable in a CUDA graph. */
pw_status pw_batch_run(pw_batch* b);

/* Synchronise and report PW_ETIMEOUT if a bounded dependency wait of a run gave up since the
 * last check (the affected outputs are invalid); clears the condition. */
pw_status pw_batch_check(pw_batch* b);

/* Slices per work item of the persistent launch (>= 4; default 8).  Rebuilds the work list
 * (synchronises). */
pw_status pw_batch_set_chunk(pw_batch* b, int chunk);
pw_status pw_batch_get_chunk(const pw_batch* b, int* chunk);

/* Execution mode: PW_BATCH_PERSISTENT or PW_BATCH_SEQUENCED (PW_EINVAL otherwise). */
pw_status pw_batch_set_mode(pw_batch* b, int mode);
pw_status pw_batch_get_mode(const pw_batch* b, int* mode);

/* Time the sequenced run and the persistent run at each candidate chunk size (4 ... 64), keep
 * the fastest mode and chunk; returns the chunk in *chunk_out if non-NULL.  Runs the batch
 * several times (synchronises). */
pw_status pw_batch_autotune(pw_batch* b, int* chunk_out);

/* Failure-detection test hook (no counterpart in the paper): leave the pass-A work of
 * `instance` out of the work list and bound every dependency wait to wait_s seconds, so that
 * the pass-B work of that instance gives up waiting and the next pw_batch_check returns
 * PW_ETIMEOUT while the other instances complete.  No device fault is involved. */
pw_status pw_batch_inject_stall(pw_batch* b, int instance, double wait_s);

/* Polychromatic intensity (Sec. 3.5: I(x) = integral of S(x, omega) over frequency; the paper
 * leaves polychromatic light to future work, Sec. 6): dev_I (N x N float32, device) =
 * sum_i weights[i] S_i(x) over all instances, with weights[i] (host, n doubles, copied before the
 * call returns) carrying the spectrum S0(omega_i) and the quadrature weight.  Needs a common
 * output grid: every instance with the same N and the same output sampling lambda_i z_i /
 * (N dxi_i) to 1e-9 relative (e.g. z_i = z0 lambda0 / lambda_i); PW_EINVAL otherwise.  Enqueued
 * on the batch's stream; reads the S of the last pw_batch_run. */
pw_status pw_batch_spectral_sum(pw_batch* b, const double* weights, float* dev_I);

/* Synchronise the stream and free the host-side state (the workspace belongs to the caller). */
pw_status pw_batch_destroy(pw_batch* b);

/* Allocation-free Fresnel propagation of a GSM source (the paper has no counterpart).
 * For callers that cannot allocate device memory: applications whose framework reserves all
 * device memory in its own pool and does not let libraries call the CUDA allocator, and
 * latency-critical loops that cannot afford the implicit device synchronisation of
 * cudaMalloc / cudaFree.  It computes what pw_csd_create + pw_source_gsm + pw_source_aperture
 * + pw_source_lens + pw_source_mask + pw_propagate_fresnel + pw_spectral_density compute on a
 * new handle, without a handle: the half-transformed CSDA and the small tables live in one
 * fixed device array inside the library (8 MiB + 12.5 KiB, held by every device that loads the
 * library until the process exits), so N is limited to 2 <= N <= 32 (even, pw_supported_n);
 * larger N returns PW_EINVAL with a message naming the limit.
 *   N, dxi_m, lambda_m, z_m, sigma_S_m, sigma_mu_m, amplitude  as for the handle calls
 *   aperture_m  radius of the inclusive circular aperture, <= 0 for none
 *   lens_f_m    focal length of the thin lens in the source plane, 0 for none
 *   dev_mask    N x N complex64 device mask applied as m*(xi1) W m(xi2), or NULL; 8-byte aligned
 *   dev_W_out   device buffer of >= N^4 * 8 bytes (W_bytes) receiving the propagated CSDA;
 *               16-byte aligned (it is written by bulk copies)
 *   dev_S_out   device buffer of N x N float32 receiving S of the output plane; 4-byte aligned
 * A misaligned pointer returns PW_EINVAL before anything is launched.
 *   stream      cudaStream_t (NULL = legacy default stream); work is asynchronous on it
 * The output sampling is lambda z / (N dxi).  The first call on a device looks up the
 * device address of the internal array (cudaGetSymbolAddress); make that first call before
 * any stream capture.  Every call on a device reuses the same array, so calls whose work
 * overlaps on the GPU (other streams, other threads) race and must be serialised by the
 * caller.  Each call overwrites every byte of the array that it reads later, so no state is
 * carried from one call to the next.  Allocates nothing: no cudaMalloc, no cudaFree. */
pw_status pw_propagate_gsm_fresnel_noalloc(int N, double dxi_m, double lambda_m, double z_m,
                                           double sigma_S_m, double sigma_mu_m, double amplitude,
                                           double aperture_m, double lens_f_m,
                                           const pw_c32* dev_mask, pw_c32* dev_W_out,
                                           size_t W_bytes, float* dev_S_out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PYWOLF_GB_H */
