/*
 * gbsmps — pure bosonic Gaussian state -> matrix product state, on one GB300.
 *
 * C ABI of the library that implements the method of arXiv:2512.10643
 * ("Efficient simulation of low-entanglement bosonic Gaussian states in
 * polynomial time"): the iterative Gaussian SVD of Sec. II B, the kept
 * subspace and projected-creation-operator (PCO) mapping of Sec. II C and
 * App. B, and MPS consumers (amplitudes, conditional sampling) of the
 * finished tensors.  Every step runs in CUDA kernels for sm_103a; the host
 * code only validates arguments, sizes buffers and orders launches.
 *
 * Conventions (Sec. II A): a_j = (x_j + i p_j)/sqrt(2); the covariance matrix
 * Gamma = (1/2)<{dR, dR}> with R = (x_1..x_N, p_1..p_N) ("xxpp"), so the vacuum
 * has Gamma = I/2.  Complex numbers are interleaved (re, im) doubles.
 *
 * Memory and ownership.  Every pointer argument is tagged by a mem_kind:
 * GBSMPS_MEM_HOST (ordinary or pinned host memory) or GBSMPS_MEM_DEVICE
 * (device memory of the context's GPU).  The caller owns every buffer it
 * passes; the library copies what it needs before returning, so inputs may be
 * freed after the call.  Calls are ordered on the context's CUDA stream: a
 * call whose outputs are device memory returns once its work is enqueued; a
 * call with host outputs synchronises the stream before returning.  The
 * library owns every gbsmps_mps_t and its device memory until
 * gbsmps_release.  Calls on one context must not run concurrently from
 * several host threads.
 *
 * Errors.  Every entry point returns 0 (GBSMPS_OK) or a positive error code;
 * gbsmps_strerror gives its text, and gbsmps_last_error_detail a one-line
 * description of the last failure on the calling thread.  No entry point
 * aborts or throws.  Device-side failures (a Jacobi sweep limit, an index
 * bound) are recorded in a device status word and returned by the next call
 * that synchronises.
 */
#ifndef GBSMPS_H
#define GBSMPS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ------------------------------------------------------ */
#define GBSMPS_OK 0
#define GBSMPS_ERR_ARG 1            /* bad argument (null, size, range)         */
#define GBSMPS_ERR_NOT_SYMMETRIC 2  /* Gamma not symmetric                       */
#define GBSMPS_ERR_NOT_PURE 3       /* (2 Gamma Omega)^2 != -1 within tolerance  */
#define GBSMPS_ERR_OOM 4            /* device allocation failed                  */
#define GBSMPS_ERR_NOT_CONVERGED 5  /* eigensolver sweep limit reached           */
#define GBSMPS_ERR_BOUNDS 6         /* n_e or a basis size exceeds a built limit */
#define GBSMPS_ERR_CUDA 7           /* CUDA runtime error                        */
#define GBSMPS_ERR_NUMERIC 8        /* non-finite value, singular matrix         */
#define GBSMPS_ERR_STATE 9          /* object in the wrong state for the call    */
#define GBSMPS_ERR_TIMEOUT 10       /* a bounded wait (device mbarrier, server
                                       wait) ran out                            */

#define GBSMPS_MEM_HOST 0
#define GBSMPS_MEM_DEVICE 1

/* Arithmetic of the tensor build, environments and sampling.  The Gaussian
 * SVD, symplectic orthogonalisation and normalisation are FP64 in both. */
#define GBSMPS_PREC_FP64 0
#define GBSMPS_PREC_MIXED 1   /* FP32 PCO passes with FP64 output sums,
                                 environments on the tensor cores with exact
                                 accumulation of bf16 integer slices (double-
                                 float on the FP32 pipes with GBSMPS_ENV_TC=0),
                                 split-FP16 tcgen05 sampling GEMMs */

/* Largest number of entangled mode pairs at one cut (n_e of Sec. II A). */
#define GBSMPS_NE_MAX 24

typedef struct gbsmps_ctx* gbsmps_ctx_t;
typedef struct gbsmps_mps* gbsmps_mps_t;

typedef struct {
  int32_t d;               /* physical Fock cutoff: p = 0..d-1 (Sec. II C)      */
  int32_t chi_max;         /* bond dimension cap chi (D of Sec. II C)            */
  double eps_trunc;        /* target discarded weight eps; D_m = min(chi, D(eps)),
                              eps = 0 means chi alone (Sec. II C, D(eps) rule)   */
  double lambda2_freeze;   /* modes with Lambda^2 <= this are frozen: the D*
                              tolerance of Sec. II A, expressed on Lambda^2     */
  int32_t precision;       /* GBSMPS_PREC_FP64 or GBSMPS_PREC_MIXED              */
  int32_t validate;        /* 1: check symmetry and purity of the input         */
  double purity_tol;       /* max |(2 Gamma Omega)^2 + 1| accepted              */
} gbsmps_opts;

/* Fill *o with defaults: d = 4, chi = 64, eps = 0, lambda2_freeze = 1e-13,
 * FP64, validate = 1, purity_tol = 1e-9.  Returns GBSMPS_ERR_ARG on null. */
int gbsmps_opts_default(gbsmps_opts* o);

/* Create a context on CUDA device `device`, ordering all work on `stream`
 * (a cudaStream_t; NULL = the legacy default stream).  *out receives the
 * handle.  Errors: ARG (null out, bad device), CUDA. */
int gbsmps_create(int device, void* stream, gbsmps_ctx_t* out);
int gbsmps_destroy(gbsmps_ctx_t ctx);

/* Build the MPS of the N-mode pure Gaussian state with covariance `gamma`
 * (2N x 2N, xxpp, row-major FP64; Sec. II A, Eq. (GammaMat)).  Runs the
 * iterative GSVD (Sec. II B: Williamson form Eq. (symDiag), Bogoliubov map
 * Eq. (MUV), regularised paired form of App. A), the kept-basis selection
 * and truncation error (Sec. II C, Sec. III A), the PCO mapping of every
 * local tensor (Sec. II C, App. B), the right environments and the
 * normalisation (norm 1, all-vacuum amplitude real positive).
 * N >= 1; 1 <= d <= 255; 1 <= chi_max <= 4096.  *out receives a new handle.
 * Errors: ARG, NOT_SYMMETRIC, NOT_PURE (validate = 1), BOUNDS (n_e > NE_MAX),
 * NOT_CONVERGED, NUMERIC, OOM, CUDA.  Synchronises the stream once (bond
 * sizes are read back to size the tensors). */
int gbsmps_build_from_cov(gbsmps_ctx_t ctx, int32_t N, const double* gamma,
                          int mem_kind, const gbsmps_opts* opts,
                          gbsmps_mps_t* out);

/* Same from the paired-form (A-)matrix Q of Eq. (paired-form): the state is
 * proportional to exp(1/2 sum Q_ij a_i^dag a_j^dag)|0>, Q (N x N, complex
 * symmetric, row-major interleaved, all singular values < 1).  The GBS
 * "A-matrix" of a pure state is Q (+) Q^*; pass its first block.  Q is turned
 * into Gamma on the device (N = (1 - Q^*Q)^{-1} - 1, M = Q(1 + N)). */
int gbsmps_build_from_Q(gbsmps_ctx_t ctx, int32_t N, const double* Q,
                        int mem_kind, const gbsmps_opts* opts,
                        gbsmps_mps_t* out);

/* Build `count` MPSs of independent states in one pass (same results as
 * gbsmps_build_from_cov on each, up to the rounding order of the environment
 * products).  Ns[i], gammas[i] (all in mem_kind memory) and opts[i] describe
 * state i; out[i] receives its handle.  The sequential parts of the method run
 * side by side across the batch: all GSVD chains (Sec. II B) in one launch,
 * the PCO tensors of all sites together (Sec. II C), and the right-
 * environment chains of the mixed-precision states in one persistent launch;
 * bond sizes are read back once.  On error no handle is returned.  Errors as
 * gbsmps_build_from_cov.  count = 0 is a no-op. */
int gbsmps_build_batch(gbsmps_ctx_t ctx, int32_t count, const int32_t* Ns,
                       const double* const* gammas, int mem_kind,
                       const gbsmps_opts* opts, gbsmps_mps_t* out);

/* Sizes of a built MPS (host outputs, any may be NULL):
 * bond_dims[N+1] (D_0 = D_N = 1), n_e[N-1] (entangled pairs per cut),
 * eps_m[N-1] (discarded weight per bond, Sec. III A), *N_out, *d_out. */
int gbsmps_info(gbsmps_mps_t mps, int32_t* N_out, int32_t* d_out,
                int32_t* bond_dims, int32_t* n_e, double* eps_m);

/* Copy tensor A^site (0-based) as row-major [alpha][p][beta] complex128
 * (beta fastest), size D_site * d * D_{site+1} * 16 bytes, into dst.
 * Errors: ARG (site range, dst_bytes too small). */
int gbsmps_get_tensor(gbsmps_mps_t mps, int32_t site, void* dst,
                      size_t dst_bytes, int mem_kind);

/* Symplectic spectra and entanglement data of the GSVD, for checks:
 * lam2[(N-1) * NE_MAX] (Lambda_q^2 of active modes, descending, zero padded),
 * Qm[N * (2 NE_MAX + 1)^2] complex (local paired forms over c_m =
 * (r_{m-1}, a_m, l_m), row stride 2 NE_MAX + 1), c_m[N].  Host outputs. */
int gbsmps_get_gsvd(gbsmps_mps_t mps, double* lam2, double* Qm, double* c_m);

/* The kept basis of bond b (0..N; bond b is the cut after site b-1, bonds 0
 * and N hold only the vacuum), Sec. II C "The kept subspace and projection":
 * occ[D_b * n_e_b] uint8, row j = the occupation vector n_beta of kept state
 * j over the n_e_b Schmidt modes of the cut (E order, ties lexicographic;
 * index 0 is the vacuum), and E[D_b] its entanglement energy
 * E_beta = sum_q n_q (-ln Lambda_q^2).  Host outputs, either may be NULL;
 * sizes from gbsmps_info.  Synchronises.  Errors: ARG (bond range). */
int gbsmps_get_basis(gbsmps_mps_t mps, int32_t bond, uint8_t* occ, double* E);

/* Amplitudes <n_1..n_N|psi> (Eq. (Am_definition) contracted along the chain)
 * of P patterns (P x N uint8, row-major) into out (P x 2 doubles).  Patterns
 * with any n_i >= d give 0.  P = 0 is a no-op.  Errors: ARG, CUDA. */
int gbsmps_amplitudes(gbsmps_mps_t mps, int64_t P, const uint8_t* patterns,
                      double* out, int mem_kind);

/* Draw S photon-count patterns (S x N uint8, row-major) by exact sequential
 * conditional sampling of the normalised MPS: at site m the weights
 * q_p = w_p R_{m+1} w_p^dag of w_p = v A^m[p] (right environment R), the
 * first p with u Z < C_p (C the prefix sums, Z the total) is chosen and
 * v = w_p / sqrt(q_p).  Uniforms: `uniforms` (S x N doubles in [0,1),
 * row-major, same mem_kind) if non-NULL; otherwise Philox4x32-10 keyed by
 * seed with counter (counter0 + sample, site), 53 bits per draw.
 * `flags` (S bytes, may be NULL) receives 1 where a draw fell within 1e-12 Z
 * of a CDF boundary.  S = 0 is a no-op.  Errors: ARG, OOM, CUDA. */
int gbsmps_sample(gbsmps_mps_t mps, int64_t S, uint64_t seed,
                  uint64_t counter0, const double* uniforms, uint8_t* out,
                  uint8_t* flags, int mem_kind);

/* Build and sample a stream of `count` states: state k is built as by
 * gbsmps_build_from_cov (Ns[k], gammas[k], opts[k]) and S patterns are drawn
 * from it as by gbsmps_sample with Philox keys seeds[k], counters from
 * counter0s[k] (no uniforms, no flags) into outs[k] (S x Ns[k] bytes).  The
 * Gaussian SVD chain of Sec. II B is sequential and runs on one SM; here the
 * chain of state k+1 runs while state k is sampled on the other SMs, and the
 * rest of build k+1 waits for that sampling to finish.  The patterns are
 * the ones the two separate calls give.  gammas and outs are in mem_kind
 * memory (host buffers are best page-locked: pageable copies block the
 * overlap).  Returns when every state is sampled; the handles are released
 * internally.  On error the remaining states are skipped.  Errors as
 * gbsmps_build_from_cov and gbsmps_sample.  count = 0 is a no-op. */
int gbsmps_build_sample_stream(gbsmps_ctx_t ctx, int32_t count, const int32_t* Ns,
                               const double* const* gammas, const gbsmps_opts* opts,
                               int64_t S, const uint64_t* seeds,
                               const uint64_t* counter0s, uint8_t* const* outs,
                               int mem_kind);

/* Mixed -> pure decomposition of lossy-experiment covariances (Sec. III,
 * Eq. (decompose); App. C): each Gamma_th (2N x 2N, xxpp, row-major, FP64)
 * is split as Gamma_p + W with Gamma_p = S S^T / 2 pure (S symplectic) and
 * W >= 0, by Riemannian gradient descent on Sp(2N) of the loss
 * L(S) = -lambda_min(Gamma_th - S S^T / 2) (Eq. (loss)) from S = I: the
 * unit gradient in sp(2N) under the Frobenius norm (the appendix's
 * "two-form norm" is not defined further), the retraction
 * S <- S exp(-alpha G) with fixed step alpha, stop once L <= eps or after
 * max_iter steps.  A batch of `count` states of equal N runs in one launch,
 * one state per SM, FP64.  gamma_th and S_out: count x (2N)^2 doubles, both
 * host or both device (mem_kind); iters and loss: host arrays of count
 * entries (may be NULL) receiving the steps taken and the final L.
 * The pure part's covariance is S_out S_out^T / 2.  Synchronises.
 * Limits: N <= GBSMPS_FILTER_MAX_N.  Errors: ARG, BOUNDS, CUDA. */
#define GBSMPS_FILTER_MAX_N 64
int gbsmps_filter(gbsmps_ctx_t ctx, int32_t count, int32_t N, const double* gamma_th,
                  double alpha, double eps, int32_t max_iter, double* S_out,
                  int32_t* iters, double* loss, int mem_kind);

/* Out-of-core sampling of an MPS that need not fit the GPU's memory: the
 * paper's sampling estimate (Sec. III B) has the bond tensors of large
 * states exceed one device's memory.  Moves a mixed-precision MPS's sampler
 * planes (every site's right-canonical tensor as split-FP16 planes) to
 * pinned host memory and frees every other device array of its tensors
 * (tensors, environments and their factors); later gbsmps_sample calls
 * stream the planes site by site through a ring of three device slots on a
 * copy stream of their own, each site's copy overlapping the GEMMs of the
 * sites before it, and draw exactly the patterns the resident MPS draws.
 * Device memory then held for the MPS: the ring (three sites' planes) and
 * the per-sample work buffers of the sampling.  gbsmps_get_tensor and
 * gbsmps_amplitudes of an offloaded MPS return GBSMPS_ERR_STATE; info,
 * get_gsvd and get_basis still work.  A second call is a no-op.
 * *host_bytes (may be NULL) receives the size of the host copy: the bytes
 * each sampling streams to the device.  Synchronises.  Errors: ARG (FP64
 * MPS), OOM/CUDA (pinned allocation). */
int gbsmps_offload(gbsmps_mps_t mps, size_t* host_bytes);

/* Release an MPS and its device memory (and its pinned host copy when
 * offloaded). */
int gbsmps_release(gbsmps_mps_t mps);

/* Expert entry: PCO build of one local tensor (Sec. II C, App. B) from a
 * given paired form Qm ((nl + 1 + nr)^2 complex, mode order (r_1..r_nl, a,
 * l_1..l_nr)) and kept bases given as occupation vectors occ_l (Dl x nl
 * uint8) and occ_r (Dr x nr uint8) that must be closed under removing one
 * quantum and start with the vacuum.  out: Dl x d x Dr complex128, scaled by
 * c.  All pointers are of mem_kind.  precision selects FP64 or FP32 PCO
 * arithmetic (the output is FP64 either way). */
int gbsmps_build_site(gbsmps_ctx_t ctx, int32_t nl, int32_t nr, int32_t d,
                      const double* Qm, double c, int32_t Dl,
                      const uint8_t* occ_l, int32_t Dr, const uint8_t* occ_r,
                      int32_t precision, double* out, int mem_kind);

/* Allocation-free variant of gbsmps_build_site.  The paper has no
 * counterpart; this is a service of the library.  It computes exactly what
 * gbsmps_build_site computes, but performs no device allocation, for callers
 * that must not allocate while they run: a serving process that reserved its
 * device memory up front (for resident tensors and admission by free memory)
 * and must not have a call fail or fragment that reserve, latency-critical
 * loops for which cudaMalloc / cudaFree are unacceptable because they can
 * synchronise the device and stall other streams, and hosts whose own
 * allocator owns all device memory.
 * All pointers are device memory of the context's GPU: Qm ((nl+1+nr)^2
 * complex, row-major, mode order (r_1..r_nl, a, l_1..l_nr)), occ_l (Dl x nl
 * uint8) and occ_r (Dr x nr uint8), vacuum first and closed under removing
 * one quantum, out (Dl x d x Dr complex128, scaled by c).
 * Working memory is one static device array of GBSMPS_NOALLOC_SCRATCH_BYTES
 * that every GPU which loads the library holds until the process exits.
 * Limit: Dl and Dr <= GBSMPS_NOALLOC_MAX_D; larger sizes are rejected with
 * GBSMPS_ERR_BOUNDS before any GPU work.  The first call on a device looks up
 * the array's device address once (cudaGetSymbolAddress, with that device
 * current); make that first call before any stream capture.  Every call
 * reuses the same array, which keeps the previous call's contents (a call
 * rewrites everything it reads), so calls that overlap on the GPU (from
 * several streams or host threads) race and must be serialised by the
 * caller.  Synchronises the context's stream.  Errors: ARG, BOUNDS, CUDA. */
#define GBSMPS_NOALLOC_MAX_D 128
#define GBSMPS_NOALLOC_SCRATCH_BYTES (1280 * 1024)
int gbsmps_build_site_noalloc(gbsmps_ctx_t ctx, int32_t nl, int32_t nr, int32_t d,
                              const double* Qm, double c, int32_t Dl, const uint8_t* occ_l,
                              int32_t Dr, const uint8_t* occ_r, int32_t precision,
                              double* out);

/* Text of an error code (static storage). */
const char* gbsmps_strerror(int code);
/* One-line detail of the last error on the calling thread. */
const char* gbsmps_last_error_detail(void);

/* Number of kernels the library has enqueued since it was loaded (all
 * contexts), for launch accounting. */
int64_t gbsmps_launch_count(gbsmps_ctx_t ctx);

/* Tracing of the dominant kernel, the tcgen05 split-FP16 complex GEMM of the
 * mixed-precision sampler (one launch per site): gbsmps_trace(ctx, 1) clears
 * the record and records a CUDA event pair around every later launch on the
 * launching stream; gbsmps_trace(ctx, 0) stops recording.  gbsmps_trace_read
 * synchronises on the recorded events and returns the summed device time,
 * the launch count, and the launches' algorithmic work: 8 M N K real flops
 * per complex M x N x K product and the operand/result bytes at their storage
 * width.  Outputs may be NULL.  Not part of the numerical path. */
int gbsmps_trace(gbsmps_ctx_t ctx, int enable);
int gbsmps_trace_read(gbsmps_ctx_t ctx, double* total_ms, int64_t* launches,
                      double* flops, double* bytes);

/* The same record for one of three traced kernels: which = 0, the sampler
 * GEMM above (gbsmps_trace_read); which = 1, the products of the
 * right-environment chain R_m = sum_p A^m[p] R_{m+1} A^m[p]^dag (the norm,
 * and the standard MPS sampling that Sec. I and Sec. III defer to), two
 * traced passes per site: on the tensor cores (the default) each pass is
 * the slicing of its operands, the GEMM and the k-split reduction; with
 * GBSMPS_ENV_TC=0 each is one grouped double-float GEMM launch.  The work
 * counts 8 real flops per complex multiply-add of the lower triangle of a
 * Hermitian result and of every element otherwise, and the bytes are the
 * operands and results at 16 bytes per complex element; which = 2, the
 * PCO tensor build of a state (Sec. II C, App. B; one launch per wave of
 * sites), time and launch count only (its algorithmic work is counted by the
 * caller from the kept bases, gbsmps_get_basis).  Recording is switched on
 * and cleared for all three by gbsmps_trace.  GBSMPS_ERR_ARG for another
 * `which`.  Not part of the numerical path. */
int gbsmps_trace_read_kernel(gbsmps_ctx_t ctx, int32_t which, double* total_ms,
                             int64_t* launches, double* flops, double* bytes);

/* ---- serving: continuous batching of build + sampling requests -----------
 * Not a step of the paper's method: a request loop around it.  A server owns
 * `slots` worker threads, each with its own non-blocking CUDA stream and
 * context on `device`.  Requests queue in arrival order; a free slot admits
 * the first of the next 8 queued requests whose device-memory estimate
 * (gbsmps_estimate_bytes) fits the budget that the jobs on the device leave
 * free, and a request passed over 32 times blocks later ones until it fits.
 * An admitted job runs build (gbsmps_build_from_cov, host Gamma) and sampling
 * (gbsmps_sample, Philox keyed by seed/counter0) on its slot's stream, with
 * the MPS resident on the device in between, and writes the S x N patterns to
 * req.out; jobs on different slots overlap on the GPU, and a job's result is
 * bitwise the result of the same calls made alone.  With batch_max > 1 a
 * slot that admits a job also admits up to batch_max - 1 more admissible
 * queued jobs and builds them all in one gbsmps_build_batch call (every GSVD
 * chain in one launch, every PCO tensor together, the environment chains in
 * one persistent launch), then samples them one after another, each job
 * completing when its own patterns are out; the environment products of a
 * batch sum in another order, so such a result equals the job run alone up
 * to rounding (samples bit-exact except draws that req.flags marks).  The
 * caller keeps req.gamma, req.out and req.flags valid until the job is done.
 * Latency is submit -> done on the server's monotonic clock. */
typedef struct gbsmps_server* gbsmps_server_t;

typedef struct {
  int32_t slots;                 /* concurrent jobs (1..64), default 4          */
  size_t hbm_budget;             /* bytes the admitted jobs may hold together;
                                    0: 80% of the free device memory at creation;
                                    capped at 90% of it                          */
  double simulate_s_per_tensor;  /* > 0: jobs do not touch a GPU, each sleeps
                                    N x this many seconds and writes zeros
                                    (tests of the scheduler without a device);
                                    needs hbm_budget > 0                        */
  int32_t batch_max;             /* jobs one slot builds in one batched call
                                    (1..64), default 1                          */
} gbsmps_server_opts;

typedef struct {
  const double* gamma;   /* host 2N x 2N covariance (xxpp, row-major)           */
  int32_t N;
  gbsmps_opts opts;
  int64_t samples;       /* S >= 0                                              */
  uint64_t seed, counter0;
  uint8_t* out;          /* host S x N uint8, written by the job                */
  uint8_t* flags;        /* optional host S bytes: 1 where a draw lay within the
                            sampler's boundary window (as gbsmps_sample)       */
} gbsmps_request;

typedef struct {
  int32_t state;         /* 0 queued, 1 running, 2 done, 3 failed               */
  int32_t error;         /* the job's error code (0 when done)                  */
  int32_t slot;          /* slot that ran it, -1 before admission               */
  double t_submit, t_admit, t_done;   /* seconds since server creation          */
  size_t hbm_bytes;      /* admission estimate                                  */
  char detail[128];      /* error detail of a failed job                        */
  int32_t batch;         /* jobs built in the same batched call (1: alone)      */
} gbsmps_job_info;

typedef struct {
  int64_t submitted, completed, failed, running, queued;
  double p50_ms, p99_ms, mean_ms;   /* submit -> done, completed jobs (nearest rank) */
  double busy_s;                    /* first admission -> last completion       */
  double tensors, samples;          /* totals over completed jobs               */
  size_t hbm_in_use, hbm_budget, hbm_peak;
} gbsmps_server_stats;

int gbsmps_server_opts_default(gbsmps_server_opts* o);
/* Errors: ARG (slots out of range, bad device), CUDA. */
int gbsmps_server_create(int device, const gbsmps_server_opts* o, gbsmps_server_t* out);
/* Queue a request; *id identifies it.  Errors: ARG, OOM (estimate larger than
 * the whole budget), STATE (server stopping). */
int gbsmps_server_submit(gbsmps_server_t srv, const gbsmps_request* req, int64_t* id);
/* Wait for request `id` (timeout_s < 0: no limit); returns the job's error
 * code, or TIMEOUT.  info (may be NULL) receives its record. */
int gbsmps_server_wait(gbsmps_server_t srv, int64_t id, double timeout_s, gbsmps_job_info* info);
/* Wait until no request is queued or running.  Errors: TIMEOUT. */
int gbsmps_server_drain(gbsmps_server_t srv, double timeout_s);
int gbsmps_server_stats_read(gbsmps_server_t srv, gbsmps_server_stats* st);
/* Finish every queued request, stop the workers, free the contexts. */
int gbsmps_server_destroy(gbsmps_server_t srv);

/* Upper bound of the device bytes one build + sampling call of this size
 * holds at its peak (every bond at chi_max), as used for admission; 0 for
 * invalid arguments. */
size_t gbsmps_estimate_bytes(int32_t N, const gbsmps_opts* opts, int64_t samples);

#ifdef __cplusplus
}
#endif
#endif /* GBSMPS_H */
