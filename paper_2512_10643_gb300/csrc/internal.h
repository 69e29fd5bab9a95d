// Internal declarations shared by the gbsmps kernel files (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>
#include "../../include/gbsmps.h"

#define NEM GBSMPS_NE_MAX          // max entangled pairs per cut
#define NLM (NEM + 1)              // max modes of L_m = (r_{m-1}, a_m)
#define N2M (2 * NLM)              // max quadratures of L_m
#define QS (2 * NEM + 1)           // row stride of stored local paired forms
#define TIE_MARGIN 64              // extra basis candidates kept for tie groups
#define TIE_TOL 1e-12              // relative tolerance of an energy tie

// device status word bits (first failure wins, see set_status)
#define ST_NOT_CONVERGED 1
#define ST_BOUNDS 2
#define ST_NUMERIC 4
#define ST_NOT_SYMMETRIC 8
#define ST_NOT_PURE 16
#define ST_TIMEOUT 32

// ---- Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): uniform in [0,1)
// with 53 bits from the first two output words; key = seed, counter =
// (sample lo, sample hi, site, 0) ---------------------------------------------
__device__ inline void philox_round(uint32_t c[4], uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  uint32_t hi0 = __umulhi(M0, c[0]), lo0 = M0 * c[0];
  uint32_t hi1 = __umulhi(M1, c[2]), lo1 = M1 * c[2];
  uint32_t n0 = hi1 ^ c[1] ^ k0, n1 = lo1, n2 = hi0 ^ c[3] ^ k1, n3 = lo0;
  c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
}
__device__ inline double philox_uniform(uint64_t seed, uint64_t sample, uint32_t site) {
  uint32_t c[4] = {(uint32_t)sample, (uint32_t)(sample >> 32), site, 0u};
  uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  for (int r = 0; r < 10; ++r) {
    philox_round(c, k0, k1);
    k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
  }
  uint64_t a = c[0] >> 5, b = c[1] >> 6;     // 27 + 26 bits
  return (double)(a * 67108864ull + b) * (1.0 / 9007199254740992.0);
}

// ---- complex helpers on double2 -------------------------------------------
__host__ __device__ inline double2 cmk(double r, double i) { return make_double2(r, i); }
__host__ __device__ inline double2 cadd(double2 a, double2 b) { return cmk(a.x + b.x, a.y + b.y); }
__host__ __device__ inline double2 csub(double2 a, double2 b) { return cmk(a.x - b.x, a.y - b.y); }
__host__ __device__ inline double2 cmul(double2 a, double2 b) {
  return cmk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ inline double2 cconj(double2 a) { return cmk(a.x, -a.y); }
__host__ __device__ inline double2 cscale(double2 a, double s) { return cmk(a.x * s, a.y * s); }
__host__ __device__ inline double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }
// a += b * c
__host__ __device__ inline void cfma(double2& a, double2 b, double2 c) {
  a.x = fma(b.x, c.x, fma(-b.y, c.y, a.x));
  a.y = fma(b.x, c.y, fma(b.y, c.x, a.y));
}

// float2 versions (FP32 arithmetic of the mixed-precision path)
__host__ __device__ inline float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ inline float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ inline float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__host__ __device__ inline void cfma(float2& a, float2 b, float2 c) {
  a.x = fmaf(b.x, c.x, fmaf(-b.y, c.y, a.x));
  a.y = fmaf(b.x, c.y, fmaf(b.y, c.x, a.y));
}

// complex type of a real type
template <typename T> struct Cx;
template <> struct Cx<double> { using type = double2; };
template <> struct Cx<float> { using type = float2; };
template <typename C2> __host__ __device__ inline C2 to_c(double2 v);
template <> __host__ __device__ inline double2 to_c<double2>(double2 v) { return v; }
template <> __host__ __device__ inline float2 to_c<float2>(double2 v) {
  return make_float2((float)v.x, (float)v.y);
}
__host__ __device__ inline double2 to_d(double2 v) { return v; }
__host__ __device__ inline double2 to_d(float2 v) { return make_double2(v.x, v.y); }

__device__ inline void set_status(int* st, int bit) { atomicOr(st, bit); }

// ---- per-bond basis storage ----------------------------------------------
// For bond b (0..N): occupations occ[b*cap*NEM + i*NEM + q] (uint8),
// energies E[b*cap + i], lowering maps low[(b*NEM + q)*cap + i] = index of
// state i minus one quantum of mode q (or -1), D[b] kept size, ne[b] modes.
struct BondArrays {
  int cap;            // capacity per bond (chi + TIE_MARGIN)
  uint8_t* occ;
  double* E;
  int* low;
  int* D;             // kept dims (device)
  int* ne;            // entangled pairs (device)
  int* maxocc;        // [b*NEM + q] max occupation of mode q in the kept basis
  double* lam2;       // [b*NEM + q] Lambda^2 (bond b = cut after site b-1)
  double* eps;        // [b] discarded weight
  int* pidx;          // [b*cap + j]: kept states of bond b, even total photon number
                      // first, the E order kept within each class
  int* pcnt;          // [2b + c]: kept states of bond b with photon-number parity c
};

// ---- opt-in kernel tracing: CUDA events around every launch of one kernel
// family on its own stream, summed with the launches' algorithmic work -------
#include <atomic>
#include <mutex>
#include <vector>
struct KernelTrace {
  std::atomic<bool> on{false};
  std::mutex mu;
  std::vector<cudaEvent_t> ev;   // begin/end pairs
  double flops = 0.0, bytes = 0.0;
  long long launches = 0;
  cudaEvent_t begin(cudaStream_t s) {
    if (!on.load()) return nullptr;
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    cudaEventRecord(e, s);
    return e;
  }
  void end(cudaEvent_t b0, cudaStream_t s, double f, double b) {
    if (!b0) return;
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) { cudaEventDestroy(b0); return; }
    cudaEventRecord(e, s);
    std::lock_guard<std::mutex> lk(mu);
    ev.push_back(b0);
    ev.push_back(e);
    flops += f; bytes += b; ++launches;
  }
  void add_work(double f, double b) {        // work known only after the launches ran
    if (!on.load()) return;
    std::lock_guard<std::mutex> lk(mu);
    flops += f; bytes += b;
  }
  double total_ms() {
    std::lock_guard<std::mutex> lk(mu);
    double t = 0.0;
    for (size_t i = 0; i + 1 < ev.size(); i += 2) {
      cudaEventSynchronize(ev[i + 1]);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ev[i], ev[i + 1]);
      t += ms;
    }
    return t;
  }
  void reset() {
    std::lock_guard<std::mutex> lk(mu);
    for (auto e : ev) cudaEventDestroy(e);
    ev.clear(); flops = bytes = 0.0; launches = 0;
  }
};
extern KernelTrace g_tc_trace;    // the tcgen05 sampler GEMM
extern KernelTrace g_env_trace;   // the double-float environment GEMM
extern KernelTrace g_pco_trace;   // the PCO tensor build

// ---- launchers (each returns cudaError_t of the launch) -------------------
// g_kernel_launches counts every kernel the library enqueues.
extern std::atomic<unsigned long long> g_kernel_launches;
#define COUNT_LAUNCH(n) (g_kernel_launches += (n))
cudaError_t launch_check_input(const double* gamma, int N, double purity_tol,
                               double* work, int* status, cudaStream_t s);
cudaError_t launch_q_to_gamma(const double2* Q, int N, double* gamma, double2* work,
                              int* status, cudaStream_t s);
cudaError_t launch_bandwidth(const double* gamma, int N, int* bw, cudaStream_t s);
// one state of a batched GSVD chain launch (device pointers of that state)
struct ChainJob {
  const double* gamma;
  int N;
  const int* bw;
  double freeze;
  double* G;
  BondArrays ba;
  double2* Qm;
  double* cm;
};
cudaError_t launch_gsvd_chain_batch(const ChainJob* jobs_dev, int count, int maxN, int* status,
                                    cudaStream_t s);
cudaError_t launch_gsvd_chain(const double* gamma, int N, const int* bw,
                              double lambda2_freeze, double* Gscratch,
                              BondArrays ba, double2* Qm, double* cm, int* status,
                              cudaStream_t s);
cudaError_t launch_basis(BondArrays ba, int nbonds, int chi, double eps,
                         int* status, cudaStream_t s);
cudaError_t launch_maps(BondArrays ba, int nbonds, int* status, cudaStream_t s);

struct SiteTask {       // one local tensor to build
  int nl, nr, Dl, Dr;
  const double2* Q;     // (nl+1+nr)^2 with row stride qs
  int qs;
  double c;
  const uint8_t* occl; const int* lowl; int capl;   // left basis (stride NEM)
  const uint8_t* occr; const int* lowr; int capr;   // right basis
  double2* out;         // Dl x d x Dr
  size_t scratch_off;   // offset (complex elements) into the scratch arena
  // photon-number parity classes of the two bonds (optional): the kept
  // states of each bond listed even class first, and the class sizes
  const int* pl = nullptr;
  const int* pr = nullptr;
  int kl[2] = {0, 0}, kr[2] = {0, 0};
};
cudaError_t launch_maps_brute(const uint8_t* occ, int D, int n, int* low, int cap,
                              int* status, cudaStream_t s);
cudaError_t launch_pco(const SiteTask* tasks_dev, int ntasks, int d, int precision,
                       double2* scratch, int* status, cudaStream_t s);
size_t pco_scratch_elems(int Dl, int Dr);
// persistent variant for many sites: `grid` CTAs (pco_dynamic_grid(): as many
// as fit on the GPU at once), each with a scratch slot of slot_elems
int pco_dynamic_grid();
cudaError_t launch_pco_dynamic(const SiteTask* tasks_dev, int ntasks, int d, int precision,
                               double2* scratch, size_t slot_elems, int grid, int* counter,
                               int* status, cudaStream_t s);

// complex FP64 GEMM: C[M x N] = alpha * op(A) * op(B) + beta * C, row-major,
// op = 'N' or 'C' (conjugate transpose), batched with element strides.
cudaError_t launch_zgemm(char opa, char opb, int M, int N, int K, double2 alpha,
                         const double2* A, int lda, long long sA,
                         const double2* B, int ldb, long long sB, double2 beta,
                         double2* C, int ldc, long long sC, int batch, cudaStream_t s);
cudaError_t launch_zscale(double2* x, size_t n, const double2* factor, cudaStream_t s);
cudaError_t launch_norm_phase(const double2* R0, const double2* amp0, double2* factor,
                              int* status, cudaStream_t s);

// A complex double as a double-float pair (hi, lo) per part: float4
// (re_hi, re_lo, im_hi, im_lo), 16 bytes like a double2.  The mixed path
// stores the energy-gauge tensors and the environment products' first
// factor this way, so the double-float GEMM loads them without converting
// on GB300's slow FP64 pipe.
__device__ __forceinline__ float4 df_pack(double2 v) {
  const float rh = (float)v.x, ih = (float)v.y;
  return make_float4(rh, (float)(v.x - (double)rh), ih, (float)(v.y - (double)ih));
}
__host__ __device__ __forceinline__ double2 df_unpack(float4 w) {
  return make_double2((double)w.x + (double)w.y, (double)w.z + (double)w.w);
}

// Parity-compact layout of the mixed path's per-site tensors (energy gauge,
// environment products, canonical transforms).  A^m[alpha, p, beta] is zero
// unless n_alpha + p + n_beta is even, so site m is stored as two class
// blocks: rows = the class-c states of the left bond (kl[c] of them, in the
// order of the bond's parity list), row length K_c = ceil(d/2) kr[c] +
// floor(d/2) kr[c^1], and column block p = the class c^(p&1) states of the
// right bond, starting at floor(p/2) D_r + (p odd ? kr[c] : 0).  Class 0
// rows come first.  Environments and their factors are stored per bond as
// two diagonal blocks (class 0 then class 1, each row-major with its own
// leading dimension).
struct ParitySite {
  const int* pl;           // parity list of the left bond (class 0 then class 1), device
  const int* pr;           // the same for the right bond
  int kl[2], kr[2];
};
__host__ __device__ inline long long pk_len(int d, const int* kr, int c) {
  return (long long)((d + 1) / 2) * kr[c] + (long long)(d / 2) * kr[c ^ 1];
}
__host__ __device__ inline long long pk_off(int p, int Dr, const int* kr, int c) {
  return (long long)(p >> 1) * Dr + ((p & 1) ? kr[c] : 0);
}
__host__ __device__ inline long long pk_size(int d, const int* kl, const int* kr) {
  return (long long)kl[0] * pk_len(d, kr, 0) + (long long)kl[1] * pk_len(d, kr, 1);
}
// compact index idx of a site -> (class c, row a, p, column j, right class cr)
__device__ inline void pk_locate(const ParitySite& P, int d, long long idx, int& c, int& a, int& p,
                                 int& j, int& cr) {
  const long long n0 = (long long)P.kl[0] * pk_len(d, P.kr, 0);
  const int Dr = P.kr[0] + P.kr[1];
  c = idx < n0 ? 0 : 1;
  const long long loc = c ? idx - n0 : idx;
  const long long K = pk_len(d, P.kr, c);
  a = (int)(loc / K);
  const long long k = loc - (long long)a * K;
  const int pp = (int)(k / Dr), rem = (int)(k - (long long)pp * Dr);
  const int odd = rem >= P.kr[c] ? 1 : 0;
  p = 2 * pp + odd;
  j = odd ? rem - P.kr[c] : rem;
  cr = c ^ odd;
}

struct NormJob {         // one state of the batched normalisation
  int N, d;
  const int* D;            // bond dimensions [N + 1] (device)
  const long long* toff;   // tensor offsets [N] (device)
  double2* T;              // FP64 tensors; A^1 is rescaled in place
  const double2* R0;       // norm^2
  double2* Ah;             // mixed path: energy-gauge tensors (A^1 rewritten), else null
  const double* E1;        // e^{-E/2} of bond 1's states (mixed path)
  ParitySite P0;           // mixed path: parity-compact layout of site 0
};
cudaError_t launch_vac_norm_batch(const NormJob* jobs_dev, int count, int maxD, int* status,
                                  cudaStream_t s);
struct ChainView {       // view of an MPS for the amplitude kernels
  int N, d;
  const int* D;          // host: N+1 bond dims
  const long long* toff; // host: N tensor offsets (complex elements)
  const double2* T;      // device: tensors
};
cudaError_t launch_amplitudes(ChainView cv, long long P, const uint8_t* pats,
                              double2* out, double2* work, int maxD, cudaStream_t s);
cudaError_t launch_init_ones(double2* V, long long P, int ld, cudaStream_t s);
cudaError_t launch_init_ones_f(float2* V, long long P, cudaStream_t s);
cudaError_t launch_sample_select_mixed(int S, int d, int Dm, const float2* W, const float2* Y,
                                       const double* u, int ustride, int site, uint64_t seed,
                                       uint64_t counter0, float2* vnew, uint8_t* out, int N,
                                       uint8_t* flags, double flag_tol, cudaStream_t s);
struct GaugeTask {        // one site of a batched energy-gauge launch
  const double2* A;       // FP64 tensor, E order
  int Dl, Dr;
  const double* El;       // e^{+E/2} of the left bond's states (launch_gauge_scale)
  const double* Er;       // e^{-E/2} of the right bond's states
  double2* Ah;            // parity-compact output, double-float pairs (df_pack)
  ParitySite P;
};
cudaError_t launch_energy_gauge_batch(const GaugeTask* tasks_dev, int ntasks, int d, int max_elems,
                                      cudaStream_t s);
// G[i] = e^{E[i]/2}, G[n + i] = e^{-E[i]/2}: the energy gauge's factors
cudaError_t launch_gauge_scale(const double* E, long long n, double* G, cudaStream_t s);
// El, Er: e^{+E/2} of the left bond's states, e^{-E/2} of the right bond's
cudaError_t launch_energy_gauge(const double2* A, int Dl, int d, int Dr, const double* El,
                                const double* Er, const ParitySite& P, double2* Ah, cudaStream_t s);
// allocation-free single-site build (noalloc.cu)
int noalloc_build_site(int device, cudaStream_t s, int* status_dev, int32_t nl, int32_t nr,
                       int32_t d, const double* Qm, double cscale, int32_t Dl,
                       const uint8_t* occ_l, int32_t Dr, const uint8_t* occ_r, int32_t precision,
                       double* out, const char** detail);
// complex GEMM in double-float arithmetic (k_df64.cu), FP64 operands/result
// many independent double-float products in one launch (grouped k split,
// partials reduced in FP64 in k order); products with M or N = 0 are skipped
struct DfSub {
  int opa, opb, M, N, K;
  const double2* A; long long lda;
  const double2* B; long long ldb;
  double2* C; long long ldc;
  int herm;                // C Hermitian (M == N): lower triangle computed, mirrored
  int asplit = 0, bsplit = 0, csplit = 0;   // A, B, C as double-float pairs (df_pack)
};
// The workspace starts with DFG_CNT_BYTES of tile counters, which the caller
// zeroes once; every launch leaves them zero.  Partials follow.
constexpr size_t DFG_CNT_BYTES = 256 << 10;
cudaError_t launch_zgemm_df64_grouped(const DfSub* subs, int n, cudaStream_t s, void* work,
                                      size_t work_bytes);
// The same products on the tensor cores with exact accumulation (k_envtc.cu):
// operands sliced into bf16 integer planes; arenas and tensor maps per
// launch slot (0: Ahat R, 1: X Ahat^dag), sized once per build from the
// products of every step.
constexpr int ETC_MAX = 16;           // products per launch
struct EtcNeeds {
  bool ok = true;
  int W[2] = {0, 0};                  // real k (bf16 per arena row)
  long long rowsA[2] = {0, 0}, rowsB[2] = {0, 0}, expo[2] = {0, 0};
  long long part = 0;                 // split-K partials (complex elements)
};
// running maxima over the steps; enc: complex columns per tile (48 or 64)
void envtc_needs(const DfSub* s1, int n1, const DfSub* s2, int n2, int enc, EtcNeeds* acc);
int envtc_slices(int enc);                                    // slices per operand
size_t envtc_arena_bytes(int W, long long rows, int nsl);
struct EnvTcPlan {
  alignas(64) unsigned char mapA[2][128], mapB[2][128];
  int W[2] = {0, 0};
  long long rowsA[2] = {0, 0}, rowsB[2] = {0, 0};
  void* arenaA[2] = {nullptr, nullptr};
  void* arenaB[2] = {nullptr, nullptr};
  int* expo[2] = {nullptr, nullptr};
  long long expo_cap[2] = {0, 0};
  float4* work = nullptr;             // split-K partials: (Re pair, Im pair) per element
  long long work_cap = 0;
  // the configuration: seven slices per operand; 48 complex columns and five
  // accumulators (slice pairs with s + t <= 3 summed exactly), or 64 columns
  // and four (s + t <= 2)
  int enc = 48, nsl = 7;
};
int envtc_setup(EnvTcPlan* P, int slot, int W, long long rowsA, long long rowsB, void* arenaA,
                void* arenaB);
// one environment step (both products); cudaErrorNotSupported (nothing
// enqueued) when a product does not fit the plan
cudaError_t launch_envtc_step(const EnvTcPlan& P, const DfSub* s1, int n1, const DfSub* s2, int n2,
                              int* status, cudaStream_t s);
// herm: C (square) is Hermitian; only i >= j is computed, C[j][i] = conj(C[i][j])
// one state of the batched persistent environment chain (device pointers)
struct EnvJob {
  int N, d;
  const int* D;            // bond dimensions [N + 1]
  const long long* toff;   // tensor offsets [N]
  const long long* eoff;   // environment offsets [N + 1]
  const double2* Ah;       // energy-gauge tensors
  double2* R;              // environments, two parity blocks per bond, as double-float pairs
                           // (R^0 in FP64; R^N = 1 on entry)
  double2* X;              // scratch, >= d maxD^2 complex
  const int* pc;           // parity class sizes [2 (N + 1)] (device); Ah is parity-compact
};
// cfg: tile shape 0 = 64x64, 1 = 32x64, 2 = 32x32 (all give the same result);
// cfg < 0 picks the fastest for the batch class, measured once per process
cudaError_t launch_env_chain_batch(const EnvJob* jobs_dev, int count, int maxN, int maxD, int cfg,
                                   cudaStream_t s, int* chosen);
int env_chain_tile_configs();
// right-canonical mixed sampling (k_canon.cu)
#include <cuda_fp16.h>
int canon_make_map(void* map128, const void* planes, int Kp, long long rows);
// mixed -> pure decomposition (k_filter.cu): one CTA per state of a batch
size_t filter_smem_bytes(int n);
cudaError_t launch_filter(int count, int n, const double* gth, double* S, double* W, double alpha,
                          double eps, int max_iter, int refresh, int* iters, double* loss,
                          int* status, cudaStream_t s);
// Parity groups.  Every PCO adds two quanta, so A^m[alpha, p, beta] = 0
// unless n_alpha + p + n_beta is even; the environments, their Cholesky
// factors and the canonical tensors inherit the block structure, and a
// sampled state lies in one parity class of its bond.  The sampler keeps the
// samples of each class in a group of its own and multiplies only the
// nonzero blocks.  Within group pi of site m the K index runs over the class
// pi states of bond m, and column block p over the class pi^(p&1) states of
// bond m+1, padded to 16 complex columns (widths wself for even p, wother for
// odd p, blocks in p order).
// The state planes are indexed by sample: row s of a class's planes holds
// sample s's state whenever s is in that class's list, so a pass moves only
// sample indices, never a state row.  A stored state may carry a per-sample
// scale (the p = 0 pre-pass stores w_0 and its 1 / |w_0| beside it).
struct TcGroup {          // one group of the two-group sampler GEMM
  int nkb, ntn;           // K blocks of 64 and N tiles of 128 (real fp16 elements)
  const int* cnt;         // rows of the group (device; nullptr: mcap)
  int mcap;               // row capacity
  const int* rows;        // state row (sample index) of each GEMM row
  const __half* A; long long apl;  // state planes: row stride nkb * 64, plane stride apl
  const float* rsc;       // per-sample scale of the stored states (nullptr: 1)
  float* W; long long ldw;       // output rows, real floats per row (nullptr: Vn instead)
  float* part; long long ldp;    // per-row norms of 32-real-column chunks
  __half* Vn; long long vnpl;    // else: output written as fp16 planes into row rows[i] of Vn
  int Kpn, wv;            // (row stride Kpn; real columns >= wv written as zeros, >= Kpn skipped)
};
struct SelGroup {         // one group as the selection pass reads it
  const int* cnt; const int* sid;
  const float2* W; long long ldw;  // complex per row
  const float* part; long long ldp;
  int wself, wother;
};
struct NextGroup {        // one class of the next bond as the selection pass writes it
  __half* V; long long vpl; int Kp;  // sample-indexed state planes
  int* sid; int D;                   // the class's sample list (appended to)
  float* rs;                         // per-sample scale of the stored states
};
struct RestGroup {        // the samples of one group that the p = 0 pre-pass leaves
  int* sid; int* cnt;
};
cudaError_t launch_select_pre(int Scap, const SelGroup& g0, const SelGroup& g1, const NextGroup& n0,
                              const NextGroup& n1, int* cnt_next, const RestGroup& r0,
                              const RestGroup& r1, const unsigned long long* regmax, double reg_ok,
                              const double* u, int ustride, int site, uint64_t seed,
                              uint64_t counter0, uint8_t* out, int N, double margin, cudaStream_t s);
cudaError_t launch_parity_classes(BondArrays ba, int nb, cudaStream_t s);
cudaError_t launch_canon_gemm(const void* mapB0, const void* mapB1, const TcGroup& g0,
                              const TcGroup& g1, const __half* B0, long long bpl0, const __half* B1,
                              long long bpl1, int use_tc, int* status, int sm_reserve,
                              cudaStream_t s);
struct PackJob {          // the planes of one (site, group) from its compact tensor
  const float2* At;       // kc rows of length K
  int kc, kr0, kr1, K, w0, w1, Kp, Np;
  __half* Bp; long long bpl;
};
cudaError_t launch_pack_compact_batch(const PackJob* jobs_dev, int njobs, int d, cudaStream_t s);
cudaError_t launch_sampler_init(__half* V, long long vpl, int Spad, int Kp, int* sid, float* rs,
                                int* cnt, int S, cudaStream_t s);
cudaError_t launch_select_groups(int Scap, int d, const SelGroup& g0, const SelGroup& g1,
                                 const NextGroup& n0, const NextGroup& n1, int* cnt_next,
                                 const double* u, int ustride, int site, uint64_t seed,
                                 uint64_t counter0, uint8_t* out, int N, uint8_t* flags,
                                 double flag_tol, cudaStream_t s);
// Factor and inverse of every diagonal block in one launch, each block in
// shared memory (double-float arithmetic): for blocks of at most
// chol_inv_smem's limit (chol_inv_smem(maxd) == 0 above it); L and L^{-1}
// are written in FP64 like launch_chol and launch_trinv
size_t chol_inv_smem(int maxd);
cudaError_t launch_chol_inv(const double2* src, double2* L, double2* X, const long long* off,
                            const int* Dv, int b0, int nb, int maxd, double* dused,
                            unsigned long long* regmax, int* status, cudaStream_t s);
// src: the environments as double-float pairs (one float4 per complex element)
cudaError_t launch_chol(const double2* src, double2* dst, const long long* off, const int* Dv,
                        int b0, int nb, double* dused, unsigned long long* regmax, int* status,
                        cudaStream_t s);
cudaError_t launch_trinv(const double2* L, double2* X, const long long* off, const int* Dv, int b0,
                         int nb, int maxd, cudaStream_t s);
// complex GEMM in FP32 on the CUDA cores (k_f32gemm.cu): C (FP32) = A B with
// A, B FP64 (a64/b64 = 1) or FP32, row-major, batched by strides
// many independent FP32 products C = A B (A, B FP64 or FP32 as a64 / b64,
// a64 = 2: A as double-float pairs; C FP32) in one launch; the device table is sorted by c0, the first CTA of
// each product, with tn = its column tiles; ctas = the total
struct F32Prob {
  int M, N, K, tn;
  const void* A; long long lda;
  const void* B; long long ldb;
  float2* C; long long ldc;
  long long c0;
};
int f32_tile_rows();
int f32_tile_cols();
cudaError_t launch_zgemm_f32_grouped(const F32Prob* probs_dev, int np, long long ctas, int a64,
                                     int b64, cudaStream_t s);
cudaError_t launch_zgemm_f32(int M, int N, int K, const void* A, int a64, long long lda, long long sA,
                             const void* B, int b64, long long ldb, long long sB, float2* C,
                             long long ldc, long long sC, int batch, cudaStream_t s);
cudaError_t launch_sample_select(int S, int d, int Dm, const double2* W,
                                 const double2* Y, const double* u, int ustride,
                                 int site, uint64_t seed, uint64_t counter0,
                                 double2* vnew, uint8_t* out, int N, uint8_t* flags,
                                 cudaStream_t s);
