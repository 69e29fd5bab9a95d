// Library objects shared by the host translation units (api.cu, batch.cu):
// contexts, stream-ordered device buffers, MPS handles, error reporting and
// the opt-in stage timer.  Host code only.
#pragma once
#include "internal.h"
#include <array>
#include <cstdio>
#include <cstdlib>
#include <memory>
#include <string>
#include <vector>

extern thread_local std::string g_detail;


inline int fail(int code, const std::string& what) {
  g_detail = what;
  return code;
}

#define CK(expr)                                                                   \
  do {                                                                             \
    cudaError_t e_ = (expr);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      return fail(e_ == cudaErrorMemoryAllocation ? GBSMPS_ERR_OOM : GBSMPS_ERR_CUDA, \
                  std::string(#expr) + ": " + cudaGetErrorString(e_));            \
    }                                                                              \
  } while (0)

// Opt-in stage tracing: with GBSMPS_PROFILE=1 every pipeline records CUDA
// events between its stages and prints the elapsed times to stderr.
struct StageTimer {
  bool on = false;
  cudaStream_t s = nullptr;
  std::vector<std::pair<std::string, cudaEvent_t>> ev;
  explicit StageTimer(cudaStream_t st) : s(st) {
    const char* e = getenv("GBSMPS_PROFILE");
    on = e && e[0] == '1';
    mark("start");
  }
  int* dbg_status = nullptr;       // GBSMPS_DEBUG=1: status word checked at every mark
  std::string failed_stage;
  void mark(const char* name) {
    if (dbg_status && failed_stage.empty()) {
      int st = 0;
      cudaMemcpyAsync(&st, dbg_status, sizeof(int), cudaMemcpyDeviceToHost, s);
      cudaStreamSynchronize(s);
      if (st) {
        failed_stage = name;
        fprintf(stderr, "[gbsmps] device status %d raised in stage '%s'\n", st, name);
      }
    }
    if (!on) return;
    cudaEvent_t e;
    cudaEventCreate(&e);
    cudaEventRecord(e, s);
    ev.emplace_back(name, e);
  }
  ~StageTimer() {
    if (!on) return;
    cudaEventSynchronize(ev.back().second);
    for (size_t i = 1; i < ev.size(); ++i) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ev[i - 1].second, ev[i].second);
      fprintf(stderr, "[gbsmps] %-14s %9.3f ms\n", ev[i].first.c_str(), ms);
    }
    for (auto& p : ev) cudaEventDestroy(p.second);
  }
};

inline int status_to_code(int st) {
  if (st & ST_NOT_SYMMETRIC) return GBSMPS_ERR_NOT_SYMMETRIC;
  if (st & ST_NOT_PURE) return GBSMPS_ERR_NOT_PURE;
  if (st & ST_BOUNDS) return GBSMPS_ERR_BOUNDS;
  if (st & ST_NOT_CONVERGED) return GBSMPS_ERR_NOT_CONVERGED;
  if (st & ST_NUMERIC) return GBSMPS_ERR_NUMERIC;
  if (st & ST_TIMEOUT) return GBSMPS_ERR_TIMEOUT;
  return st ? GBSMPS_ERR_CUDA : GBSMPS_OK;
}

struct gbsmps_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int* d_status = nullptr;
  unsigned long long launches_at_create = 0;
  // extra streams for work that overlaps the main chain, created on first use
  std::vector<cudaStream_t> sides;
  cudaStream_t side_stream(int k = 0) {
    while ((int)sides.size() <= k) {
      cudaStream_t st = nullptr;
      if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return nullptr;
      sides.push_back(st);
    }
    return sides[k];
  }
  ~gbsmps_ctx() {
    for (auto st : sides) cudaStreamDestroy(st);
  }
};

struct DevBuf {                // stream-ordered device allocation
  void* p = nullptr;
  cudaStream_t s = nullptr;
  cudaError_t alloc(size_t bytes, cudaStream_t st) {
    s = st;
    if (bytes == 0) bytes = 16;
    return cudaMallocAsync(&p, bytes, st);
  }
  void release() {
    if (p) cudaFreeAsync(p, s);
    p = nullptr;
  }
  template <class T> T* as() const { return reinterpret_cast<T*>(p); }
};

struct gbsmps_mps {
  gbsmps_ctx* ctx = nullptr;
  int N = 0, d = 0, chi = 0, precision = 0;
  std::vector<int> D, ne;
  std::vector<double> eps;
  std::vector<long long> toff, eoff;
  int maxD = 1;
  long long ttot = 0, etot = 0;   // complex elements of all tensors / all environments
  DevBuf tensors, env, gsvd, bonds;
  DevBuf tens_mixed;        // mixed path: tensors in the energy gauge (parity-compact pairs)
  DevBuf gscale;            // mixed path: e^{+E/2} then e^{-E/2} of every bond's states
  DevBuf vacamp;            // mixed path: the all-vacuum amplitude from the environment chain (FP64)
  // mixed path, right-canonical sampler: Cholesky factors of the environments,
  // their inverses, and every site's canonical tensor as fp16 planes + TMA map
  DevBuf eoff_dev, lchol, linv, bpack;
  DevBuf creg;                    // largest relative Cholesky regulariser (double bits, device)
  std::vector<int> pcnt;          // [2b + c]: kept states of bond b with parity c
  struct SiteGroups {             // the two parity groups of one site's sampler GEMM
    int Kp[2], Np[2];             // group pi: K (real, multiple of 64), N (real, of 128)
    int w[2];                     // column-block width (complex, multiple of 16) of the
                                  // class c states of the right bond
    long long boff[2];            // group pi's packed planes in bpack (halves)
    std::array<unsigned char, 128> map[2];
  };
  std::vector<SiteGroups> sg;
  BondArrays ba{};
  double* lam2 = nullptr;
  double2* Qm = nullptr;
  double* cm = nullptr;
  // out of core (gbsmps_offload): the sampler planes in pinned host memory,
  // streamed site by site through a ring of device slots by a copy stream;
  // the MPS then holds no tensor on the device
  static constexpr int RING = 3;
  __half* host_bpack = nullptr;
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ring_ready[RING] = {}, ring_free[RING] = {}, ring_start = nullptr;
  long long site_halves(int m) const {        // both parity groups' planes of site m
    return 2LL * sg[m].Np[0] * sg[m].Kp[0] + 2LL * sg[m].Np[1] * sg[m].Kp[1];
  }
  ~gbsmps_mps() {
    tensors.release(); env.release(); gsvd.release(); bonds.release(); tens_mixed.release();
    gscale.release();
    vacamp.release();
    eoff_dev.release(); lchol.release(); linv.release(); bpack.release(); creg.release();
    if (host_bpack) {            // pinned memory: no copy or sampling may still read it
      if (copy_stream) cudaStreamSynchronize(copy_stream);
      if (ctx) cudaStreamSynchronize(ctx->stream);
      cudaFreeHost(host_bpack);
    }
    for (int k = 0; k < RING; ++k) {
      if (ring_ready[k]) cudaEventDestroy(ring_ready[k]);
      if (ring_free[k]) cudaEventDestroy(ring_free[k]);
    }
    if (ring_start) cudaEventDestroy(ring_start);
    if (copy_stream) cudaStreamDestroy(copy_stream);
  }
};

inline int sync_status(gbsmps_ctx* c) {
  int st = 0;
  CK(cudaMemcpyAsync(&st, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (st) {
    CK(cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream));
    return fail(status_to_code(st), "device status word " + std::to_string(st));
  }
  return GBSMPS_OK;
}

inline int check_opts(const gbsmps_opts* o) {
  if (!o) return fail(GBSMPS_ERR_ARG, "opts is NULL");
  if (o->d < 1 || o->d > 255) return fail(GBSMPS_ERR_ARG, "d out of range [1,255]");
  if (o->chi_max < 1 || o->chi_max > 4096) return fail(GBSMPS_ERR_ARG, "chi_max out of range [1,4096]");
  if (!(o->eps_trunc >= 0.0 && o->eps_trunc < 1.0)) return fail(GBSMPS_ERR_ARG, "eps_trunc not in [0,1)");
  if (!(o->lambda2_freeze >= 0.0 && o->lambda2_freeze < 1.0))
    return fail(GBSMPS_ERR_ARG, "lambda2_freeze not in [0,1)");
  if (o->precision != GBSMPS_PREC_FP64 && o->precision != GBSMPS_PREC_MIXED)
    return fail(GBSMPS_ERR_ARG, "unknown precision");
  return GBSMPS_OK;
}


// ---- build pipeline stages (pipeline.cu), shared by single and batched builds
namespace gbs {
struct Front {                  // per-state device scratch of the GSVD stage
  double* Gs = nullptr;
  int* dbw = nullptr;
  double* work = nullptr;
};
struct Readback {               // host copies of the bond sizes and scale factors
  std::vector<int> D, ne, pcnt;
  std::vector<double> eps, cm;
};
int alloc_front(gbsmps_mps* M, gbsmps_ctx* c, int N, const gbsmps_opts* o, Front* f);
int launch_checks(gbsmps_ctx* c, gbsmps_mps* M, const double* dgamma, const gbsmps_opts* o,
                  const Front& f);
int launch_bases(gbsmps_ctx* c, gbsmps_mps* M, const gbsmps_opts* o);
int enqueue_readback(gbsmps_mps* M, Readback* r, cudaStream_t s);
void finish_readback(gbsmps_mps* M, const Readback& r);
int alloc_tensors(gbsmps_mps* M, cudaStream_t s, size_t* scr_max);
void site_tasks(gbsmps_mps* M, const std::vector<double>& cm, std::vector<SiteTask>& out);
int run_pco(gbsmps_ctx* c, std::vector<SiteTask>& tasks, size_t scr_max, int d, int precision);
int env_single(gbsmps_ctx* c, gbsmps_mps* M, StageTimer& tm);
int normalise_single(gbsmps_ctx* c, gbsmps_mps* M);
struct CanonWork {               // temporaries of the right-canonical packing
  DevBuf du;                     // regulariser used per diagonal block
  ~CanonWork() { du.release(); }
};
ParitySite parity_site(const gbsmps_mps* M, int m);   // site m's parity-compact layout
int canon_prepare(gbsmps_mps* M, CanonWork* w, cudaStream_t s);
int canon_bonds(gbsmps_ctx* c, gbsmps_mps* M, CanonWork* w, int b0, int nb, cudaStream_t s);
int canon_sites_grouped(gbsmps_mps* M, CanonWork* w0, cudaStream_t st);
int canonical_stage(gbsmps_ctx* c, gbsmps_mps* M, StageTimer& tm);
int finish(gbsmps_ctx* c, gbsmps_mps* M);
// a build split in two: the front (validation, GSVD chain, bases, bond
// read-back enqueued) on one context, the rest on another once the front is
// done; build_single runs both on one context.  gate (may be null): the
// rest's stream waits for it before the stages that occupy every SM
struct FrontState {
  std::unique_ptr<gbsmps_mps> M;
  Front f;
  Readback rb;
  gbsmps_opts opts{};
  gbsmps_ctx* cf = nullptr;      // the context the front ran on
};
int build_front(gbsmps_ctx* cf, int N, const double* dgamma, const gbsmps_opts* o, FrontState* fs);
int build_rest(gbsmps_ctx* c, FrontState* fs, cudaEvent_t gate, gbsmps_mps_t* out);
// the rest in its three parts: PCO (long CTAs), environments (short CTAs:
// may run beside a sampling), canonical form + hand-over
int rest_pco(gbsmps_ctx* c, FrontState* fs, cudaEvent_t gate);
int rest_env(gbsmps_ctx* c, FrontState* fs);
int rest_canon(gbsmps_ctx* c, FrontState* fs, cudaEvent_t gate, gbsmps_mps_t* out);
int build_single(gbsmps_ctx* c, int N, const double* dgamma, const gbsmps_opts* o,
                 gbsmps_mps_t* out, cudaEvent_t gate = nullptr);
int sample_impl(gbsmps_mps* m, cudaStream_t s, int* status, int sm_reserve, int sync_host,
                int64_t S, uint64_t seed, uint64_t counter0, const double* uniforms, uint8_t* out,
                uint8_t* flags, int mem_kind);
}  // namespace gbs
