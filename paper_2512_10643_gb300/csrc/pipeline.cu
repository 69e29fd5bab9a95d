// Stages of the build pipeline (Gamma on the device -> normalised MPS), shared
// by the single-state entry points and the batched build: allocation of the
// GSVD and bond arrays, input checks, kept bases, the host read-back of the
// bond sizes, tensor storage, the PCO waves, the per-state environment chain
// and normalisation, and the right-canonical packing of the mixed sampler.
#include "objects.h"
#include <algorithm>
#include <cstring>

namespace gbs {

int alloc_front(gbsmps_mps* M, gbsmps_ctx* c, int N, const gbsmps_opts* o, Front* f) {
  cudaStream_t s = c->stream;
  M->ctx = c; M->N = N; M->d = o->d; M->chi = o->chi_max; M->precision = o->precision;
  const int cap = o->chi_max + TIE_MARGIN;
  const int nb = N + 1;
  // GSVD outputs and the carried correlation block in one allocation
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t r = off; off += (bytes + 255) & ~size_t(255); return r; };
  size_t o_Q = take(sizeof(double2) * (size_t)N * QS * QS);
  size_t o_c = take(sizeof(double) * N);
  size_t o_G = take(sizeof(double) * 2 * 2 * NEM * 2 * (size_t)std::max(N, 1));
  size_t o_bw = take(sizeof(int) * 4);
  size_t o_work = take(sizeof(double) * 8);
  CK(M->gsvd.alloc(off, s));
  char* g0 = M->gsvd.as<char>();
  M->Qm = reinterpret_cast<double2*>(g0 + o_Q);
  M->cm = reinterpret_cast<double*>(g0 + o_c);
  f->Gs = reinterpret_cast<double*>(g0 + o_G);
  f->dbw = reinterpret_cast<int*>(g0 + o_bw);
  f->work = reinterpret_cast<double*>(g0 + o_work);
  // kept bases, maps and per-bond scalars in one allocation
  off = 0;
  size_t o_occ = take((size_t)nb * cap * NEM);
  size_t o_E = take(sizeof(double) * (size_t)nb * cap);
  size_t o_low = take(sizeof(int) * (size_t)nb * NEM * cap);
  size_t o_D = take(sizeof(int) * nb);
  size_t o_ne = take(sizeof(int) * nb);
  size_t o_mo = take(sizeof(int) * (size_t)nb * NEM);
  size_t o_l2 = take(sizeof(double) * (size_t)nb * NEM);
  size_t o_eps = take(sizeof(double) * nb);
  size_t o_pidx = take(sizeof(int) * (size_t)nb * cap);
  size_t o_pcnt = take(sizeof(int) * 2 * (size_t)nb);
  CK(M->bonds.alloc(off, s));
  char* b0 = M->bonds.as<char>();
  BondArrays& ba = M->ba;
  ba.cap = cap;
  ba.occ = reinterpret_cast<uint8_t*>(b0 + o_occ);
  ba.E = reinterpret_cast<double*>(b0 + o_E);
  ba.low = reinterpret_cast<int*>(b0 + o_low);
  ba.D = reinterpret_cast<int*>(b0 + o_D);
  ba.ne = reinterpret_cast<int*>(b0 + o_ne);
  ba.maxocc = reinterpret_cast<int*>(b0 + o_mo);
  ba.lam2 = reinterpret_cast<double*>(b0 + o_l2);
  ba.eps = reinterpret_cast<double*>(b0 + o_eps);
  ba.pidx = reinterpret_cast<int*>(b0 + o_pidx);
  ba.pcnt = reinterpret_cast<int*>(b0 + o_pcnt);
  M->lam2 = ba.lam2;
  CK(cudaMemsetAsync(b0, 0, off, s));
  CK(cudaMemsetAsync(M->Qm, 0, sizeof(double2) * (size_t)N * QS * QS, s));
  return GBSMPS_OK;
}

int launch_checks(gbsmps_ctx* c, gbsmps_mps* M, const double* dgamma, const gbsmps_opts* o,
                  const Front& f) {
  cudaStream_t s = c->stream;
  if (o->validate) {
    CK(launch_check_input(dgamma, M->N, o->purity_tol, f.work, c->d_status, s));
    COUNT_LAUNCH(2);
  }
  CK(launch_bandwidth(dgamma, M->N, f.dbw, s));
  COUNT_LAUNCH(1);
  return GBSMPS_OK;
}

int launch_bases(gbsmps_ctx* c, gbsmps_mps* M, const gbsmps_opts* o) {
  cudaStream_t s = c->stream;
  const int nb = M->N + 1;
  CK(launch_basis(M->ba, nb, o->chi_max, o->eps_trunc, c->d_status, s));
  CK(launch_maps(M->ba, nb, c->d_status, s));
  CK(launch_parity_classes(M->ba, nb, s));
  COUNT_LAUNCH(3);
  return GBSMPS_OK;
}

int enqueue_readback(gbsmps_mps* M, Readback* r, cudaStream_t s) {
  const int N = M->N, nb = N + 1;
  r->D.assign(nb, 1);
  r->ne.assign(nb, 0);
  r->eps.assign(nb, 0.0);
  r->cm.assign(N, 0.0);
  r->pcnt.assign(2 * nb, 0);
  CK(cudaMemcpyAsync(r->D.data(), M->ba.D, sizeof(int) * nb, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(r->pcnt.data(), M->ba.pcnt, sizeof(int) * 2 * nb, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(r->ne.data(), M->ba.ne, sizeof(int) * nb, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(r->eps.data(), M->ba.eps, sizeof(double) * nb, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(r->cm.data(), M->cm, sizeof(double) * N, cudaMemcpyDeviceToHost, s));
  return GBSMPS_OK;
}

void finish_readback(gbsmps_mps* M, const Readback& r) {
  const int N = M->N;
  M->D = r.D;
  M->ne = r.ne;
  M->pcnt = r.pcnt;
  M->eps.assign(r.eps.begin() + 1, r.eps.end() - 1);
  M->D[0] = 1; M->D[N] = 1;
}

int alloc_tensors(gbsmps_mps* M, cudaStream_t s, size_t* scr_max) {
  const int N = M->N, d = M->d;
  M->toff.resize(N);
  long long tot = 0;
  size_t sm = 0;
  M->maxD = 1;
  for (int m = 0; m < N; ++m) {
    M->toff[m] = tot;
    tot += (long long)M->D[m] * d * M->D[m + 1];
    sm = std::max(sm, pco_scratch_elems(M->D[m], M->D[m + 1]));
    M->maxD = std::max(M->maxD, M->D[m]);
  }
  M->eoff.resize(N + 1);
  long long etot = 0;
  for (int m = 0; m <= N; ++m) { M->eoff[m] = etot; etot += (long long)M->D[m] * M->D[m]; }
  M->ttot = tot;
  M->etot = etot;
  CK(M->tensors.alloc(sizeof(double2) * tot, s));
  CK(M->env.alloc(sizeof(double2) * (etot + 8), s));
  if (scr_max) *scr_max = std::max(*scr_max, sm);
  return GBSMPS_OK;
}

void site_tasks(gbsmps_mps* M, const std::vector<double>& cm, std::vector<SiteTask>& out) {
  const int N = M->N, cap = M->ba.cap;
  for (int m = 0; m < N; ++m) {
    SiteTask t;
    t.nl = M->ne[m]; t.nr = M->ne[m + 1]; t.Dl = M->D[m]; t.Dr = M->D[m + 1];
    t.Q = M->Qm + (size_t)m * QS * QS; t.qs = QS;
    t.c = cm[m];
    t.occl = M->ba.occ + (size_t)m * cap * NEM; t.lowl = M->ba.low + (size_t)m * NEM * cap; t.capl = cap;
    t.occr = M->ba.occ + (size_t)(m + 1) * cap * NEM; t.lowr = M->ba.low + (size_t)(m + 1) * NEM * cap;
    t.capr = cap;
    t.out = M->tensors.as<double2>() + M->toff[m];
    t.scratch_off = 0;
    if ((int)M->pcnt.size() == 2 * (N + 1)) {
      t.pl = M->ba.pidx + (size_t)m * cap;
      t.pr = M->ba.pidx + (size_t)(m + 1) * cap;
      t.kl[0] = M->pcnt[2 * m]; t.kl[1] = M->pcnt[2 * m + 1];
      t.kr[0] = M->pcnt[2 * m + 2]; t.kr[1] = M->pcnt[2 * m + 3];
    }
    out.push_back(t);
  }
}

int run_pco(gbsmps_ctx* c, std::vector<SiteTask>& tasks, size_t scr_max, int d, int precision) {
  // GBSMPS_PCO_FP64=1 runs a mixed build's passes in FP64 (its other stages
  // unchanged): the mixed path's error without the PCO's FP32 part
  if (precision == GBSMPS_PREC_MIXED) {
    const char* e = getenv("GBSMPS_PCO_FP64");
    if (e && e[0] == '1') precision = GBSMPS_PREC_FP64;
  }
  // FP64 passes for FP64 states; the mixed path runs the passes in FP32 and
  // accumulates the tensors in FP64 (GB300's FP64 pipe is 1/64 of its FP32
  // rate; the mixed path's amplitudes are held to 1e-5 of the FP64 path's).
  // Up to one resident wave of sites: one CTA per site; more: persistent
  // CTAs (below)
  cudaStream_t s = c->stream;
  const int n = (int)tasks.size();
  if (n == 0) return GBSMPS_OK;
  const int grid = pco_dynamic_grid();
  if (grid > 0 && n > grid) {
    // more sites than resident CTAs (a batch, or a long chain): persistent
    // CTAs pull the sites largest first, each with its own scratch slot
    std::sort(tasks.begin(), tasks.end(), [](const SiteTask& a, const SiteTask& b) {
      const double ca = (double)a.Dl * a.Dr * (a.nl + a.nr + 1), cb = (double)b.Dl * b.Dr * (b.nl + b.nr + 1);
      return ca > cb;
    });
    DevBuf scr, tk, ctr;
    CK(scr.alloc(sizeof(double2) * scr_max * grid, s));
    CK(tk.alloc(sizeof(SiteTask) * n, s));
    CK(ctr.alloc(sizeof(int), s));
    CK(cudaMemcpyAsync(tk.p, tasks.data(), sizeof(SiteTask) * n, cudaMemcpyHostToDevice, s));
    cudaEvent_t tr0 = g_pco_trace.begin(s);
    CK(launch_pco_dynamic(tk.as<SiteTask>(), n, d, precision, scr.as<double2>(), scr_max, grid,
                          ctr.as<int>(), c->d_status, s));
    g_pco_trace.end(tr0, s, 0.0, 0.0);
    COUNT_LAUNCH(1);
    scr.release();
    tk.release();
    ctr.release();
    return GBSMPS_OK;
  }
  const int wave = std::min(n, 304);
  for (int k = 0; k < n; ++k) tasks[k].scratch_off = (size_t)(k % wave) * scr_max;
  DevBuf scr, tk;
  CK(scr.alloc(sizeof(double2) * scr_max * wave, s));
  CK(tk.alloc(sizeof(SiteTask) * n, s));
  CK(cudaMemcpyAsync(tk.p, tasks.data(), sizeof(SiteTask) * n, cudaMemcpyHostToDevice, s));
  for (int k0 = 0; k0 < n; k0 += wave) {
    const int cnt = std::min(wave, n - k0);
    cudaEvent_t tr0 = g_pco_trace.begin(s);
    CK(launch_pco(tk.as<SiteTask>() + k0, cnt, d, precision, scr.as<double2>(), c->d_status, s));
    g_pco_trace.end(tr0, s, 0.0, 0.0);
    COUNT_LAUNCH(1);
  }
  scr.release();
  tk.release();
  return GBSMPS_OK;
}

ParitySite parity_site(const gbsmps_mps* M, int m) {
  const int cap = M->ba.cap;
  ParitySite P;
  P.pl = M->ba.pidx + (size_t)m * cap;
  P.pr = M->ba.pidx + (size_t)(m + 1) * cap;
  P.kl[0] = M->pcnt[2 * m]; P.kl[1] = M->pcnt[2 * m + 1];
  P.kr[0] = M->pcnt[2 * m + 2]; P.kr[1] = M->pcnt[2 * m + 3];
  return P;
}

// one step of the parity-compact environment chain: R_m from R_{m+1}.
// Product 1, per class c and p: X_c[:, block p] = Ahat_c[:, block p] R_{m+1, c^(p&1)};
// product 2, per class c: R_{m, c} = X_c Ahat_c^dag (Hermitian)
// One step of the environment chain on the parity blocks.  With ui set it
// also carries the all-vacuum amplitude from the right: uo = Ahat^m[0] ui on
// the class-0 states (the vacuum pattern keeps every bond state in the even
// class; in the energy gauge the end bonds' energies are 0, so at m = 0 the
// product is the amplitude itself), written as pairs, or in FP64 at m = 0.
void env_subs(const gbsmps_mps* M, int m, const double2* Ah, double2* R, double2* X,
              const double2* ui, double2* uo, std::vector<DfSub>& s1, std::vector<DfSub>& s2) {
  const int d = M->d;
  const ParitySite P = parity_site(M, m);
  const int Dr = P.kr[0] + P.kr[1];
  const long long K[2] = {pk_len(d, P.kr, 0), pk_len(d, P.kr, 1)};
  const long long o1 = (long long)P.kl[0] * K[0];
  const double2* A = Ah + M->toff[m];
  const double2* Rr = R + M->eoff[m + 1];
  s1.clear();
  s2.clear();
  for (int c = 0; c < 2; ++c)
    for (int p = 0; p < d; ++p) {
      const int cr = c ^ (p & 1);
      const long long off = (c ? o1 : 0) + pk_off(p, Dr, P.kr, c);
      // Ahat, R (bonds 1 .. N) and X as double-float pairs
      s1.push_back(DfSub{0, 0, P.kl[c], P.kr[cr], P.kr[cr], A + off, K[c],
                         Rr + (cr ? (long long)P.kr[0] * P.kr[0] : 0), P.kr[cr], X + off, K[c], 0,
                         1, 1, 1});
    }
  if (ui && uo)       // block p = 0 of class 0: the first kr[0] columns of its rows
    s1.push_back(DfSub{0, 0, P.kl[0], 1, P.kr[0], A, K[0], ui, 1, uo, 1, 0, 1, 1, m > 0 ? 1 : 0});
  for (int c = 0; c < 2; ++c) {
    const long long off = c ? o1 : 0;
    // R_m as pairs too, but R_0 (the squared norm) in FP64
    s2.push_back(DfSub{0, 1, P.kl[c], P.kl[c], (int)K[c], X + off, K[c], A + off, K[c],
                       R + M->eoff[m] + (c ? (long long)P.kl[0] * P.kl[0] : 0), P.kl[c], 1, 1, 1,
                       m > 0 ? 1 : 0});
  }
}

// One step of the environment chain on the parity blocks.  With ui set it
// also carries the all-vacuum amplitude from the right: uo = Ahat^m[0] ui on
// the class-0 states (the vacuum pattern keeps every bond state in the even
// class; in the energy gauge the end bonds' energies are 0, so at m = 0 the
// product is the amplitude itself), written as pairs, or in FP64 at m = 0.
// The products run on the tensor cores when a plan is given (and they fit
// it), else in double-float on the FP32 pipes.
int env_step_blocks(gbsmps_mps* M, int m, const double2* Ah, double2* R, double2* X, void* work,
                    size_t wbytes, cudaStream_t s, const double2* ui, double2* uo,
                    const EnvTcPlan* tp, int* status) {
  std::vector<DfSub> s1, s2;
  env_subs(M, m, Ah, R, X, ui, uo, s1, s2);
  if (tp) {
    const cudaError_t e =
        launch_envtc_step(*tp, s1.data(), (int)s1.size(), s2.data(), (int)s2.size(), status, s);
    if (e != cudaErrorNotSupported) {
      CK(e);
      return GBSMPS_OK;
    }
  }
  CK(launch_zgemm_df64_grouped(s1.data(), (int)s1.size(), s, work, wbytes));
  CK(launch_zgemm_df64_grouped(s2.data(), (int)s2.size(), s, work, wbytes));
  return GBSMPS_OK;
}

// The environment products: GBSMPS_ENV_TC=1 (default) the tensor cores with
// 48-column tiles and slice pairs s + t <= 3 summed exactly, =2 64-column
// tiles with s + t <= 2 exact (4x less accurate over the 144-mode chain),
// =0 the double-float GEMM on the FP32 pipes (the most accurate chain:
// 6.8e-14 of the largest amplitude against 1.2e-12 for =1, with FP64 PCO
// passes).  Returns the tile width, 0 for double-float.
int env_tc_mode() {
  const char* e = getenv("GBSMPS_ENV_TC");
  if (e && e[0] == '0') return 0;
  if (e && e[0] == '2') return 64;
  return 48;
}

// arenas, exponents, partials and counters for every step of one chain
struct EnvTcBufs {
  EnvTcPlan plan;
  DevBuf arA[2], arB[2], ex, wk;
  ~EnvTcBufs() { release(); }
  void release() {
    for (int k = 0; k < 2; ++k) { arA[k].release(); arB[k].release(); }
    ex.release(); wk.release();
  }
};

int env_tc_prepare(const gbsmps_mps* M, const double2* Ah, double2* R, double2* X,
                   const double2* ui, double2* uo, int enc, EnvTcBufs& B, cudaStream_t s, bool* ok) {
  EtcNeeds nd;
  std::vector<DfSub> s1, s2;
  for (int m = M->N - 1; m >= 0; --m) {
    env_subs(M, m, Ah, R, X, ui, uo, s1, s2);
    envtc_needs(s1.data(), (int)s1.size(), s2.data(), (int)s2.size(), enc, &nd);
  }
  *ok = nd.ok;
  if (!nd.ok) return GBSMPS_OK;
  EnvTcPlan& P = B.plan;
  P.enc = enc;
  P.nsl = envtc_slices(enc);
  for (int k = 0; k < 2; ++k) {
    const size_t ba = envtc_arena_bytes(nd.W[k], nd.rowsA[k], P.nsl);
    const size_t bb = envtc_arena_bytes(nd.W[k], nd.rowsB[k], P.nsl);
    CK(B.arA[k].alloc(ba, s));
    CK(B.arB[k].alloc(bb, s));
    // padding rows are never written by the slicing: zero them once
    CK(cudaMemsetAsync(B.arA[k].p, 0, ba, s));
    CK(cudaMemsetAsync(B.arB[k].p, 0, bb, s));
    if (envtc_setup(&P, k, nd.W[k], nd.rowsA[k], nd.rowsB[k], B.arA[k].p, B.arB[k].p))
      return GBSMPS_ERR_CUDA;
  }
  CK(B.ex.alloc(sizeof(int) * (nd.expo[0] + nd.expo[1] + 2), s));
  P.expo[0] = B.ex.as<int>();
  P.expo[1] = P.expo[0] + nd.expo[0] + 1;
  P.expo_cap[0] = nd.expo[0];
  P.expo_cap[1] = nd.expo[1];
  CK(B.wk.alloc(sizeof(float4) * (nd.part + 1), s));
  P.work = B.wk.as<float4>();
  P.work_cap = nd.part;
  return GBSMPS_OK;
}

int env_single(gbsmps_ctx* c, gbsmps_mps* M, StageTimer& tm) {
  cudaStream_t s = c->stream;
  const int N = M->N, d = M->d, cap = M->ba.cap;
  double2* R = M->env.as<double2>();
  const double2 one = cmk(1.0, 0.0), zero = cmk(0.0, 0.0);
  // R_N = 1 (as a double-float pair on the mixed path)
  static const float4 one_pair = make_float4(1.f, 0.f, 0.f, 0.f);
  if (M->precision == GBSMPS_PREC_MIXED)
    CK(cudaMemcpyAsync(R + M->eoff[N], &one_pair, sizeof(float4), cudaMemcpyHostToDevice, s));
  else
    CK(cudaMemcpyAsync(R + M->eoff[N], &one, sizeof(double2), cudaMemcpyHostToDevice, s));
  size_t xmax = 0;
  for (int m = 0; m < N; ++m) xmax = std::max(xmax, (size_t)M->D[m] * d * M->D[m + 1]);
  DevBuf xb;
  CK(xb.alloc(sizeof(double2) * (xmax + 8), s));
  double2* X = xb.as<double2>();
  if (M->precision == GBSMPS_PREC_MIXED) {
    // energy gauge (FP64) and environments in double-float arithmetic on the
    // FP32 pipes (~44-bit): the chain of N dependent products sets the norm,
    // so its per-step error must stay far below the tensor cores' FP32
    // accumulation error
    // tensors in the parity-compact layout: the environments are then two
    // diagonal blocks per bond and every product a quarter of the dense one
    CK(M->tens_mixed.alloc(sizeof(double2) * M->ttot, s));
    double2* Ah = M->tens_mixed.as<double2>();
    const long long ne = (long long)(N + 1) * cap;
    CK(M->gscale.alloc(sizeof(double) * 2 * ne, s));
    CK(launch_gauge_scale(M->ba.E, ne, M->gscale.as<double>(), s));
    COUNT_LAUNCH(1);
    const double* Gup = M->gscale.as<double>();
    const double* Gdn = Gup + ne;
    {
      // every site in one launch
      std::vector<GaugeTask> gt(N);
      int gmax = 1;
      for (int m = 0; m < N; ++m) {
        gt[m] = GaugeTask{M->tensors.as<double2>() + M->toff[m], M->D[m], M->D[m + 1],
                          Gup + (size_t)m * cap, Gdn + (size_t)(m + 1) * cap, Ah + M->toff[m],
                          parity_site(M, m)};
        gmax = std::max(gmax, M->D[m] * d * M->D[m + 1]);
      }
      DevBuf gb;
      CK(gb.alloc(sizeof(GaugeTask) * N, s));
      CK(cudaMemcpyAsync(gb.p, gt.data(), sizeof(GaugeTask) * N, cudaMemcpyHostToDevice, s));
      CK(launch_energy_gauge_batch(gb.as<GaugeTask>(), N, d, gmax, s));
      COUNT_LAUNCH(1);
      gb.release();
    }
    tm.mark("energy_gauge");
    const size_t wbytes = ((size_t)64 << 20) + DFG_CNT_BYTES;   // tile counters, split-K partials
    DevBuf kw, ub;
    CK(kw.alloc(wbytes, s));
    CK(cudaMemsetAsync(kw.p, 0, DFG_CNT_BYTES, s));
    // the all-vacuum amplitude rides along: u_N = 1, u_m = Ahat^m[0] u_{m+1}
    CK(ub.alloc(sizeof(float4) * 2 * ((size_t)M->maxD + 8), s));
    CK(M->vacamp.alloc(sizeof(double2), s));
    double2* ua = ub.as<double2>();
    double2* ubn = ua + M->maxD + 8;
    static const float4 one_u = make_float4(1.f, 0.f, 0.f, 0.f);
    CK(cudaMemcpyAsync(ua, &one_u, sizeof(float4), cudaMemcpyHostToDevice, s));
    // (plain FP32 products were measured at 4.4e-5 (N = 144) and 2.8e-4
    // (N = 1024) amplitude error against FP64: the norm needs more bits)
    // exact-accumulation tensor-core products (the plan is sized from the
    // products of every step before the first)
    EnvTcBufs tcb;
    const int enc = env_tc_mode();
    bool use_tc = enc > 0;
    if (use_tc) {
      const int rc = env_tc_prepare(M, Ah, R, X, ua, ubn, enc, tcb, s, &use_tc);
      if (rc) return rc;
    }
    for (int m = N - 1; m >= 0; --m) {
      const int rc = env_step_blocks(M, m, Ah, R, X, kw.p, wbytes, s, ua,
                                     m > 0 ? ubn : M->vacamp.as<double2>(),
                                     use_tc ? &tcb.plan : nullptr, c->d_status);
      if (rc) return rc;
      std::swap(ua, ubn);
    }
    tcb.release();
    kw.release();
    ub.release();
  } else {
    for (int m = N - 1; m >= 0; --m) {
      int Dl = M->D[m], Dr = M->D[m + 1];
      const double2* A = M->tensors.as<double2>() + M->toff[m];
      CK(launch_zgemm('N', 'N', Dl * d, Dr, Dr, one, A, Dr, 0, R + M->eoff[m + 1], Dr, 0, zero, X,
                      Dr, 0, 1, s));
      CK(launch_zgemm('N', 'C', Dl, Dl, d * Dr, one, X, d * Dr, 0, A, d * Dr, 0, zero,
                      R + M->eoff[m], Dl, 0, 1, s));
      COUNT_LAUNCH(2);
    }
  }
  xb.release();
  return GBSMPS_OK;
}

int normalise_single(gbsmps_ctx* c, gbsmps_mps* M) {
  // vacuum amplitude, then A^1 *= conj(phase)/sqrt(norm^2)
  cudaStream_t s = c->stream;
  const int N = M->N, d = M->d, cap = M->ba.cap;
  double2* R = M->env.as<double2>();
  DevBuf ab;
  CK(ab.alloc(sizeof(double2) * (2 * (size_t)M->maxD + 8) + N, s));
  double2* awork = ab.as<double2>();
  double2* amp0 = awork + 2 * M->maxD;
  double2* fac = amp0 + 1;
  uint8_t* zpat = reinterpret_cast<uint8_t*>(fac + 2);
  if (M->precision == GBSMPS_PREC_MIXED && M->vacamp.p) {
    amp0 = M->vacamp.as<double2>();          // carried along the environment chain
  } else {
    CK(cudaMemsetAsync(zpat, 0, N, s));
    ChainView cv{N, d, M->D.data(), M->toff.data(), M->tensors.as<double2>()};
    CK(launch_amplitudes(cv, 1, zpat, amp0, awork, M->maxD, s));
    COUNT_LAUNCH(2 + N);
  }
  CK(launch_norm_phase(R + M->eoff[0], amp0, fac, c->d_status, s));
  CK(launch_zscale(M->tensors.as<double2>(), (size_t)M->D[0] * d * M->D[1], fac, s));
  COUNT_LAUNCH(2);
  if (M->precision == GBSMPS_PREC_MIXED) {   // the normalised first tensor in the energy gauge
    const double* Gup = M->gscale.as<double>();
    const double* Gdn = Gup + (long long)(N + 1) * cap;
    CK(launch_energy_gauge(M->tensors.as<double2>(), 1, d, M->D[1], Gup, Gdn + cap,
                           parity_site(M, 0), M->tens_mixed.as<double2>(), s));
    COUNT_LAUNCH(1);
  }
  ab.release();
  return GBSMPS_OK;
}

// ---- right-canonical form for the tensor-core sampler ----------------------
// R_m = L_m L_m^dag (bonds 1..N-1), L_0 = L_N = 1 for the normalised state;
// At^m = L_m^{-1} Ahat^m L_{m+1}; packed as fp16 planes per site.  Bond b
// needs only R_b, site m only L_m, L_m^{-1}, L_{m+1} and Ahat^m, so the
// stages below can run per bond / per site as soon as their inputs exist.
int canon_prepare(gbsmps_mps* M, CanonWork* w, cudaStream_t s) {
  const int N = M->N, d = M->d;
  if ((int)M->pcnt.size() != 2 * (N + 1)) return fail(GBSMPS_ERR_CUDA, "parity classes missing");
  // the environments' diagonal blocks (bond b, class c at 2b + c): offsets,
  // then sizes; the factors and inverses use the same places
  {
    const int nbk = 2 * (N + 1);
    std::vector<long long> tab(nbk + (nbk + 1) / 2, 0);
    int* dims = reinterpret_cast<int*>(tab.data() + nbk);
    for (int b = 0; b <= N; ++b)
      for (int c = 0; c < 2; ++c) {
        tab[2 * b + c] = M->eoff[b] + (c ? (long long)M->pcnt[2 * b] * M->pcnt[2 * b] : 0);
        dims[2 * b + c] = M->pcnt[2 * b + c];
      }
    CK(M->eoff_dev.alloc(sizeof(long long) * tab.size(), s));
    CK(cudaMemcpyAsync(M->eoff_dev.p, tab.data(), sizeof(long long) * tab.size(),
                       cudaMemcpyHostToDevice, s));
  }
  CK(M->lchol.alloc(sizeof(double2) * (M->etot + 8), s));
  CK(M->linv.alloc(sizeof(double2) * (M->etot + 8), s));
  CK(w->du.alloc(sizeof(double) * 2 * (N + 1), s));
  CK(cudaMemsetAsync(w->du.p, 0, sizeof(double) * 2 * (N + 1), s));
  CK(M->creg.alloc(sizeof(unsigned long long), s));
  CK(cudaMemsetAsync(M->creg.p, 0, sizeof(unsigned long long), s));
  const double2 one = cmk(1.0, 0.0);
  for (int b : {0, N}) {
    CK(cudaMemcpyAsync(M->lchol.as<double2>() + M->eoff[b], &one, sizeof(double2),
                       cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(M->linv.as<double2>() + M->eoff[b], &one, sizeof(double2),
                       cudaMemcpyHostToDevice, s));
  }
  // the sampler's two parity groups per site: group pi multiplies the class
  // pi rows of the left bond into column blocks p of the class pi^(p&1)
  // states of the right bond
  if ((int)M->pcnt.size() != 2 * (N + 1)) return fail(GBSMPS_ERR_CUDA, "parity classes missing");
  for (int b = 0; b <= N; ++b)
    if (M->pcnt[2 * b] + M->pcnt[2 * b + 1] != M->D[b] || M->pcnt[2 * b] < 0 || M->pcnt[2 * b + 1] < 0)
      return fail(GBSMPS_ERR_CUDA, "parity class sizes do not add up to the bond dimension");
  M->sg.resize(N);
  long long btot = 0;
  for (int m = 0; m < N; ++m) {
    gbsmps_mps::SiteGroups& G = M->sg[m];
    for (int c = 0; c < 2; ++c) G.w[c] = (M->pcnt[2 * (m + 1) + c] + 15) / 16 * 16;
    for (int pi = 0; pi < 2; ++pi) {
      G.Kp[pi] = std::max(64, (2 * M->pcnt[2 * m + pi] + 63) / 64 * 64);
      const long long ncx = (long long)((d + 1) / 2) * G.w[pi] + (long long)(d / 2) * G.w[pi ^ 1];
      G.Np[pi] = (int)std::max<long long>(128, (2 * ncx + 127) / 128 * 128);
      G.boff[pi] = btot;
      btot += 2LL * G.Np[pi] * G.Kp[pi];
    }
  }
  CK(M->bpack.alloc(sizeof(__half) * (btot + 64), s));
  return GBSMPS_OK;
}

int canon_bonds(gbsmps_ctx* c, gbsmps_mps* M, CanonWork* w, int b0, int nb, cudaStream_t s) {
  // one CTA per diagonal parity block of R: factor and inverse together in
  // shared memory with double-float updates when the blocks fit (classes of
  // up to 160 states), else the FP64 kernels in global memory
  if (nb <= 0) return GBSMPS_OK;
  const long long* off = M->eoff_dev.as<long long>();
  const int* dims = reinterpret_cast<const int*>(off + 2 * (M->N + 1));
  int maxd = 1;
  for (int b = b0; b < b0 + nb; ++b) maxd = std::max({maxd, M->pcnt[2 * b], M->pcnt[2 * b + 1]});
  const char* ce = getenv("GBSMPS_CHOL_SMEM");
  if (chol_inv_smem(maxd) && !(ce && ce[0] == '0')) {
    CK(launch_chol_inv(M->env.as<double2>(), M->lchol.as<double2>(), M->linv.as<double2>(), off, dims,
                       2 * b0, 2 * nb, maxd, w->du.as<double>(), M->creg.as<unsigned long long>(),
                       c->d_status, s));
    COUNT_LAUNCH(1);
    return GBSMPS_OK;
  }
  CK(launch_chol(M->env.as<double2>(), M->lchol.as<double2>(), off, dims, 2 * b0, 2 * nb,
                 w->du.as<double>(), M->creg.as<unsigned long long>(), c->d_status, s));
  CK(launch_trinv(M->lchol.as<double2>(), M->linv.as<double2>(), off, dims, 2 * b0, 2 * nb, maxd, s));
  COUNT_LAUNCH(2);
  return GBSMPS_OK;
}

void canon_report(gbsmps_mps* M, CanonWork* w, StageTimer& tm, cudaStream_t s) {
  if (!tm.on) return;
  std::vector<double> h(2 * (M->N + 1));
  cudaMemcpyAsync(h.data(), w->du.p, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  double mx = 0.0;
  for (double v : h) mx = std::max(mx, v);
  fprintf(stderr, "[gbsmps] largest Cholesky regulariser: %.1e of max diag\n", mx);
}

int canonical_stage(gbsmps_ctx* c, gbsmps_mps* M, StageTimer& tm) {
  cudaStream_t s = c->stream;
  CanonWork w;
  int rc = canon_prepare(M, &w, s);
  if (!rc) rc = canon_bonds(c, M, &w, 1, M->N - 1, s);
  if (rc) return rc;
  canon_report(M, &w, tm, s);
  tm.mark("cholesky");
  rc = canon_sites_grouped(M, &w, s);
  if (rc) return rc;
  tm.mark("canonical_pack");
  return GBSMPS_OK;
}

// The transforms and packing of every site as three grouped launches per
// chunk of sites (the chunk's T and At fit a byte budget): all products
// T_c[:, block p] = Ahat_c[:, block p] L_{m+1, c^(p&1)}, then all
// At_c = L_{m, c}^{-1} T_c (site 0: At = T, L_0 = 1), then the planes.
int canon_sites_grouped(gbsmps_mps* M, CanonWork* w0, cudaStream_t st) {
  (void)w0;
  const int N = M->N, d = M->d;
  const int TM = f32_tile_rows(), TN = f32_tile_cols();
  const size_t budget = (size_t)1 << 27;          // complex elements of T (and of At) per chunk
  std::vector<long long> cofs(N + 1, 0);          // compact offset of each site in a chunk
  DevBuf Tg, Ag, tab;
  size_t cap_el = 0;
  for (int m = 0; m < N; ++m) {
    const ParitySite P = parity_site(M, m);
    cap_el = std::max(cap_el, (size_t)pk_size(d, P.kl, P.kr));
  }
  cap_el = std::max(cap_el, std::min(budget, (size_t)M->ttot));
  CK(Tg.alloc(sizeof(float2) * (cap_el + 8), st));
  CK(Ag.alloc(sizeof(float2) * (cap_el + 8), st));
  float2* T = Tg.as<float2>();
  float2* At = Ag.as<float2>();
  const double2* Ahb = M->tens_mixed.as<double2>();
  const double2* Lb = M->lchol.as<double2>();
  const double2* Lib = M->linv.as<double2>();
  std::vector<F32Prob> pt, pa;
  std::vector<PackJob> pj;
  for (int m0 = 0; m0 < N;) {
    // the chunk: sites m0 .. m1-1
    int m1 = m0;
    long long tot = 0;
    while (m1 < N) {
      const ParitySite P = parity_site(M, m1);
      const long long sz = pk_size(d, P.kl, P.kr);
      if (m1 > m0 && (size_t)(tot + sz) > cap_el) break;
      cofs[m1 - m0] = tot;
      tot += sz;
      ++m1;
    }
    pt.clear(); pa.clear(); pj.clear();
    long long ct = 0, ca = 0;
    for (int m = m0; m < m1; ++m) {
      const ParitySite P = parity_site(M, m);
      const int Dr = P.kr[0] + P.kr[1];
      const long long K[2] = {pk_len(d, P.kr, 0), pk_len(d, P.kr, 1)};
      const long long o1 = (long long)P.kl[0] * K[0], base = cofs[m - m0];
      const double2* Ah = Ahb + M->toff[m];
      for (int c = 0; c < 2; ++c) {
        if (P.kl[c] == 0) continue;
        for (int p = 0; p < d; ++p) {
          const int cr = c ^ (p & 1);
          if (P.kr[cr] == 0) continue;
          const long long off = (c ? o1 : 0) + pk_off(p, Dr, P.kr, c);
          F32Prob q{P.kl[c], P.kr[cr], P.kr[cr], (P.kr[cr] + TN - 1) / TN, Ah + off, K[c],
                    Lb + M->eoff[m + 1] + (cr ? (long long)P.kr[0] * P.kr[0] : 0), P.kr[cr],
                    T + base + off, K[c], ct};
          ct += (long long)((q.M + TM - 1) / TM) * q.tn;
          pt.push_back(q);
        }
        if (m > 0) {
          F32Prob q{P.kl[c], (int)K[c], P.kl[c], (int)((K[c] + TN - 1) / TN),
                    Lib + M->eoff[m] + (c ? (long long)P.kl[0] * P.kl[0] : 0), P.kl[c],
                    T + base + (c ? o1 : 0), K[c], At + base + (c ? o1 : 0), K[c], ca};
          ca += (long long)((q.M + TM - 1) / TM) * q.tn;
          pa.push_back(q);
        }
      }
      gbsmps_mps::SiteGroups& G = M->sg[m];
      for (int pi = 0; pi < 2; ++pi) {
        const float2* src = (m > 0 ? At : T) + base + (pi ? o1 : 0);
        pj.push_back(PackJob{src, P.kl[pi], P.kr[pi], P.kr[pi ^ 1], (int)K[pi], G.w[pi], G.w[pi ^ 1],
                             G.Kp[pi], G.Np[pi], M->bpack.as<__half>() + G.boff[pi],
                             (long long)G.Np[pi] * G.Kp[pi]});
      }
    }
    const size_t tb = sizeof(F32Prob) * (pt.size() + pa.size()) + sizeof(PackJob) * pj.size() + 64;
    tab.release();
    CK(tab.alloc(tb, st));
    F32Prob* dpt = tab.as<F32Prob>();
    F32Prob* dpa = dpt + pt.size();
    PackJob* dpj = reinterpret_cast<PackJob*>(dpa + pa.size());
    if (!pt.empty()) CK(cudaMemcpyAsync(dpt, pt.data(), sizeof(F32Prob) * pt.size(), cudaMemcpyHostToDevice, st));
    if (!pa.empty()) CK(cudaMemcpyAsync(dpa, pa.data(), sizeof(F32Prob) * pa.size(), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(dpj, pj.data(), sizeof(PackJob) * pj.size(), cudaMemcpyHostToDevice, st));
    // the canonical tensors feed fp16x2 planes: FP32 products suffice
    CK(launch_zgemm_f32_grouped(dpt, (int)pt.size(), ct, 2, 1, st));   // Ahat as pairs
    CK(launch_zgemm_f32_grouped(dpa, (int)pa.size(), ca, 1, 0, st));
    CK(launch_pack_compact_batch(dpj, (int)pj.size(), d, st));
    for (int m = m0; m < m1; ++m)
      for (int pi = 0; pi < 2; ++pi) {
        gbsmps_mps::SiteGroups& G = M->sg[m];
        if (canon_make_map(G.map[pi].data(), M->bpack.as<__half>() + G.boff[pi], G.Kp[pi], G.Np[pi]))
          return fail(GBSMPS_ERR_CUDA, "tensor map encoding failed for the packed tensors");
      }
    m0 = m1;
  }
  tab.release();
  Tg.release();
  Ag.release();
  return GBSMPS_OK;
}

int finish(gbsmps_ctx* c, gbsmps_mps* M) {
  // R_0 of the normalised state is 1
  const double2 one = cmk(1.0, 0.0);
  CK(cudaMemcpyAsync(M->env.as<double2>() + M->eoff[0], &one, sizeof(double2),
                     cudaMemcpyHostToDevice, c->stream));
  return GBSMPS_OK;
}

// The front of one build on context cf: validation, the GSVD chain, the kept
// bases and maps.  Nothing here waits on the host (the bond sizes are read
// back by build_rest: a copy into pageable memory would block until the
// chain is done).  Only Gamma is read on the device; the state lives in fs.
int build_front(gbsmps_ctx* cf, int N, const double* dgamma, const gbsmps_opts* o, FrontState* fs) {
  cudaStream_t s = cf->stream;
  StageTimer tm(s);
  {
    const char* dbg = getenv("GBSMPS_DEBUG");
    if (dbg && dbg[0] == '1') tm.dbg_status = cf->d_status;
  }
  fs->M.reset(new gbsmps_mps());
  fs->opts = *o;
  fs->cf = cf;
  gbsmps_mps* M = fs->M.get();
  int rc = alloc_front(M, cf, N, o, &fs->f);
  if (rc) return rc;
  // a1 validation, a2-a3 GSVD chain
  rc = launch_checks(cf, M, dgamma, o, fs->f);
  if (rc) return rc;
  tm.mark("validate");
  CK(launch_gsvd_chain(dgamma, N, fs->f.dbw, o->lambda2_freeze, fs->f.Gs, M->ba, M->Qm, M->cm,
                       cf->d_status, s));
  COUNT_LAUNCH(1);
  tm.mark("gsvd_chain");
  // a4-a5 kept bases and index maps
  rc = launch_bases(cf, M, o);
  if (rc) return rc;
  tm.mark("basis_maps");
  return GBSMPS_OK;
}

// The rest of the build on context c, once its front has finished, in three
// parts that the stream entry point schedules around the sampling of the
// previous state.  (a) the bond read-back (the host waits for the front's
// stream and status word), the tensors and the PCO build: long FP64 CTAs.
// gate (may be null): c's stream waits for it first.
int rest_pco(gbsmps_ctx* c, FrontState* fs, cudaEvent_t gate) {
  cudaStream_t s = c->stream;
  gbsmps_mps* M = fs->M.get();
  int rc = enqueue_readback(M, &fs->rb, fs->cf->stream);
  if (!rc) rc = sync_status(fs->cf);
  if (rc) return rc;
  finish_readback(M, fs->rb);
  M->ctx = c;
  StageTimer tm(s);
  if (gate) CK(cudaStreamWaitEvent(s, gate, 0));
  // a6 PCO build
  size_t scr_max = 0;
  rc = alloc_tensors(M, s, &scr_max);
  if (rc) return rc;
  std::vector<SiteTask> tasks;
  site_tasks(M, fs->rb.cm, tasks);
  rc = run_pco(c, tasks, scr_max, fs->opts.d, fs->opts.precision);
  if (rc) return rc;
  tm.mark("pco");
  return GBSMPS_OK;
}

// (b) the energy gauge, the environments and the normalisation: short CTAs
// only, so this part may run beside the sampling of another state
int rest_env(gbsmps_ctx* c, FrontState* fs) {
  gbsmps_mps* M = fs->M.get();
  StageTimer tm(c->stream);
  int rc = env_single(c, M, tm);
  if (rc) return rc;
  tm.mark("environments");
  rc = normalise_single(c, M);
  if (rc) return rc;
  tm.mark("normalise");
  return GBSMPS_OK;
}

// (c) the sampler's right-canonical form (factors of the diagonal blocks,
// one CTA per block, then the transforms and planes), then the host waits
// for c's stream and hands the MPS over.  gate (may be null): c's stream
// waits for it first.
int rest_canon(gbsmps_ctx* c, FrontState* fs, cudaEvent_t gate, gbsmps_mps_t* out) {
  cudaStream_t s = c->stream;
  gbsmps_mps* M = fs->M.get();
  StageTimer tm(s);
  if (gate) CK(cudaStreamWaitEvent(s, gate, 0));
  int rc = GBSMPS_OK;
  if (fs->opts.precision == GBSMPS_PREC_MIXED) {
    CanonWork w;
    rc = canon_prepare(M, &w, s);
    if (!rc) rc = canon_bonds(c, M, &w, 1, M->N - 1, s);
    if (rc) return rc;
    canon_report(M, &w, tm, s);
    tm.mark("cholesky");
    rc = canon_sites_grouped(M, &w, s);
    if (rc) return rc;
    tm.mark("canonical_pack");
  }
  rc = finish(c, M);
  if (rc) return rc;
  rc = sync_status(c);
  if (rc) return rc;
  *out = fs->M.release();
  return GBSMPS_OK;
}

int build_rest(gbsmps_ctx* c, FrontState* fs, cudaEvent_t gate, gbsmps_mps_t* out) {
  int rc = rest_pco(c, fs, gate);
  if (!rc) rc = rest_env(c, fs);
  if (!rc) rc = rest_canon(c, fs, nullptr, out);
  return rc;
}

// the whole pipeline for one state whose covariance is on the device
int build_single(gbsmps_ctx* c, int N, const double* dgamma, const gbsmps_opts* o,
                 gbsmps_mps_t* out, cudaEvent_t gate) {
  FrontState fs;
  int rc = build_front(c, N, dgamma, o, &fs);
  if (rc) return rc;
  return build_rest(c, &fs, gate, out);
}

}  // namespace gbs
