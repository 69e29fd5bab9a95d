// C ABI of gbsmps (include/gbsmps.h): argument checks, device buffers and the
// launch order of the build / amplitude / sampling pipelines.  All numerics run
// in the kernels of k_gsvd.cu, k_basis.cu, k_pco.cu and k_mps.cu.
#include "objects.h"
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <array>
#include <memory>
#include <string>
#include <vector>

std::atomic<unsigned long long> g_kernel_launches{0};
KernelTrace g_tc_trace;
KernelTrace g_env_trace;
KernelTrace g_pco_trace;

thread_local std::string g_detail;

extern "C" {

int gbsmps_opts_default(gbsmps_opts* o) {
  if (!o) return fail(GBSMPS_ERR_ARG, "opts is NULL");
  o->d = 4; o->chi_max = 64; o->eps_trunc = 0.0; o->lambda2_freeze = 1e-13;
  o->precision = GBSMPS_PREC_FP64; o->validate = 1; o->purity_tol = 1e-9;
  return GBSMPS_OK;
}

int gbsmps_create(int device, void* stream, gbsmps_ctx_t* out) {
  if (!out) return fail(GBSMPS_ERR_ARG, "out is NULL");
  int n = 0;
  CK(cudaGetDeviceCount(&n));
  if (device < 0 || device >= n) return fail(GBSMPS_ERR_ARG, "bad device index");
  CK(cudaSetDevice(device));
  auto* c = new gbsmps_ctx();
  c->device = device;
  c->stream = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMalloc(&c->d_status, sizeof(int));
  if (e) { delete c; return fail(GBSMPS_ERR_CUDA, cudaGetErrorString(e)); }
  e = cudaMemset(c->d_status, 0, sizeof(int));
  if (e) { cudaFree(c->d_status); delete c; return fail(GBSMPS_ERR_CUDA, cudaGetErrorString(e)); }
  c->launches_at_create = g_kernel_launches.load();
  *out = c;
  return GBSMPS_OK;
}

int gbsmps_destroy(gbsmps_ctx_t c) {
  if (!c) return fail(GBSMPS_ERR_ARG, "ctx is NULL");
  cudaStreamSynchronize(c->stream);
  cudaFree(c->d_status);
  delete c;
  return GBSMPS_OK;
}

int gbsmps_build_from_cov(gbsmps_ctx_t c, int32_t N, const double* gamma, int mem_kind,
                          const gbsmps_opts* o, gbsmps_mps_t* out) {
  if (!c || !gamma || !out) return fail(GBSMPS_ERR_ARG, "NULL argument");
  if (N < 1 || N > 1000000) return fail(GBSMPS_ERR_ARG, "N out of range");
  if (mem_kind != GBSMPS_MEM_HOST && mem_kind != GBSMPS_MEM_DEVICE) return fail(GBSMPS_ERR_ARG, "mem_kind");
  int rc = check_opts(o);
  if (rc) return rc;
  CK(cudaSetDevice(c->device));
  const size_t bytes = sizeof(double) * 4 * (size_t)N * N;
  DevBuf g;
  const double* dg = gamma;
  if (mem_kind == GBSMPS_MEM_HOST) {
    CK(g.alloc(bytes, c->stream));
    CK(cudaMemcpyAsync(g.p, gamma, bytes, cudaMemcpyHostToDevice, c->stream));
    dg = g.as<double>();
  }
  rc = gbs::build_single(c, N, dg, o, out);
  g.release();
  return rc;
}

int gbsmps_build_from_Q(gbsmps_ctx_t c, int32_t N, const double* Q, int mem_kind,
                        const gbsmps_opts* o, gbsmps_mps_t* out) {
  if (!c || !Q || !out) return fail(GBSMPS_ERR_ARG, "NULL argument");
  if (N < 1 || N > 65536) return fail(GBSMPS_ERR_ARG, "N out of range");
  if (mem_kind != GBSMPS_MEM_HOST && mem_kind != GBSMPS_MEM_DEVICE) return fail(GBSMPS_ERR_ARG, "mem_kind");
  int rc = check_opts(o);
  if (rc) return rc;
  CK(cudaSetDevice(c->device));
  cudaStream_t s = c->stream;
  const size_t qbytes = sizeof(double2) * (size_t)N * N;
  DevBuf qb, gb, wb;
  const double2* dq = reinterpret_cast<const double2*>(Q);
  if (mem_kind == GBSMPS_MEM_HOST) {
    CK(qb.alloc(qbytes, s));
    CK(cudaMemcpyAsync(qb.p, Q, qbytes, cudaMemcpyHostToDevice, s));
    dq = qb.as<double2>();
  }
  CK(gb.alloc(sizeof(double) * 4 * (size_t)N * N, s));
  CK(wb.alloc(qbytes + sizeof(double2) * 2 * (size_t)N, s));
  CK(launch_q_to_gamma(dq, N, gb.as<double>(), wb.as<double2>(), c->d_status, s));
  COUNT_LAUNCH(2 + 2 * (unsigned long long)N);
  rc = sync_status(c);
  if (rc == GBSMPS_OK) rc = gbs::build_single(c, N, gb.as<double>(), o, out);
  qb.release(); gb.release(); wb.release();
  return rc;
}

int gbsmps_info(gbsmps_mps_t m, int32_t* N_out, int32_t* d_out, int32_t* bond_dims,
                int32_t* n_e, double* eps_m) {
  if (!m) return fail(GBSMPS_ERR_ARG, "mps is NULL");
  if (N_out) *N_out = m->N;
  if (d_out) *d_out = m->d;
  if (bond_dims) for (int i = 0; i <= m->N; ++i) bond_dims[i] = m->D[i];
  if (n_e) for (int i = 1; i < m->N; ++i) n_e[i - 1] = m->ne[i];
  if (eps_m) for (int i = 0; i + 1 < m->N; ++i) eps_m[i] = m->eps[i];
  return GBSMPS_OK;
}

int gbsmps_get_tensor(gbsmps_mps_t m, int32_t site, void* dst, size_t dst_bytes, int mem_kind) {
  if (!m || !dst) return fail(GBSMPS_ERR_ARG, "NULL argument");
  if (m->host_bpack) return fail(GBSMPS_ERR_STATE, "the MPS is offloaded: only sampling remains");
  if (site < 0 || site >= m->N) return fail(GBSMPS_ERR_ARG, "site out of range");
  size_t bytes = sizeof(double2) * (size_t)m->D[site] * m->d * m->D[site + 1];
  if (dst_bytes < bytes) return fail(GBSMPS_ERR_ARG, "dst too small");
  CK(cudaSetDevice(m->ctx->device));
  CK(cudaMemcpyAsync(dst, m->tensors.as<double2>() + m->toff[site], bytes,
                     mem_kind == GBSMPS_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                     m->ctx->stream));
  if (mem_kind == GBSMPS_MEM_HOST) CK(cudaStreamSynchronize(m->ctx->stream));
  return GBSMPS_OK;
}

int gbsmps_get_gsvd(gbsmps_mps_t m, double* lam2, double* Qm, double* c_m) {
  if (!m) return fail(GBSMPS_ERR_ARG, "mps is NULL");
  CK(cudaSetDevice(m->ctx->device));
  cudaStream_t s = m->ctx->stream;
  if (lam2 && m->N > 1)
    CK(cudaMemcpyAsync(lam2, m->lam2 + NEM, sizeof(double) * NEM * (size_t)(m->N - 1),
                       cudaMemcpyDeviceToHost, s));
  if (Qm) CK(cudaMemcpyAsync(Qm, m->Qm, sizeof(double2) * (size_t)m->N * QS * QS, cudaMemcpyDeviceToHost, s));
  if (c_m) CK(cudaMemcpyAsync(c_m, m->cm, sizeof(double) * m->N, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return GBSMPS_OK;
}

int gbsmps_get_basis(gbsmps_mps_t m, int32_t bond, uint8_t* occ, double* E) {
  if (!m) return fail(GBSMPS_ERR_ARG, "mps is NULL");
  if (bond < 0 || bond > m->N) return fail(GBSMPS_ERR_ARG, "bond out of range");
  CK(cudaSetDevice(m->ctx->device));
  cudaStream_t s = m->ctx->stream;
  const int D = m->D[bond];
  const int ne = (bond == 0 || bond == m->N) ? 0 : m->ne[bond];
  const size_t cap = (size_t)m->ba.cap;
  std::vector<uint8_t> rows((size_t)D * NEM);
  if (occ && ne > 0)
    CK(cudaMemcpyAsync(rows.data(), m->ba.occ + (size_t)bond * cap * NEM, rows.size(),
                       cudaMemcpyDeviceToHost, s));
  if (E) CK(cudaMemcpyAsync(E, m->ba.E + (size_t)bond * cap, sizeof(double) * D,
                            cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (occ)
    for (int j = 0; j < D; ++j)
      for (int q = 0; q < ne; ++q) occ[(size_t)j * ne + q] = rows[(size_t)j * NEM + q];
  return GBSMPS_OK;
}

int gbsmps_amplitudes(gbsmps_mps_t m, int64_t P, const uint8_t* patterns, double* out, int mem_kind) {
  if (!m) return fail(GBSMPS_ERR_ARG, "mps is NULL");
  if (P < 0) return fail(GBSMPS_ERR_ARG, "P < 0");
  if (P == 0) return GBSMPS_OK;
  if (!patterns || !out) return fail(GBSMPS_ERR_ARG, "NULL argument");
  if (m->host_bpack) return fail(GBSMPS_ERR_STATE, "the MPS is offloaded: only sampling remains");
  CK(cudaSetDevice(m->ctx->device));
  cudaStream_t s = m->ctx->stream;
  DevBuf pb, ob, wb;
  const uint8_t* dp = patterns;
  double2* dout = reinterpret_cast<double2*>(out);
  if (mem_kind == GBSMPS_MEM_HOST) {
    CK(pb.alloc((size_t)P * m->N, s));
    CK(cudaMemcpyAsync(pb.p, patterns, (size_t)P * m->N, cudaMemcpyHostToDevice, s));
    dp = pb.as<uint8_t>();
    CK(ob.alloc(sizeof(double2) * P, s));
    dout = ob.as<double2>();
  }
  CK(wb.alloc(sizeof(double2) * 2 * (size_t)P * m->maxD, s));
  ChainView cv{m->N, m->d, m->D.data(), m->toff.data(), m->tensors.as<double2>()};
  CK(launch_amplitudes(cv, P, dp, dout, wb.as<double2>(), m->maxD, s));
  COUNT_LAUNCH(2 + m->N);
  if (mem_kind == GBSMPS_MEM_HOST)
    CK(cudaMemcpyAsync(out, dout, sizeof(double2) * P, cudaMemcpyDeviceToHost, s));
  pb.release(); ob.release(); wb.release();
  if (mem_kind == GBSMPS_MEM_HOST) return sync_status(m->ctx);
  return GBSMPS_OK;
}

}  // extern "C"

namespace gbs {
// Sampling of a built MPS on stream s; device errors go to status.  sm_reserve
// SMs are left free of the tensor-core GEMM's persistent CTAs (another
// stream's single-SM chain kernel runs there).  With sync_host = 0 a host
// output is copied asynchronously and the caller synchronises s.
int sample_impl(gbsmps_mps* m, cudaStream_t s, int* status, int sm_reserve, int sync_host,
                int64_t S, uint64_t seed, uint64_t counter0, const double* uniforms, uint8_t* out,
                uint8_t* flags, int mem_kind) {
  if (!m) return fail(GBSMPS_ERR_ARG, "mps is NULL");
  if (S < 0) return fail(GBSMPS_ERR_ARG, "S < 0");
  if (S == 0) return GBSMPS_OK;
  if (!out) return fail(GBSMPS_ERR_ARG, "out is NULL");
  if (S > (int64_t)1 << 31) return fail(GBSMPS_ERR_ARG, "S too large for one call");
  CK(cudaSetDevice(m->ctx->device));
  const int N = m->N, d = m->d;
  // samples are processed in chunks that bound the W/Y work buffers
  const size_t per = (size_t)d * m->maxD;
  int64_t chunk;
  if (m->precision == GBSMPS_PREC_MIXED) {
    // per sample: four state planes (two fp16 planes of up to Kp halves each),
    // six index lists, two scales, and per parity group a row of W and its
    // chunk norms; up to 32 GB of them per chunk (a chunk re-runs every site;
    // an offloaded MPS streams its planes once per chunk, so it takes the
    // largest chunks)
    int Kpm = 64, Npm = 128;
    for (int i = 0; i < N; ++i)
      for (int pi = 0; pi < 2; ++pi) {
        Kpm = std::max(Kpm, m->sg[i].Kp[pi]);
        Npm = std::max(Npm, m->sg[i].Np[pi]);
      }
    const double ps = 2.0 * 2.0 * 4.0 * Kpm + 4.0 * 6.0 + 4.0 * 2.0 + 2.0 * (4.0 * Npm + 4.0 * (Npm / 32));
    chunk = std::max<int64_t>(1, std::min<int64_t>(S, (int64_t)(32.0 * (double)(1ll << 30) / ps)));
    if (!m->host_bpack) {
      // resident MPS: balanced chunks of at most ~576 MB of state planes
      // (16 Kp bytes per sample); measured on GB300: one chunk for 100k
      // samples of the 144-mode state (Kp = 320: 18.3 ms; 23.0 ms in two),
      // ~50k for the 1024-mode state (Kp = 640, 1M samples: 2.83 s; 4.14 s
      // in one chunk, whose gathered rows and scattered next-state writes
      // miss L2)
      const double planes = 16.0 * Kpm;
      const int64_t nch = std::max<int64_t>(1, (int64_t)std::ceil((double)S * planes / (576.0 * (1 << 20))));
      chunk = std::min<int64_t>(chunk, (S + nch - 1) / nch);
    }
  } else {
    chunk = std::max<int64_t>(1, std::min<int64_t>(S, (int64_t)((size_t)6 << 30) / (int64_t)(sizeof(double2) * 2 * per + 32 * m->maxD)));
  }
  // GBSMPS_SAMPLE_CHUNK caps the samples per chunk (the patterns do not
  // depend on it: every sample's arithmetic is its own)
  if (const char* ce = getenv("GBSMPS_SAMPLE_CHUNK")) {
    const long long cap = atoll(ce);
    if (cap > 0) chunk = std::min<int64_t>(chunk, cap);
  }
  DevBuf ub, obuf, fbuf, vb, wb, yb;
  if (m->precision != GBSMPS_PREC_MIXED) {
    CK(vb.alloc(sizeof(double2) * 2 * (size_t)chunk * m->maxD, s));
    CK(wb.alloc(sizeof(double2) * (size_t)chunk * per, s));
    CK(yb.alloc(sizeof(double2) * (size_t)chunk * per, s));
  }
  const double* du = uniforms;
  uint8_t* dout = out;
  uint8_t* dfl = flags;
  if (mem_kind == GBSMPS_MEM_HOST) {
    if (uniforms) {
      CK(ub.alloc(sizeof(double) * (size_t)S * N, s));
      CK(cudaMemcpyAsync(ub.p, uniforms, sizeof(double) * (size_t)S * N, cudaMemcpyHostToDevice, s));
      du = ub.as<double>();
    }
    CK(obuf.alloc((size_t)S * N, s));
    dout = obuf.as<uint8_t>();
    if (flags) { CK(fbuf.alloc((size_t)S, s)); dfl = fbuf.as<uint8_t>(); }
  }
  if (dfl) CK(cudaMemsetAsync(dfl, 0, (size_t)S, s));
  const double2* R = m->env.as<double2>();
  const double2 one = cmk(1, 0), zero = cmk(0, 0);
  StageTimer tm(s);
  // mixed path: per parity class the fp16 state planes of the current and
  // the next bond (row s = sample s), the class lists of sample indices
  // (current, next, rest), the per-sample scales (current, next), W and the
  // chunk norms per group; list counts per bond
  DevBuf cv[4], csid[6], crs[2], cw[2], cpart[2], ccnt, crest, ring;
  const char* tce = getenv("GBSMPS_TC");
  const int use_tc = !(tce && tce[0] == '0');
  // the p = 0 pre-pass (on unless GBSMPS_P0PASS=0): block 0 of every sample
  // first, the full product only for the samples it cannot decide
  const char* p0e = getenv("GBSMPS_P0PASS");
  const bool p0pass = !(p0e && p0e[0] == '0') && d > 1;
  std::vector<int> hrest;
  std::vector<int> hcnt;                  // group row counts, read back for the trace
  for (int64_t s0 = 0; s0 < S; s0 += chunk) {
    const int cs = (int)std::min<int64_t>(chunk, S - s0);
    if (m->precision == GBSMPS_PREC_MIXED) {
      // right-canonical tensors: per site a two-group tensor-core GEMM over
      // the class lists (block 0 first with the pre-pass), q_p = |w_p|^2 from
      // the chunk norms, each sample appended to the list of its next class
      const int Spad = (int)((chunk + 127) / 128 * 128);
      int Kpmax = 64, Npmax = 128;
      for (int i = 0; i < N; ++i)
        for (int pi = 0; pi < 2; ++pi) {
          Kpmax = std::max(Kpmax, m->sg[i].Kp[pi]);
          Npmax = std::max(Npmax, m->sg[i].Np[pi]);
        }
      if (!ccnt.p) {
        for (int k = 0; k < 4; ++k) CK(cv[k].alloc(sizeof(__half) * 2 * (size_t)Spad * Kpmax, s));
        for (int k = 0; k < 6; ++k) CK(csid[k].alloc(sizeof(int) * (size_t)Spad, s));
        for (int k = 0; k < 2; ++k) {
          CK(crs[k].alloc(sizeof(float) * (size_t)Spad, s));
          CK(cw[k].alloc(sizeof(float) * (size_t)chunk * Npmax, s));
          CK(cpart[k].alloc(sizeof(float) * (size_t)chunk * (Npmax / 32), s));
        }
        CK(ccnt.alloc(sizeof(int) * 2 * (size_t)(N + 1), s));
        CK(crest.alloc(sizeof(int) * 2 * (size_t)(N + 1), s));
      }
      // out of core: the planes of sites m and m + 1 are copied ahead, each
      // copy waiting until the GEMMs of the site that used its slot before
      // are done (a ring of three slots)
      const bool ooc = m->host_bpack != nullptr;
      long long slot_h = 0;
      if (ooc) {
        for (int i = 0; i < N; ++i) slot_h = std::max(slot_h, m->site_halves(i));
        if (!ring.p) CK(ring.alloc(sizeof(__half) * (size_t)(gbsmps_mps::RING * slot_h + 64), s));
        CK(cudaEventRecord(m->ring_start, s));          // earlier readers of the ring
        CK(cudaStreamWaitEvent(m->copy_stream, m->ring_start, 0));
      }
      auto issue_copy = [&](int site) -> int {
        const int k = site % gbsmps_mps::RING;
        CK(cudaStreamWaitEvent(m->copy_stream, m->ring_free[k], 0));
        CK(cudaMemcpyAsync(ring.as<__half>() + k * slot_h, m->host_bpack + m->sg[site].boff[0],
                           sizeof(__half) * (size_t)m->site_halves(site), cudaMemcpyHostToDevice,
                           m->copy_stream));
        CK(cudaEventRecord(m->ring_ready[k], m->copy_stream));
        return GBSMPS_OK;
      };
      if (ooc) {
        for (int i = 0; i < std::min(N, gbsmps_mps::RING - 1); ++i) {
          const int rc0 = issue_copy(i);
          if (rc0) return rc0;
        }
      }
      int* cnt = ccnt.as<int>();
      int* rcnt = crest.as<int>();
      CK(cudaMemsetAsync(cnt, 0, sizeof(int) * 2 * (size_t)(N + 1), s));
      CK(cudaMemsetAsync(rcnt, 0, sizeof(int) * 2 * (size_t)(N + 1), s));
      int cur[2] = {0, 1}, nxt[2] = {2, 3};   // planes
      int lc[2] = {0, 1}, ln[2] = {2, 3};     // lists
      int rc = 0, rn = 1;                     // scales
      CK(launch_sampler_init(cv[cur[0]].as<__half>(), (long long)Spad * m->sg[0].Kp[0], Spad,
                             m->sg[0].Kp[0], csid[lc[0]].as<int>(), crs[rc].as<float>(), cnt, cs, s));
      COUNT_LAUNCH(1);
      for (int site = 0; site < N; ++site) {
        const gbsmps_mps::SiteGroups& G = m->sg[site];
        TcGroup tg[2];
        SelGroup sl[2];
        NextGroup ng[2];
        for (int pi = 0; pi < 2; ++pi) {
          const int Kpn = site + 1 < N ? m->sg[site + 1].Kp[pi] : 64;
          tg[pi] = TcGroup{G.Kp[pi] / 64, G.Np[pi] / 128, cnt + 2 * site + pi, cs,
                           csid[lc[pi]].as<int>(), cv[cur[pi]].as<__half>(), (long long)Spad * G.Kp[pi],
                           crs[rc].as<float>(), cw[pi].as<float>(), (long long)G.Np[pi],
                           cpart[pi].as<float>(), (long long)(G.Np[pi] / 32), nullptr, 0, 0, 0};
          sl[pi] = SelGroup{cnt + 2 * site + pi, csid[lc[pi]].as<int>(), cw[pi].as<float2>(),
                            (long long)(G.Np[pi] / 2), cpart[pi].as<float>(),
                            (long long)(G.Np[pi] / 32), G.w[pi], G.w[pi ^ 1]};
          ng[pi] = NextGroup{cv[nxt[pi]].as<__half>(), (long long)Spad * Kpn, Kpn,
                             csid[ln[pi]].as<int>(), m->pcnt[2 * (site + 1) + pi], crs[rn].as<float>()};
        }
        const __half* B0;
        const __half* B1;
        const unsigned char* map0 = G.map[0].data();
        const unsigned char* map1 = G.map[1].data();
        alignas(64) unsigned char rmap[2][128];
        if (ooc) {
          if (site + gbsmps_mps::RING - 1 < N) {
            const int rc0 = issue_copy(site + gbsmps_mps::RING - 1);
            if (rc0) return rc0;
          }
          CK(cudaStreamWaitEvent(s, m->ring_ready[site % gbsmps_mps::RING], 0));
          B0 = ring.as<__half>() + (site % gbsmps_mps::RING) * slot_h;
          B1 = B0 + 2LL * G.Np[0] * G.Kp[0];
          if (canon_make_map(rmap[0], B0, G.Kp[0], G.Np[0]) || canon_make_map(rmap[1], B1, G.Kp[1], G.Np[1]))
            return fail(GBSMPS_ERR_CUDA, "tensor map encoding failed for a ring slot");
          map0 = rmap[0];
          map1 = rmap[1];
        } else {
          B0 = m->bpack.as<__half>() + G.boff[0];
          B1 = m->bpack.as<__half>() + G.boff[1];
        }
        const long long bpl0 = (long long)G.Np[0] * G.Kp[0], bpl1 = (long long)G.Np[1] * G.Kp[1];
        const double* uu = du ? du + (size_t)s0 * N : nullptr;
        if (p0pass) {
          // block 0 only (the first column tiles of each group's planes),
          // written as the next state of the same class
          TcGroup ta[2] = {tg[0], tg[1]};
          RestGroup rg[2];
          for (int pi = 0; pi < 2; ++pi) {
            ta[pi].ntn = std::min(G.Np[pi] / 128, (2 * G.w[pi] + 127) / 128);
            ta[pi].W = nullptr;
            ta[pi].Vn = ng[pi].V;
            ta[pi].vnpl = ng[pi].vpl;
            ta[pi].Kpn = ng[pi].Kp;
            ta[pi].wv = 2 * G.w[pi];
            rg[pi] = RestGroup{csid[4 + pi].as<int>(), rcnt + 2 * site + pi};
          }
          CK(launch_canon_gemm(map0, map1, ta[0], ta[1], B0, bpl0, B1, bpl1,
                               use_tc, status, sm_reserve, s));
          CK(launch_select_pre(cs, sl[0], sl[1], ng[0], ng[1], cnt + 2 * (site + 1), rg[0], rg[1],
                               m->creg.as<unsigned long long>(), 1e-10, uu, N, site, seed,
                               counter0 + (uint64_t)s0, dout + (size_t)s0 * N, N, 1e-5, s));
          COUNT_LAUNCH(1);
          // the full product and selection for the rest
          TcGroup tb[2] = {tg[0], tg[1]};
          SelGroup sb[2] = {sl[0], sl[1]};
          for (int pi = 0; pi < 2; ++pi) {
            tb[pi].cnt = rcnt + 2 * site + pi;
            tb[pi].rows = csid[4 + pi].as<int>();
            sb[pi].cnt = rcnt + 2 * site + pi;
            sb[pi].sid = csid[4 + pi].as<int>();
          }
          CK(launch_canon_gemm(map0, map1, tb[0], tb[1], B0, bpl0, B1, bpl1,
                               use_tc, status, sm_reserve, s));
          if (ooc) CK(cudaEventRecord(m->ring_free[site % gbsmps_mps::RING], s));
          CK(launch_select_groups(cs, d, sb[0], sb[1], ng[0], ng[1], cnt + 2 * (site + 1), uu, N,
                                  site, seed, counter0 + (uint64_t)s0, dout + (size_t)s0 * N, N,
                                  dfl ? dfl + s0 : nullptr, 1e-5, s));
          COUNT_LAUNCH(1);
        } else {
          CK(launch_canon_gemm(map0, map1, tg[0], tg[1], B0, bpl0, B1, bpl1,
                               use_tc, status, sm_reserve, s));
          if (ooc) CK(cudaEventRecord(m->ring_free[site % gbsmps_mps::RING], s));
          CK(launch_select_groups(cs, d, sl[0], sl[1], ng[0], ng[1], cnt + 2 * (site + 1), uu, N,
                                  site, seed, counter0 + (uint64_t)s0, dout + (size_t)s0 * N, N,
                                  dfl ? dfl + s0 : nullptr, 1e-5, s));
          COUNT_LAUNCH(1);
        }
        std::swap(cur, nxt);
        std::swap(lc, ln);
        std::swap(rc, rn);
      }
      if (g_tc_trace.on.load()) {
        // algorithmic work of the GEMMs: 8 real flops per complex product of a
        // sample's class-pi state with the nonzero blocks of At
        // (with the pre-pass: block 0 of every sample, all blocks of the rest)
        hcnt.assign(2 * (N + 1), 0);
        hrest.assign(2 * (N + 1), 0);
        CK(cudaMemcpyAsync(hcnt.data(), cnt, sizeof(int) * 2 * (N + 1), cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(hrest.data(), rcnt, sizeof(int) * 2 * (N + 1), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        // bytes: the gathered state rows (two fp16 planes), the packed
        // tensor's planes, and the outputs (the next state's planes for the
        // pre-pass, FP32 rows of W otherwise) with their chunk norms
        double f = 0.0, by = 0.0;
        for (int site = 0; site < N; ++site)
          for (int pi = 0; pi < 2; ++pi) {
            const gbsmps_mps::SiteGroups& G = m->sg[site];
            double cols = 0.0;
            for (int p = 0; p < d; ++p) cols += m->pcnt[2 * (site + 1) + (pi ^ (p & 1))];
            const double kl = m->pcnt[2 * site + pi];
            const double rows = hcnt[2 * site + pi], rest = hrest[2 * site + pi];
            const double Kp = G.Kp[pi], Np = G.Np[pi];
            if (p0pass) {
              const double Np0 = 128.0 * std::min(G.Np[pi] / 128, (2 * G.w[pi] + 127) / 128);
              const double Kpn = site + 1 < N ? m->sg[site + 1].Kp[pi] : 64;
              f += 8.0 * kl * (rows * (double)m->pcnt[2 * (site + 1) + pi] + rest * cols);
              by += rows * (4.0 * Kp + 4.0 * Kpn + Np0 / 8.0) + 4.0 * Np0 * Kp;
              by += rest * (4.0 * Kp + 4.0 * Np + Np / 8.0) + (rest > 0 ? 4.0 * Np * Kp : 0.0);
            } else {
              f += 8.0 * rows * kl * cols;
              by += rows * (4.0 * Kp + 4.0 * Np + Np / 8.0) + 4.0 * Np * Kp;
            }
          }
        g_tc_trace.add_work(f, by);
      }
      continue;
    }
    double2* V = vb.as<double2>();
    double2* Vn = V + (size_t)chunk * m->maxD;
    // v = [1] for every sample (D_0 = 1)
    CK(launch_init_ones(V, cs, 1, s));
    COUNT_LAUNCH(1);
    for (int site = 0; site < N; ++site) {
      const int Dl = m->D[site], Dr = m->D[site + 1];
      const double2* A = m->tensors.as<double2>() + m->toff[site];
      double2* W = wb.as<double2>();
      double2* Y = yb.as<double2>();
      CK(launch_zgemm('N', 'N', cs, d * Dr, Dl, one, V, Dl, 0, A, d * Dr, 0, zero, W, d * Dr, 0, 1, s));
      CK(launch_zgemm('N', 'N', cs * d, Dr, Dr, one, W, Dr, 0, R + m->eoff[site + 1], Dr, 0, zero, Y,
                      Dr, 0, 1, s));
      CK(launch_sample_select(cs, d, Dr, W, Y, du ? du + (size_t)s0 * N : nullptr, N, site, seed,
                              counter0 + (uint64_t)s0, Vn, dout + (size_t)s0 * N, N,
                              dfl ? dfl + s0 : nullptr, s));
      COUNT_LAUNCH(3);
      std::swap(V, Vn);
    }
  }
  tm.mark("sample");
  if (mem_kind == GBSMPS_MEM_HOST) {
    CK(cudaMemcpyAsync(out, dout, (size_t)S * N, cudaMemcpyDeviceToHost, s));
    if (flags) CK(cudaMemcpyAsync(flags, dfl, (size_t)S, cudaMemcpyDeviceToHost, s));
  }
  ub.release(); obuf.release(); fbuf.release(); vb.release(); wb.release(); yb.release();
  for (auto& b : cv) b.release();
  for (auto& b : csid) b.release();
  for (auto& b : crs) b.release();
  for (auto& b : cw) b.release();
  for (auto& b : cpart) b.release();
  ccnt.release();
  crest.release();
  ring.release();
  if (mem_kind == GBSMPS_MEM_HOST && sync_host) return sync_status(m->ctx);
  return GBSMPS_OK;
}
}  // namespace gbs

extern "C" {

int gbsmps_sample(gbsmps_mps_t m, int64_t S, uint64_t seed, uint64_t counter0,
                  const double* uniforms, uint8_t* out, uint8_t* flags, int mem_kind) {
  if (!m) return fail(GBSMPS_ERR_ARG, "mps is NULL");
  return gbs::sample_impl(m, m->ctx->stream, m->ctx->d_status, 0, 1, S, seed, counter0, uniforms,
                          out, flags, mem_kind);
}

int gbsmps_build_sample_stream(gbsmps_ctx_t c, int32_t count, const int32_t* Ns,
                               const double* const* gammas, const gbsmps_opts* opts, int64_t S,
                               const uint64_t* seeds, const uint64_t* counter0s,
                               uint8_t* const* outs, int mem_kind) {
  // SMs the sampler's persistent GEMM leaves to the next state's chain and
  // build while it runs (a performance knob, GBSMPS_STREAM_RESERVE: the
  // patterns do not depend on it)
  const char* sre = getenv("GBSMPS_STREAM_RESERVE");
  const int stream_reserve = sre ? std::max(0, std::min(128, atoi(sre))) : 12;
  // the sampler's stream priority against the next build's (GBSMPS_STREAM_PRIO:
  // 1 = the sampler first, 0 = equal)
  const char* spe = getenv("GBSMPS_STREAM_PRIO");
  // GBSMPS_STREAM_BUILD_PRIO=1: the builds' parts run on a stream of the
  // highest priority instead of c's, and the sampler on the lowest
  const char* bpe = getenv("GBSMPS_STREAM_BUILD_PRIO");
  const bool build_hi = bpe ? atoi(bpe) != 0 : false;
  const bool sampler_hi = build_hi ? false : (spe ? atoi(spe) != 0 : true);
  if (!c) return fail(GBSMPS_ERR_ARG, "ctx is NULL");
  if (count < 0) return fail(GBSMPS_ERR_ARG, "count < 0");
  if (count == 0) return GBSMPS_OK;
  if (!Ns || !gammas || !opts || !seeds || !counter0s || !outs)
    return fail(GBSMPS_ERR_ARG, "NULL argument");
  if (mem_kind != GBSMPS_MEM_HOST && mem_kind != GBSMPS_MEM_DEVICE) return fail(GBSMPS_ERR_ARG, "mem_kind");
  if (S < 0) return fail(GBSMPS_ERR_ARG, "S < 0");
  size_t gmax = 0;
  for (int k = 0; k < count; ++k) {
    if (Ns[k] < 1 || Ns[k] > 1000000) return fail(GBSMPS_ERR_ARG, "N out of range");
    if (!gammas[k] || (S > 0 && !outs[k])) return fail(GBSMPS_ERR_ARG, "NULL gamma or out");
    const int rc = check_opts(&opts[k]);
    if (rc) return rc;
    gmax = std::max(gmax, sizeof(double) * 4 * (size_t)Ns[k] * Ns[k]);
  }
  CK(cudaSetDevice(c->device));
  // Per state the build runs in four parts: the front (validation, GSVD
  // chain on one SM, bases) on one of NF contexts of its own, launched NF - 1
  // states ahead (it has NF - 2 steps before its PCO; a 144-mode chain takes
  // about two); then on c's stream the PCO build, the environments and the
  // canonical form.  Iteration k runs PCO(k+1) alone, then the sampling of
  // state k (its own stream, high priority, own status word) beside the
  // environments and the canonical form of state k+1.  The PCO's CTAs hold
  // 47 KB of shared memory for milliseconds and would keep the sampler's
  // persistent GEMM CTAs (218 KB) off their SMs, so the PCO never overlaps a
  // sampling; every CTA of the other two parts is short, or fits on an SM
  // beside a GEMM CTA.  The chain hides behind all of it.
  int rc = GBSMPS_OK;
  auto ck = [&](cudaError_t e) {
    if (e != cudaSuccess && rc == GBSMPS_OK) rc = fail(GBSMPS_ERR_CUDA, cudaGetErrorString(e));
    return e == cudaSuccess;
  };
  // fronts run NF - 1 states ahead (GBSMPS_STREAM_AHEAD, 1 .. NFMAX - 1)
  constexpr int NFMAX = 6;
  const char* sae = getenv("GBSMPS_STREAM_AHEAD");
  const int NF = 1 + (sae ? std::max(1, std::min(NFMAX - 1, atoi(sae))) : 4);
  cudaStream_t ss = nullptr;
  cudaEvent_t pco_done = nullptr, sampled = nullptr;
  gbsmps_ctx cf[NFMAX];
  gbsmps_ctx cbx;                        // the builds' own context when build_hi
  gbsmps_ctx* cb = c;
  DevBuf st, fst, g[NFMAX];
  gbs::FrontState fs[NFMAX];
  gbsmps_mps* cur = nullptr;
  int lo = 0, hi = 0;
  bool ok = ck(cudaDeviceGetStreamPriorityRange(&lo, &hi)) &&
            ck(cudaStreamCreateWithPriority(&ss, cudaStreamNonBlocking, sampler_hi ? hi : lo)) &&
            ck(cudaEventCreateWithFlags(&pco_done, cudaEventDisableTiming)) &&
            ck(cudaEventCreateWithFlags(&sampled, cudaEventDisableTiming)) &&
            ck(st.alloc(sizeof(int), c->stream)) && ck(fst.alloc(NF * sizeof(int), c->stream)) &&
            ck(cudaMemsetAsync(st.p, 0, sizeof(int), c->stream)) &&
            ck(cudaMemsetAsync(fst.p, 0, NF * sizeof(int), c->stream));
  for (int i = 0; i < NF && ok; ++i) {
    cf[i].device = c->device;
    cf[i].d_status = fst.as<int>() + i;
    ok = ck(cudaStreamCreateWithFlags(&cf[i].stream, cudaStreamNonBlocking)) &&
         (mem_kind == GBSMPS_MEM_DEVICE || ck(g[i].alloc(gmax, c->stream)));
  }
  if (ok && build_hi) {
    cbx.device = c->device;
    cbx.d_status = c->d_status;
    ok = ck(cudaStreamCreateWithPriority(&cbx.stream, cudaStreamNonBlocking, hi));
    if (ok) cb = &cbx;
  }
  ok = ok && ck(cudaStreamSynchronize(c->stream));
  auto keep = [&](int r) {
    if (r && rc == GBSMPS_OK) rc = r;
    return r == GBSMPS_OK;
  };
  // the front of state k on context k % NF (a host Gamma is copied first)
  auto front = [&](int k) {
    gbsmps_ctx* x = &cf[k % NF];
    const double* dg = gammas[k];
    if (mem_kind == GBSMPS_MEM_HOST) {
      if (!ck(cudaMemcpyAsync(g[k % NF].p, gammas[k], sizeof(double) * 4 * (size_t)Ns[k] * Ns[k],
                              cudaMemcpyHostToDevice, x->stream)))
        return false;
      dg = g[k % NF].as<double>();
    }
    return keep(gbs::build_front(x, Ns[k], dg, &opts[k], &fs[k % NF]));
  };
  for (int i = 0; i < std::min(count, NF - 1) && ok; ++i) ok = front(i);
  // state 0 alone
  if (ok) ok = keep(gbs::rest_pco(cb, &fs[0], nullptr)) && keep(gbs::rest_env(cb, &fs[0])) &&
               keep(gbs::rest_canon(cb, &fs[0], nullptr, &cur));
  for (int k = 0; k < count && ok; ++k) {
    // state k is built; state k-1's sampling finished before it was handed over
    if (k + NF - 1 < count && !front(k + NF - 1)) break;
    // (sampling k-1 has finished: the loop waited for it)
    if (k + 1 < count && !keep(gbs::rest_pco(cb, &fs[(k + 1) % NF], nullptr))) break;
    // the sampling starts after PCO(k+1): no long CTA beside the sampler
    if (!ck(cudaEventRecord(pco_done, cb->stream)) || !ck(cudaStreamWaitEvent(ss, pco_done, 0))) break;
    if (!keep(gbs::sample_impl(cur, ss, st.as<int>(), k + 1 < count ? stream_reserve : 0, 0, S, seeds[k],
                               counter0s[k], nullptr, outs[k], nullptr, mem_kind)))
      break;
    if (!ck(cudaEventRecord(sampled, ss))) break;
    gbsmps_mps_t next = nullptr;
    if (k + 1 < count) {
      // beside sampling k: every CTA of these parts fits on an SM next to a
      // sampler GEMM CTA, or is short
      if (!keep(gbs::rest_env(cb, &fs[(k + 1) % NF]))) break;
      if (!keep(gbs::rest_canon(cb, &fs[(k + 1) % NF], nullptr, &next))) break;
    }
    // state k's MPS is freed once its sampling is done
    if (!ck(cudaStreamSynchronize(ss))) break;
    delete cur;
    cur = next;
  }
  if (ss) ck(cudaStreamSynchronize(ss));
  if (cbx.stream) ck(cudaStreamSynchronize(cbx.stream));
  for (int i = 0; i < NF; ++i)
    if (cf[i].stream) ck(cudaStreamSynchronize(cf[i].stream));
  delete cur;
  for (auto& f : fs) f.M.reset();
  int hst[1 + NFMAX] = {0};
  if (st.p) ck(cudaMemcpyAsync(hst, st.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  if (fst.p) ck(cudaMemcpyAsync(hst + 1, fst.p, NF * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  ck(cudaStreamSynchronize(c->stream));
  for (int i = 0; i < 1 + NF; ++i)
    if (hst[i] && rc == GBSMPS_OK) rc = fail(status_to_code(hst[i]), "device status word " + std::to_string(hst[i]));
  st.release();
  fst.release();
  for (auto& b : g) b.release();
  ck(cudaStreamSynchronize(c->stream));
  for (int i = 0; i < NF; ++i)
    if (cf[i].stream) { cudaStreamDestroy(cf[i].stream); cf[i].stream = nullptr; }
  if (cbx.stream) { cudaStreamDestroy(cbx.stream); cbx.stream = nullptr; }
  if (sampled) cudaEventDestroy(sampled);
  if (pco_done) cudaEventDestroy(pco_done);
  if (ss) cudaStreamDestroy(ss);
  return rc;
}

int gbsmps_filter(gbsmps_ctx_t c, int32_t count, int32_t N, const double* gamma_th, double alpha,
                  double eps, int32_t max_iter, double* S_out, int32_t* iters, double* loss,
                  int mem_kind) {
  if (!c) return fail(GBSMPS_ERR_ARG, "ctx is NULL");
  if (count < 0) return fail(GBSMPS_ERR_ARG, "count < 0");
  if (count == 0) return GBSMPS_OK;
  if (!gamma_th || !S_out) return fail(GBSMPS_ERR_ARG, "NULL argument");
  if (N < 1 || N > GBSMPS_FILTER_MAX_N) return fail(GBSMPS_ERR_BOUNDS, "N out of range [1, 64]");
  if (!(alpha > 0.0) || !(eps >= 0.0) || max_iter < 0) return fail(GBSMPS_ERR_ARG, "bad alpha, eps or max_iter");
  if (mem_kind != GBSMPS_MEM_HOST && mem_kind != GBSMPS_MEM_DEVICE) return fail(GBSMPS_ERR_ARG, "bad mem_kind");
  CK(cudaSetDevice(c->device));
  cudaStream_t s = c->stream;
  const int n = 2 * N;
  const size_t mat = sizeof(double) * (size_t)n * n * count;
  DevBuf gb, sb, wb, ib, lb;
  const double* dg = gamma_th;
  double* ds = S_out;
  if (mem_kind == GBSMPS_MEM_HOST) {
    CK(gb.alloc(mat, s));
    CK(cudaMemcpyAsync(gb.p, gamma_th, mat, cudaMemcpyHostToDevice, s));
    dg = gb.as<double>();
    CK(sb.alloc(mat, s));
    ds = sb.as<double>();
  }
  CK(wb.alloc(mat, s));
  CK(ib.alloc(sizeof(int) * count, s));
  CK(lb.alloc(sizeof(double) * count, s));
  CK(launch_filter(count, n, dg, ds, wb.as<double>(), alpha, eps, max_iter, 64, ib.as<int>(),
                   lb.as<double>(), c->d_status, s));
  COUNT_LAUNCH(1);
  if (mem_kind == GBSMPS_MEM_HOST) CK(cudaMemcpyAsync(S_out, ds, mat, cudaMemcpyDeviceToHost, s));
  if (iters) CK(cudaMemcpyAsync(iters, ib.p, sizeof(int) * count, cudaMemcpyDeviceToHost, s));
  if (loss) CK(cudaMemcpyAsync(loss, lb.p, sizeof(double) * count, cudaMemcpyDeviceToHost, s));
  gb.release(); sb.release(); wb.release(); ib.release(); lb.release();
  return sync_status(c);
}

int gbsmps_offload(gbsmps_mps_t m, size_t* host_bytes) {
  if (!m) return fail(GBSMPS_ERR_ARG, "mps is NULL");
  if (m->precision != GBSMPS_PREC_MIXED || m->sg.empty())
    return fail(GBSMPS_ERR_ARG, "only a mixed-precision MPS samples from packed planes");
  const int N = m->N;
  const long long halves = m->sg[N - 1].boff[0] + m->site_halves(N - 1);
  if (host_bytes) *host_bytes = sizeof(__half) * (size_t)halves;
  if (m->host_bpack) return GBSMPS_OK;
  CK(cudaSetDevice(m->ctx->device));
  cudaStream_t s = m->ctx->stream;
  __half* host = nullptr;
  CK(cudaMallocHost(reinterpret_cast<void**>(&host), sizeof(__half) * (size_t)halves));
  cudaError_t e = cudaMemcpyAsync(host, m->bpack.p, sizeof(__half) * (size_t)halves,
                                  cudaMemcpyDeviceToHost, s);
  if (!e) e = cudaStreamSynchronize(s);
  if (!e) e = cudaStreamCreateWithFlags(&m->copy_stream, cudaStreamNonBlocking);
  for (int k = 0; k < gbsmps_mps::RING && !e; ++k) {
    e = cudaEventCreateWithFlags(&m->ring_ready[k], cudaEventDisableTiming);
    if (!e) e = cudaEventCreateWithFlags(&m->ring_free[k], cudaEventDisableTiming);
  }
  if (!e) e = cudaEventCreateWithFlags(&m->ring_start, cudaEventDisableTiming);
  if (e) {
    cudaFreeHost(host);
    return fail(GBSMPS_ERR_CUDA, std::string("offload: ") + cudaGetErrorString(e));
  }
  m->host_bpack = host;
  // nothing but the planes is read by the sampling: the tensors, the
  // environments and their factors leave the device
  m->bpack.release(); m->tensors.release(); m->env.release(); m->tens_mixed.release();
  m->gscale.release(); m->eoff_dev.release(); m->lchol.release(); m->linv.release();
  return sync_status(m->ctx);
}

int gbsmps_release(gbsmps_mps_t m) {
  if (!m) return fail(GBSMPS_ERR_ARG, "mps is NULL");
  cudaSetDevice(m->ctx->device);
  cudaStream_t s = m->ctx->stream;
  delete m;
  cudaStreamSynchronize(s);
  return GBSMPS_OK;
}

int gbsmps_build_site(gbsmps_ctx_t c, int32_t nl, int32_t nr, int32_t d, const double* Qm,
                      double cscale, int32_t Dl, const uint8_t* occ_l, int32_t Dr,
                      const uint8_t* occ_r, int32_t precision, double* out, int mem_kind) {
  if (!c || !Qm || !out) return fail(GBSMPS_ERR_ARG, "NULL argument");
  if (nl < 0 || nr < 0 || nl > NEM || nr > NEM) return fail(GBSMPS_ERR_ARG, "nl/nr out of range");
  if (d < 1 || d > 255 || Dl < 1 || Dr < 1 || Dl > 65536 || Dr > 65536)
    return fail(GBSMPS_ERR_ARG, "sizes out of range");
  if ((nl > 0 && !occ_l) || (nr > 0 && !occ_r)) return fail(GBSMPS_ERR_ARG, "missing occupations");
  CK(cudaSetDevice(c->device));
  cudaStream_t s = c->stream;
  const int nm = nl + 1 + nr;
  // host-side repacking of the (small) inputs into the NEM-strided layout
  std::vector<double2> q(nm * nm);
  std::vector<uint8_t> ol((size_t)Dl * NEM, 0), orr((size_t)Dr * NEM, 0);
  std::vector<uint8_t> hl((size_t)Dl * std::max(nl, 1)), hr((size_t)Dr * std::max(nr, 1));
  auto kind = mem_kind == GBSMPS_MEM_HOST ? cudaMemcpyHostToHost : cudaMemcpyDeviceToHost;
  CK(cudaMemcpyAsync(q.data(), Qm, sizeof(double2) * nm * nm, kind, s));
  if (nl) CK(cudaMemcpyAsync(hl.data(), occ_l, (size_t)Dl * nl, kind, s));
  if (nr) CK(cudaMemcpyAsync(hr.data(), occ_r, (size_t)Dr * nr, kind, s));
  CK(cudaStreamSynchronize(s));
  for (int i = 0; i < Dl; ++i) for (int k = 0; k < nl; ++k) ol[(size_t)i * NEM + k] = hl[(size_t)i * nl + k];
  for (int i = 0; i < Dr; ++i) for (int k = 0; k < nr; ++k) orr[(size_t)i * NEM + k] = hr[(size_t)i * nr + k];
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t r = off; off += (bytes + 255) & ~size_t(255); return r; };
  size_t o_q = take(sizeof(double2) * nm * nm);
  size_t o_ol = take(ol.size());
  size_t o_or = take(orr.size());
  size_t o_ll = take(sizeof(int) * (size_t)NEM * Dl);
  size_t o_lr = take(sizeof(int) * (size_t)NEM * Dr);
  size_t o_t = take(sizeof(SiteTask));
  size_t o_s = take(sizeof(double2) * pco_scratch_elems(Dl, Dr));
  size_t o_o = take(sizeof(double2) * (size_t)Dl * d * Dr);
  DevBuf buf;
  CK(buf.alloc(off, s));
  char* b = buf.as<char>();
  CK(cudaMemcpyAsync(b + o_q, q.data(), sizeof(double2) * nm * nm, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(b + o_ol, ol.data(), ol.size(), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(b + o_or, orr.data(), orr.size(), cudaMemcpyHostToDevice, s));
  CK(launch_maps_brute(reinterpret_cast<uint8_t*>(b + o_ol), Dl, nl, reinterpret_cast<int*>(b + o_ll), Dl, c->d_status, s));
  CK(launch_maps_brute(reinterpret_cast<uint8_t*>(b + o_or), Dr, nr, reinterpret_cast<int*>(b + o_lr), Dr, c->d_status, s));
  COUNT_LAUNCH(2);
  // a basis that is not closed under lowering leaves -1 in the maps: stop here
  {
    int rc0 = sync_status(c);
    if (rc0) { buf.release(); return rc0; }
  }
  SiteTask t;
  t.nl = nl; t.nr = nr; t.Dl = Dl; t.Dr = Dr;
  t.Q = reinterpret_cast<double2*>(b + o_q); t.qs = nm; t.c = cscale;
  t.occl = reinterpret_cast<uint8_t*>(b + o_ol); t.lowl = reinterpret_cast<int*>(b + o_ll); t.capl = Dl;
  t.occr = reinterpret_cast<uint8_t*>(b + o_or); t.lowr = reinterpret_cast<int*>(b + o_lr); t.capr = Dr;
  double2* dout = mem_kind == GBSMPS_MEM_DEVICE ? reinterpret_cast<double2*>(out)
                                                : reinterpret_cast<double2*>(b + o_o);
  t.out = dout;
  t.scratch_off = 0;
  CK(cudaMemcpyAsync(b + o_t, &t, sizeof(SiteTask), cudaMemcpyHostToDevice, s));
  CK(launch_pco(reinterpret_cast<SiteTask*>(b + o_t), 1, d, precision,
                reinterpret_cast<double2*>(b + o_s), c->d_status, s));
  COUNT_LAUNCH(1);
  if (mem_kind == GBSMPS_MEM_HOST)
    CK(cudaMemcpyAsync(out, dout, sizeof(double2) * (size_t)Dl * d * Dr, cudaMemcpyDeviceToHost, s));
  buf.release();
  return sync_status(c);
}

int gbsmps_build_site_noalloc(gbsmps_ctx_t c, int32_t nl, int32_t nr, int32_t d, const double* Qm,
                              double cscale, int32_t Dl, const uint8_t* occ_l, int32_t Dr,
                              const uint8_t* occ_r, int32_t precision, double* out) {
  if (!c) return fail(GBSMPS_ERR_ARG, "ctx is NULL");
  const char* detail = "";
  int rc = noalloc_build_site(c->device, c->stream, c->d_status, nl, nr, d, Qm, cscale, Dl, occ_l,
                              Dr, occ_r, precision, out, &detail);
  if (rc) return fail(rc, detail);
  return GBSMPS_OK;
}

size_t gbsmps_estimate_bytes(int32_t N, const gbsmps_opts* o, int64_t S) {
  // mirrors the allocations of the build pipeline and gbsmps_sample with every bond
  // at chi_max (D_m <= chi); transient buffers are counted as if all were live
  if (N < 1 || S < 0 || check_opts(o) != GBSMPS_OK) return 0;
  const double n = N, d = o->d, chi = o->chi_max, cap = chi + TIE_MARGIN;
  const double c2 = chi * chi, site = 16.0 * d * c2;          // one complex128 tensor
  double b = 0.0;
  b += 16.0 * n * QS * QS + 64.0 * NEM * n;                   // GSVD outputs and carried block
  b += (n + 1) * cap * (NEM + 8.0 + 4.0 * NEM) + 64.0 * NEM * (n + 1);   // bases, maps
  b += n * site + 16.0 * (n + 1) * c2;                        // tensors, environments
  b += std::min(n, 304.0) * 16.0 * (4.0 * chi + 4.0 * c2);    // PCO scratch (one wave)
  b += site;                                                  // environment step product
  const double kp = std::ceil(2.0 * chi / 64.0) * 64.0;
  if (o->precision == GBSMPS_PREC_MIXED) {
    b += n * site + 2.0 * 16.0 * (n + 1) * c2;                // energy gauge, L, L^-1
    // two parity groups per site, each bounded by one class holding all chi states
    const double npg = std::ceil(2.0 * d * std::ceil(chi / 16.0) * 16.0 / 128.0) * 128.0;
    b += n * 2.0 * 2.0 * npg * kp * 2.0;                      // packed fp16 planes
    b += 2.0 * 8.0 * d * c2 + 2.0 * (64 << 20);               // transform buffers, split-K
    const double sp = std::ceil(S / 128.0) * 128.0;
    b += 4.0 * 2.0 * sp * kp * 2.0 + 8.0 * 4.0 * sp;          // state planes; lists, scales
    b += 2.0 * (S * npg * 4.0 + S * (npg / 32.0) * 4.0);      // W, chunk norms
  } else {
    const double per = d * chi;
    const double chunk = std::max(1.0, std::min((double)S, 6.0 * (1 << 30) / (32.0 * per + 32.0 * chi)));
    b += 32.0 * chunk * chi + 32.0 * chunk * per;
  }
  b += (double)S * n * 2.0 + S;                               // patterns, flags
  b = b * 1.1 + (64 << 20);                                   // allocator granularity
  return (size_t)b;
}

const char* gbsmps_strerror(int code) {
  switch (code) {
    case GBSMPS_OK: return "ok";
    case GBSMPS_ERR_ARG: return "invalid argument";
    case GBSMPS_ERR_NOT_SYMMETRIC: return "covariance matrix not symmetric";
    case GBSMPS_ERR_NOT_PURE: return "covariance matrix not of a pure state";
    case GBSMPS_ERR_OOM: return "device out of memory";
    case GBSMPS_ERR_NOT_CONVERGED: return "eigensolver did not converge";
    case GBSMPS_ERR_BOUNDS: return "size limit exceeded";
    case GBSMPS_ERR_CUDA: return "CUDA error";
    case GBSMPS_ERR_NUMERIC: return "numerical failure";
    case GBSMPS_ERR_STATE: return "invalid state";
    case GBSMPS_ERR_TIMEOUT: return "bounded device wait timed out";
    default: return "unknown error";
  }
}

const char* gbsmps_last_error_detail(void) { return g_detail.c_str(); }

int64_t gbsmps_launch_count(gbsmps_ctx_t) { return (int64_t)g_kernel_launches.load(); }

int gbsmps_trace(gbsmps_ctx_t c, int enable) {
  if (!c) return fail(GBSMPS_ERR_ARG, "ctx is NULL");
  g_tc_trace.reset();
  g_tc_trace.on = enable != 0;
  g_env_trace.reset();
  g_env_trace.on = enable != 0;
  g_pco_trace.reset();
  g_pco_trace.on = enable != 0;
  return GBSMPS_OK;
}

int gbsmps_trace_read(gbsmps_ctx_t c, double* total_ms, int64_t* launches, double* flops,
                      double* bytes) {
  if (!c) return fail(GBSMPS_ERR_ARG, "ctx is NULL");
  if (total_ms) *total_ms = g_tc_trace.total_ms();
  if (launches) *launches = g_tc_trace.launches;
  if (flops) *flops = g_tc_trace.flops;
  if (bytes) *bytes = g_tc_trace.bytes;
  return GBSMPS_OK;
}

int gbsmps_trace_read_kernel(gbsmps_ctx_t c, int32_t which, double* total_ms, int64_t* launches,
                             double* flops, double* bytes) {
  if (!c) return fail(GBSMPS_ERR_ARG, "ctx is NULL");
  if (which < 0 || which > 2) return fail(GBSMPS_ERR_ARG, "which must be 0, 1 or 2");
  KernelTrace& t = which == 2 ? g_pco_trace : which == 1 ? g_env_trace : g_tc_trace;
  if (total_ms) *total_ms = t.total_ms();
  if (launches) *launches = t.launches;
  if (flops) *flops = t.flops;
  if (bytes) *bytes = t.bytes;
  return GBSMPS_OK;
}

}  // extern "C"
