// Batched build of many independent states (gbsmps_build_batch).
//
// The per-state pipeline has two sequential chains, the GSVD over the cuts
// (left to right) and the right environments (right to left); everything
// else is parallel over sites.  A batch runs the chains of all states side by
// side instead of one after another: every GSVD chain in one launch (one CTA
// per state), the PCO tensors of all sites of all states in one persistent
// launch (largest sites first), the energy gauge of all sites in one launch, the environment
// chains of all mixed-precision states in one persistent cooperative launch
// (step k takes site N_s - 1 - k of every state, grid-wide barriers between
// the two products of a step), and the normalisations in one launch (one CTA
// per state).  Bond sizes are read back once for the whole batch.  The
// right-canonical packing of the sampler then runs per state, the states
// spread over side streams.
#include "objects.h"
#include <algorithm>
#include <map>

namespace {

template <class T>
int upload(DevBuf& b, const std::vector<T>& v, cudaStream_t s) {
  CK(b.alloc(sizeof(T) * std::max<size_t>(v.size(), 1), s));
  if (!v.empty()) CK(cudaMemcpyAsync(b.p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, s));
  return GBSMPS_OK;
}

}  // namespace

extern "C" int gbsmps_build_batch(gbsmps_ctx_t c, int32_t count, const int32_t* Ns,
                                  const double* const* gammas, int mem_kind,
                                  const gbsmps_opts* opts, gbsmps_mps_t* out) {
  if (!c) return fail(GBSMPS_ERR_ARG, "ctx is NULL");
  if (count < 0) return fail(GBSMPS_ERR_ARG, "count < 0");
  if (count == 0) return GBSMPS_OK;
  if (!Ns || !gammas || !opts || !out) return fail(GBSMPS_ERR_ARG, "NULL argument");
  if (mem_kind != GBSMPS_MEM_HOST && mem_kind != GBSMPS_MEM_DEVICE) return fail(GBSMPS_ERR_ARG, "mem_kind");
  for (int i = 0; i < count; ++i) {
    if (!gammas[i]) return fail(GBSMPS_ERR_ARG, "gammas[" + std::to_string(i) + "] is NULL");
    if (Ns[i] < 1 || Ns[i] > 1000000) return fail(GBSMPS_ERR_ARG, "N out of range");
    int rc = check_opts(&opts[i]);
    if (rc) return rc;
    out[i] = nullptr;
  }
  CK(cudaSetDevice(c->device));
  cudaStream_t s = c->stream;
  StageTimer tm(s);
  std::vector<DevBuf> gin(count);
  std::vector<const double*> dg(count);
  for (int i = 0; i < count; ++i) {
    dg[i] = gammas[i];
    if (mem_kind == GBSMPS_MEM_HOST) {
      const size_t bytes = sizeof(double) * 4 * (size_t)Ns[i] * Ns[i];
      CK(gin[i].alloc(bytes, s));
      CK(cudaMemcpyAsync(gin[i].p, gammas[i], bytes, cudaMemcpyHostToDevice, s));
      dg[i] = gin[i].as<double>();
    }
  }
  auto release_inputs = [&] { for (auto& b : gin) b.release(); };
  std::vector<std::unique_ptr<gbsmps_mps>> Ms(count);
  std::vector<gbs::Front> F(count);
  int rc = GBSMPS_OK;
  for (int i = 0; i < count && !rc; ++i) {
    Ms[i].reset(new gbsmps_mps());
    rc = gbs::alloc_front(Ms[i].get(), c, Ns[i], &opts[i], &F[i]);
    if (!rc) rc = gbs::launch_checks(c, Ms[i].get(), dg[i], &opts[i], F[i]);
  }
  if (rc) { release_inputs(); return rc; }
  tm.mark("validate");
  // a2-a3: all GSVD chains in one launch
  {
    std::vector<ChainJob> cj(count);
    for (int i = 0; i < count; ++i) {
      gbsmps_mps* M = Ms[i].get();
      cj[i] = ChainJob{dg[i], Ns[i], F[i].dbw, opts[i].lambda2_freeze, F[i].Gs, M->ba, M->Qm, M->cm};
    }
    DevBuf jb;
    rc = upload(jb, cj, s);
    if (rc) { release_inputs(); return rc; }
    int maxN = 0;
    for (const ChainJob& j : cj) maxN = std::max(maxN, j.N);
    CK(launch_gsvd_chain_batch(jb.as<ChainJob>(), count, maxN, c->d_status, s));
    COUNT_LAUNCH(1);
    jb.release();
  }
  tm.mark("gsvd_chain");
  // a4-a5 kept bases and maps; one read-back of the bond sizes for the batch
  for (int i = 0; i < count && !rc; ++i) rc = gbs::launch_bases(c, Ms[i].get(), &opts[i]);
  if (rc) { release_inputs(); return rc; }
  std::vector<gbs::Readback> rb(count);
  for (int i = 0; i < count && !rc; ++i) rc = gbs::enqueue_readback(Ms[i].get(), &rb[i], s);
  if (!rc) rc = sync_status(c);
  release_inputs();
  if (rc) return rc;
  for (int i = 0; i < count; ++i) gbs::finish_readback(Ms[i].get(), rb[i]);
  tm.mark("basis_maps");
  // a6: PCO tensors of every site of every state (one wave set per cutoff d)
  size_t scr_max = 0;
  for (int i = 0; i < count && !rc; ++i) rc = gbs::alloc_tensors(Ms[i].get(), s, &scr_max);
  if (rc) return rc;
  {
    // grouped by (d, precision): mixed states take the FP32 passes
    std::map<std::pair<int, int>, std::vector<SiteTask>> by_d;
    for (int i = 0; i < count; ++i)
      gbs::site_tasks(Ms[i].get(), rb[i].cm, by_d[{opts[i].d, opts[i].precision}]);
    for (auto& kv : by_d) {
      rc = gbs::run_pco(c, kv.second, scr_max, kv.first.first, kv.first.second);
      if (rc) return rc;
    }
  }
  tm.mark("pco");
  // a7: environments and normalisation
  std::vector<int> mixed;
  for (int i = 0; i < count; ++i) {
    gbsmps_mps* M = Ms[i].get();
    if (opts[i].precision == GBSMPS_PREC_MIXED) {
      mixed.push_back(i);
      continue;
    }
    rc = gbs::env_single(c, M, tm);
    if (!rc) rc = gbs::normalise_single(c, M);
    if (rc) return rc;
  }
  if (!mixed.empty()) {
    // energy gauge of every site, one launch per cutoff d
    std::map<int, std::vector<GaugeTask>> gt;
    std::map<int, int> gmax;
    for (int i : mixed) {
      gbsmps_mps* M = Ms[i].get();
      CK(M->tens_mixed.alloc(sizeof(double2) * M->ttot, s));
      const int cap = M->ba.cap;
      const long long ne = (long long)(M->N + 1) * cap;
      CK(M->gscale.alloc(sizeof(double) * 2 * ne, s));
      CK(launch_gauge_scale(M->ba.E, ne, M->gscale.as<double>(), s));
      COUNT_LAUNCH(1);
      const double* Gup = M->gscale.as<double>();
      const double* Gdn = Gup + ne;
      for (int m = 0; m < M->N; ++m) {
        gt[M->d].push_back(GaugeTask{M->tensors.as<double2>() + M->toff[m], M->D[m], M->D[m + 1],
                                     Gup + (size_t)m * cap, Gdn + (size_t)(m + 1) * cap,
                                     M->tens_mixed.as<double2>() + M->toff[m],
                                     gbs::parity_site(M, m)});
        gmax[M->d] = std::max(gmax[M->d], M->D[m] * M->d * M->D[m + 1]);
      }
    }
    std::vector<DevBuf> gb(gt.size());
    int gi = 0;
    for (auto& kv : gt) {
      rc = upload(gb[gi], kv.second, s);
      if (rc) return rc;
      CK(launch_energy_gauge_batch(gb[gi].as<GaugeTask>(), (int)kv.second.size(), kv.first,
                                   gmax[kv.first], s));
      COUNT_LAUNCH(1);
      ++gi;
    }
    tm.mark("energy_gauge");
    // per-state device offset tables and product scratch
    const size_t nm = mixed.size();
    std::vector<DevBuf> offs(nm), xs(nm);
    std::vector<EnvJob> ej(nm);
    std::vector<NormJob> nj(nm);
    int maxN = 0, maxD = 1;
    for (size_t k = 0; k < nm; ++k) {
      gbsmps_mps* M = Ms[mixed[k]].get();
      const int N = M->N;
      std::vector<long long> tab(M->toff);
      tab.insert(tab.end(), M->eoff.begin(), M->eoff.end());
      rc = upload(offs[k], tab, s);
      if (rc) return rc;
      CK(xs[k].alloc(sizeof(double2) * ((size_t)M->d * M->maxD * M->maxD + 8), s));
      double2* R = M->env.as<double2>();
      static const float4 one_pair = make_float4(1.f, 0.f, 0.f, 0.f);   // R_N = 1 as a pair
      CK(cudaMemcpyAsync(R + M->eoff[N], &one_pair, sizeof(float4), cudaMemcpyHostToDevice, s));
      const long long* toff_d = offs[k].as<long long>();
      ej[k] = EnvJob{N, M->d, M->ba.D, toff_d, toff_d + N, M->tens_mixed.as<double2>(), R,
                     xs[k].as<double2>(), M->ba.pcnt};
      nj[k] = NormJob{N, M->d, M->ba.D, toff_d, M->tensors.as<double2>(), R,
                      M->tens_mixed.as<double2>(),
                      M->gscale.as<double>() + (long long)(N + 1) * M->ba.cap + M->ba.cap,
                      gbs::parity_site(M, 0)};
      maxN = std::max(maxN, N);
      maxD = std::max(maxD, M->maxD);
    }
    DevBuf ejb, njb;
    rc = upload(ejb, ej, s);
    if (!rc) rc = upload(njb, nj, s);
    if (rc) return rc;
    int cfg = -1;                                   // autotuned tile shape
    if (const char* e = getenv("GBSMPS_ENV_TILE")) cfg = atoi(e);
    if (cfg >= env_chain_tile_configs()) return fail(GBSMPS_ERR_ARG, "GBSMPS_ENV_TILE out of range");
    CK(launch_env_chain_batch(ejb.as<EnvJob>(), (int)nm, maxN, maxD, cfg, s, nullptr));
    tm.mark("environments");
    CK(launch_vac_norm_batch(njb.as<NormJob>(), (int)nm, maxD, c->d_status, s));
    tm.mark("normalise");
    // stream order keeps the scratch alive until the launches above are done
    for (auto& b : xs) b.release();
    for (auto& b : offs) b.release();
    for (auto& b : gb) b.release();
    ejb.release();
    njb.release();
    // right-canonical packing: the states' factorisations and transforms are
    // independent, so they are spread over side streams (storage is allocated
    // on the main stream first; the main stream waits for every side stream
    // before the temporaries are freed)
    constexpr int NSIDE = 8;
    std::vector<std::unique_ptr<gbs::CanonWork>> cw(nm);
    for (size_t k = 0; k < nm; ++k) {
      cw[k].reset(new gbs::CanonWork());
      rc = gbs::canon_prepare(Ms[mixed[k]].get(), cw[k].get(), s);
      if (rc) return rc;
    }
    const int nside = (int)std::min<size_t>(NSIDE, nm);
    std::vector<cudaEvent_t> evs(nside + 1, nullptr);
    for (auto& e : evs)
      if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) e = nullptr;
    auto drop_events = [&] { for (auto e : evs) if (e) cudaEventDestroy(e); };
    if (std::any_of(evs.begin(), evs.end(), [](cudaEvent_t e) { return e == nullptr; })) {
      drop_events();
      return fail(GBSMPS_ERR_CUDA, "event creation failed");
    }
    std::vector<cudaStream_t> side(nside);
    cudaEventRecord(evs[nside], s);
    for (int j = 0; j < nside; ++j) {
      side[j] = c->side_stream(j);
      if (!side[j]) { drop_events(); return fail(GBSMPS_ERR_CUDA, "could not create a side stream"); }
      cudaStreamWaitEvent(side[j], evs[nside], 0);
    }
    for (size_t k = 0; k < nm && !rc; ++k) {
      gbsmps_mps* M = Ms[mixed[k]].get();
      cudaStream_t st = side[k % nside];
      rc = gbs::canon_bonds(c, M, cw[k].get(), 1, M->N - 1, st);
      if (!rc) rc = gbs::canon_sites_grouped(M, cw[k].get(), st);
    }
    for (int j = 0; j < nside; ++j) {           // join (also on an error above)
      cudaEventRecord(evs[j], side[j]);
      cudaStreamWaitEvent(s, evs[j], 0);
    }
    drop_events();
    cw.clear();
    if (rc) return rc;
    tm.mark("canonical_pack");
  }
  for (int i = 0; i < count && !rc; ++i) rc = gbs::finish(c, Ms[i].get());
  if (!rc) rc = sync_status(c);
  if (rc) return rc;
  for (int i = 0; i < count; ++i) out[i] = Ms[i].release();
  return GBSMPS_OK;
}
