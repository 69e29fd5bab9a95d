// Mixed-precision sampling in right-canonical form (tcgen05 + TMA).
//
// Exact conditional sampling (q_p = w_p R_{m+1} w_p^dag, w_p = v A^m[p]) is
// rewritten with the Cholesky factors of the right environments of the
// energy-gauge tensors, R_m = L_m L_m^dag: the tensors
//     At^m[p] = L_m^{-1} A^m[p] L_{m+1}
// satisfy sum_p At^m[p] At^m[p]^dag = 1, the sampled state is vt = v L_m,
// and the weights become q_p = |vt At^m[p]|^2.  One site of sampling is then a
// single complex GEMM W = Vt At^m (S x D_{m-1} by D_{m-1} x d D_m) followed by
// a selection pass that reads only the chosen block of W.
//
// The GEMM runs on the 5th-generation tensor cores: operands are stored as
// three bf16 planes (x = h + m + l), K-major, in global memory; TMA copies
// 128 x 64 tiles of every plane into 128-byte-swizzled shared memory; one
// thread issues tcgen05.mma (M = 128, N = 128, K = 16, FP32 accumulators in
// tensor memory) for the six cross products hh, hm, mh, hl, mm, lh; the four
// warps read the accumulators back with tcgen05.ld and write W plus the
// per-tile row norms.  Every wait on an mbarrier is bounded in time; on a
// timeout the kernel records ST_TIMEOUT and releases its tensor memory.
#include "internal.h"
#include <cuda.h>
#include <cuda_bf16.h>
#include <algorithm>
#include <cstring>

namespace {

constexpr int TBM = 128, TBN = 128, TBK = 64;     // tile in bf16 elements (real)
constexpr int NPL = 3;                            // bf16 planes per operand
constexpr int TSTAGES = 2;
constexpr int PLANE_BYTES = TBM * TBK * 2;        // 16 KB (TBN == TBM)
constexpr int STAGE_BYTES = 2 * NPL * PLANE_BYTES;
constexpr int TC_SMEM = TSTAGES * STAGE_BYTES + 1024 + 256;
constexpr unsigned long long WAIT_NS = 2000000000ull;   // 2 s

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t su32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// bounded wait: false after WAIT_NS
__device__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  if (mbar_try(bar, parity)) return true;
  const unsigned long long t0 = gtimer();
  while (!mbar_try(bar, parity)) {
    if (gtimer() - t0 > WAIT_NS) return false;
  }
  return true;
}
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, uint32_t bar,
                                            int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, "
      "%4, %5}], [%2];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(x), "r"(y), "r"(z)
      : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (start address, LBO = 16 B, SBO = 1024 B, version 1,
// layout SWIZZLE_128B)
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}
__device__ __forceinline__ void umma_bf16(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc,
                                          uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void split3(float x, __nv_bfloat16& h, __nv_bfloat16& m,
                                       __nv_bfloat16& l) {
  h = __float2bfloat16_rn(x);
  float r = x - __bfloat162float(h);
  m = __float2bfloat16_rn(r);
  l = __float2bfloat16_rn(r - __bfloat162float(m));
}

// ---------------------------------------------------------------- tcgen05 GEMM
// W[row, n] (complex, row-major, ldw complex) and part[row, tile] = sum |W|^2
// over the tile's 64 complex columns.
__global__ void __launch_bounds__(128, 1)
canon_gemm_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                     int nkb, int nterms, float2* __restrict__ W, long long ldw, int M,
                     float* __restrict__ part, int ntiles, int* status) {
  extern __shared__ __align__(1024) uint8_t smraw[];
  const uint32_t raw = su32(smraw);
  const uint32_t sbase = (raw + 1023u) & ~1023u;
  uint8_t* sp = smraw + (sbase - raw);
  uint64_t* bars = reinterpret_cast<uint64_t*>(sp + TSTAGES * STAGE_BYTES);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 2 * TSTAGES + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * TBM, n0 = blockIdx.x * TBN;
  const uint32_t full0 = su32(bars), empty0 = full0 + 8 * TSTAGES, accb = full0 + 16 * TSTAGES;
  if (threadIdx.x == 0) {
    for (int s = 0; s < TSTAGES; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    mbar_init(accb, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(su32(tslot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  // product terms (plane of A, plane of B), small first; nterms 3 keeps the last 3
  const int ta[6] = {2, 1, 0, 1, 0, 0};
  const int tb[6] = {0, 1, 2, 0, 1, 0};
  const int q0 = nterms == 3 ? 3 : 0;
  if (warp == 0 && lane == 0) {                       // TMA producer
    for (int kb = 0; kb < nkb; ++kb) {
      const int st = kb % TSTAGES, r = kb / TSTAGES;
      if (r > 0 && !mbar_wait(empty0 + 8 * st, (r - 1) & 1)) { set_status(status, ST_TIMEOUT); break; }
      mbar_expect_tx(full0 + 8 * st, STAGE_BYTES);
      const uint32_t sA = sbase + st * STAGE_BYTES, sB = sA + NPL * PLANE_BYTES;
      for (int p = 0; p < NPL; ++p) {
        tma_load_3d(sA + p * PLANE_BYTES, &tmA, full0 + 8 * st, kb * TBK, m0, p);
        tma_load_3d(sB + p * PLANE_BYTES, &tmB, full0 + 8 * st, kb * TBK, n0, p);
      }
    }
  } else if (warp == 1 && lane == 0) {                // MMA issuer
    // D f32, A bf16, B bf16, both K-major, N = 128, M = 128
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TBN >> 3) << 17) |
                           ((uint32_t)(TBM >> 4) << 24);
    bool ok = true;
    for (int kb = 0; kb < nkb; ++kb) {
      const int st = kb % TSTAGES, r = kb / TSTAGES;
      if (!mbar_wait(full0 + 8 * st, r & 1)) { set_status(status, ST_TIMEOUT); ok = false; break; }
      tc_fence_after();
      const uint32_t sA = sbase + st * STAGE_BYTES, sB = sA + NPL * PLANE_BYTES;
      for (int k16 = 0; k16 < TBK / 16; ++k16) {
        for (int q = q0; q < 6; ++q) {
          const uint64_t ad = sdesc(sA + ta[q] * PLANE_BYTES + k16 * 32);
          const uint64_t bd = sdesc(sB + tb[q] * PLANE_BYTES + k16 * 32);
          umma_bf16(tmem, ad, bd, idesc, (kb | k16 | (q - q0)) != 0 ? 1u : 0u);
        }
      }
      umma_commit(empty0 + 8 * st);
    }
    if (ok) umma_commit(accb);
  }
  __syncwarp();
  // epilogue: every warp reads its 32 TMEM lanes (= tile rows)
  const bool got = mbar_wait(accb, 0);
  __syncwarp();
  tc_fence_after();
  if (got) {
    const int row = m0 + warp * 32 + lane;
    float nrm = 0.f;
#pragma unroll 1
    for (int c0 = 0; c0 < TBN; c0 += 32) {
      uint32_t r[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, r);
      if (row < M) {
        float2* dst = W + (long long)row * ldw + (n0 + c0) / 2;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          float re = __uint_as_float(r[2 * j]), im = __uint_as_float(r[2 * j + 1]);
          dst[j] = make_float2(re, im);
          nrm = fmaf(re, re, fmaf(im, im, nrm));
        }
      }
    }
    if (row < M) part[(long long)row * ntiles + blockIdx.x] = nrm;
  } else if (threadIdx.x == 0) {
    set_status(status, ST_TIMEOUT);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tmem) : "memory");
  }
}

// SIMT reference on the same packed planes (cross-check of the tcgen05 path)
__global__ void canon_gemm_ref_kernel(const __nv_bfloat16* __restrict__ Ap, long long apl, int Kp,
                                      const __nv_bfloat16* __restrict__ Bp, long long bpl, int Np,
                                      int nterms, float2* __restrict__ W, long long ldw, int M) {
  const int ta[6] = {2, 1, 0, 1, 0, 0};
  const int tb[6] = {0, 1, 2, 0, 1, 0};
  const int q0 = nterms == 3 ? 3 : 0;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < (long long)M * (Np / 2);
       idx += (long long)gridDim.x * blockDim.x) {
    const int row = idx / (Np / 2), nc = idx % (Np / 2);
    float re = 0.f, im = 0.f;
    for (int q = q0; q < 6; ++q) {
      const __nv_bfloat16* a = Ap + ta[q] * apl + (long long)row * Kp;
      const __nv_bfloat16* b0 = Bp + tb[q] * bpl + (long long)(2 * nc) * Kp;
      const __nv_bfloat16* b1 = b0 + Kp;
      for (int k = 0; k < Kp; ++k) {
        float av = __bfloat162float(a[k]);
        re = fmaf(av, __bfloat162float(b0[k]), re);
        im = fmaf(av, __bfloat162float(b1[k]), im);
      }
    }
    W[(long long)row * ldw + nc] = make_float2(re, im);
  }
}

__global__ void canon_part_ref_kernel(const float2* __restrict__ W, long long ldw, int M,
                                      float* __restrict__ part, int ntiles) {
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < (long long)M * ntiles;
       idx += (long long)gridDim.x * blockDim.x) {
    const int row = idx / ntiles, t = idx % ntiles;
    float s = 0.f;
    for (int j = 0; j < 64; ++j) {
      float2 v = W[(long long)row * ldw + t * 64 + j];
      s = fmaf(v.x, v.x, fmaf(v.y, v.y, s));
    }
    part[idx] = s;
  }
}

// ---------------------------------------------------------------- packing
// B planes of one site: row n_r = 2 (p Drp + b) + c, column k_r = 2 a + e;
// [[Re, -Im], [Im, Re]] blocks of At[a, p, b] (zero in the padding)
__global__ void pack_b_kernel(const float2* __restrict__ At, int Dl, int d, int Dr, int Drp, int Kp,
                              __nv_bfloat16* __restrict__ Bp, long long bpl) {
  const long long ncx = (long long)d * Drp;                 // complex columns
  const long long total = ncx * (Kp / 2);
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long nc = idx / (Kp / 2);
    const int a = idx % (Kp / 2);
    const int p = nc / Drp, b = nc % Drp;
    float2 v = make_float2(0.f, 0.f);
    if (a < Dl && b < Dr) v = At[((long long)a * d + p) * Dr + b];
    __nv_bfloat16 rh, rm, rl, ih, im_, il;
    split3(v.x, rh, rm, rl);
    split3(v.y, ih, im_, il);
    const __nv_bfloat16 rr[3] = {rh, rm, rl}, ii[3] = {ih, im_, il};
    for (int s = 0; s < NPL; ++s) {
      __nv_bfloat16* row0 = Bp + s * bpl + (2 * nc) * Kp + 2 * a;
      __nv_bfloat16* row1 = row0 + Kp;
      __nv_bfloat162 x0, x1;
      x0.x = rr[s]; x0.y = __hneg(ii[s]);
      x1.x = ii[s]; x1.y = rr[s];
      *reinterpret_cast<__nv_bfloat162*>(row0) = x0;
      *reinterpret_cast<__nv_bfloat162*>(row1) = x1;
    }
  }
}

// first site: vt = [1] (D_0 = 1) for every sample, zero padding
__global__ void vinit_kernel(__nv_bfloat16* V, long long vpl, int Spad, int Kp) {
  const long long total = (long long)Spad * Kp;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int k = idx % Kp;
    for (int s = 0; s < NPL; ++s)
      V[s * vpl + idx] = __float2bfloat16_rn((s == 0 && k == 0) ? 1.f : 0.f);
  }
}

// one warp per sample: q_p from the tile norms (fixed order), choose p*,
// write vt' = w_{p*} / sqrt(q_{p*}) as bf16 planes for the next site
__global__ void select_canon_kernel(int S, int d, int Dr, int Drp, const float2* __restrict__ W,
                                    const float* __restrict__ part, int ntiles,
                                    const double* __restrict__ u, int ustride, int site,
                                    uint64_t seed, uint64_t counter0, __nv_bfloat16* __restrict__ V,
                                    long long vpl, int Kpn, uint8_t* __restrict__ out, int N,
                                    uint8_t* flags, double flag_tol);

}  // namespace

namespace {
__global__ void select_canon_kernel(int S, int d, int Dr, int Drp, const float2* __restrict__ W,
                                    const float* __restrict__ part, int ntiles,
                                    const double* __restrict__ u, int ustride, int site,
                                    uint64_t seed, uint64_t counter0, __nv_bfloat16* __restrict__ V,
                                    long long vpl, int Kpn, uint8_t* __restrict__ out, int N,
                                    uint8_t* flags, double flag_tol) {
  const int lane = threadIdx.x & 31;
  const long long s = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  if (s >= S) return;
  const int tpp = Drp / 64;
  double Z = 0.0;
  for (int p = 0; p < d; ++p)
    for (int t = 0; t < tpp; ++t) Z += part[s * ntiles + p * tpp + t];
  const double uu = u ? u[(size_t)s * ustride + site] : philox_uniform(seed, counter0 + s, (uint32_t)site);
  const double tt = uu * Z;
  int pstar = -1, plast = 0;
  double C = 0.0, qsel = 0.0;
  bool flag = false;
  for (int p = 0; p < d; ++p) {
    double q = 0.0;
    for (int t = 0; t < tpp; ++t) q += part[s * ntiles + p * tpp + t];
    C += q;
    if (fabs(tt - C) <= flag_tol * Z) flag = true;
    if (q > 0.0) plast = p;
    if (pstar < 0 && tt < C) { pstar = p; qsel = q; }
  }
  if (pstar < 0) {
    pstar = plast;
    qsel = 0.0;
    for (int t = 0; t < tpp; ++t) qsel += part[s * ntiles + pstar * tpp + t];
  }
  const float inv = qsel > 0.0 ? (float)(1.0 / sqrt(qsel)) : 0.f;
  const float2* w = W + s * (long long)d * Drp + (long long)pstar * Drp;
  for (int b = lane; b < Kpn / 2; b += 32) {
    float2 v = b < Dr ? w[b] : make_float2(0.f, 0.f);
    __nv_bfloat16 h0, m0_, l0, h1, m1, l1;
    split3(v.x * inv, h0, m0_, l0);
    split3(v.y * inv, h1, m1, l1);
    const __nv_bfloat16 rr[3] = {h0, m0_, l0}, ii[3] = {h1, m1, l1};
    for (int pl = 0; pl < NPL; ++pl) {
      __nv_bfloat162 x;
      x.x = rr[pl]; x.y = ii[pl];
      *reinterpret_cast<__nv_bfloat162*>(V + pl * vpl + s * Kpn + 2 * b) = x;
    }
  }
  if (lane == 0) {
    out[(size_t)s * N + site] = (uint8_t)pstar;
    if (flags && flag) flags[s] = 1;
  }
}

// ---------------------------------------------------------------- Cholesky
// one CTA per bond: R + delta 1 = L L^dag (lower, FP64 complex), R overwritten
// by L.  delta = reg * max diag(R) regularises the bond states the truncated
// right part barely reaches (near-null directions of R, which the mixed
// path's FP32-accurate environments resolve only to ~1e-7 |R|): a sampled
// state carries no weight there, so the weights q_p / Z move by O(delta)
// absolute.  A pivot that is still not positive flags ST_NUMERIC.
__global__ void chol_kernel(const double2* __restrict__ src, double2* __restrict__ dst,
                            const long long* __restrict__ off, const int* __restrict__ Dv, int b0,
                            double* __restrict__ dused, int* status) {
  const int b = b0 + blockIdx.x;
  const int D = Dv[b];
  const double2* Sm = src + off[b];
  double2* R = dst + off[b];
  const int tid = threadIdx.x, nt = blockDim.x;
  __shared__ double dmax;
  if (tid == 0) {
    double m = 0.0;
    for (int i = 0; i < D; ++i) m = fmax(m, Sm[(long long)i * D + i].x);
    dmax = m;
  }
  __syncthreads();
  // the smallest regulariser in 1e-12 .. 1e-4 (x100 steps) that factorises
  double reg = 1e-12;
  bool okf = false;
  double delta = 0.0;
  for (int attempt = 0; attempt < 5 && !okf; ++attempt, reg *= 100.0) {
    delta = reg * dmax;
    for (long long idx = tid; idx < (long long)D * D; idx += nt) {
      double2 v = Sm[idx];
      if (idx / D == idx % D) v.x += delta;
      R[idx] = v;
    }
    __syncthreads();
    okf = true;
    for (int k = 0; k < D; ++k) {
      const double akk = R[(long long)k * D + k].x;
      if (!(akk > 0.0)) { okf = false; break; }   // same value in every thread
      const double lkk = sqrt(akk), il = 1.0 / lkk;
    __syncthreads();
    for (int i = k + 1 + tid; i < D; i += nt) R[(long long)i * D + k] = cscale(R[(long long)i * D + k], il);
    if (tid == 0) R[(long long)k * D + k] = cmk(lkk, 0.0);
    __syncthreads();
    const int w = D - k - 1;
    for (long long idx = tid; idx < (long long)w * w; idx += nt) {
      const int i = k + 1 + idx / w, j = k + 1 + idx % w;
      if (j > i) continue;
      double2 v = R[(long long)i * D + j];
      const double2 a = R[(long long)i * D + k], c = cconj(R[(long long)j * D + k]);
      v = csub(v, cmul(a, c));
      R[(long long)i * D + j] = v;
    }
    __syncthreads();
    }
    __syncthreads();
  }
  if (!okf && tid == 0) set_status(status, ST_NUMERIC);
  if (tid == 0) dused[b] = okf ? delta / fmax(dmax, 1e-300) : -1.0;
  for (long long idx = tid; idx < (long long)D * D; idx += nt) {
    const int i = idx / D, j = idx % D;
    if (j > i) R[idx] = cmk(0.0, 0.0);
  }
}

// one CTA per bond: X = L^{-1} (lower), one column per thread
__global__ void trinv_kernel(const double2* __restrict__ Lb, double2* __restrict__ Xb,
                             const long long* __restrict__ off, const int* __restrict__ Dv, int b0) {
  const int b = b0 + blockIdx.x;
  const int D = Dv[b];
  const double2* L = Lb + off[b];
  double2* X = Xb + off[b];
  for (int j = threadIdx.x; j < D; j += blockDim.x) {
    for (int i = 0; i < j; ++i) X[(long long)i * D + j] = cmk(0.0, 0.0);
    const double2 ljj = L[(long long)j * D + j];
    X[(long long)j * D + j] = cmk(1.0 / ljj.x, 0.0);
    for (int i = j + 1; i < D; ++i) {
      double2 s = cmk(0.0, 0.0);
      for (int k = j; k < i; ++k) cfma(s, L[(long long)i * D + k], X[(long long)k * D + j]);
      X[(long long)i * D + j] = cscale(s, -1.0 / L[(long long)i * D + i].x);
    }
  }
}

typedef CUresult (*EncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                             const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                             CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                             CUtensorMapFloatOOBfill);

EncodeFn encode_fn() {
  static EncodeFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeFn>(p);
  }
  return fn;
}

}  // namespace

// ---- host side --------------------------------------------------------------
int canon_make_map(void* map128, const void* planes, int Kp, long long rows) {
  EncodeFn fn = encode_fn();
  if (!fn) return 1;
  // TMA: 16-byte aligned base, 16-byte multiple strides, box inner extent 128 B
  if ((reinterpret_cast<uintptr_t>(planes) & 15) || (Kp % TBK) || (rows % TBM)) return 2;
  cuuint64_t dims[3] = {(cuuint64_t)Kp, (cuuint64_t)rows, (cuuint64_t)NPL};
  cuuint64_t strides[2] = {(cuuint64_t)Kp * 2, (cuuint64_t)Kp * 2 * rows};
  cuuint32_t box[3] = {TBK, TBM, 1};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = fn(reinterpret_cast<CUtensorMap*>(map128), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3,
                  const_cast<void*>(planes), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : 3;
}

cudaError_t launch_canon_gemm(const void* mapA, const void* mapB, const __nv_bfloat16* Ap,
                              long long apl, const __nv_bfloat16* Bp, long long bpl, int Kp,
                              int Np, int M, int Mpad, int nterms, float2* W, float* part,
                              int use_tc, double alg_flops, int* status, cudaStream_t s) {
  const int ntiles = Np / TBN;
  COUNT_LAUNCH(1);
  double flops = alg_flops;
  double bytes = (double)NPL * 2 * ((double)Mpad * Kp + (double)Np * Kp) + (double)M * Np * 4;
  g_tc_trace.begin(s);
  if (use_tc) {
    static bool attr = false;
    if (!attr) {
      cudaError_t e = cudaFuncSetAttribute(canon_gemm_tc_kernel,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
      if (e) return e;
      attr = true;
    }
    CUtensorMap a, b;
    memcpy(&a, mapA, sizeof(CUtensorMap));
    memcpy(&b, mapB, sizeof(CUtensorMap));
    dim3 grid(ntiles, Mpad / TBM);
    canon_gemm_tc_kernel<<<grid, 128, TC_SMEM, s>>>(a, b, Kp / TBK, nterms, W, Np / 2, M, part,
                                                    ntiles, status);
  } else {
    long long n = (long long)M * (Np / 2);
    int blocks = (int)std::min<long long>((n + 255) / 256, 16384);
    canon_gemm_ref_kernel<<<blocks, 256, 0, s>>>(Ap, apl, Kp, Bp, bpl, Np, nterms, W, Np / 2, M);
    long long n2 = (long long)M * ntiles;
    int b2 = (int)std::min<long long>((n2 + 255) / 256, 8192);
    canon_part_ref_kernel<<<b2, 256, 0, s>>>(W, Np / 2, M, part, ntiles);
    COUNT_LAUNCH(1);
  }
  g_tc_trace.end(s, flops, bytes);
  return cudaGetLastError();
}

cudaError_t launch_pack_b(const float2* At, int Dl, int d, int Dr, int Drp, int Kp,
                          __nv_bfloat16* Bp, long long bpl, cudaStream_t s) {
  long long total = (long long)d * Drp * (Kp / 2);
  int blocks = (int)std::min<long long>((total + 255) / 256, 8192);
  pack_b_kernel<<<blocks, 256, 0, s>>>(At, Dl, d, Dr, Drp, Kp, Bp, bpl);
  return cudaGetLastError();
}

cudaError_t launch_vinit(__nv_bfloat16* V, long long vpl, int Spad, int Kp, cudaStream_t s) {
  long long total = (long long)Spad * Kp;
  int blocks = (int)std::min<long long>((total + 255) / 256, 8192);
  vinit_kernel<<<blocks, 256, 0, s>>>(V, vpl, Spad, Kp);
  return cudaGetLastError();
}

cudaError_t launch_select_canon(int S, int d, int Dr, int Drp, const float2* W, const float* part,
                                int ntiles, const double* u, int ustride, int site, uint64_t seed,
                                uint64_t counter0, __nv_bfloat16* V, long long vpl, int Kpn,
                                uint8_t* out, int N, uint8_t* flags, double flag_tol,
                                cudaStream_t s) {
  long long threads = (long long)S * 32;
  int blocks = (int)((threads + 255) / 256);
  select_canon_kernel<<<blocks, 256, 0, s>>>(S, d, Dr, Drp, W, part, ntiles, u, ustride, site, seed,
                                             counter0, V, vpl, Kpn, out, N, flags, flag_tol);
  return cudaGetLastError();
}

cudaError_t launch_chol(const double2* src, double2* dst, const long long* off, const int* Dv,
                        int b0, int nb, double* dused, int* status, cudaStream_t s) {
  if (nb <= 0) return cudaSuccess;
  chol_kernel<<<nb, 512, 0, s>>>(src, dst, off, Dv, b0, dused, status);
  return cudaGetLastError();
}

cudaError_t launch_trinv(const double2* L, double2* X, const long long* off, const int* Dv, int b0,
                         int nb, cudaStream_t s) {
  if (nb <= 0) return cudaSuccess;
  trinv_kernel<<<nb, 256, 0, s>>>(L, X, off, Dv, b0);
  return cudaGetLastError();
}
