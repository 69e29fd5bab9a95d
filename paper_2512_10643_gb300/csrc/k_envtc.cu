// Right-environment products on the tensor cores with exact accumulation.
//
// The environments R_m = sum_p Ahat^m[p] R_{m+1} Ahat^m[p]^dag are a chain of
// N dependent complex products whose last value is the squared norm of the
// state, so the rounding of one step compounds over the chain: tensor-core
// FP32 accumulation of full-precision operands biases each step by ~2e-7,
// which is why the chain otherwise runs in double-float arithmetic on the
// FP32 pipes.  Here every product is split in the way of Ozaki, Ogita, Oishi
// and Rump ("Error-free transformations of matrix multiplication by using
// fast routines of matrix multiplication", Numer. Algorithms 59, 2012).
//
// * Complex as real: C = A B is [Re C | Im C] = [Re A, Im A] Bt with
//   Bt = [[Re B, Im B], [-Im B, Re B]] (k = 2K real terms).
// * Every row of [Re A, Im A] and every column pair of Bt is scaled by a
//   power of two 2^e (e the exponent of its largest entry) and cut, exactly
//   from the double-float operand, into seven integer slices of seven bits,
//   x = 2^(e-7) sum_t s_t 2^(-7t), |s_0| <= 128, |s_t| <= 64.  The slices are
//   stored as bf16 values s_t 2^(-7t) (eight significant bits: exact).
// * Products of slice pairs (s, t) are exact in the tensor cores; pairs with
//   s + t = 0, 1, 2 go to one FP32 tensor-memory accumulator each, whose
//   partial sums over at most 512 real k are integers (times 2^(-7g)) below
//   2^24 and therefore exact; the pairs with 3 <= s + t <= 6 share a fourth
//   accumulator (their FP32 rounding is 2^-24 of a sum that is already below
//   2^-21 of the leading one); pairs with s + t > 6 are dropped (2^-49 of the
//   row and column maxima).
// * The four accumulators are summed in double-float registers, scaled by
//   2^(e_row + e_col - 14) and written as pairs; a k split writes partials
//   that a reduction kernel sums in k order.
//
// Kernels: a slicing pass (one CTA per operand row, its exponent from a
// block max) writes the bf16 planes of a launch's operands into arenas
// (K-major rows, seven planes, zero-padded k); the GEMM runs one CTA per
// (product, 128-row x 64-complex-column tile, k split): one thread brings
// 32-k stages of both operands' seven planes by TMA (64-byte swizzle) through
// a two-stage ring, one thread issues the 28 slice-pair MMAs (M = 128,
// N = 128) per 16 k into the four accumulators (all 512 tensor-memory
// columns), and four epilogue warps fold them into double-float and write the
// outputs or partials; the reduction sums partials coalesced.  Every
// mbarrier wait is bounded.
#include "internal.h"
#include "objects.h"
#include "tc_ptx.h"
#include <cuda.h>
#include <cuda_bf16.h>
#include <algorithm>
#include <cstring>
#include <utility>
#include <vector>

namespace {

using namespace tcx;

constexpr int EM = 128;                        // complex rows of A per tile (tensor-memory lanes)
constexpr int EK = 32;                         // real k per stage (64-byte rows)
constexpr int SBITS = 7;                       // bits per slice
constexpr int NSL_MAX = 8;
constexpr int CHUNK = 16;                      // stages summed exactly (512 real k)
constexpr int ESTG = 2;
constexpr int PLANE_A = EM * EK * 2;           // 8 KB
constexpr int ENBAR = 2 * ESTG + 2;            // full, empty, accumulators full, drain
constexpr int E_THREADS = 320;                 // load warp, MMA warp, eight epilogue warps
constexpr int E_TMEM = 512;
constexpr int SL_THREADS = 128;
constexpr int SL_K = 2 * SL_THREADS;            // complex k per slicing CTA (two per thread)
constexpr int RED_THREADS = 256;

// Two configurations.  NSL slices per operand (pairs with s + t <= NSL - 1
// are multiplied), ENC complex columns per tile (ENR = 2 ENC real MMA
// columns: Re of the ENC, then Im) and NACC tensor-memory accumulators: pairs
// with s + t < NACC - 1 one exact accumulator each, the rest the last.
// <7, 48, 5>: s + t = 0..3 exact (their sums over a 512-k chunk stay below
// 2^24), 480 columns; <7, 64, 4>: s + t = 0..2 exact, 512 columns, wider
// tiles.  Measured over the 144-mode chain (mixed build with FP64 PCO passes
// against the FP64 build): 1.2e-12 and 5.3e-12 of the largest amplitude
// (double-float products: 6.8e-14).  An eighth slice does not help (2.3e-12:
// more products in the rounded accumulator); the error is that of the
// per-row/column scaling, which bounds each term by the row and column
// maxima rather than by the term itself.
template <int NSL_, int ENC_, int NACC_>
struct EtcCfg {
  static constexpr int NSL = NSL_, ENC = ENC_, ENR = 2 * ENC_, NACC = NACC_;
  static constexpr int PLANE_B = ENR * EK * 2;
  static constexpr int A_BYTES = NSL * PLANE_A;
  static constexpr int ESTAGE = NSL * (PLANE_A + PLANE_B);
  static constexpr int SMEM = ESTG * ESTAGE + 1024 + 256;
  static constexpr int SROW = ENC + 1;         // staged output row (float4), padded
  static constexpr int HC = ENC / 2;           // columns per epilogue warp
  static_assert(NACC * ENR <= E_TMEM, "accumulators fit the tensor memory");
  static_assert(ENR % 16 == 0 && ENR <= 256 && HC % 8 == 0 && HC <= 32, "MMA and epilogue shape");
  static_assert(4 * 32 * SROW * 16 <= ESTG * ESTAGE, "the output staging fits the operand stages");
  static_assert(ESTAGE % 1024 == 0 && PLANE_B % 512 == 0, "swizzle atoms");
  static_assert(SMEM <= 232448, "shared memory per CTA");
  static_assert(NSL <= NSL_MAX, "slice planes");
};
using CfgExact = EtcCfg<7, 48, 5>;
using CfgWide = EtcCfg<7, 64, 4>;

__host__ __device__ inline long long pad_to(long long x, long long m) { return (x + m - 1) / m * m; }

// Packed pairs of FP32 values (Blackwell's f32x2 add/sub/mul, each lane
// correctly rounded): the slicing cuts the Re and Im parts of an element,
// and the epilogue folds the Re and Im values of a column, together at half
// the instruction count.
typedef unsigned long long f2x;
__device__ __forceinline__ f2x pk(float a, float b) {
  f2x d;
  asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(a), "f"(b));
  return d;
}
__device__ __forceinline__ float2 upk(f2x v) {
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
  return r;
}
__device__ __forceinline__ f2x add2(f2x a, f2x b) {
  f2x d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2x sub2(f2x a, f2x b) {
  f2x d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2x mul2(f2x a, f2x b) {
  f2x d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
// ---- slicing ------------------------------------------------------------------
struct SlJob {
  const float4* src;          // double-float complex pairs; element (r, k) at src[r * ld + k * es]
  long long ld, es;
  int rows, K, kind, conj;    // kind 0: A rows [Re | Im]; 1: B columns (Re and Im rows of Bt)
  __nv_bfloat16* arena;
  long long plane, dst;       // plane stride (elements), first arena row
  int W, enc;                 // enc: complex columns per B tile (kind 1)
  int* expo;
  long long b0;               // first CTA
};
struct SlSet {
  int n;
  SlJob j[3 * ETC_MAX];
};

// (re, im) = (v.x + v.y, v.z + v.w) 2^sh, each cut into NS slices s_t,
// handed over as bf16 values s_t 2^(-7t) (put(t, re_t, im_t)); the pair's
// arithmetic runs packed.  Cutting -x gives the negated slices of x (round
// to nearest even and TwoSum are odd functions), so a negated part is stored
// from the same slices.
template <int NS, class Put>
__device__ __forceinline__ void slice_pair(float4 v, int sh, Put&& put) {
  f2x hs = pk(ldexpf(v.x, sh), ldexpf(v.z, sh)), ls = pk(ldexpf(v.y, sh), ldexpf(v.w, sh));
  const f2x k128 = pk((float)(1 << SBITS), (float)(1 << SBITS));
  float w = 1.f;
#pragma unroll
  for (int t = 0; t < NS; ++t) {
    const float2 h2 = upk(hs);
    const float sr = rintf(h2.x), si = rintf(h2.y);
    put(t, __float2bfloat16_rn(sr * w), __float2bfloat16_rn(si * w));   // |s| <= 128: exact
    hs = sub2(hs, pk(sr, si));                        // exact
    const f2x u = add2(hs, ls);                       // TwoSum: (hs, ls) renormalised exactly
    const f2x vv = sub2(u, hs);
    const f2x e = add2(sub2(hs, sub2(u, vv)), sub2(ls, vv));
    hs = mul2(u, k128);
    ls = mul2(e, k128);
    w *= 1.f / (float)(1 << SBITS);
  }
}

__device__ __forceinline__ int find_job(const SlSet& js, long long b) {
  int lo = 0, hi = js.n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (js.j[mid].b0 <= b) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// One CTA per (operand row, segment of SL_K complex k): every CTA of a row
// takes the row's maximum (the same exponent), then slices its segment, two
// consecutive k per thread so that the planes are written as bf16 pairs.
template <int NS>
__global__ void __launch_bounds__(SL_THREADS) etc_slice_kernel(const __grid_constant__ SlSet js) {
  __shared__ float red[SL_THREADS / 32];
  // a register copy: the stores below go through generic pointers, which
  // would otherwise make every field a reload from parameter space
  const SlJob J = js.j[find_job(js, blockIdx.x)];
  // launched as a programmatic dependent: no global access before the wait
  griddep_wait();
  griddep_launch();
  const long long bl = blockIdx.x - J.b0;
  const int segs = (J.K + SL_K - 1) / SL_K;
  const int r = (int)(bl / segs), seg = (int)(bl % segs);
  const int tid = threadIdx.x;
  const float4* row = J.src + (long long)r * J.ld;
  float mx = 0.f;
  for (int k = tid; k < J.K; k += SL_THREADS) {
    const float4 v = row[(long long)k * J.es];
    mx = fmaxf(mx, fmaxf(fabsf(v.x), fabsf(v.z)));
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((tid & 31) == 0) red[tid >> 5] = mx;
  __syncthreads();
  mx = fmaxf(fmaxf(red[0], red[1]), fmaxf(red[2], red[3]));
  int E = 0;
  if (mx > 0.f) frexpf(mx, &E);                      // |x| < 2^E (the low word cannot cross it)
  if (tid == 0 && seg == 0) J.expo[r] = E;
  const int sh = SBITS - E;
  const long long r0 = J.kind == 0 ? J.dst + r : J.dst + (long long)(r / J.enc) * 2 * J.enc + r % J.enc;
  __nv_bfloat16* p0 = J.arena + r0 * J.W;
  __nv_bfloat16* p1 = p0 + (long long)J.enc * J.W;   // kind 1: the Im row of the column
  const int k0 = seg * SL_K + 2 * tid;
  if (k0 < J.K) {
    const bool two = k0 + 1 < J.K;
    float4 v0 = row[(long long)k0 * J.es];
    float4 v1 = two ? row[(long long)(k0 + 1) * J.es] : make_float4(0.f, 0.f, 0.f, 0.f);
    if (J.conj) { v0.z = -v0.z; v0.w = -v0.w; v1.z = -v1.z; v1.w = -v1.w; }
    __nv_bfloat16 re0[NS], im0[NS], re1[NS], im1[NS];
    slice_pair<NS>(v0, sh, [&](int t, __nv_bfloat16 re, __nv_bfloat16 im) { re0[t] = re; im0[t] = im; });
    slice_pair<NS>(v1, sh, [&](int t, __nv_bfloat16 re, __nv_bfloat16 im) { re1[t] = re; im1[t] = im; });
    const long long pl = J.plane;
    // a pair of k at an even offset as one 4-byte store, else one by one
    auto put2 = [&](__nv_bfloat16* p, long long off, __nv_bfloat16 a, __nv_bfloat16 b) {
      if (two && !(off & 1)) {
        *reinterpret_cast<__nv_bfloat162*>(p + off) = __halves2bfloat162(a, b);
      } else {
        p[off] = a;
        if (two) p[off + 1] = b;
      }
    };
#pragma unroll
    for (int t = 0; t < NS; ++t) {
      if (J.kind == 0) {                             // [Re | Im]
        put2(p0, t * pl + k0, re0[t], re1[t]);
        put2(p0, t * pl + J.K + k0, im0[t], im1[t]);
      } else {                                       // Re row [Re | -Im], Im row [Im | Re]
        put2(p0, t * pl + k0, re0[t], re1[t]);
        put2(p0, t * pl + J.K + k0, __hneg(im0[t]), __hneg(im1[t]));
        put2(p1, t * pl + k0, im0[t], im1[t]);
        put2(p1, t * pl + J.K + k0, re0[t], re1[t]);
      }
    }
  }
  if (seg == segs - 1) {                             // zeros up to the end of the last 32-k stage
    const int kend = (int)pad_to(2LL * J.K, EK);
    const __nv_bfloat16 z = __float2bfloat16_rn(0.f);
    for (int x = 2 * J.K + tid; x < kend; x += SL_THREADS)
      for (int t = 0; t < NS; ++t) {
        p0[t * J.plane + x] = z;
        if (J.kind == 1) p1[t * J.plane + x] = z;
      }
  }
}

// ---- the GEMM -------------------------------------------------------------------
struct EtcProb {
  int M, N, nst;              // complex rows, complex columns, 32-k stages of the real k = 2K
  long long arow, brow;       // first arena rows
  const int* ea;              // exponents of A's rows and of B's columns
  const int* eb;
  void* C; long long ldc;     // output: double-float pairs (csplit) or FP64
  int herm, csplit;
  int tm, tn, ks, kst;        // tiles; k splits of kst stages
  long long u0;               // first CTA
  float4* part;               // partials [ks][M][N] when ks > 1
};
struct EtcGroup {
  int np;
  EtcProb p[ETC_MAX];
};

__device__ __forceinline__ void dfa(float& h, float& l, float x) {   // (h, l) += x, TwoSum
  const float t = h + x;
  const float v = t - h;
  l += (h - (t - v)) + (x - v);
  h = t;
}
__device__ __forceinline__ float2 df_norm(float h, float l) {
  const float s = h + l;
  const float v = s - h;
  return make_float2(s, (h - (s - v)) + (l - v));
}

__device__ __forceinline__ void dfa2x(f2x& h, f2x& l, f2x x) {   // (h, l) += x lane-wise, TwoSum
  const f2x t = add2(h, x);
  const f2x v = sub2(t, h);
  l = add2(l, add2(sub2(h, sub2(t, v)), sub2(x, v)));
  h = t;
}
// (h + l) 2^e as normalised pairs, for the two lanes at once
__device__ __forceinline__ float4 scale_pair2(f2x h, f2x l, int e) {
  if (e >= -126 && e <= 127) {
    const float p = __int_as_float((e + 127) << 23);
    const f2x pp = pk(p, p);
    h = mul2(h, pp);
    l = mul2(l, pp);
    const f2x sm = add2(h, l);
    const f2x v = sub2(sm, h);
    const f2x er = add2(sub2(h, sub2(sm, v)), sub2(l, v));
    const float2 a = upk(sm), b = upk(er);
    return make_float4(a.x, b.x, a.y, b.y);
  }
  const float2 a = upk(h), b = upk(l);
  const float2 re = df_norm(ldexpf(a.x, e), ldexpf(b.x, e)), im = df_norm(ldexpf(a.y, e), ldexpf(b.y, e));
  return make_float4(re.x, re.y, im.x, im.y);
}

template <class CF>
__global__ void __launch_bounds__(E_THREADS, 1)
envtc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
             const __grid_constant__ EtcGroup g, int* status) {
  const long long b = blockIdx.x;
  int lo = 0, hi = g.np - 1;
  while (lo < hi) {                                   // last product with u0 <= b
    const int mid = (lo + hi + 1) >> 1;
    if (g.p[mid].u0 <= b) lo = mid; else hi = mid - 1;
  }
  const EtcProb P = g.p[lo];                          // in registers (see the slicing kernel)
  const long long l = b - P.u0;
  const int kz = (int)(l % P.ks);
  const int tile = (int)(l / P.ks);
  const int tmi = tile / P.tn, tni = tile % P.tn;
  constexpr int ENC = CF::ENC, ENR = CF::ENR, NACC = CF::NACC, SROW = CF::SROW, HC = CF::HC;
  constexpr int ESTAGE = CF::ESTAGE, PLANE_B = CF::PLANE_B, NSL = CF::NSL, A_BYTES = CF::A_BYTES;
  if (P.herm && tni * ENC > tmi * EM + EM - 1) return;   // a tile above the diagonal: nothing kept
  const int s_beg = kz * P.kst;
  const int nstage = max(0, min(P.nst, s_beg + P.kst) - s_beg);   // <= CHUNK

  extern __shared__ __align__(1024) uint8_t smraw[];
  const uint32_t raw = su32(smraw);
  const uint32_t sbase = (raw + 1023u) & ~1023u;
  uint8_t* sp = smraw + (sbase - raw);
  uint64_t* bars = reinterpret_cast<uint64_t*>(sp + ESTG * ESTAGE);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + ENBAR);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t full0 = su32(bars), empty0 = full0 + 8 * ESTG;
  const uint32_t afull = empty0 + 8 * ESTG, drain = afull + 8;
  if (threadIdx.x == 0) {
    for (int s = 0; s < ESTG; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    mbar_init(afull, 1);
    mbar_init(drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tslot)),
                 "r"(E_TMEM)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  // the setup above overlaps the preceding kernel; no global access before the wait
  griddep_wait();
  griddep_launch();
  if (warp == 0) {
    if (lane == 0) {                                  // loads: both operands' seven planes per stage
      int i = 0;
      for (; i < nstage; ++i) {
        const int st = i % ESTG, r = i / ESTG;
        if (r > 0 && !mbar_wait(empty0 + 8 * st, (r - 1) & 1)) {
          set_status(status, ST_TIMEOUT);
          break;
        }
        const uint32_t sA = sbase + st * ESTAGE, sB = sA + A_BYTES;
        mbar_expect_tx(full0 + 8 * st, ESTAGE);
        const int x = (s_beg + i) * EK;
        tma_load_3d(sA, &tmA, full0 + 8 * st, x, (int)(P.arow + tmi * EM), 0);
        tma_load_3d(sB, &tmB, full0 + 8 * st, x, (int)(P.brow + tni * ENR), 0);
      }
      // the last copy issued into each stage has landed before the CTA exits
      for (int st = 0; st < ESTG && st < i; ++st) {
        const int lastg = st + ESTG * ((i - 1 - st) / ESTG);
        if (!mbar_wait(full0 + 8 * st, (lastg / ESTG) & 1)) set_status(status, ST_TIMEOUT);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {                                  // MMA issuer
      // D f32, A and B bf16, both K-major, N = ENR, M = 128
      const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(ENR >> 3) << 17) |
                             ((uint32_t)(EM >> 4) << 24);
      unsigned init = 0;
      for (int i = 0; i < nstage; ++i) {
        const int st = i % ESTG, r = i / ESTG;
        if (!mbar_wait(full0 + 8 * st, r & 1)) {
          set_status(status, ST_TIMEOUT);
          break;
        }
        tc_fence_after();
        const uint32_t sA = sbase + st * ESTAGE, sB = sA + A_BYTES;
#pragma unroll
        for (int k16 = 0; k16 < EK / 16; ++k16)
#pragma unroll
          for (int ia = 0; ia < NSL; ++ia)
#pragma unroll
            for (int jb = 0; ia + jb < NSL; ++jb) {
              const int a = min(ia + jb, NACC - 1);
              const uint64_t ad = sdesc_sw(sA + ia * PLANE_A + k16 * 32, 512, 4);
              const uint64_t bd = sdesc_sw(sB + jb * PLANE_B + k16 * 32, 512, 4);
              umma_f16(tmem + (uint32_t)(a * ENR), ad, bd, idesc, (init >> a) & 1u);
              init |= 1u << a;
            }
        umma_commit(empty0 + 8 * st);
      }
      umma_commit(afull);                             // every MMA issued here has completed
    }
  } else {
    // epilogue: warps 2..9; tensor-memory lane quadrant warp % 4, columns
    // half * HC .. half * HC + HC - 1 of the tile
    const int q = warp & 3, half = (warp - 2) >> 2;
    const int i = tmi * EM + q * 32 + lane;           // complex output row
    const bool rvalid = i < P.M;
    // exponents while the MMAs run: the row's, and one column's per lane
    const int er = rvalid ? P.ea[i] : 0;
    const int jl = tni * ENC + half * HC + lane;
    const int ebl = (lane < HC && jl < P.N) ? P.eb[jl] : 0;
    const bool got = __all_sync(0xffffffffu, mbar_wait(afull, 0));
    if (!got) {
      if (lane == 0) set_status(status, ST_TIMEOUT);
    } else {
      tc_fence_after();
      // Every MMA has completed, so the operand stages are free: the 32 rows
      // x ENC complex results of a quadrant go through them (rows padded by
      // one element: conflict-free) and leave as row segments.
      float4* stg = reinterpret_cast<float4*>(sp) + (size_t)q * 32 * SROW;
      const uint32_t tb = tmem + ((uint32_t)(q * 32) << 16);
#pragma unroll 1
      for (int ch = 0; ch < HC / 8; ++ch) {
        const int c0 = half * HC + ch * 8;            // first tile column of the 8
        uint32_t v[NACC][8], w[NACC][8];
#pragma unroll
        for (int a = 0; a < NACC; ++a) {
          tmem_ld8_nw(tb + (uint32_t)(a * ENR + c0), v[a]);          // Re
          tmem_ld8_nw(tb + (uint32_t)(a * ENR + ENC + c0), w[a]);    // Im
        }
        tmem_wait_ld();
#pragma unroll
        for (int x = 0; x < 8; ++x) {
          f2x ah = pk(__uint_as_float(v[0][x]), __uint_as_float(w[0][x])), al = 0ull;
#pragma unroll
          for (int a = 1; a < NACC; ++a)
            dfa2x(ah, al, pk(__uint_as_float(v[a][x]), __uint_as_float(w[a][x])));
          const int e = er + __shfl_sync(0xffffffffu, ebl, ch * 8 + x) - 2 * SBITS;
          stg[lane * SROW + c0 + x] = scale_pair2(ah, al, e);
        }
      }
      const bool bulk = P.ks > 1 || (P.csplit && !P.herm);
      if (bulk) fence_proxy_async();                  // the staged rows, visible to the bulk copies
      named_bar(1 + q, 64);                           // both halves of the quadrant staged
      const int ncol = min(ENC, P.N - tni * ENC);
      if (bulk) {
        // one bulk copy per row: rows half * 16 .. half * 16 + 15 of the quadrant
        const int rr = half * 16 + lane;
        const int ii = tmi * EM + q * 32 + rr;
        if (lane < 16 && ii < P.M) {
          float4* dst = P.ks > 1 ? P.part + ((long long)kz * P.M + ii) * P.N + tni * ENC
                                 : reinterpret_cast<float4*>(P.C) + (long long)ii * P.ldc + tni * ENC;
          bulk_s2g(dst, su32(stg + rr * SROW), (uint32_t)ncol * 16u);
          bulk_commit();
          bulk_wait_all();
        }
      } else {
        for (int r = 0; r < 16; ++r) {
          const int rr = half * 16 + r;
          const int ii = tmi * EM + q * 32 + rr;
          if (ii >= P.M) break;
#pragma unroll
          for (int cc = 0; cc < ENC; cc += 32) {
            const int c = cc + lane, j = tni * ENC + c;
            if (c >= ncol || (P.herm && j > ii)) continue;
            const float4 w = stg[rr * SROW + c];
            if (P.csplit) {
              float4* C4 = reinterpret_cast<float4*>(P.C);
              C4[(long long)ii * P.ldc + j] = w;
              if (P.herm && ii > j) C4[(long long)j * P.ldc + ii] = make_float4(w.x, w.y, -w.z, -w.w);
            } else {
              double2* Cd = reinterpret_cast<double2*>(P.C);
              const double vr = (double)w.x + (double)w.y, vi = (double)w.z + (double)w.w;
              Cd[(long long)ii * P.ldc + j] = make_double2(vr, vi);
              if (P.herm && ii > j) Cd[(long long)j * P.ldc + ii] = make_double2(vr, -vi);
            }
          }
        }
      }
    }
  }
  __syncwarp();
  tc_fence_before();
  __syncthreads();
  if (warp == 1 && lane == 0 && nstage > 0) {         // nothing of ours in flight before the dealloc
    umma_commit(drain);
    if (!mbar_wait(drain, 0)) set_status(status, ST_TIMEOUT);
  }
  __syncthreads();
  if (warp == 0) {
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(E_TMEM)
                 : "memory");
  }
}

// ---- k-split reduction --------------------------------------------------------------
struct RedJob {
  const float4* part;
  int ks, M, N;
  void* C; long long ldc;
  int herm, csplit;
  long long e0;               // first element of the launch
};
struct RedSet {
  int n;
  RedJob j[ETC_MAX];
};

// `split` (1, 2 or 4) threads per complex output, each summing every
// split-th partial; their sums are combined in a fixed order (deterministic)
__global__ void __launch_bounds__(RED_THREADS) etc_reduce_kernel(const __grid_constant__ RedSet rs,
                                                                 int split) {
  const long long t = ((long long)blockIdx.x * RED_THREADS + threadIdx.x) / split;
  const int sub = threadIdx.x % split;
  int lo = 0, hi = rs.n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (rs.j[mid].e0 <= t) lo = mid; else hi = mid - 1;
  }
  const RedJob J = rs.j[lo];
  griddep_wait();
  griddep_launch();
  const long long x = t - J.e0;
  const long long MN = (long long)J.M * J.N;
  const bool live = x < MN && !(J.herm && (x % J.N) > (x / J.N));
  float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
  if (live) {
    constexpr int U = 8;                              // loads in flight per thread
    for (int k0 = sub; k0 < J.ks; k0 += U * split) {
      float4 w[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int kz = k0 + u * split;
        w[u] = kz < J.ks ? __ldcg(J.part + kz * MN + x) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        dfa(rh, rl, w[u].x);
        rl += w[u].y;
        dfa(ih, il, w[u].z);
        il += w[u].w;
      }
    }
  }
  for (int o = 1; o < split; o <<= 1) {               // the partial sums, fixed order
    const float a = __shfl_xor_sync(0xffffffffu, rh, o), b = __shfl_xor_sync(0xffffffffu, rl, o);
    const float c = __shfl_xor_sync(0xffffffffu, ih, o), d = __shfl_xor_sync(0xffffffffu, il, o);
    dfa(rh, rl, a);
    rl += b;
    dfa(ih, il, c);
    il += d;
  }
  if (!live || sub) return;
  const int i = (int)(x / J.N), j = (int)(x % J.N);
  const float2 re = df_norm(rh, rl), im = df_norm(ih, il);
  if (J.csplit) {
    float4* C4 = reinterpret_cast<float4*>(J.C);
    C4[(long long)i * J.ldc + j] = make_float4(re.x, re.y, im.x, im.y);
    if (J.herm && i > j) C4[(long long)j * J.ldc + i] = make_float4(re.x, re.y, -im.x, -im.y);
  } else {
    double2* Cd = reinterpret_cast<double2*>(J.C);
    const double vr = (double)re.x + (double)re.y, vi = (double)im.x + (double)im.y;
    Cd[(long long)i * J.ldc + j] = make_double2(vr, vi);
    if (J.herm && i > j) Cd[(long long)j * J.ldc + i] = make_double2(vr, -vi);
  }
}

// ---- host helpers -------------------------------------------------------------------------
typedef CUresult (*EncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                             const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                             CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                             CUtensorMapFloatOOBfill);

EncodeFn encode_fn() {
  static const EncodeFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<EncodeFn>(p);
    return static_cast<EncodeFn>(nullptr);
  }();
  return fn;
}

// arena of W bf16 per row, `rows` rows, seven planes; box of 32 k x box_rows rows x 7 planes
int make_arena_map(void* map128, const void* arena, int W, long long rows, int box_rows, int nsl) {
  EncodeFn fn = encode_fn();
  if (!fn) return 1;
  if ((reinterpret_cast<uintptr_t>(arena) & 15) || (W % EK)) return 2;
  cuuint64_t dims[3] = {(cuuint64_t)W, (cuuint64_t)rows, (cuuint64_t)nsl};
  cuuint64_t strides[2] = {(cuuint64_t)W * 2, (cuuint64_t)W * 2 * rows};
  cuuint32_t box[3] = {EK, (cuuint32_t)box_rows, (cuuint32_t)nsl};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = fn(reinterpret_cast<CUtensorMap*>(map128), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3,
                  const_cast<void*>(arena), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : 3;
}

int sm_count() {
  static std::atomic<int> cache[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
  int v = cache[dev].load();
  if (!v) {
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 148;
    cache[dev].store(v);
  }
  return v;
}

struct Lay {
  int sub;
  long long arow, brow, ea, eb, part;
  bool slice_b;
  int tm, tn, nst, ks, kst;
};

// Arena rows, exponent slots and k splits of one launch's products; a B
// operand equal to an earlier product's (same matrix and reading) is sliced
// once.  -1 when a product is not of the sliced form.
int etc_layout(const DfSub* subs, int n, int enc, Lay* L, int& W, long long& rowsA,
               long long& rowsB, long long& expo, long long& part) {
  int np = 0;
  long long arow = 0, brow = 0, eo = 0, pt = 0;
  int T = 0;
  W = 0;
  for (int i = 0; i < n; ++i) {
    const DfSub& u = subs[i];
    if (u.M <= 0 || u.N <= 0) continue;
    if (u.opa != 0 || !u.asplit || !u.bsplit || u.K <= 0 || np >= ETC_MAX) return -1;
    if (u.herm && u.M != u.N) return -1;
    Lay& l = L[np];
    l.sub = i;
    l.arow = arow;
    l.ea = eo;
    eo += u.M;
    arow += pad_to(u.M, EM);
    l.slice_b = true;
    for (int j = 0; j < np; ++j) {
      const DfSub& v = subs[L[j].sub];
      if (v.B == u.B && v.ldb == u.ldb && v.N == u.N && v.K == u.K && v.opb == u.opb) {
        l.brow = L[j].brow;
        l.eb = L[j].eb;
        l.slice_b = false;
        break;
      }
    }
    if (l.slice_b) {
      l.brow = brow;
      l.eb = eo;
      eo += u.N;
      brow += pad_to(u.N, enc) / enc * 2 * enc;
    }
    l.tm = (int)(pad_to(u.M, EM) / EM);
    l.tn = (int)(pad_to(u.N, enc) / enc);
    l.nst = (int)(pad_to(2LL * u.K, EK) / EK);
    W = std::max(W, l.nst * EK);
    T += l.tm * l.tn;
    ++np;
  }
  // k splits: about one CTA per SM over the launch; at most one exactly
  // summed chunk per CTA
  const int per = std::max(1, sm_count() / std::max(1, T));
  for (int q = 0; q < np; ++q) {
    Lay& l = L[q];
    const int ks0 = std::max(std::min(per, l.nst), (l.nst + CHUNK - 1) / CHUNK);
    l.kst = (l.nst + ks0 - 1) / ks0;
    l.ks = (l.nst + l.kst - 1) / l.kst;
    l.part = pt;
    if (l.ks > 1) pt += (long long)l.ks * subs[l.sub].M * subs[l.sub].N;
  }
  rowsA = arow;
  rowsB = brow;
  expo = eo;
  part = pt;
  return np;
}

// slicing jobs of one launch's A operands (kind 0) or B operands (kind 1)
void add_slice_jobs(const EnvTcPlan& P, int slot, const DfSub* subs, const Lay* L, int np, int kind,
                    SlSet& js, long long& blocks) {
  __nv_bfloat16* arena =
      reinterpret_cast<__nv_bfloat16*>(kind == 0 ? P.arenaA[slot] : P.arenaB[slot]);
  const long long plane = (long long)P.W[slot] * (kind == 0 ? P.rowsA[slot] : P.rowsB[slot]);
  for (int q = 0; q < np; ++q) {
    const Lay& l = L[q];
    const DfSub& u = subs[l.sub];
    if (kind == 1 && !l.slice_b) continue;
    SlJob J;
    J.K = u.K;
    J.kind = kind;
    J.arena = arena;
    J.plane = plane;
    J.W = P.W[slot];
    J.enc = P.enc;
    J.b0 = blocks;
    if (kind == 0) {
      J.src = reinterpret_cast<const float4*>(u.A);
      J.ld = u.lda; J.es = 1; J.conj = 0;
      J.rows = u.M;
      J.dst = l.arow;
      J.expo = P.expo[slot] + l.ea;
    } else {
      J.src = reinterpret_cast<const float4*>(u.B);
      if (u.opb == 0) { J.ld = 1; J.es = u.ldb; J.conj = 0; }       // column j: stride ldb
      else { J.ld = u.ldb; J.es = 1; J.conj = 1; }                  // B = Y^dag: conj(row j of Y)
      J.rows = u.N;
      J.dst = l.brow;
      J.expo = P.expo[slot] + l.eb;
    }
    js.j[js.n++] = J;
    blocks += (long long)J.rows * ((J.K + SL_K - 1) / SL_K);
  }
}

// every launch of a step is a programmatic dependent of the one before it
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kern)(KArgs...), unsigned grid, unsigned block, size_t smem,
                       cudaStream_t s, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

cudaError_t launch_slices(const SlSet& js, long long blocks, int nsl, cudaStream_t s) {
  if (js.n == 0 || blocks == 0) return cudaSuccess;
  COUNT_LAUNCH(1);
  if (nsl == 8) return launch_pdl(etc_slice_kernel<8>, (unsigned)blocks, SL_THREADS, 0, s, js);
  if (nsl == 7) return launch_pdl(etc_slice_kernel<7>, (unsigned)blocks, SL_THREADS, 0, s, js);
  return cudaErrorInvalidValue;
}

template <class CF>
cudaError_t launch_gemm(const EnvTcPlan& P, int slot, const DfSub* subs, const Lay* L, int np,
                        int* status, cudaStream_t s, double& fl, double& by) {
  static std::atomic<int> attr_set[64];
  EtcGroup G;
  RedSet rs;
  G.np = np;
  rs.n = 0;
  long long units = 0, elems = 0;
  int maxks = 1;
  for (int q = 0; q < np; ++q) {
    const Lay& l = L[q];
    const DfSub& u = subs[l.sub];
    EtcProb& p = G.p[q];
    p.M = u.M; p.N = u.N; p.nst = l.nst;
    p.arow = l.arow; p.brow = l.brow;
    p.ea = P.expo[slot] + l.ea;
    p.eb = P.expo[slot] + l.eb;
    p.C = u.C; p.ldc = u.ldc; p.herm = u.herm; p.csplit = u.csplit;
    p.tm = l.tm; p.tn = l.tn; p.ks = l.ks; p.kst = l.kst;
    p.u0 = units;
    p.part = P.work + l.part;
    units += (long long)l.tm * l.tn * l.ks;
    if (l.ks > 1) {
      rs.j[rs.n++] = RedJob{p.part, l.ks, u.M, u.N, u.C, u.ldc, u.herm, u.csplit, elems};
      maxks = std::max(maxks, l.ks);
      elems += (long long)u.M * u.N;
    }
    fl += 8.0 * u.M * (u.herm ? (u.N + 1) / 2.0 : (double)u.N) * u.K;
    by += 16.0 * ((double)u.M * u.K + (double)u.K * u.N + (double)u.M * u.N);
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!attr_set[dev].load()) {
    e = cudaFuncSetAttribute(envtc_kernel<CF>, cudaFuncAttributeMaxDynamicSharedMemorySize, CF::SMEM);
    if (e) return e;
    attr_set[dev].store(1);
  }
  CUtensorMap ma, mb;
  memcpy(&ma, P.mapA[slot], sizeof(CUtensorMap));
  memcpy(&mb, P.mapB[slot], sizeof(CUtensorMap));
  e = launch_pdl(envtc_kernel<CF>, (unsigned)units, E_THREADS, CF::SMEM, s, ma, mb, G, status);
  COUNT_LAUNCH(1);
  if (e) return e;
  if (rs.n) {
    // threads per output: enough loads in flight for the longest k split
    const int split = maxks >= 16 ? 4 : maxks >= 8 ? 2 : 1;
    const long long thr = elems * split;
    e = launch_pdl(etc_reduce_kernel, (unsigned)((thr + RED_THREADS - 1) / RED_THREADS), RED_THREADS, 0,
                   s, rs, split);
    COUNT_LAUNCH(1);
  }
  return e;
}

cudaError_t launch_gemm_any(const EnvTcPlan& P, int slot, const DfSub* subs, const Lay* L, int np,
                            int* status, cudaStream_t s, double& fl, double& by) {
  if (P.enc == CfgExact::ENC) return launch_gemm<CfgExact>(P, slot, subs, L, np, status, s, fl, by);
  if (P.enc == CfgWide::ENC) return launch_gemm<CfgWide>(P, slot, subs, L, np, status, s, fl, by);
  return cudaErrorInvalidValue;
}

}  // namespace

// ---- host side ------------------------------------------------------------------------------
void envtc_needs(const DfSub* s1, int n1, const DfSub* s2, int n2, int enc, EtcNeeds* acc) {
  Lay L[ETC_MAX];
  const DfSub* s[2] = {s1, s2};
  const int n[2] = {n1, n2};
  for (int k = 0; k < 2; ++k) {
    int W;
    long long ra, rb, ex, pt;
    if (etc_layout(s[k], n[k], enc, L, W, ra, rb, ex, pt) < 0) {
      acc->ok = false;
      continue;
    }
    acc->W[k] = std::max(acc->W[k], W);
    acc->rowsA[k] = std::max(acc->rowsA[k], ra);
    acc->rowsB[k] = std::max(acc->rowsB[k], rb);
    acc->expo[k] = std::max(acc->expo[k], ex);
    acc->part = std::max(acc->part, pt);
  }
}

int envtc_slices(int enc) { return enc == CfgExact::ENC ? CfgExact::NSL : CfgWide::NSL; }

size_t envtc_arena_bytes(int W, long long rows, int nsl) {
  return sizeof(__nv_bfloat16) * (size_t)pad_to(std::max(W, EK), EK) *
             (size_t)pad_to(std::max<long long>(rows, EM), EM) * nsl + 256;
}

int envtc_setup(EnvTcPlan* P, int slot, int W, long long rowsA, long long rowsB, void* arenaA,
                void* arenaB) {
  if (slot < 0 || slot > 1 || (P->enc != CfgExact::ENC && P->enc != CfgWide::ENC) ||
      P->nsl != envtc_slices(P->enc))
    return 1;
  P->W[slot] = (int)pad_to(std::max(W, EK), EK);
  P->rowsA[slot] = pad_to(std::max<long long>(rowsA, EM), EM);
  P->rowsB[slot] = pad_to(std::max<long long>(rowsB, EM), EM);
  P->arenaA[slot] = arenaA;
  P->arenaB[slot] = arenaB;
  if (make_arena_map(P->mapA[slot], arenaA, P->W[slot], P->rowsA[slot], EM, P->nsl)) return 2;
  if (make_arena_map(P->mapB[slot], arenaB, P->W[slot], P->rowsB[slot], 2 * P->enc, P->nsl)) return 3;
  return 0;
}

// One environment step: X = Ahat R (products s1), R_m = X Ahat^dag (s2).
// Launches, each a programmatic dependent of the one before: slices of s1's
// operands and of s2's B (Ahat rows, independent of X), the first GEMM (and
// its k-split reduction), slices of X, the second GEMM (and reduction).
// cudaErrorNotSupported (nothing enqueued) when a product does not fit the
// plan; the caller then takes the double-float GEMM.
cudaError_t launch_envtc_step(const EnvTcPlan& P, const DfSub* s1, int n1, const DfSub* s2, int n2,
                              int* status, cudaStream_t s) {
  Lay L1[ETC_MAX], L2[ETC_MAX];
  int W1, W2;
  long long ra1, rb1, ex1, pt1, ra2, rb2, ex2, pt2;
  const int np1 = etc_layout(s1, n1, P.enc, L1, W1, ra1, rb1, ex1, pt1);
  const int np2 = etc_layout(s2, n2, P.enc, L2, W2, ra2, rb2, ex2, pt2);
  if (np1 < 0 || np2 < 0 || W1 > P.W[0] || W2 > P.W[1] || ra1 > P.rowsA[0] || rb1 > P.rowsB[0] ||
      ra2 > P.rowsA[1] || rb2 > P.rowsB[1] || ex1 > P.expo_cap[0] || ex2 > P.expo_cap[1] ||
      pt1 > P.work_cap || pt2 > P.work_cap)
    return cudaErrorNotSupported;
  // traced per product pass: its slicing, GEMM and k-split reduction
  SlSet js;
  long long blocks = 0;
  double fl = 0.0, by = 0.0;
  js.n = 0;
  add_slice_jobs(P, 0, s1, L1, np1, 0, js, blocks);
  add_slice_jobs(P, 0, s1, L1, np1, 1, js, blocks);
  add_slice_jobs(P, 1, s2, L2, np2, 1, js, blocks);
  cudaEvent_t tr0 = g_env_trace.begin(s);
  cudaError_t e = launch_slices(js, blocks, P.nsl, s);
  if (!e && np1) e = launch_gemm_any(P, 0, s1, L1, np1, status, s, fl, by);
  g_env_trace.end(tr0, s, fl, by);
  if (e) return e;
  js.n = 0;
  blocks = 0;
  fl = by = 0.0;
  add_slice_jobs(P, 1, s2, L2, np2, 0, js, blocks);
  tr0 = g_env_trace.begin(s);
  e = launch_slices(js, blocks, P.nsl, s);
  if (!e && np2) e = launch_gemm_any(P, 1, s2, L2, np2, status, s, fl, by);
  g_env_trace.end(tr0, s, fl, by);
  return e;
}
