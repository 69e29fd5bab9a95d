// Complex GEMM in double-float arithmetic on the FP32 pipes.
//
// The right environments R_m = sum_p A^m[p] R_{m+1} A^m[p]^dag are a chain of
// N dependent products; the norm of the state is R_0, so a one-sided error
// per step (the tensor cores' FP32 accumulation) compounds over the chain.
// GB300 runs FP64 at a small fraction of its FP32 rate, so these products use
// double-float numbers x = hi + lo (two FP32 words, ~44 significant bits):
// every real multiply-add forms the product exactly with FMA (p = ah bh,
// e = fma(ah, bh, -p) + ah bl + al bh) and adds it with Knuth's TwoSum.
// Operands are read as stored pairs, or in FP64 and split into (hi, lo) on
// the way to shared memory; partial sums over k-chunks (split-K, for
// parallelism in the short sequential products) are written as pairs and
// summed in k order by the last CTA of each output tile.  Tiles of
// TM x TN complex outputs (16 to 64 square), 8 complex k per stage, 256
// threads.  Two drivers: a grouped launch of many independent products (one
// environment step of one state on its parity blocks), and a persistent
// cooperative kernel that runs the whole chains of a batch of states.
#include "internal.h"
#include <algorithm>
#include <cooperative_groups.h>
#include <array>
#include <map>
#include <mutex>

namespace cg = cooperative_groups;

namespace {

constexpr int DK = 8;                         // k per shared-memory stage

struct Df { float h, l; };

__device__ __forceinline__ void df_mac(float& h, float& l, float xh, float xl, float yh, float yl) {
  const float p = xh * yh;
  float e = fmaf(xh, yh, -p);
  e = fmaf(xh, yl, e);
  e = fmaf(xl, yh, e);
  const float t = h + p;
  const float v = t - h;
  const float err = (h - (t - v)) + (p - v);
  l += err + e;
  h = t;
}

// s + e = h + l exactly (TwoSum), s = fl(h + l): a normalised pair
__device__ __forceinline__ void df_norm(float h, float l, float& s, float& e) {
  s = h + l;
  const float v = s - h;
  e = (h - (s - v)) + (l - v);
}
// (h, l) += (xh, xl) in double-float arithmetic (TwoSum on the high words)
__device__ __forceinline__ void df_acc(float& h, float& l, float xh, float xl) {
  const float t = h + xh;
  const float v = t - h;
  const float err = (h - (t - v)) + (xh - v);
  l += err + xl;
  h = t;
}

__device__ __forceinline__ Df df_split(double x) {
  Df r;
  r.h = (float)x;
  r.l = (float)(x - (double)r.h);
  return r;
}

// one 64 x 64 complex output tile of C = op(A) op(B) over k in [kbeg, kend),
// written to C[gi * ldc + gj] (the whole CTA calls it together)
struct DfTile {
  int M, N, opa, opb;
  const double2* A; long long lda;
  const double2* B; long long ldb;
  double2* C; long long ldc;
  int herm = 0;     // Hermitian C: only elements i >= j are stored from this tile...
  int mirror = 0;   // ...and, if set, C[j][i] = conj(C[i][j]) for i > j as well
  int asplit = 0, bsplit = 0, csplit = 0;   // stored as double-float pairs (df_pack)
};

// TM x TN tile on 16 x 16 threads, (TM/16) x (TN/16) outputs each.  Every
// output sums k in the same order whatever the tile shape, so the result does
// not depend on it (the shape is a pure performance choice).  Stages of DK k
// run through two shared-memory buffers: the next stage's operands are read
// into registers before the current stage's arithmetic and stored to the
// other buffer after it, so one barrier per stage suffices.
template <int TM, int TN, int SK = DK>
__device__ __forceinline__ void df_tile(const DfTile& p, int i0, int j0, int kbeg, int kend,
                                        float (*As)[SK][TM + 1][4], float (*Bs)[SK][TN + 1][4]) {
  constexpr int RM = TM / 16, RN = TN / 16;
  constexpr int NA = (SK * TM + 255) / 256, NB = (SK * TN + 255) / 256;   // elements per thread
  // Hermitian result: a tile strictly above the diagonal is never needed
  // (its elements are the mirrors of lower ones), whatever the tile shape
  if (p.herm && i0 + TM - 1 < j0) return;
  const double2* A = p.A;
  const double2* B = p.B;
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  float ah[RM][RN][2], al[RM][RN][2];   // [row][col][re/im] hi and lo accumulators
#pragma unroll
  for (int r = 0; r < RM; ++r)
#pragma unroll
    for (int c = 0; c < RN; ++c) {
      ah[r][c][0] = ah[r][c][1] = 0.f;
      al[r][c][0] = al[r][c][1] = 0.f;
    }
  // Each thread's share of a stage: fixed (row, k) slots of the A and B
  // tiles.  Their addresses, shared-memory places and row bounds are set
  // once here; a stage only advances the pointers by SK k.
  float4 ra[NA], rb[NB];
  const float4* pa[NA];
  const double2* pa64[NA];
  long long sa[NA];                          // element step per stage
  int ka[NA], sta[NA];                       // k within the stage; shared-memory slot (kk * (TM + 1) + ii)
  bool va[NA];
#pragma unroll
  for (int q = 0; q < NA; ++q) {
    const int e = tid + 256 * q;
    int kk = 0, ii = 0;
    if (p.opa == 0) { ii = e / SK; kk = e % SK; } else { kk = e / TM; ii = e % TM; }
    const int gi = i0 + ii;
    va[q] = e < SK * TM && gi < p.M;
    ka[q] = kk;
    sta[q] = kk * (TM + 1) + ii;
    const long long at = va[q] ? (p.opa == 0 ? (long long)gi * p.lda + kbeg + kk
                                             : (long long)(kbeg + kk) * p.lda + gi)
                               : 0;
    sa[q] = p.opa == 0 ? SK : (long long)SK * p.lda;
    pa[q] = reinterpret_cast<const float4*>(A) + at;
    pa64[q] = A + at;
  }
  const float4* pb[NB];
  const double2* pb64[NB];
  long long sb[NB];
  int kb[NB], stb[NB];
  bool vb[NB];
#pragma unroll
  for (int q = 0; q < NB; ++q) {
    const int e = tid + 256 * q;
    int kk = 0, jj = 0;
    if (p.opb == 0) { kk = e / TN; jj = e % TN; } else { jj = e / SK; kk = e % SK; }
    const int gj = j0 + jj;
    vb[q] = e < SK * TN && gj < p.N;
    kb[q] = kk;
    stb[q] = kk * (TN + 1) + jj;
    const long long at = vb[q] ? (p.opb == 0 ? (long long)(kbeg + kk) * p.ldb + gj
                                             : (long long)gj * p.ldb + kbeg + kk)
                               : 0;
    sb[q] = p.opb == 0 ? (long long)SK * p.ldb : SK;
    pb[q] = reinterpret_cast<const float4*>(B) + at;
    pb64[q] = B + at;
  }
  const bool nega = p.opa != 0, negb = p.opb != 0;
  // operands of the stage starting at k0 (stage index st = (k0 - kbeg) / SK)
  auto load = [&](int k0, long long st) {
#pragma unroll
    for (int q = 0; q < NA; ++q) {
      float4 w = make_float4(0.f, 0.f, 0.f, 0.f);
      if (va[q] && k0 + ka[q] < kend) {
        if (p.asplit) {
          w = pa[q][st * sa[q]];
        } else {
          const double2 v = pa64[q][st * sa[q]];
          const Df re = df_split(v.x), im = df_split(v.y);
          w = make_float4(re.h, re.l, im.h, im.l);
        }
        if (nega) { w.z = -w.z; w.w = -w.w; }
      }
      ra[q] = w;
    }
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      float4 w = make_float4(0.f, 0.f, 0.f, 0.f);
      if (vb[q] && k0 + kb[q] < kend) {
        if (p.bsplit) {
          w = pb[q][st * sb[q]];
        } else {
          const double2 v = pb64[q][st * sb[q]];
          const Df re = df_split(v.x), im = df_split(v.y);
          w = make_float4(re.h, re.l, im.h, im.l);
        }
        if (negb) { w.z = -w.z; w.w = -w.w; }
      }
      rb[q] = w;
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int q = 0; q < NA; ++q)
      if (tid + 256 * q < SK * TM) *reinterpret_cast<float4*>(&As[buf][0][0][0] + 4 * sta[q]) = ra[q];
#pragma unroll
    for (int q = 0; q < NB; ++q)
      if (tid + 256 * q < SK * TN) *reinterpret_cast<float4*>(&Bs[buf][0][0][0] + 4 * stb[q]) = rb[q];
  };
  if (kbeg < kend) {
    load(kbeg, 0);
    store(0);
  }
  __syncthreads();
  int buf = 0;
  long long st = 0;
  for (int k0 = kbeg; k0 < kend; k0 += SK, buf ^= 1, ++st) {
    const bool more = k0 + SK < kend;
    if (more) load(k0 + SK, st + 1);         // in flight during the arithmetic below
#pragma unroll 2
    for (int kk = 0; kk < SK; ++kk) {
      float a[RM][4], b[RN][4];
#pragma unroll
      for (int r = 0; r < RM; ++r) {
        const float4 v = *reinterpret_cast<const float4*>(&As[buf][kk][ty + 16 * r][0]);
        a[r][0] = v.x; a[r][1] = v.y; a[r][2] = v.z; a[r][3] = v.w;
      }
#pragma unroll
      for (int c = 0; c < RN; ++c) {
        const float4 v = *reinterpret_cast<const float4*>(&Bs[buf][kk][tx + 16 * c][0]);
        b[c][0] = v.x; b[c][1] = v.y; b[c][2] = v.z; b[c][3] = v.w;
      }
#pragma unroll
      for (int r = 0; r < RM; ++r)
#pragma unroll
        for (int c = 0; c < RN; ++c) {
          // re += ar br - ai bi ; im += ar bi + ai br
          df_mac(ah[r][c][0], al[r][c][0], a[r][0], a[r][1], b[c][0], b[c][1]);
          df_mac(ah[r][c][0], al[r][c][0], -a[r][2], -a[r][3], b[c][2], b[c][3]);
          df_mac(ah[r][c][1], al[r][c][1], a[r][0], a[r][1], b[c][2], b[c][3]);
          df_mac(ah[r][c][1], al[r][c][1], a[r][2], a[r][3], b[c][0], b[c][1]);
        }
    }
    // the other buffer was last read before the previous barrier
    if (more) store(buf ^ 1);
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < RM; ++r) {
    const int gi = i0 + ty + 16 * r;
    if (gi >= p.M) continue;
#pragma unroll
    for (int c = 0; c < RN; ++c) {
      const int gj = j0 + tx + 16 * c;
      if (gj >= p.N) continue;
      if (p.herm && gi < gj) continue;
      if (p.csplit) {                             // normalised pairs, no FP64 arithmetic
        float4 w;
        df_norm(ah[r][c][0], al[r][c][0], w.x, w.y);
        df_norm(ah[r][c][1], al[r][c][1], w.z, w.w);
        if (p.herm && p.mirror && gi > gj)
          reinterpret_cast<float4*>(p.C)[(long long)gj * p.ldc + gi] = make_float4(w.x, w.y, -w.z, -w.w);
        reinterpret_cast<float4*>(p.C)[(long long)gi * p.ldc + gj] = w;
      } else {
        const double2 v = make_double2((double)ah[r][c][0] + (double)al[r][c][0],
                                       (double)ah[r][c][1] + (double)al[r][c][1]);
        if (p.herm && p.mirror && gi > gj) p.C[(long long)gj * p.ldc + gi] = cconj(v);
        p.C[(long long)gi * p.ldc + gj] = v;
      }
    }
  }
}

// Many independent products C_i = op(A_i) op(B_i) in one launch (the blocks
// of a parity-compact environment step).  CTAs are dealt to the products in
// order (c0 = first CTA of a product); each product has its own tile grid and
// k split.  A CTA of a split product writes its partial tile as double-float
// pairs to the workspace, then takes a ticket from the tile's counter; the
// CTA that draws the last ticket sums the tile's partials in k order
// (double-float additions), writes the output and resets the counter, so no
// FP64 arithmetic and no second launch are needed.  No CTA waits for another.
constexpr int DFG_MAX = 40;
struct DfProb {
  DfTile t;                 // operands, dims, ops; C / ldc = the final output
  int K, ksplit, kchunk, tn;
  long long c0;             // first CTA of this product
  long long part;           // its partials in the workspace (ksplit > 1), in complex elements
  int cbase;                // its tile counters (ksplit > 1)
};
struct DfGroup {
  int np;
  float4* work;             // partials, one pair of pairs per complex element
  int* cnt;                 // tile counters: zero between launches
  DfProb p[DFG_MAX];
};

constexpr int RED_ILP = 4;                    // partial loads in flight per thread in a tile's reduction

// Resident CTAs per SM the register allocation is held to (measured for the
// 144-mode chi = 256 chain with 16 x 16 tiles: 4, 5, 6, 8 CTAs give 18.7,
// 17.3, 16.5, 17.8 ms)

template <int TM, int TN, int SK>
__global__ void __launch_bounds__(256, TM == 16 ? 6 : (TM == 32 ? 4 : 2)) zgemm_df64_grouped_kernel(const __grid_constant__ DfGroup g) {
  __shared__ __align__(16) float As[2][SK][TM + 1][4];
  __shared__ __align__(16) float Bs[2][SK][TN + 1][4];
  __shared__ int last;
  const long long b = blockIdx.x;
  int lo = 0, hi = g.np - 1;
  while (lo < hi) {                           // last product with c0 <= b
    const int mid = (lo + hi + 1) >> 1;
    if (g.p[mid].c0 <= b) lo = mid; else hi = mid - 1;
  }
  const DfProb& P = g.p[lo];
  const long long l = b - P.c0;
  const int kz = (int)(l % P.ksplit);
  const long long tl = l / P.ksplit;
  const int i0 = (int)(tl / P.tn) * TM, j0 = (int)(tl % P.tn) * TN;
  const int kbeg = kz * P.kchunk, kend = min(P.K, kbeg + P.kchunk);
  DfTile t = P.t;
  const bool split = P.ksplit > 1;
  const long long MN = (long long)t.M * t.N;
  if (split) {
    t.C = reinterpret_cast<double2*>(g.work + P.part + (long long)kz * MN);
    t.ldc = t.N;
    t.mirror = 0;
    t.csplit = 1;
  }
  df_tile<TM, TN, SK>(t, i0, j0, kbeg, kend, As, Bs);
  if (!split || (t.herm && i0 + TM - 1 < j0)) return;   // (a tile above a Hermitian diagonal: unused)
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(g.cnt + P.cbase + tl, 1) == P.ksplit - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  const DfTile& o = P.t;
  for (int e = threadIdx.x; e < TM * TN; e += blockDim.x) {
    const int gi = i0 + e / TN, gj = j0 + e % TN;
    if (gi >= o.M || gj >= o.N || (o.herm && gi < gj)) continue;
    const float4* src = g.work + P.part + (long long)gi * o.N + gj;
    float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
    for (int k0 = 0; k0 < P.ksplit; k0 += RED_ILP) {   // RED_ILP loads in flight, summed in k order
      float4 w[RED_ILP];
#pragma unroll
      for (int k = 0; k < RED_ILP; ++k)
        w[k] = k0 + k < P.ksplit ? __ldcg(src + (long long)(k0 + k) * MN) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int k = 0; k < RED_ILP; ++k) {
        if (k0 + k >= P.ksplit) break;
        df_acc(rh, rl, w[k].x, w[k].y);
        df_acc(ih, il, w[k].z, w[k].w);
      }
    }
    if (o.csplit) {
      float4 w;
      df_norm(rh, rl, w.x, w.y);
      df_norm(ih, il, w.z, w.w);
      float4* C4 = reinterpret_cast<float4*>(o.C);
      C4[(long long)gi * o.ldc + gj] = w;
      if (o.herm && gi > gj) C4[(long long)gj * o.ldc + gi] = make_float4(w.x, w.y, -w.z, -w.w);
    } else {
      const double2 v = make_double2((double)rh + (double)rl, (double)ih + (double)il);
      o.C[(long long)gi * o.ldc + gj] = v;
      if (o.herm && gi > gj) o.C[(long long)gj * o.ldc + gi] = cconj(v);
    }
  }
  if (threadIdx.x == 0) g.cnt[P.cbase + tl] = 0;
}

// Right-environment chains of many states in one persistent cooperative
// launch.  Step k handles site m = N_s - 1 - k of every state s with N_s > k:
// phase 0: X_s = Ahat^m (D_m d x D_{m+1}) R^{m+1}; phase 1: R^m = X_s
// (D_m x d D_{m+1}) Ahat^m^dag.  The output tiles of all states in a phase are
// dealt round-robin to the CTAs, and a grid-wide barrier separates phases
// (all CTAs are co-resident by construction of the cooperative launch).
template <int TM, int TN>
__global__ void __launch_bounds__(256) env_chain_kernel(const EnvJob* __restrict__ jobs, int count,
                                                       int maxN) {
  // rows padded by one 16-byte element: the k-major fills of A (and of B^dag)
  // then fall into different banks
  __shared__ __align__(16) float As[2][DK][TM + 1][4];
  __shared__ __align__(16) float Bs[2][DK][TN + 1][4];
  cg::grid_group grid = cg::this_grid();
  for (int k = 0; k < maxN; ++k) {
    for (int phase = 0; phase < 2; ++phase) {
      long long base = 0, t = blockIdx.x;
      for (int j = 0; j < count; ++j) {
        const EnvJob J = jobs[j];
        if (k >= J.N) continue;
        const int m = J.N - 1 - k;
        // parity blocks: phase 0 per class c and p, phase 1 per class c
        const int kl[2] = {J.pc[2 * m], J.pc[2 * m + 1]};
        const int kr[2] = {J.pc[2 * m + 2], J.pc[2 * m + 3]};
        const int Dr = kr[0] + kr[1];
        const long long Kc[2] = {pk_len(J.d, kr, 0), pk_len(J.d, kr, 1)};
        const long long o1 = (long long)kl[0] * Kc[0];
        const double2* A = J.Ah + J.toff[m];
        const int nsub = phase == 0 ? 2 * J.d : 2;
        for (int q = 0; q < nsub; ++q) {
          DfTile p;
          int K;
          if (phase == 0) {
            const int c = q / J.d, pp = q % J.d, cr = c ^ (pp & 1);
            const long long off = (c ? o1 : 0) + pk_off(pp, Dr, kr, c);
            p = DfTile{kl[c], kr[cr], 0, 0, A + off, Kc[c],
                       J.R + J.eoff[m + 1] + (cr ? (long long)kr[0] * kr[0] : 0), kr[cr], J.X + off,
                       Kc[c]};
            p.asplit = 1;                                    // Ahat, R and X as pairs
            p.bsplit = 1;
            p.csplit = 1;
            K = kr[cr];
          } else {
            const int c = q;
            const long long off = c ? o1 : 0;
            p = DfTile{kl[c], kl[c], 0, 1, J.X + off, Kc[c], A + off, Kc[c],
                       J.R + J.eoff[m] + (c ? (long long)kl[0] * kl[0] : 0), kl[c], 1, 1};
            p.asplit = 1;
            p.bsplit = 1;
            p.csplit = m > 0 ? 1 : 0;                        // R^0 (the squared norm) in FP64
            K = (int)Kc[c];                                  // R^m is Hermitian
          }
          if (p.M <= 0 || p.N <= 0) continue;
          const long long tn = (p.N + TN - 1) / TN;
          const long long nt = ((p.M + TM - 1) / TM) * tn;
          for (; t < base + nt; t += gridDim.x) {
            const long long l = t - base;
            df_tile<TM, TN>(p, (int)(l / tn) * TM, (int)(l % tn) * TN, 0, K, As, Bs);
          }
          base += nt;
        }
      }
      grid.sync();
    }
  }
}

}  // namespace


cudaError_t launch_zgemm_df64_grouped(const DfSub* subs, int n, cudaStream_t s, void* work,
                                      size_t work_bytes) {
  // SM count of the current device, cached per device index
  static std::atomic<int> nsm_cache[64];
  int dev = 0;
  cudaError_t ed = cudaGetDevice(&dev);
  if (ed) return ed;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  int nsm = nsm_cache[dev].load();
  if (!nsm) {
    ed = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (ed) return ed;
    nsm_cache[dev].store(nsm);
  }
  std::vector<DfSub> live;
  for (int i = 0; i < n; ++i)
    if (subs[i].M > 0 && subs[i].N > 0) live.push_back(subs[i]);
  for (size_t g0 = 0; g0 < live.size(); g0 += DFG_MAX) {
    const int np = (int)std::min<size_t>(DFG_MAX, live.size() - g0);
    // tile shape: the largest of 64, 32 and 16 square that still gives two
    // waves of tiles (16 x 16 for the 144-mode chi = 256 chain: 19.6 ms
    // against 20.2 ms with 32 x 32)
    long long t64 = 0, t32 = 0;
    for (int i = 0; i < np; ++i) {
      const DfSub& u = live[g0 + i];
      t64 += (long long)((u.M + 63) / 64) * ((u.N + 63) / 64);
      t32 += (long long)((u.M + 31) / 32) * ((u.N + 31) / 32);
    }
    // Knobs.  GBSMPS_DFG_TILE = 16, 32 or 64 forces the tile shape, a pure
    // performance choice: every output sums k in the same order and the k
    // split below does not depend on it.  GBSMPS_DFG_WAVES (CTA target in
    // multiples of the SM count) and GBSMPS_DFG_MINK (least k chunk, in
    // stages of DK) set the k split, and with it the FP64 partial sums'
    // grouping: deterministic for each setting, equal to within rounding
    // across settings.
    auto knob = [](const char* name, int dflt) {
      const char* e = getenv(name);
      return e ? atoi(e) : dflt;
    };
    const int env_tile = knob("GBSMPS_DFG_TILE", 0);
    const int env_waves = std::max(1, knob("GBSMPS_DFG_WAVES", 4));
    const int env_mink = std::max(1, knob("GBSMPS_DFG_MINK", 4));
    // k per shared-memory stage of the 16 x 16 tiles (GBSMPS_DFG_SK = 8 or 16;
    // the k order of every sum is the same)
    const int env_sk = knob("GBSMPS_DFG_SK", 8) == 16 ? 16 : 8;
    const int T = env_tile == 16 || env_tile == 32 || env_tile == 64
                      ? env_tile
                      : (t64 >= 2LL * nsm ? 64 : (t32 >= 2LL * nsm ? 32 : 16));
    long long tref = 0;                           // the k split follows a fixed 32 x 32 tiling
    for (int i = 0; i < np; ++i) {
      const DfSub& u = live[g0 + i];
      tref += (long long)((u.M + 31) / 32) * ((u.N + 31) / 32);
    }
    // k split toward four waves of CTAs of the 32 x 32 reference tiling
    // (144-mode chain: 29 ms at two waves with the first form of this
    // kernel; now 16.9 ms at four against 17.1 at eight), chunks of >= 4
    // stages, within the workspace
    int target = (int)std::max<long long>(1, ((long long)env_waves * nsm + tref - 1) / tref);
    DfGroup G;
    G.np = np;
    // workspace: tile counters (zeroed by the caller once), then partials
    if (work && work_bytes <= DFG_CNT_BYTES) return cudaErrorInvalidValue;
    G.cnt = reinterpret_cast<int*>(work);
    G.work = work ? reinterpret_cast<float4*>(static_cast<char*>(work) + DFG_CNT_BYTES) : nullptr;
    const size_t part_bytes = work ? work_bytes - DFG_CNT_BYTES : 0;
    for (;;) {
      long long c0 = 0, part = 0, ncnt = 0;
      for (int i = 0; i < np; ++i) {
        const DfSub& u = live[g0 + i];
        DfProb& P = G.p[i];
        P.t = DfTile{u.M, u.N, u.opa, u.opb, u.A, u.lda, u.B, u.ldb, u.C, u.ldc, u.herm, u.herm,
                     u.asplit, u.bsplit, u.csplit};
        P.K = u.K;
        int ks = std::max(1, std::min(target, u.K / (env_mink * DK)));
        if (!work) ks = 1;
        int kchunk = u.K > 0 ? ((u.K + ks - 1) / ks + DK - 1) / DK * DK : DK;
        ks = u.K > 0 ? (u.K + kchunk - 1) / kchunk : 1;
        P.ksplit = ks;
        P.kchunk = kchunk;
        P.tn = (u.N + T - 1) / T;
        P.c0 = c0;
        P.part = part;
        P.cbase = (int)ncnt;
        const long long tiles = (long long)((u.M + T - 1) / T) * P.tn;
        c0 += tiles * ks;
        if (ks > 1) {
          part += (long long)ks * u.M * u.N;
          ncnt += tiles;
        }
      }
      const bool fits = (size_t)part * sizeof(float4) <= part_bytes &&
                        (size_t)ncnt * sizeof(int) <= DFG_CNT_BYTES;
      if (fits || target == 1) {
        if (!fits) return cudaErrorInvalidValue;
        if (c0 > 0x7fffffffLL) return cudaErrorInvalidValue;
        double fl = 0.0, by = 0.0;               // algorithmic work, for the trace
        for (int i = 0; i < np; ++i) {
          const DfSub& u = live[g0 + i];
          const double outs = u.herm ? 0.5 * u.M * (u.M + 1.0) : (double)u.M * u.N;
          fl += 8.0 * outs * u.K;
          by += 16.0 * ((double)u.M * u.K + (double)u.K * u.N + outs);
        }
        cudaEvent_t tr0 = g_env_trace.begin(s);
        if (T == 64)
          zgemm_df64_grouped_kernel<64, 64, DK><<<(unsigned)c0, 256, 0, s>>>(G);
        else if (T == 32)
          zgemm_df64_grouped_kernel<32, 32, DK><<<(unsigned)c0, 256, 0, s>>>(G);
        else if (env_sk == 8)
          zgemm_df64_grouped_kernel<16, 16, 8><<<(unsigned)c0, 256, 0, s>>>(G);
        else
          zgemm_df64_grouped_kernel<16, 16, 16><<<(unsigned)c0, 256, 0, s>>>(G);
        g_env_trace.end(tr0, s, fl, by);
        COUNT_LAUNCH(1);
        break;
      }
      target = std::max(1, target / 2);
    }
    cudaError_t e = cudaGetLastError();
    if (e) return e;
  }
  return cudaSuccess;
}

namespace {

template <int TM, int TN>
cudaError_t env_chain_launch(const EnvJob* jobs_dev, int count, int maxN, cudaStream_t s) {
  int dev = 0, nsm = 0, per = 0, coop = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e) return e;
  if ((e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev))) return e;
  if (!coop) return cudaErrorNotSupported;
  if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev))) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, env_chain_kernel<TM, TN>, 256, 0)))
    return e;
  if (per < 1) return cudaErrorInvalidConfiguration;
  void* args[] = {(void*)&jobs_dev, (void*)&count, (void*)&maxN};
  e = cudaLaunchCooperativeKernel((const void*)env_chain_kernel<TM, TN>, dim3(nsm * per), dim3(256),
                                  args, 0, s);
  COUNT_LAUNCH(1);
  return e;
}

cudaError_t env_chain_cfg(int cfg, const EnvJob* jobs_dev, int count, int maxN, cudaStream_t s) {
  switch (cfg) {
    case 0: return env_chain_launch<64, 64>(jobs_dev, count, maxN, s);
    case 1: return env_chain_launch<32, 64>(jobs_dev, count, maxN, s);
    default: return env_chain_launch<32, 32>(jobs_dev, count, maxN, s);
  }
}

// tile-shape choices per batch class (count, largest bond, longest chain,
// each rounded up to a power of two), measured on the first batch of a class
std::mutex g_tune_mu;
std::map<std::array<int, 3>, int> g_tune;

int pow2(int x) { int r = 1; while (r < x) r <<= 1; return r; }

}  // namespace

int env_chain_tile_configs() { return 3; }

cudaError_t launch_env_chain_batch(const EnvJob* jobs_dev, int count, int maxN, int maxD, int cfg,
                                   cudaStream_t s, int* chosen) {
  if (count <= 0 || maxN <= 0) return cudaSuccess;
  if (cfg < 0) {
    const std::array<int, 3> key{pow2(count), pow2(maxD), pow2(maxN)};
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      auto it = g_tune.find(key);
      if (it != g_tune.end()) cfg = it->second;
    }
    if (cfg < 0) {
      // every shape computes the same result, so the candidates simply run on
      // the batch itself; the last run leaves the environments in place
      cudaEvent_t e0, e1;
      cudaEventCreate(&e0);
      cudaEventCreate(&e1);
      float best = 1e30f;
      int bi = 0;
      for (int c = 0; c < env_chain_tile_configs(); ++c) {
        cudaEventRecord(e0, s);
        cudaError_t e = env_chain_cfg(c, jobs_dev, count, maxN, s);
        cudaEventRecord(e1, s);
        if (e) { cudaEventDestroy(e0); cudaEventDestroy(e1); return e; }
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) { best = ms; bi = c; }
      }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune[key] = bi;
      }
      if (chosen) *chosen = bi;
      return cudaGetLastError();
    }
  }
  if (chosen) *chosen = cfg;
  return env_chain_cfg(cfg, jobs_dev, count, maxN, s);
}
