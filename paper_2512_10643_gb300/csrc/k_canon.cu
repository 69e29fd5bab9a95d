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
// The GEMM runs on the 5th-generation tensor cores.  Both operands are
// bounded by 1 in magnitude (vt has norm at most 1, the rows of the packed
// At are orthonormal), and each is stored as two fp16 planes, x = h + 2^-11 l
// with h = fp16(x), l = fp16(2^11 (x - h)): 22 significant bits above the
// fp16 normal range and an absolute floor near 2^-35 below it.  The product
// is h_a h_b + 2^-11 (h_a l_b + l_a h_b) (the dropped l_a l_b term is
// 2^-22 of the scale), three tcgen05.mma per K step into two FP32
// accumulators in tensor memory.  The kernel is persistent and
// warp-specialised: one warp loads a three-stage ring (a TMA copy of the
// 128 x 64 packed-tensor tile of both planes, and a gather of the 128 state
// rows by sample index with 16-byte cp.async copies into the same
// 128-byte-swizzled layout), one thread issues the MMAs (M = N = 128,
// K = 16), and eight epilogue warps (two per lane quadrant of tensor memory,
// each with half the columns) drain the other of two accumulator buffers
// (tcgen05.ld, W = s (hh + 2^-11 x) with the row's stored scale s, per-tile
// row norms, rows transposed through shared memory into coalesced stores:
// FP32 rows of W, or fp16 planes straight into the sampled rows of the next
// bond's state), so the epilogue of one tile overlaps the MMAs of the next.
// The state rows never move: row s of a class's planes is sample s, and the
// passes exchange lists of sample indices.  Every wait on an mbarrier is
// bounded in time; on a timeout the kernel records ST_TIMEOUT, waits
// (bounded) for its own copies and MMAs in flight, and frees its tensor
// memory.
#include "internal.h"
#include "tc_ptx.h"
#include <cuda.h>
#include <cuda_fp16.h>
#include <algorithm>
#include <cstring>

namespace {

using namespace tcx;

constexpr int TBM = 128, TBN = 128, TBK = 64;     // tile in fp16 elements (real)
constexpr int NPL = 2;                            // fp16 planes per operand: h, l
constexpr int TSTAGES = 3;
constexpr int PLANE_BYTES = TBM * TBK * 2;        // 16 KB (TBN == TBM)
constexpr int STAGE_BYTES = 2 * NPL * PLANE_BYTES;
constexpr int EPI_WARPS = 8;                      // two per TMEM lane quadrant
constexpr int EPI_LD = 16;                        // floats per staged row (16 columns; float4 index
                                                  // XOR-swizzled by row, conflict-free without a pad)
constexpr int EPI_BYTES = EPI_WARPS * 32 * EPI_LD * 4;
constexpr int NBAR = 2 * TSTAGES + 2 + 2 + 1;     // full, empty, acc full, acc empty, drain
constexpr int TC_SMEM = TSTAGES * STAGE_BYTES + EPI_BYTES + 1024 + 256;
constexpr int NPROD = TSTAGES;                    // load warps: warp 0 and the last two, one per stage
constexpr int TC_THREADS = 32 * (2 + EPI_WARPS + NPROD - 1);   // + MMA warp, epilogue warps
constexpr int TMEM_COLS = 4 * TBN;                // 2 buffers x (hh, cross) accumulators
constexpr float LO_SCALE = 2048.f, LO_INV = 1.f / 2048.f;

__device__ __forceinline__ void split2(float x, __half& h, __half& l) {
  h = __float2half_rn(x);
  l = __float2half_rn((x - __half2float(h)) * LO_SCALE);
}

// ---------------------------------------------------------------- tcgen05 GEMM
// Two independent GEMMs (the parity groups) in one persistent launch.  For
// group g: W_g[row, n] (real view: row-major, ldw floats; complex pairs
// interleaved) and part_g[row, c] = sum of W_g^2 over real columns
// 32c .. 32c + 31.  The row counts are read on the device (the previous
// selection pass wrote them).  Tiles run over group 0, then group 1; tile t
// of a group's ntm x ntn grid is (t / ntn, t % ntn): consecutive tiles share
// the A row block, so the streamed operand is read from HBM once while the
// packed tensor (a few MB) stays in L2.
struct TileRef { int g, m0, nb; };
__device__ __forceinline__ TileRef tile_of(int t, int T0, int ntn0, int ntn1) {
  TileRef r;
  r.g = t >= T0 ? 1 : 0;
  const int tt = r.g ? t - T0 : t, ntn = r.g ? ntn1 : ntn0;
  r.m0 = (tt / ntn) * TBM;
  r.nb = tt % ntn;
  return r;
}
__device__ __forceinline__ int group_rows(const TcGroup& g) {
  const int m = g.cnt ? *g.cnt : g.mcap;
  return max(0, min(m, g.mcap));
}

__global__ void __launch_bounds__(TC_THREADS, 1)
canon_gemm_tc_kernel(const __grid_constant__ CUtensorMap tmB0, const __grid_constant__ CUtensorMap tmB1,
                     const TcGroup g0, const TcGroup g1, int* status) {
  extern __shared__ __align__(1024) uint8_t smraw[];
  const uint32_t raw = su32(smraw);
  const uint32_t sbase = (raw + 1023u) & ~1023u;
  uint8_t* sp = smraw + (sbase - raw);
  float* epi = reinterpret_cast<float*>(sp + TSTAGES * STAGE_BYTES);
  uint64_t* bars = reinterpret_cast<uint64_t*>(sp + TSTAGES * STAGE_BYTES + EPI_BYTES);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + NBAR);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t full0 = su32(bars), empty0 = full0 + 8 * TSTAGES;
  const uint32_t afull0 = empty0 + 8 * TSTAGES, aempty0 = afull0 + 16, drain = aempty0 + 16;
  const int M0 = group_rows(g0), M1 = group_rows(g1);
  const int T0 = ((M0 + TBM - 1) / TBM) * g0.ntn;
  const int ntiles = T0 + ((M1 + TBM - 1) / TBM) * g1.ntn;
  if (threadIdx.x == 0) {
    for (int s = 0; s < TSTAGES; ++s) {
      mbar_init(full0 + 8 * s, 2);                   // B copy (tx bytes) + A gather
      mbar_init(empty0 + 8 * s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(afull0 + 8 * b, 1);
      mbar_init(aempty0 + 8 * b, EPI_WARPS);
    }
    mbar_init(drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tslot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  if (warp == 0 || warp >= 2 + EPI_WARPS) {
    // Loads.  Stage g of the ring belongs to load warp g % NPROD (warp 0,
    // then the warps after the epilogue warps).  Lane 0 issues the TMA copy
    // of the packed-tensor tile (B); the warp gathers the 128 state rows of
    // the A tile by sample index, 16 bytes a lane (eight lanes per 128-byte
    // row, four rows per instruction), into the 128-byte-swizzled layout TMA
    // would write: chunk j of row r at r * 128 + 16 (j ^ (r & 7)).  Rows past
    // the group's count read zeros.  Once its copies have landed the warp
    // makes them visible to the async proxy and releases the stage, so every
    // stage of the ring can be in flight at once.
    const int pid = warp == 0 ? 0 : warp - (1 + EPI_WARPS);
    int g = 0;
    bool ok = true;
    const int j = lane & 7;
    for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      const TileRef tr = tile_of(t, T0, g0.ntn, g1.ntn);
      const TcGroup& gg = tr.g ? g1 : g0;
      const int Mg = tr.g ? M1 : M0;
      const int m0 = tr.m0, n0 = tr.nb * TBN, nkb = gg.nkb;
      const long long Kp = (long long)nkb * TBK;
      const CUtensorMap* mB = tr.g ? &tmB1 : &tmB0;
      int ridx[4];                                    // sample of row m0 + lane + 32 k
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int r = m0 + lane + 32 * k;
        ridx[k] = r < Mg ? gg.rows[r] : -1;
      }
      for (int kb = 0; kb < nkb; ++kb, ++g) {
        if (g % NPROD != pid) continue;
        const int st = g % TSTAGES, r = g / TSTAGES;
        const bool free_ = r == 0 || mbar_wait(empty0 + 8 * st, (r - 1) & 1);
        if (!__all_sync(0xffffffffu, free_)) {
          if (lane == 0) set_status(status, ST_TIMEOUT);
          ok = false;
          break;
        }
        const uint32_t sA = sbase + st * STAGE_BYTES, sB = sA + NPL * PLANE_BYTES;
        if (lane == 0) {
          mbar_expect_tx(full0 + 8 * st, NPL * PLANE_BYTES);
          tma_load_3d(sB, mB, full0 + 8 * st, kb * TBK, n0, 0);    // box: both planes
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {                 // rows 32 k .. 32 k + 31
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const int row = 32 * k + (lane >> 3) + 4 * i;
            const int src = __shfl_sync(0xffffffffu, ridx[k], row & 31);
            const __half* p = gg.A + (long long)max(src, 0) * Kp + kb * TBK + 8 * j;
            const uint32_t dst = sA + row * 128 + ((j ^ (row & 7)) << 4);
            const uint32_t nb = src >= 0 ? 16u : 0u;
            cp_async16(dst, p, nb);
            cp_async16(dst + PLANE_BYTES, p + gg.apl, nb);
          }
        }
        cp_async_commit();
        cp_async_wait<0>();
        fence_proxy_async();
        __syncwarp();
        if (lane == 0) mbar_arrive(full0 + 8 * st);
      }
    }
    cp_async_wait<0>();
    if (warp == 0 && lane == 0) {
      // the last TMA copy issued into each stage has landed before the CTA exits
      for (int st = 0; st < TSTAGES && st < g; ++st) {
        const int last = st + TSTAGES * ((g - 1 - st) / TSTAGES);
        if (!mbar_wait(full0 + 8 * st, (last / TSTAGES) & 1)) set_status(status, ST_TIMEOUT);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {                                  // MMA issuer
      // D f32, A f16, B f16, both K-major, N = 128, M = 128
      const uint32_t idesc =
          (1u << 4) | ((uint32_t)(TBN >> 3) << 17) | ((uint32_t)(TBM >> 4) << 24);
      int g = 0, i = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++i) {
        const int buf = i & 1, u = i >> 1;
        if (u > 0 && !mbar_wait(aempty0 + 8 * buf, (u - 1) & 1)) {
          set_status(status, ST_TIMEOUT);
          break;
        }
        tc_fence_after();
        const uint32_t dhh = tmem + (uint32_t)(buf * 2 * TBN), dx = dhh + TBN;
        const int nkb = tile_of(t, T0, g0.ntn, g1.ntn).g ? g1.nkb : g0.nkb;
        for (int kb = 0; kb < nkb; ++kb, ++g) {
          const int st = g % TSTAGES, r = g / TSTAGES;
          if (!mbar_wait(full0 + 8 * st, r & 1)) {
            set_status(status, ST_TIMEOUT);
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sA = sbase + st * STAGE_BYTES, sB = sA + NPL * PLANE_BYTES;
#pragma unroll
          for (int k16 = 0; k16 < TBK / 16; ++k16) {
            const uint64_t ah = sdesc(sA + k16 * 32), al = sdesc(sA + PLANE_BYTES + k16 * 32);
            const uint64_t bh = sdesc(sB + k16 * 32), bl = sdesc(sB + PLANE_BYTES + k16 * 32);
            const uint32_t acc = (kb | k16) != 0 ? 1u : 0u;
            umma_f16(dhh, ah, bh, idesc, acc);
            umma_f16(dx, ah, bl, idesc, acc);
            umma_f16(dx, al, bh, idesc, 1u);
          }
          umma_commit(empty0 + 8 * st);
        }
        if (!ok) break;
        umma_commit(afull0 + 8 * buf);
      }
      if (g > 0) {                                    // every MMA issued here has completed
        umma_commit(drain);
        if (!mbar_wait(drain, 0)) set_status(status, ST_TIMEOUT);
      }
    }
  } else if (warp >= 2 && warp < 2 + EPI_WARPS) {    // epilogue warps
    const int q = warp & 3;                           // TMEM lanes 32q .. 32q + 31
    const int cb = ((warp - 2) >> 2) * (TBN / 2);     // this warp's half of the columns
    float* stg = epi + (warp - 2) * 32 * EPI_LD;
    int i = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++i) {
      const int buf = i & 1, u = i >> 1;
      const bool got = __all_sync(0xffffffffu, mbar_wait(afull0 + 8 * buf, u & 1));
      if (!got) {
        if (lane == 0) set_status(status, ST_TIMEOUT);
        break;
      }
      tc_fence_after();
      const TileRef tr = tile_of(t, T0, g0.ntn, g1.ntn);
      const TcGroup& gg = tr.g ? g1 : g0;
      const int M = tr.g ? M1 : M0;
      float* __restrict__ W = gg.W;
      const bool vout = W == nullptr;                 // fp16 planes into the sampled rows
      const long long ldw = gg.ldw;
      const int nb = tr.nb, n0 = nb * TBN;
      const int rbase = tr.m0 + q * 32;
      int smp = 0;                                    // sample of this lane's row
      float rsc = 1.f;
      if (rbase + lane < M) {
        smp = gg.rows[rbase + lane];
        if (gg.rsc) rsc = gg.rsc[smp];
      }
#pragma unroll 1
      for (int c0 = cb; c0 < cb + TBN / 2; c0 += 32) {
        float nrm = 0.f;
        uint32_t h[32], x[32];
        const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * 2 * TBN + c0);
        tmem_ld32(ta, h);
        tmem_ld32(ta + TBN, x);
        float4* srow = reinterpret_cast<float4*>(stg + lane * EPI_LD);
#pragma unroll
        for (int hf = 0; hf < 2; ++hf) {                // 16 columns at a time through shared memory
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            float v[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const int k = 16 * hf + 4 * j + e;
              v[e] = rsc * fmaf(LO_INV, __uint_as_float(x[k]), __uint_as_float(h[k]));
              nrm = fmaf(v[e], v[e], nrm);
            }
            if (!vout) {
              srow[j ^ ((lane >> 1) & 3)] = make_float4(v[0], v[1], v[2], v[3]);
            } else {                                  // {h01, h23, l01, l23} of four columns
              const bool in = n0 + c0 + 16 * hf + 4 * j < gg.wv;
              __half hh[4], ll[4];
#pragma unroll
              for (int e = 0; e < 4; ++e) split2(in ? v[e] : 0.f, hh[e], ll[e]);
              const __half2 a0 = __halves2half2(hh[0], hh[1]), a1 = __halves2half2(hh[2], hh[3]);
              const __half2 b0 = __halves2half2(ll[0], ll[1]), b1 = __halves2half2(ll[2], ll[3]);
              uint4 pk;
              pk.x = *reinterpret_cast<const uint32_t*>(&a0);
              pk.y = *reinterpret_cast<const uint32_t*>(&a1);
              pk.z = *reinterpret_cast<const uint32_t*>(&b0);
              pk.w = *reinterpret_cast<const uint32_t*>(&b1);
              reinterpret_cast<uint4*>(srow)[j ^ ((lane >> 1) & 3)] = pk;
            }
          }
          __syncwarp();
#pragma unroll
          for (int it = 0; it < 4; ++it) {
            const int r = it * 8 + (lane >> 2), c4 = lane & 3;
            const int sr = __shfl_sync(0xffffffffu, smp, r);
            const float4 val = *reinterpret_cast<const float4*>(stg + r * EPI_LD + 4 * (c4 ^ ((r >> 1) & 3)));
            const int col = n0 + c0 + 16 * hf + c4 * 4;
            if (rbase + r < M) {
              if (!vout) {
                *reinterpret_cast<float4*>(W + (long long)(rbase + r) * ldw + col) = val;
              } else if (col < gg.Kpn) {
                __half* dst = gg.Vn + (long long)sr * gg.Kpn + col;
                *reinterpret_cast<uint2*>(dst) = make_uint2(__float_as_uint(val.x), __float_as_uint(val.y));
                *reinterpret_cast<uint2*>(dst + gg.vnpl) =
                    make_uint2(__float_as_uint(val.z), __float_as_uint(val.w));
              }
            }
          }
          __syncwarp();
        }
        if (rbase + lane < M) gg.part[(long long)(rbase + lane) * gg.ldp + (n0 + c0) / 32] = nrm;
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(aempty0 + 8 * buf);  // buffer free for tile i + 2
    }
  }
  __syncwarp();
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS)
                 : "memory");
  }
}

// SIMT reference on the same packed planes (cross-check of the tcgen05 path):
// the same three products, FP32 accumulation in k order, the same scale and
// outputs; one thread per row and 32-real-column chunk; rows beyond the
// group's device-side count are skipped
__global__ void canon_gemm_ref_kernel(const __half* __restrict__ Bp, long long bpl, int Np,
                                      const TcGroup g) {
  const int M = group_rows(g);
  const int Kp = g.nkb * TBK, nch = Np / 32;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < (long long)M * nch;
       idx += (long long)gridDim.x * blockDim.x) {
    const int row = idx / nch, c = idx % nch;
    const int smp = g.rows[row];
    const float sc = g.rsc ? g.rsc[smp] : 1.f;
    const __half* ah = g.A + (long long)smp * Kp;
    const __half* al = ah + g.apl;
    float nrm = 0.f;
    for (int jj = 0; jj < 16; ++jj) {
      const int nc = 16 * c + jj;
      float hh[2] = {0.f, 0.f}, xx[2] = {0.f, 0.f};
      for (int e = 0; e < 2; ++e) {
        const __half* bh = Bp + (long long)(2 * nc + e) * Kp;
        const __half* bl = bh + bpl;
        for (int k = 0; k < Kp; ++k) {
          const float a0 = __half2float(ah[k]), a1 = __half2float(al[k]);
          const float b0 = __half2float(bh[k]), b1 = __half2float(bl[k]);
          hh[e] = fmaf(a0, b0, hh[e]);
          xx[e] = fmaf(a0, b1, fmaf(a1, b0, xx[e]));
        }
      }
      const float vr = sc * fmaf(LO_INV, xx[0], hh[0]), vi = sc * fmaf(LO_INV, xx[1], hh[1]);
      nrm = fmaf(vi, vi, fmaf(vr, vr, nrm));
      if (g.W) {
        reinterpret_cast<float2*>(g.W)[(long long)row * (g.ldw / 2) + nc] = make_float2(vr, vi);
      } else if (2 * nc < g.Kpn) {
        const bool in = 2 * nc < g.wv;
        __half hr[NPL], hi[NPL];
        split2(in ? vr : 0.f, hr[0], hr[1]);
        split2(in ? vi : 0.f, hi[0], hi[1]);
        for (int pl = 0; pl < NPL; ++pl)
          *reinterpret_cast<__half2*>(g.Vn + pl * g.vnpl + (long long)smp * g.Kpn + 2 * nc) =
              __halves2half2(hr[pl], hi[pl]);
      }
    }
    g.part[(long long)row * g.ldp + c] = nrm;
  }
}

// ---------------------------------------------------------------- parity classes
// one warp per bond: the kept states by photon-number parity (sum of the
// occupations), even class first, each class in the kept (E) order
__global__ void parity_classes_kernel(BondArrays ba, int nb) {
  const int b = blockIdx.x, lane = threadIdx.x;
  const bool edge = b == 0 || b == nb - 1;       // vacuum-only end bonds
  const int D = edge ? 1 : ba.D[b];
  const int ne = edge ? 0 : ba.ne[b];
  const uint8_t* occ = ba.occ + (size_t)b * ba.cap * NEM;
  int* out = ba.pidx + (size_t)b * ba.cap;
  int k = 0;
  for (int c = 0; c < 2; ++c) {
    const int k0 = k;
    for (int i0 = 0; i0 < D; i0 += 32) {
      const int i = i0 + lane;
      bool hit = false;
      if (i < D) {
        int n = 0;
        for (int q = 0; q < ne; ++q) n += occ[(size_t)i * NEM + q];
        hit = (n & 1) == c;
      }
      const unsigned m = __ballot_sync(0xffffffffu, hit);
      if (hit) out[k + __popc(m & ((1u << lane) - 1u))] = i;
      k += __popc(m);
    }
    if (lane == 0) ba.pcnt[2 * b + c] = k - k0;
  }
}

// ---------------------------------------------------------------- packing
// B planes of group pi of one site from its parity-compact canonical tensor
// (At_pi: kc rows of length K): complex column nc = (p, j) in the group's
// 16-padded block layout, real rows 2 nc + c; K index a (real 2a + e) = row
// a; [[Re, -Im], [Im, Re]] blocks; zero in the padding.  Block p of a
// compact row starts at floor(p/2) (kr0 + kr1) + (p odd ? kr0 : 0), with kr0
// (kr1) states of the right bond in the class of even (odd) p.
// the packing of many (site, group) planes in one launch: blockIdx.y = job
__global__ void pack_compact_batch_kernel(const PackJob* __restrict__ jobs, int d) {
  const PackJob J = jobs[blockIdx.y];
  const long long total = (long long)(J.Np / 2) * (J.Kp / 2);
  const int P2 = J.w0 + J.w1, Dr = J.kr0 + J.kr1;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int nc = (int)(idx / (J.Kp / 2));
    const int a = (int)(idx % (J.Kp / 2));
    const int pp = nc / P2, rem = nc - pp * P2;
    const bool odd = rem >= J.w0;
    const int p = 2 * pp + (odd ? 1 : 0), j = odd ? rem - J.w0 : rem;
    float2 v = make_float2(0.f, 0.f);
    if (p < d && a < J.kc && j < (odd ? J.kr1 : J.kr0))
      v = J.At[(long long)a * J.K + (long long)pp * Dr + (odd ? J.kr0 : 0) + j];
    __half rr[NPL], ii[NPL];
    split2(v.x, rr[0], rr[1]);
    split2(v.y, ii[0], ii[1]);
    for (int sp = 0; sp < NPL; ++sp) {
      __half* row0 = J.Bp + sp * J.bpl + (2LL * nc) * J.Kp + 2 * a;
      __half* row1 = row0 + J.Kp;
      __half2 x0, x1;
      x0.x = rr[sp]; x0.y = __hneg(ii[sp]);
      x1.x = ii[sp]; x1.y = rr[sp];
      *reinterpret_cast<__half2*>(row0) = x0;
      *reinterpret_cast<__half2*>(row1) = x1;
    }
  }
}

// first site: every sample in group 0 (D_0 = 1, the vacuum) with vt = [1]
__global__ void sampler_init_kernel(__half* V, long long vpl, int Spad, int Kp, int* sid, float* rs,
                                    int* cnt, int S) {
  const long long total = (long long)Spad * Kp;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int k = idx % Kp;
    for (int sp = 0; sp < NPL; ++sp)
      V[sp * vpl + idx] = __float2half_rn((sp == 0 && k == 0) ? 1.f : 0.f);
    if (k == 0 && idx / Kp < S) {
      sid[idx / Kp] = (int)(idx / Kp);
      rs[idx / Kp] = 1.f;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) { cnt[0] = S; cnt[1] = 0; }
}

// One lane per sample for the draw, one warp per spw samples for the copy.
// Lane l < spw of warp w takes global row t = spw w + l: row t of group 0 or, past
// its count, row t - count0 of group 1 (the counts add up to S).  The lane
// sums q_p from the chunk norms (fixed order), draws u, takes the first p
// with u Z < C_p (C the running sum in p order, Z the total), and flags the
// draw if u Z lies within flag_tol Z of any C_p.  The warp reserves its rows
// of each next group with one atomic per group, then copies the 32 chosen
// blocks w_{p*} / sqrt(q_{p*}) as fp16 planes (coalesced, sample by sample)
// into row s (the sample's index) of the next class's planes, with scale 1.
// The order of a next list depends on the order of the reservations; no
// arithmetic depends on it.
constexpr int SEL_THREADS = 256;
constexpr int SEL_SPW_DEFAULT = 4;   // samples per warp (the warp copies their rows one by one)
__global__ void __launch_bounds__(SEL_THREADS)
select_groups_kernel(int S, int spw, int d, const SelGroup g0, const SelGroup g1, const NextGroup n0,
                     const NextGroup n1, int* cnt_next, const double* __restrict__ u, int ustride,
                     int site, uint64_t seed, uint64_t counter0, uint8_t* __restrict__ out, int N,
                     uint8_t* flags, double flag_tol) {
  const int lane = threadIdx.x & 31;
  const int M0 = max(0, min(*g0.cnt, S)), M1 = max(0, min(*g1.cnt, S));
  // warps stride over the spw-sample groups up to the device-side counts
  // (the grid is sized for a few waves, not for S)
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long wg = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
       wg * spw < (long long)M0 + M1; wg += nwarps) {   // warp-uniform: the warp syncs below
    const long long t = wg * spw + lane;          // lanes 0 .. spw-1 take a sample each
    const int grp = t >= M0 ? 1 : 0;
    const int r = (int)(t - (grp ? M0 : 0));
    const bool active = lane < spw && t < S && r < (grp ? M1 : M0);
    const SelGroup& g = grp ? g1 : g0;
    int pstar = 0, np = 0, s = 0;
    float inv = 0.f;
    if (active) {
      s = g.sid[r];
      const float* ps = g.part + (long long)r * g.ldp;
      const int P2 = g.wself + g.wother;
      auto qp = [&](int p) {
        const int c0 = ((p >> 1) * P2 + ((p & 1) ? g.wself : 0)) / 16;
        const int nch = ((p & 1) ? g.wother : g.wself) / 16;
        float q = 0.f;
  #pragma unroll 8
        for (int k = 0; k < nch; ++k) q += ps[c0 + k];
        return q;
      };
      // FP32 weights: W is FP32-accurate, and a draw whose margin to a CDF
      // boundary is below flag_tol Z (>> FP32 rounding) is flagged anyway
      float Z = 0.f;
      for (int p = 0; p < d; ++p) Z += qp(p);
      const double uu = u ? u[(size_t)s * ustride + site] : philox_uniform(seed, counter0 + s, (uint32_t)site);
      const float tt = (float)uu * Z;
      const float ftol = (float)flag_tol * Z;
      float C = 0.f, qsel = 0.f;
      int plast = 0;
      bool flag = false;
      pstar = -1;
      for (int p = 0; p < d; ++p) {
        const float q = qp(p);
        C += q;
        if (fabsf(tt - C) <= ftol) flag = true;
        if (q > 0.f) plast = p;
        if (pstar < 0 && tt < C) { pstar = p; qsel = q; }
      }
      if (pstar < 0) { pstar = plast; qsel = qp(pstar); }
      inv = qsel > 0.f ? rsqrtf(qsel) : 0.f;
      np = grp ^ (pstar & 1);
      out[(size_t)s * N + site] = (uint8_t)pstar;
      if (flags && flag) flags[s] = 1;
    }
    // rows in the next groups: one atomic per group and warp
    int pos = 0;
    for (int c = 0; c < 2; ++c) {
      const unsigned m = __ballot_sync(0xffffffffu, active && np == c);
      if (!m) continue;
      int base = 0;
      if (lane == __ffs(m) - 1) base = atomicAdd(cnt_next + c, __popc(m));
      base = __shfl_sync(0xffffffffu, base, __ffs(m) - 1);
      if (active && np == c) pos = base + __popc(m & ((1u << lane) - 1u));
    }
    // the warp copies each active lane's chosen block into its next group
    unsigned todo = __ballot_sync(0xffffffffu, active && pos < S);
    while (todo) {
      const int src = __ffs(todo) - 1;
      todo &= todo - 1;
      const int rr = __shfl_sync(0xffffffffu, r, src);
      const int gg = __shfl_sync(0xffffffffu, grp, src);
      const int ps = __shfl_sync(0xffffffffu, pstar, src);
      const int nn = __shfl_sync(0xffffffffu, np, src);
      const int po = __shfl_sync(0xffffffffu, pos, src);
      const int sd = __shfl_sync(0xffffffffu, s, src);
      const float iv = __shfl_sync(0xffffffffu, inv, src);
      const SelGroup& G = gg ? g1 : g0;
      const NextGroup& ng = nn ? n1 : n0;
      const int P2 = G.wself + G.wother;
      const float2* wr = G.W + (long long)rr * G.ldw + (long long)(ps >> 1) * P2 + ((ps & 1) ? G.wself : 0);
      for (int b = lane; b < ng.Kp / 2; b += 32) {
        const float2 v = b < ng.D ? wr[b] : make_float2(0.f, 0.f);
        __half hr[NPL], hi[NPL];
        split2(v.x * iv, hr[0], hr[1]);
        split2(v.y * iv, hi[0], hi[1]);
        for (int pl = 0; pl < NPL; ++pl)
          *reinterpret_cast<__half2*>(ng.V + pl * ng.vpl + (long long)sd * ng.Kp + 2 * b) =
              __halves2half2(hr[pl], hi[pl]);
      }
      if (lane == 0) {
        ng.sid[po] = sd;
        ng.rs[sd] = 1.f;
      }
    }
  }
}

// The p = 0 pre-pass of a site.  In right-canonical form the weights of a
// sample add up to its squared norm, sum_p q_p = |vt|^2 = 1 (to the rounding
// of the planes and transforms), so the rule "first p with u Z < C_p" picks
// p = 0 whenever u < q_0 - margin, margin >= |Z - 1|.  Only block 0 of each
// group has been multiplied: its chunk norms give q_0, and the GEMM has
// already stored w_0 in the sample's row of the next planes of the same
// class.  One lane per sample: a draw below q_0 - margin emits p = 0,
// records the row's scale 1 / sqrt(q_0) and appends the sample to the next
// list of its class; every other sample (and every sample when the build's
// largest Cholesky regulariser exceeds reg_ok, which bounds |Z - 1|) is
// appended to the rest list for the full pass, which draws and flags it.
// No state row moves; one atomic per destination list and warp.
__global__ void __launch_bounds__(SEL_THREADS)
select_pre_kernel(int S, const SelGroup g0, const SelGroup g1, const NextGroup n0,
                  const NextGroup n1, int* cnt_next, const RestGroup r0, const RestGroup r1,
                  const unsigned long long* __restrict__ regmax, double reg_ok,
                  const double* __restrict__ u, int ustride, int site, uint64_t seed,
                  uint64_t counter0, uint8_t* __restrict__ out, int N, double margin) {
  const int lane = threadIdx.x & 31;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t - lane >= S) return;                     // whole warps only: the warp syncs below
  const int M0 = max(0, min(*g0.cnt, S)), M1 = max(0, min(*g1.cnt, S));
  const int grp = t >= M0 ? 1 : 0;
  const int r = (int)(t - (grp ? M0 : 0));
  const bool active = t < S && r < (grp ? M1 : M0);
  const SelGroup& g = grp ? g1 : g0;
  const bool reg_good = __longlong_as_double((long long)*regmax) <= reg_ok;
  bool cut = false;
  int s = 0;
  if (active) {
    s = g.sid[r];
    const float* ps = g.part + (long long)r * g.ldp;
    float q0 = 0.f;
    const int nch = g.wself / 16;
#pragma unroll 8
    for (int k = 0; k < nch; ++k) q0 += ps[k];
    const double uu = u ? u[(size_t)s * ustride + site] : philox_uniform(seed, counter0 + s, (uint32_t)site);
    cut = reg_good && q0 > 0.f && uu < (double)q0 - margin;
    if (cut) {
      out[(size_t)s * N + site] = 0;
      (grp ? n1 : n0).rs[s] = rsqrtf(q0);
    }
  }
  // the next list of the same class (cut) or the rest list (not cut)
  for (int c = 0; c < 4; ++c) {
    const bool mine = active && grp == (c & 1) && cut == (c < 2);
    const unsigned m = __ballot_sync(0xffffffffu, mine);
    if (!m) continue;
    int base = 0;
    if (lane == __ffs(m) - 1) base = atomicAdd(c < 2 ? cnt_next + (c & 1) : ((c & 1) ? r1.cnt : r0.cnt), __popc(m));
    base = __shfl_sync(0xffffffffu, base, __ffs(m) - 1);
    if (mine) {
      const int pos = base + __popc(m & ((1u << lane) - 1u));
      if (pos < S) (c < 2 ? ((c & 1) ? n1.sid : n0.sid) : ((c & 1) ? r1.sid : r0.sid))[pos] = s;
    }
  }
}

// ---------------------------------------------------------------- Cholesky
// one CTA per bond: R + delta 1 = L L^dag (lower, FP64 complex) from the
// environment stored as double-float pairs, written to dst.  delta = reg * max diag(R) regularises the bond states the truncated
// right part barely reaches (near-null directions of R, which the mixed
// path's FP32-accurate environments resolve only to ~1e-7 |R|): a sampled
// state carries no weight there, so the weights q_p / Z move by O(delta)
// absolute.  A pivot that is still not positive flags ST_NUMERIC.
__global__ void chol_kernel(const double2* __restrict__ src, double2* __restrict__ dst,
                            const long long* __restrict__ off, const int* __restrict__ Dv, int b0,
                            double* __restrict__ dused, unsigned long long* regmax, int* status) {
  const int b = b0 + blockIdx.x;
  const int D = Dv[b];
  const float4* Sm = reinterpret_cast<const float4*>(src) + off[b];
  double2* R = dst + off[b];
  const int tid = threadIdx.x, nt = blockDim.x;
  __shared__ double dmax, lkk_s, il_s;
  __shared__ bool piv_ok;
  if (tid == 0) {
    double m = 0.0;
    for (int i = 0; i < D; ++i) m = fmax(m, df_unpack(Sm[(long long)i * D + i]).x);
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
      double2 v = df_unpack(Sm[idx]);
      if (idx / D == idx % D) v.x += delta;
      R[idx] = v;
    }
    __syncthreads();
    okf = true;
    for (int k = 0; k < D; ++k) {
      if (tid == 0) {                    // one thread takes the FP64 square root
        const double akk = R[(long long)k * D + k].x;
        piv_ok = akk > 0.0;
        if (piv_ok) { lkk_s = sqrt(akk); il_s = 1.0 / lkk_s; }
      }
      __syncthreads();
      if (!piv_ok) { okf = false; break; }   // same value in every thread
      const double il = il_s;
    for (int i = k + 1 + tid; i < D; i += nt) R[(long long)i * D + k] = cscale(R[(long long)i * D + k], il);
    if (tid == 0) R[(long long)k * D + k] = cmk(lkk_s, 0.0);
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
  if (tid == 0) {
    const double rel = okf ? delta / fmax(dmax, 1e-300) : -1.0;
    dused[b] = rel;
    // the largest relative regulariser of the build (bit patterns of
    // non-negative doubles order like the integers; a failure counts as huge)
    if (regmax) atomicMax(regmax, (unsigned long long)__double_as_longlong(okf ? rel : 1e300));
  }
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
  extern __shared__ double nidiag[];       // -1 / L_ii, one FP64 division per row
  for (int i = threadIdx.x; i < D; i += blockDim.x) nidiag[i] = -1.0 / L[(long long)i * D + i].x;
  __syncthreads();
  for (int j = threadIdx.x; j < D; j += blockDim.x) {
    for (int i = 0; i < j; ++i) X[(long long)i * D + j] = cmk(0.0, 0.0);
    X[(long long)j * D + j] = cmk(-nidiag[j], 0.0);
    for (int i = j + 1; i < D; ++i) {
      double2 s = cmk(0.0, 0.0);
      for (int k = j; k < i; ++k) cfma(s, L[(long long)i * D + k], X[(long long)k * D + j]);
      X[(long long)i * D + j] = cscale(s, nidiag[i]);
    }
  }
}

// ---------------------------------------------------------------- fused factor + inverse
// One CTA per diagonal parity block of a bond, the block held in shared
// memory as a packed lower triangle of double-float pairs (row i at
// i (i + 1) / 2; {re_h, re_l, im_h, im_l} per element): R + delta 1 = L L^dag
// by right-looking Cholesky, L written out in FP64, then L^{-1} in place by
// forward substitution (row i of X = L^{-1}: X_ii = 1 / L_ii,
// X_ij = -X_ii sum_{k=j}^{i-1} L_ik X_kj), written out in FP64.  Square
// roots and reciprocals of the pivots are FP64 (one thread per pivot); the
// updates are double-float multiply-adds on the FP32 pipes.  The
// regulariser search and its bookkeeping are those of chol_kernel.
constexpr int CI_THREADS = 512;
constexpr int CI_KS = 4;                  // k slices per row of the inverse (partial sums)
constexpr int CI_MAXD = 160;              // largest block: (160 * 161 / 2 + 4 * 160) * 16 B of shared memory
__device__ __forceinline__ int tri(int i) { return (i * (i + 1)) >> 1; }
// (h, l) += x y for double-float x, y (exact product by FMA, TwoSum)
__device__ __forceinline__ void ci_mac(float& h, float& l, float xh, float xl, float yh, float yl) {
  const float p = xh * yh;
  float e = fmaf(xh, yh, -p);
  e = fmaf(xh, yl, e);
  e = fmaf(xl, yh, e);
  const float t = h + p;
  const float v = t - h;
  l += ((h - (t - v)) + (p - v)) + e;
  h = t;
}
__device__ __forceinline__ void ci_norm(float& h, float& l) {
  const float s = h + l;
  const float v = s - h;
  l = (h - (s - v)) + (l - v);
  h = s;
}
// v -= a conj(c)  (all double-float complex)
__device__ __forceinline__ void ci_sub_aconjc(float4& v, const float4 a, const float4 c) {
  ci_mac(v.x, v.y, -a.x, -a.y, c.x, c.y);        // re -= ar cr
  ci_mac(v.x, v.y, -a.z, -a.w, c.z, c.w);        // re -= ai ci
  ci_mac(v.z, v.w, -a.z, -a.w, c.x, c.y);        // im -= ai cr
  ci_mac(v.z, v.w, a.x, a.y, c.z, c.w);          // im += ar ci
  ci_norm(v.x, v.y);
  ci_norm(v.z, v.w);
}
// s += a b  (double-float complex accumulators, left unnormalised)
__device__ __forceinline__ void ci_cmac(float4& s, const float4 a, const float4 b) {
  ci_mac(s.x, s.y, a.x, a.y, b.x, b.y);
  ci_mac(s.x, s.y, -a.z, -a.w, b.z, b.w);
  ci_mac(s.z, s.w, a.x, a.y, b.z, b.w);
  ci_mac(s.z, s.w, a.z, a.w, b.x, b.y);
}
__device__ __forceinline__ float4 ci_scale(const float4 a, float sh, float sl) {   // a * real (sh, sl)
  float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
  ci_mac(r.x, r.y, a.x, a.y, sh, sl);
  ci_mac(r.z, r.w, a.z, a.w, sh, sl);
  ci_norm(r.x, r.y);
  ci_norm(r.z, r.w);
  return r;
}
__device__ __forceinline__ float4 ci_pack_real(double x) {
  const float h = (float)x;
  return make_float4(h, (float)(x - (double)h), 0.f, 0.f);
}

__global__ void __launch_bounds__(CI_THREADS)
chol_inv_kernel(const float4* __restrict__ src, double2* __restrict__ Lout, double2* __restrict__ Xout,
                const long long* __restrict__ off, const int* __restrict__ Dv, int b0,
                double* __restrict__ dused, unsigned long long* regmax, int* status) {
  extern __shared__ float4 cism[];
  const int b = b0 + blockIdx.x;
  const int D = Dv[b];
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  float4* P = cism;                              // packed lower triangle
  float4* part = cism + tri(D);                  // CI_KS x D partial sums of the inverse
  const float4* Sm = src + off[b];
  __shared__ double dmax;
  __shared__ float ilh, ill;
  __shared__ bool piv_ok;
  if (D <= 0 || D > CI_MAXD) {                  // (the launcher sizes for the largest block)
    if (tid == 0) {
      if (D > CI_MAXD) set_status(status, ST_BOUNDS);
      dused[b] = 0.0;
    }
    return;
  }
  if (tid == 0) {
    double m = 0.0;
    for (int i = 0; i < D; ++i) m = fmax(m, df_unpack(Sm[(long long)i * D + i]).x);
    dmax = m;
  }
  __syncthreads();
  double reg = 1e-12, delta = 0.0;
  bool okf = false;
  for (int attempt = 0; attempt < 5 && !okf; ++attempt, reg *= 100.0) {
    delta = reg * dmax;
    for (int i = warp; i < D; i += nw)
      for (int j = lane; j <= i; j += 32) {
        float4 v = Sm[(long long)i * D + j];
        if (i == j) v = ci_pack_real(df_unpack(v).x + delta);
        P[tri(i) + j] = v;
      }
    __syncthreads();
    okf = true;
    for (int k = 0; k < D; ++k) {
      if (tid == 0) {                            // the pivot, in FP64
        const float4 d = P[tri(k) + k];
        const double akk = (double)d.x + (double)d.y;
        piv_ok = akk > 0.0;
        if (piv_ok) {
          const double lkk = sqrt(akk), il = 1.0 / lkk;
          P[tri(k) + k] = ci_pack_real(lkk);
          ilh = (float)il;
          ill = (float)(il - (double)ilh);
        }
      }
      __syncthreads();
      if (!piv_ok) { okf = false; break; }      // same value in every thread
      const float sh = ilh, sl = ill;
      for (int i = k + 1 + tid; i < D; i += nt) P[tri(i) + k] = ci_scale(P[tri(i) + k], sh, sl);
      __syncthreads();
      // trailing lower triangle: rows by warp, columns by lane
      for (int i = k + 1 + warp; i < D; i += nw) {
        const float4 a = P[tri(i) + k];
        for (int j = k + 1 + lane; j <= i; j += 32) {
          float4 v = P[tri(i) + j];
          ci_sub_aconjc(v, a, P[tri(j) + k]);
          P[tri(i) + j] = v;
        }
      }
      __syncthreads();
    }
    __syncthreads();
  }
  if (!okf && tid == 0) set_status(status, ST_NUMERIC);
  if (tid == 0) {
    const double rel = okf ? delta / fmax(dmax, 1e-300) : -1.0;
    dused[b] = rel;
    if (regmax) atomicMax(regmax, (unsigned long long)__double_as_longlong(okf ? rel : 1e300));
  }
  double2* L = Lout + off[b];
  double2* X = Xout + off[b];
  for (long long idx = tid; idx < (long long)D * D; idx += nt) {
    const int i = (int)(idx / D), j = (int)(idx % D);
    L[idx] = j <= i ? df_unpack(P[tri(i) + j]) : cmk(0.0, 0.0);
  }
  if (!okf) return;
  // L^{-1} in place, row by row
  for (int i = 0; i < D; ++i) {
    // partial sums y_j = sum_{k = j + s, j + s + KS, ..} L_ik X_kj, k < i
    for (int e = tid; e < i * CI_KS; e += nt) {
      const int j = e / CI_KS, sl = e % CI_KS;
      float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
      for (int k = j + sl; k < i; k += CI_KS) ci_cmac(acc, P[tri(i) + k], P[tri(k) + j]);
      part[sl * D + j] = acc;
    }
    if (tid == 0) {
      const float4 d = P[tri(i) + i];
      const double xi = 1.0 / ((double)d.x + (double)d.y);
      ilh = (float)xi;
      ill = (float)(xi - (double)ilh);
    }
    __syncthreads();
    const float xh = ilh, xl = ill;
    for (int j = tid; j <= i; j += nt) {
      if (j == i) {
        P[tri(i) + i] = make_float4(xh, xl, 0.f, 0.f);
      } else {
        float4 y = part[j];
        for (int q = 1; q < CI_KS; ++q) {
          const float4 w = part[q * D + j];
          ci_mac(y.x, y.y, w.x, w.y, 1.f, 0.f);
          ci_mac(y.z, y.w, w.z, w.w, 1.f, 0.f);
        }
        P[tri(i) + j] = ci_scale(y, -xh, -xl);
      }
    }
    __syncthreads();
  }
  for (long long idx = tid; idx < (long long)D * D; idx += nt) {
    const int i = (int)(idx / D), j = (int)(idx % D);
    X[idx] = j <= i ? df_unpack(P[tri(i) + j]) : cmk(0.0, 0.0);
  }
}

typedef CUresult (*EncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                             const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                             CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                             CUtensorMapFloatOOBfill);

EncodeFn encode_fn() {
  static const EncodeFn fn = [] {               // thread-safe one-time lookup
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

}  // namespace

// ---- host side --------------------------------------------------------------
int canon_make_map(void* map128, const void* planes, int Kp, long long rows) {
  EncodeFn fn = encode_fn();
  if (!fn) return 1;
  // TMA: 16-byte aligned base, 16-byte multiple strides, box inner extent 128 B
  if ((reinterpret_cast<uintptr_t>(planes) & 15) || (Kp % TBK) || (rows % TBM)) return 2;
  cuuint64_t dims[3] = {(cuuint64_t)Kp, (cuuint64_t)rows, (cuuint64_t)NPL};
  cuuint64_t strides[2] = {(cuuint64_t)Kp * 2, (cuuint64_t)Kp * 2 * rows};
  cuuint32_t box[3] = {TBK, TBM, NPL};                      // both planes in one copy
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = fn(reinterpret_cast<CUtensorMap*>(map128), CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3,
                  const_cast<void*>(planes), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : 3;
}

cudaError_t launch_canon_gemm(const void* mapB0, const void* mapB1, const TcGroup& g0,
                              const TcGroup& g1, const __half* B0, long long bpl0, const __half* B1,
                              long long bpl1, int use_tc, int* status, int sm_reserve,
                              cudaStream_t s) {
  // the row counts live on the device: the launch is sized for the capacity
  // and the kernel's tiles stop at the counts (the trace adds the
  // algorithmic work once the counts are known)
  for (int gi = 0; gi < 2; ++gi) {
    const TcGroup& g = gi ? g1 : g0;
    if (!g.rows || !g.A || !g.part || (!g.W && !g.Vn)) return cudaErrorInvalidValue;
    if (!g.W && g.ntn > 0 && (g.Kpn % 64 || g.Kpn > g.ntn * TBN)) return cudaErrorInvalidValue;
  }
  cudaEvent_t tr0 = g_tc_trace.begin(s);
  if (use_tc) {
    COUNT_LAUNCH(1);
    static std::atomic<int> nsm[64];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!nsm[dev].load()) {
      e = cudaFuncSetAttribute(canon_gemm_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               TC_SMEM);
      if (e) return e;
      int n = 0;
      e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
      if (e) return e;
      nsm[dev].store(n);
    }
    CUtensorMap b0, b1;
    memcpy(&b0, mapB0, sizeof(CUtensorMap));
    memcpy(&b1, mapB1, sizeof(CUtensorMap));
    const long long cap = ((long long)(g0.mcap + TBM - 1) / TBM) * g0.ntn +
                          ((long long)(g1.mcap + TBM - 1) / TBM) * g1.ntn;
    const int grid = (int)std::max<long long>(
        1, std::min<long long>(std::max(1, nsm[dev].load() - std::max(0, sm_reserve)), cap));
    canon_gemm_tc_kernel<<<grid, TC_THREADS, TC_SMEM, s>>>(b0, b1, g0, g1, status);
  } else {
    for (int gi = 0; gi < 2; ++gi) {
      const TcGroup& g = gi ? g1 : g0;
      const int Np = g.ntn * TBN;
      long long n = (long long)g.mcap * (Np / 32);
      int blocks = (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 16384));
      canon_gemm_ref_kernel<<<blocks, 256, 0, s>>>(gi ? B1 : B0, gi ? bpl1 : bpl0, Np, g);
      COUNT_LAUNCH(1);
    }
  }
  g_tc_trace.end(tr0, s, 0.0, 0.0);
  return cudaGetLastError();
}

cudaError_t launch_parity_classes(BondArrays ba, int nb, cudaStream_t s) {
  if (nb <= 0) return cudaSuccess;
  parity_classes_kernel<<<nb, 32, 0, s>>>(ba, nb);
  return cudaGetLastError();
}

cudaError_t launch_pack_compact_batch(const PackJob* jobs_dev, int njobs, int d, cudaStream_t s) {
  for (int j0 = 0; j0 < njobs; j0 += 65535) {
    pack_compact_batch_kernel<<<dim3(48, std::min(65535, njobs - j0)), 256, 0, s>>>(jobs_dev + j0, d);
    COUNT_LAUNCH(1);
  }
  return cudaGetLastError();
}

cudaError_t launch_sampler_init(__half* V, long long vpl, int Spad, int Kp, int* sid, float* rs,
                                int* cnt, int S, cudaStream_t s) {
  long long total = (long long)Spad * Kp;
  int blocks = (int)std::max<long long>(1, std::min<long long>((total + 255) / 256, 8192));
  sampler_init_kernel<<<blocks, 256, 0, s>>>(V, vpl, Spad, Kp, sid, rs, cnt, S);
  return cudaGetLastError();
}

// samples per warp of the selection passes (a performance knob: every value
// draws the same patterns): GBSMPS_SEL_SPW in 1 .. 32, default 4
static int sel_spw() {
  const char* e = getenv("GBSMPS_SEL_SPW");
  const int v = e ? atoi(e) : SEL_SPW_DEFAULT;
  return v < 1 ? 1 : (v > 32 ? 32 : v);
}

cudaError_t launch_select_groups(int Scap, int d, const SelGroup& g0, const SelGroup& g1,
                                 const NextGroup& n0, const NextGroup& n1, int* cnt_next,
                                 const double* u, int ustride, int site, uint64_t seed,
                                 uint64_t counter0, uint8_t* out, int N, uint8_t* flags,
                                 double flag_tol, cudaStream_t s) {
  const int spw = sel_spw();
  long long threads = ((long long)Scap + spw - 1) / spw * 32;   // spw samples per warp
  static std::atomic<int> nsm{0};
  if (!nsm.load()) {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
      nsm.store(n);
  }
  // at most four CTAs per SM: the warps loop over the counts on the device
  const long long cap = 4LL * std::max(1, nsm.load());
  const int blocks = (int)std::max<long long>(1, std::min<long long>((threads + SEL_THREADS - 1) / SEL_THREADS, cap));
  select_groups_kernel<<<blocks, SEL_THREADS, 0, s>>>(Scap, spw, d, g0, g1, n0, n1, cnt_next, u,
                                                      ustride, site, seed, counter0, out, N, flags,
                                                      flag_tol);
  return cudaGetLastError();
}

cudaError_t launch_select_pre(int Scap, const SelGroup& g0, const SelGroup& g1, const NextGroup& n0,
                              const NextGroup& n1, int* cnt_next, const RestGroup& r0,
                              const RestGroup& r1, const unsigned long long* regmax, double reg_ok,
                              const double* u, int ustride, int site, uint64_t seed,
                              uint64_t counter0, uint8_t* out, int N, double margin, cudaStream_t s) {
  const long long threads = ((long long)Scap + 31) / 32 * 32;   // one lane per sample
  const int blocks = (int)((threads + SEL_THREADS - 1) / SEL_THREADS);
  select_pre_kernel<<<blocks, SEL_THREADS, 0, s>>>(Scap, g0, g1, n0, n1, cnt_next, r0, r1, regmax,
                                                   reg_ok, u, ustride, site, seed, counter0, out, N,
                                                   margin);
  return cudaGetLastError();
}

// Both factor kernels fit on an SM beside a sampler GEMM CTA (218 KB of
// shared memory, 320 threads x 112 registers), so they may run while another
// state is sampled: 256 threads each, and shared memory for the largest
// block only.
cudaError_t launch_chol(const double2* src, double2* dst, const long long* off, const int* Dv,
                        int b0, int nb, double* dused, unsigned long long* regmax, int* status,
                        cudaStream_t s) {
  if (nb <= 0) return cudaSuccess;
  chol_kernel<<<nb, 256, 0, s>>>(src, dst, off, Dv, b0, dused, regmax, status);
  return cudaGetLastError();
}

size_t chol_inv_smem(int maxd) {
  if (maxd < 1 || maxd > CI_MAXD) return 0;
  return sizeof(float4) * ((size_t)maxd * (maxd + 1) / 2 + (size_t)CI_KS * maxd);
}

cudaError_t launch_chol_inv(const double2* src, double2* L, double2* X, const long long* off,
                            const int* Dv, int b0, int nb, int maxd, double* dused,
                            unsigned long long* regmax, int* status, cudaStream_t s) {
  if (nb <= 0) return cudaSuccess;
  const size_t smem = chol_inv_smem(maxd);
  if (!smem) return cudaErrorInvalidValue;
  static std::atomic<int> attr_set{0};
  if (!attr_set.load()) {
    cudaError_t e = cudaFuncSetAttribute(chol_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)chol_inv_smem(CI_MAXD));
    if (e) return e;
    attr_set.store(1);
  }
  chol_inv_kernel<<<nb, CI_THREADS, smem, s>>>(reinterpret_cast<const float4*>(src), L, X, off, Dv, b0,
                                               dused, regmax, status);
  return cudaGetLastError();
}

cudaError_t launch_trinv(const double2* L, double2* X, const long long* off, const int* Dv, int b0,
                         int nb, int maxd, cudaStream_t s) {
  if (nb <= 0) return cudaSuccess;
  if (maxd < 1 || maxd > 4096) return cudaErrorInvalidValue;
  trinv_kernel<<<nb, 256, sizeof(double) * maxd, s>>>(L, X, off, Dv, b0);
  return cudaGetLastError();
}
