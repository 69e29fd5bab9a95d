// Split-BF16 complex GEMM on the tensor cores, FP32 accumulation.
//
// A complex product C = op(A) op(B) (op = N or conjugate transpose) is one
// real GEMM: [Re A | Im A] (interleaved along k) times the 2x2 real blocks
// [[Re B, Im B], [-Im B, Re B]].  Every FP32 operand x is split on the fly
// into bf16 terms x = h + m + l (h = bf16(x), m = bf16(x - h), l = bf16(x -
// h - m)); NT = 3 keeps the products hh + hm + mh (~16-bit), NT = 6 adds
// hl + mm + lh (~24-bit, FP32 level).  Tile: 128 rows x 64 complex columns x
// 16 complex k per stage, 8 warps of 64 x 32 real outputs, mma.sync
// m16n8k16 bf16 with FP32 accumulators; the next stage is prefetched into
// registers while the current one is multiplied.
#include "internal.h"
#include <cuda_bf16.h>
#include <algorithm>

namespace {

constexpr int BM = 128;          // rows per CTA
constexpr int BNC = 64;          // complex columns per CTA (128 real)
constexpr int BKC = 16;          // complex k per stage (32 real)
constexpr int BNR = 2 * BNC, BKR = 2 * BKC;
constexpr int LDS = BKR + 8;     // padded smem row (bf16): conflict-free fragment loads

struct TcArgs {
  int M, N, K;                   // complex sizes of C (M x N) and the contraction
  const void* A; long long lda, sA; int a64, opa;
  const void* B; long long ldb, sB; int b64, opb;
  void* C; long long ldc, sC; int c64;
  int ksplit, kchunk;            // split-K: partial products reduced in FP64
  float2* part;
};

__device__ __forceinline__ double2 ld_c(const void* p, long long idx, int is64) {
  if (is64) return reinterpret_cast<const double2*>(p)[idx];
  float2 v = reinterpret_cast<const float2*>(p)[idx];
  return make_double2(v.x, v.y);
}

// x = o[0] + o[1] + ... (each a bf16 rounding of the remaining residual,
// residuals formed exactly in FP64): NS planes carry ~8 NS bits
template <int NS>
__device__ __forceinline__ void split(double x, __nv_bfloat16 (&o)[NS]) {
  double r = x;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    __nv_bfloat16 h = __double2bfloat16(r);
    o[s] = h;
    r -= (double)__bfloat162float(h);
  }
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                         uint32_t a3, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

template <int NT>
__global__ void __launch_bounds__(256) zgemm_tc_kernel(TcArgs p) {
  constexpr int NS = NT == 3 ? 2 : (NT == 6 ? 3 : 4);
  extern __shared__ __align__(16) unsigned char smraw[];
  auto As = reinterpret_cast<__nv_bfloat16(*)[BM][LDS]>(smraw);
  auto Bs = reinterpret_cast<__nv_bfloat16(*)[BNR][LDS]>(smraw + sizeof(__nv_bfloat16) * NS * BM * LDS);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int wm = warp & 1, wn = warp >> 1;
  const long long bz = blockIdx.z / p.ksplit;
  const int kz = blockIdx.z % p.ksplit;
  const int kbeg = kz * p.kchunk, kend = min(p.K, kbeg + p.kchunk);
  const int i0 = blockIdx.y * BM, n0 = blockIdx.x * BNC;
  const void* A = p.a64 ? (const void*)(reinterpret_cast<const double2*>(p.A) + bz * p.sA)
                        : (const void*)(reinterpret_cast<const float2*>(p.A) + bz * p.sA);
  const void* B = p.b64 ? (const void*)(reinterpret_cast<const double2*>(p.B) + bz * p.sB)
                        : (const void*)(reinterpret_cast<const float2*>(p.B) + bz * p.sB);

  float acc[4][4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;

  double2 ra[8], rb[4];
  // element coordinates owned by this thread
  auto load_stage = [&](int k0) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      int i, kc;
      if (p.opa == 0) { i = tid >> 1; kc = (tid & 1) * 8 + j; }
      else { kc = tid >> 4; i = (tid & 15) * 8 + j; }
      int gi = i0 + i, gk = k0 + kc;
      double2 v = make_double2(0.0, 0.0);
      if (gi < p.M && gk < kend) {
        if (p.opa == 0) v = ld_c(A, (long long)gi * p.lda + gk, p.a64);
        else { v = ld_c(A, (long long)gk * p.lda + gi, p.a64); v.y = -v.y; }
      }
      ra[j] = v;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int kc, nc;
      if (p.opb == 0) { kc = tid >> 4; nc = (tid & 15) * 4 + j; }
      else { nc = tid >> 2; kc = (tid & 3) * 4 + j; }
      int gn = n0 + nc, gk = k0 + kc;
      double2 v = make_double2(0.0, 0.0);
      if (gn < p.N && gk < kend) {
        if (p.opb == 0) v = ld_c(B, (long long)gk * p.ldb + gn, p.b64);
        else { v = ld_c(B, (long long)gn * p.ldb + gk, p.b64); v.y = -v.y; }
      }
      rb[j] = v;
    }
  };
  auto store_stage = [&]() {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      int i, kc;
      if (p.opa == 0) { i = tid >> 1; kc = (tid & 1) * 8 + j; }
      else { kc = tid >> 4; i = (tid & 15) * 8 + j; }
      __nv_bfloat16 sr[NS], si[NS];
      split<NS>(ra[j].x, sr);
      split<NS>(ra[j].y, si);
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        __nv_bfloat162 v;
        v.x = sr[s]; v.y = si[s];
        *reinterpret_cast<__nv_bfloat162*>(&As[s][i][2 * kc]) = v;
      }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int kc, nc;
      if (p.opb == 0) { kc = tid >> 4; nc = (tid & 15) * 4 + j; }
      else { nc = tid >> 2; kc = (tid & 3) * 4 + j; }
      __nv_bfloat16 sr[NS], si[NS];
      split<NS>(rb[j].x, sr);
      split<NS>(rb[j].y, si);
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        __nv_bfloat162 v0, v1;
        v0.x = sr[s]; v0.y = __hneg(si[s]);       // row 2nc:   ( Re,  -Im) along k
        v1.x = si[s]; v1.y = sr[s];               // row 2nc+1: ( Im,   Re)
        *reinterpret_cast<__nv_bfloat162*>(&Bs[s][2 * nc][2 * kc]) = v0;
        *reinterpret_cast<__nv_bfloat162*>(&Bs[s][2 * nc + 1][2 * kc]) = v1;
      }
    }
  };

  load_stage(kbeg);
  for (int k0 = kbeg; k0 < kend; k0 += BKC) {
    __syncthreads();
    store_stage();
    __syncthreads();
    if (k0 + BKC < kend) load_stage(k0 + BKC);
#pragma unroll
    for (int kk = 0; kk < BKR; kk += 16) {
      uint32_t af[NS][4][4], bf[NS][4][2];
#pragma unroll
      for (int s = 0; s < NS; ++s) {
#pragma unroll
        for (int mt = 0; mt < 4; ++mt) {
          int r = wm * 64 + mt * 16 + g;
          af[s][mt][0] = *reinterpret_cast<const uint32_t*>(&As[s][r][kk + 2 * t]);
          af[s][mt][1] = *reinterpret_cast<const uint32_t*>(&As[s][r + 8][kk + 2 * t]);
          af[s][mt][2] = *reinterpret_cast<const uint32_t*>(&As[s][r][kk + 8 + 2 * t]);
          af[s][mt][3] = *reinterpret_cast<const uint32_t*>(&As[s][r + 8][kk + 8 + 2 * t]);
        }
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
          int c = wn * 32 + nt * 8 + g;
          bf[s][nt][0] = *reinterpret_cast<const uint32_t*>(&Bs[s][c][kk + 2 * t]);
          bf[s][nt][1] = *reinterpret_cast<const uint32_t*>(&Bs[s][c][kk + 8 + 2 * t]);
        }
      }
      // products of total order < NS, small terms first (NT = 3, 6, 10 keep
      // the last NT entries)
      constexpr int ta[10] = {3, 2, 1, 0, 2, 1, 0, 1, 0, 0};
      constexpr int tb[10] = {0, 1, 2, 3, 0, 1, 2, 0, 1, 0};
#pragma unroll
      for (int q = 10 - NT; q < 10; ++q) {
        const int sa = ta[q], sb = tb[q];
#pragma unroll
        for (int mt = 0; mt < 4; ++mt)
#pragma unroll
          for (int nt = 0; nt < 4; ++nt)
            mma_bf16(acc[mt][nt], af[sa][mt][0], af[sa][mt][1], af[sa][mt][2], af[sa][mt][3],
                     bf[sb][nt][0], bf[sb][nt][1]);
      }
    }
  }
  // epilogue: (c0, c1) and (c2, c3) are (Re, Im) of one complex output each
#pragma unroll
  for (int mt = 0; mt < 4; ++mt) {
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      int colc = n0 + (wn * 32 + nt * 8 + 2 * t) / 2;
      if (colc >= p.N) continue;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        int row = i0 + wm * 64 + mt * 16 + g + 8 * h;
        if (row >= p.M) continue;
        float re = acc[mt][nt][2 * h], im = acc[mt][nt][2 * h + 1];
        if (p.ksplit > 1) {
          p.part[((long long)blockIdx.z * p.M + row) * p.N + colc] = make_float2(re, im);
          continue;
        }
        long long idx = bz * p.sC + (long long)row * p.ldc + colc;
        if (p.c64) reinterpret_cast<double2*>(p.C)[idx] = make_double2(re, im);
        else reinterpret_cast<float2*>(p.C)[idx] = make_float2(re, im);
      }
    }
  }
}

// C = sum over k-chunks of the FP32 partial products, summed in FP64 in a
// fixed order (deterministic)
__global__ void splitk_reduce_kernel(const float2* __restrict__ part, int ksplit, int batch,
                                     int M, int N, void* C, int c64, long long ldc, long long sC) {
  long long n = (long long)batch * M * N;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    long long b = i / ((long long)M * N), r = (i / N) % M, c = i % N;
    double re = 0.0, im = 0.0;
    for (int k = 0; k < ksplit; ++k) {
      float2 v = part[((b * ksplit + k) * M + r) * N + c];
      re += v.x;
      im += v.y;
    }
    long long idx = b * sC + r * ldc + c;
    if (c64) reinterpret_cast<double2*>(C)[idx] = make_double2(re, im);
    else reinterpret_cast<float2*>(C)[idx] = make_float2((float)re, (float)im);
  }
}

template <int NT>
cudaError_t run(const TcArgs& a, int batch, cudaStream_t s) {
  constexpr int NS = NT == 3 ? 2 : (NT == 6 ? 3 : 4);
  size_t smem = sizeof(__nv_bfloat16) * NS * (BM + BNR) * LDS;
  static std::atomic<bool> attr[64];
  int dev = 0;
  cudaError_t e0 = cudaGetDevice(&dev);
  if (e0) return e0;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!attr[dev].load()) {
    cudaError_t e = cudaFuncSetAttribute(zgemm_tc_kernel<NT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e) return e;
    attr[dev].store(true);
  }
  dim3 grid((a.N + BNC - 1) / BNC, (a.M + BM - 1) / BM, batch * a.ksplit);
  zgemm_tc_kernel<NT><<<grid, 256, smem, s>>>(a);
  if (a.ksplit > 1) {
    long long n = (long long)batch * a.M * a.N;
    int blocks = (int)std::min<long long>((n + 255) / 256, 8192);
    splitk_reduce_kernel<<<blocks, 256, 0, s>>>(a.part, a.ksplit, batch, a.M, a.N, a.C, a.c64,
                                                a.ldc, a.sC);
    COUNT_LAUNCH(1);
  }
  return cudaGetLastError();
}

}  // namespace

KernelTrace g_tc_trace;

cudaError_t launch_zgemm_tc(int nterms, char opa, char opb, int M, int N, int K,
                            const void* A, int a64, long long lda, long long sA,
                            const void* B, int b64, long long ldb, long long sB,
                            void* C, int c64, long long ldc, long long sC, int batch,
                            cudaStream_t s, void* work, size_t work_bytes) {
  if (M <= 0 || N <= 0 || batch <= 0) return cudaSuccess;
  // split K when the output tiles alone cannot fill the GPU, or K is long:
  // each chunk keeps >= 4 stages, the partials are summed in FP64
  long long tiles = (long long)((N + BNC - 1) / BNC) * ((M + BM - 1) / BM) * batch;
  int ksplit = 1;
  (void)tiles;
  if (work && K > BKC) {
    // FP64 reduction of every 16-deep stage: the FP32 tensor-core
    // accumulation never runs longer than one stage (halved while the
    // partials do not fit the workspace)
    ksplit = (K + BKC - 1) / BKC;
    while (ksplit > 1 && sizeof(float2) * (size_t)ksplit * batch * M * N > work_bytes)
      ksplit = (ksplit + 1) / 2;
  }
  int kchunk = ((K + ksplit - 1) / ksplit + BKC - 1) / BKC * BKC;
  ksplit = (K + kchunk - 1) / kchunk;
  TcArgs a{M, N, K, A, lda, sA, a64, opa == 'C' ? 1 : 0, B, ldb, sB, b64, opb == 'C' ? 1 : 0,
           C, ldc, sC, c64, ksplit, kchunk, reinterpret_cast<float2*>(work)};
  COUNT_LAUNCH(1);
  // algorithmic work of the complex product: 8 M N K real flops; bytes: one
  // read of each operand and one write of C at their storage widths
  double flops = 8.0 * M * (double)N * K * batch;
  double bytes = ((double)M * K * (a64 ? 16 : 8) + (double)K * N * (b64 ? 16 : 8) +
                  (double)M * N * (c64 ? 16 : 8)) * batch;
  (void)flops;
  (void)bytes;
  return nterms == 3 ? run<3>(a, batch, s) : nterms == 6 ? run<6>(a, batch, s) : run<10>(a, batch, s);
}
