// Complex GEMM in FP32 on the CUDA cores, for the right-canonical transforms
// of the mixed sampler (T = Ahat^m L_{m+1}, At = L_m^{-1} T).  Their output
// feeds the sampler's split-FP16 planes (2^-22 of the unit scale) and the
// sampler normalises every sample's weights by their sum, so FP32 products
// with round-to-nearest accumulation (relative error ~ sqrt(K) 2^-24, no
// bias) are accurate enough; the tensor cores' FP32 accumulation would need
// one FP64-reduced partial per 16-deep stage to match that, which costs far
// more than it saves on these small products.  Operands are FP64 or FP32 in
// memory and FP32 in shared memory; output FP32.  Batched by strides.
// Tile: 64 x 64 complex outputs, 16 complex k per stage, 256 threads of 4 x 4;
// the next stage's operands are read into registers while the current one is
// multiplied, then stored to the other of two shared-memory buffers (one
// barrier per stage).
#include "internal.h"
#include <algorithm>

namespace {

constexpr int FM = 64, FN = 64, FK = 16;

struct F32Args {
  int M, N, K, opb;
  const void* A; long long lda, sA;
  const void* B; long long ldb, sB;
  void* C; long long ldc, sC;
};

__device__ __forceinline__ float2 tof(double2 v) { return make_float2((float)v.x, (float)v.y); }
__device__ __forceinline__ float2 tof(float2 v) { return v; }
// a double-float pair (df_pack): its hi words are the FP64 value rounded to FP32
__device__ __forceinline__ float2 tof(float4 v) { return make_float2(v.x, v.z); }

__device__ __forceinline__ void store(float2* c, float2 v) { *c = v; }

// one 64 x 64 output tile of C = A op(B) (op: none, or conjugate transpose)
template <typename TA, typename TB, typename TC>
__device__ __forceinline__ void f32_tile(const F32Args& p, const TA* __restrict__ A,
                                         const TB* __restrict__ B, TC* __restrict__ C, int i0, int j0,
                                         float2 (*As)[FK][FM + 1], float2 (*Bs)[FK][FN + 1]) {
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  float2 acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = make_float2(0.f, 0.f);
  constexpr int NL = FM * FK / 256;                  // elements of each operand per thread and stage
  float2 ra[NL], rb[NL];
  auto fetch = [&](int k0) {
#pragma unroll
    for (int q = 0; q < NL; ++q) {
      const int e = tid + 256 * q;
      const int ii = e / FK, kk = e % FK, gi = i0 + ii, gk = k0 + kk;
      ra[q] = (gi < p.M && gk < p.K) ? tof(A[(long long)gi * p.lda + gk]) : make_float2(0.f, 0.f);
      int kb, jj;
      if (p.opb == 0) { kb = e / FN; jj = e % FN; } else { jj = e / FK; kb = e % FK; }
      const int gj = j0 + jj, gkb = k0 + kb;
      float2 v = make_float2(0.f, 0.f);
      if (gj < p.N && gkb < p.K) {
        if (p.opb == 0) v = tof(B[(long long)gkb * p.ldb + gj]);
        else { v = tof(B[(long long)gj * p.ldb + gkb]); v.y = -v.y; }   // B^dag
      }
      rb[q] = v;
    }
  };
  auto put = [&](int buf) {
#pragma unroll
    for (int q = 0; q < NL; ++q) {
      const int e = tid + 256 * q;
      As[buf][e % FK][e / FK] = ra[q];
      if (p.opb == 0) Bs[buf][e / FN][e % FN] = rb[q];
      else Bs[buf][e % FK][e / FK] = rb[q];
    }
  };
  fetch(0);
  put(0);
  __syncthreads();
  for (int k0 = 0, buf = 0; k0 < p.K; k0 += FK, buf ^= 1) {
    const bool more = k0 + FK < p.K;
    if (more) fetch(k0 + FK);
#pragma unroll 4
    for (int kk = 0; kk < FK; ++kk) {
      float2 a[4], b[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = As[buf][kk][ty + 16 * r];
#pragma unroll
      for (int c = 0; c < 4; ++c) b[c] = Bs[buf][kk][tx + 16 * c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          acc[r][c].x = fmaf(a[r].x, b[c].x, fmaf(-a[r].y, b[c].y, acc[r][c].x));
          acc[r][c].y = fmaf(a[r].x, b[c].y, fmaf(a[r].y, b[c].x, acc[r][c].y));
        }
    }
    if (more) put(buf ^ 1);
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int gi = i0 + ty + 16 * r;
    if (gi >= p.M) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int gj = j0 + tx + 16 * c;
      if (gj < p.N) store(C + (long long)gi * p.ldc + gj, acc[r][c]);
    }
  }
}

template <typename TA, typename TB, typename TC>
__global__ void __launch_bounds__(256) zgemm_f32_kernel(F32Args p) {
  __shared__ float2 As[2][FK][FM + 1];  // padded rows: the k-fastest fills hit distinct banks
  __shared__ float2 Bs[2][FK][FN + 1];
  const long long bz = blockIdx.z;
  f32_tile<TA, TB, TC>(p, reinterpret_cast<const TA*>(p.A) + bz * p.sA,
                       reinterpret_cast<const TB*>(p.B) + bz * p.sB,
                       reinterpret_cast<TC*>(p.C) + bz * p.sC, blockIdx.y * FM, blockIdx.x * FN, As, Bs);
}

// many independent products in one launch: CTA b works on the last product
// whose first CTA c0 <= b (the table is in device memory, sorted by c0)
template <typename TA, typename TB>
__global__ void __launch_bounds__(256) zgemm_f32_grouped_kernel(const F32Prob* __restrict__ probs,
                                                                 int np) {
  __shared__ float2 As[2][FK][FM + 1];
  __shared__ float2 Bs[2][FK][FN + 1];
  const long long b = blockIdx.x;
  int lo = 0, hi = np - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (probs[mid].c0 <= b) lo = mid; else hi = mid - 1;
  }
  const F32Prob q = probs[lo];
  const long long l = b - q.c0;
  const F32Args p{q.M, q.N, q.K, 0, q.A, q.lda, 0, q.B, q.ldb, 0, q.C, q.ldc, 0};
  f32_tile<TA, TB, float2>(p, reinterpret_cast<const TA*>(q.A), reinterpret_cast<const TB*>(q.B),
                           reinterpret_cast<float2*>(q.C), (int)(l / q.tn) * FM,
                           (int)(l % q.tn) * FN, As, Bs);
}

}  // namespace

int f32_tile_rows() { return FM; }
int f32_tile_cols() { return FN; }

cudaError_t launch_zgemm_f32_grouped(const F32Prob* probs_dev, int np, long long ctas, int a64,
                                     int b64, cudaStream_t s) {
  if (np <= 0 || ctas <= 0) return cudaSuccess;
  if (ctas > 0x7fffffffLL) return cudaErrorInvalidValue;
  if (a64 == 2 && b64) zgemm_f32_grouped_kernel<float4, double2><<<(unsigned)ctas, 256, 0, s>>>(probs_dev, np);
  else if (a64 && b64) zgemm_f32_grouped_kernel<double2, double2><<<(unsigned)ctas, 256, 0, s>>>(probs_dev, np);
  else if (a64) zgemm_f32_grouped_kernel<double2, float2><<<(unsigned)ctas, 256, 0, s>>>(probs_dev, np);
  else if (b64) zgemm_f32_grouped_kernel<float2, double2><<<(unsigned)ctas, 256, 0, s>>>(probs_dev, np);
  else zgemm_f32_grouped_kernel<float2, float2><<<(unsigned)ctas, 256, 0, s>>>(probs_dev, np);
  COUNT_LAUNCH(1);
  return cudaGetLastError();
}

cudaError_t launch_zgemm_f32(int M, int N, int K, const void* A, int a64, long long lda, long long sA,
                             const void* B, int b64, long long ldb, long long sB, float2* C,
                             long long ldc, long long sC, int batch, cudaStream_t s) {
  if (M <= 0 || N <= 0 || batch <= 0) return cudaSuccess;
  if (batch > 65535) return cudaErrorInvalidValue;
  F32Args a{M, N, K, 0, A, lda, sA, B, ldb, sB, C, ldc, sC};
  dim3 grid((N + FN - 1) / FN, (M + FM - 1) / FM, batch);
  if (a64 && b64) zgemm_f32_kernel<double2, double2, float2><<<grid, 256, 0, s>>>(a);
  else if (a64) zgemm_f32_kernel<double2, float2, float2><<<grid, 256, 0, s>>>(a);
  else if (b64) zgemm_f32_kernel<float2, double2, float2><<<grid, 256, 0, s>>>(a);
  else zgemm_f32_kernel<float2, float2, float2><<<grid, 256, 0, s>>>(a);
  COUNT_LAUNCH(1);
  return cudaGetLastError();
}
