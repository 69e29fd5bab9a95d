// MPS consumers on the finished tensors: right environments and the
// normalisation, amplitudes, and exact conditional sampling (FP64 path).
//
// Right environments R_m = sum_p A^m[p] R_{m+1} A^m[p]^dag (R_{N+1} = 1) are two
// complex GEMMs per site; sampling at site m is W = V A^m (S x D_{m-1} by
// D_{m-1} x d D_m), Y = W R_{m+1}, then per sample q_p = Re <Y_p, W_p>,
// the first p with u Z < C_p, and v = w_p / sqrt(q_p).
#include "internal.h"
#include <math.h>

namespace {

// ---- complex FP64 GEMM, 64 x 64 tile, 16-deep k slices, 4 x 4 per thread ----
constexpr int TM = 64, TN = 64, TK = 16;

__global__ void __launch_bounds__(256)
zgemm_kernel(char opa, char opb, int M, int N, int K, double2 alpha,
             const double2* __restrict__ A, int lda, long long sA,
             const double2* __restrict__ B, int ldb, long long sB, double2 beta,
             double2* __restrict__ C, int ldc, long long sC) {
  __shared__ double2 As[TK][TM + 1];
  __shared__ double2 Bs[TK][TN + 1];
  const int bz = blockIdx.z;
  A += bz * sA; B += bz * sB; C += bz * sC;
  const int i0 = blockIdx.y * TM, j0 = blockIdx.x * TN;
  const int tid = threadIdx.x;
  const int ty = tid / 16, tx = tid % 16;
  double2 acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = cmk(0, 0);
  for (int k0 = 0; k0 < K; k0 += TK) {
    for (int e = tid; e < TK * TM; e += 256) {
      int kk, ii;
      double2 v = cmk(0, 0);
      if (opa == 'N') { ii = e / TK; kk = e % TK;
        int gi = i0 + ii, gk = k0 + kk;
        if (gi < M && gk < K) v = A[(size_t)gi * lda + gk];
      } else { kk = e / TM; ii = e % TM;
        int gi = i0 + ii, gk = k0 + kk;
        if (gi < M && gk < K) v = cconj(A[(size_t)gk * lda + gi]);
      }
      As[kk][ii] = v;
    }
    for (int e = tid; e < TK * TN; e += 256) {
      int kk, jj;
      double2 v = cmk(0, 0);
      if (opb == 'N') { kk = e / TN; jj = e % TN;
        int gj = j0 + jj, gk = k0 + kk;
        if (gj < N && gk < K) v = B[(size_t)gk * ldb + gj];
      } else { jj = e / TK; kk = e % TK;
        int gj = j0 + jj, gk = k0 + kk;
        if (gj < N && gk < K) v = cconj(B[(size_t)gj * ldb + gk]);
      }
      Bs[kk][jj] = v;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < TK; ++kk) {
      double2 a[4], b[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = As[kk][ty + 16 * r];
#pragma unroll
      for (int c = 0; c < 4; ++c) b[c] = Bs[kk][tx + 16 * c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) cfma(acc[r][c], a[r], b[c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    int gi = i0 + ty + 16 * r;
    if (gi >= M) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      int gj = j0 + tx + 16 * c;
      if (gj >= N) continue;
      double2 v = cmul(alpha, acc[r][c]);
      if (beta.x != 0.0 || beta.y != 0.0) cfma(v, beta, C[(size_t)gi * ldc + gj]);
      C[(size_t)gi * ldc + gj] = v;
    }
  }
}

__global__ void zscale_kernel(double2* x, size_t n, const double2* f) {
  double2 s = *f;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    x[i] = cmul(x[i], s);
}

// factor = conj(amp0)/|amp0| / sqrt(R0): unit norm, vacuum amplitude > 0
__global__ void norm_phase_kernel(const double2* R0, const double2* amp0, double2* f, int* status) {
  double n2 = R0->x;
  double2 a = *amp0;
  double m = sqrt(cabs2(a));
  if (!(n2 > 0.0) || !isfinite(n2)) { set_status(status, ST_NUMERIC); *f = cmk(1, 0); return; }
  double s = 1.0 / sqrt(n2);
  if (m > 0.0) *f = cmk(a.x / m * s, -a.y / m * s);
  else *f = cmk(s, 0.0);
}

// Normalisation of many states in one launch (CTA = state): the all-vacuum
// amplitude v = A^1[0] A^2[0] .. A^N[0] by a chain of vector-matrix products
// in shared memory, the factor conj(v)/|v| / sqrt(R_0) applied to A^1
// (unit norm, vacuum amplitude real positive), and, for the mixed path, the
// energy-gauge copy of the rescaled A^1 (D_0 = 1, so its left energy is 0).
__global__ void vac_norm_kernel(const NormJob* __restrict__ jobs, int maxD, int* status) {
  extern __shared__ double2 vsm[];
  const NormJob J = jobs[blockIdx.x];
  double2* v = vsm;
  double2* vn = vsm + maxD;
  const int tid = threadIdx.x, nt = blockDim.x, d = J.d;
  if (tid == 0) v[0] = cmk(1.0, 0.0);
  __syncthreads();
  for (int m = 0; m < J.N; ++m) {
    const int Dl = J.D[m], Dr = J.D[m + 1];
    const double2* T = J.T + J.toff[m];
    for (int b = tid; b < Dr; b += nt) {
      double2 acc = cmk(0.0, 0.0);
      for (int a = 0; a < Dl; ++a) cfma(acc, v[a], T[((size_t)a * d) * Dr + b]);
      vn[b] = acc;
    }
    __syncthreads();
    double2* t = v; v = vn; vn = t;
  }
  __shared__ double2 fac;
  if (tid == 0) {
    const double n2 = J.R0->x;
    const double2 a = v[0];
    const double mg = sqrt(cabs2(a));
    if (!(n2 > 0.0) || !isfinite(n2)) {
      set_status(status, ST_NUMERIC);
      fac = cmk(1.0, 0.0);
    } else {
      const double s = 1.0 / sqrt(n2);
      fac = mg > 0.0 ? cmk(a.x / mg * s, -a.y / mg * s) : cmk(s, 0.0);
    }
  }
  __syncthreads();
  const int D1 = J.D[1];
  if (J.Ah) {
    // the normalised first tensor in the energy gauge, parity-compact (read
    // before the rescale below rewrites T)
    const long long n = pk_size(d, J.P0.kl, J.P0.kr);
    for (long long idx = tid; idx < n; idx += nt) {
      int c, a, p, j, cr;
      pk_locate(J.P0, d, idx, c, a, p, j, cr);
      const int be = J.P0.pr[(cr ? J.P0.kr[0] : 0) + j];
      const double g = D1 > 1 ? J.E1[be] : 1.0;
      reinterpret_cast<float4*>(J.Ah)[idx] = df_pack(cscale(cmul(J.T[(size_t)p * D1 + be], fac), g));
    }
    __syncthreads();
  }
  for (int i = tid; i < d * D1; i += nt) J.T[i] = cmul(J.T[i], fac);
}

// amplitudes: Vn[s, b] = sum_a V[s, a] A[a, n_s, b]
__global__ void amp_step_kernel(const double2* __restrict__ T, int Dl, int d, int Dr,
                                const uint8_t* __restrict__ pats, int N, int site,
                                long long P, const double2* __restrict__ V,
                                double2* __restrict__ Vn, int ld) {
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < P * Dr;
       idx += (long long)gridDim.x * blockDim.x) {
    long long s = idx / Dr;
    int b = idx % Dr;
    int p = pats[s * N + site];
    double2 acc = cmk(0, 0);
    if (p < d) {
      for (int a = 0; a < Dl; ++a) cfma(acc, V[s * ld + a], T[((size_t)a * d + p) * Dr + b]);
    }
    Vn[s * ld + b] = acc;
  }
}

// small pattern batches: one warp per output (s, b), lanes split the sum over a
__global__ void amp_step_warp_kernel(const double2* __restrict__ T, int Dl, int d, int Dr,
                                     const uint8_t* __restrict__ pats, int N, int site,
                                     long long P, const double2* __restrict__ V,
                                     double2* __restrict__ Vn, int ld) {
  const int lane = threadIdx.x & 31;
  const long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  if (w >= P * Dr) return;
  const long long s = w / Dr;
  const int b = w % Dr;
  const int p = pats[s * N + site];
  double2 acc = cmk(0, 0);
  if (p < d)
    for (int a = lane; a < Dl; a += 32) cfma(acc, V[s * ld + a], T[((size_t)a * d + p) * Dr + b]);
  for (int o = 16; o > 0; o >>= 1) {
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
  }
  if (lane == 0) Vn[s * ld + b] = acc;
}

__global__ void amp_init_kernel(double2* V, long long P, int ld) {
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < P; s += (long long)gridDim.x * blockDim.x)
    V[s * ld] = cmk(1.0, 0.0);
}

__global__ void init_ones_f_kernel(float2* V, long long P) {
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < P; s += (long long)gridDim.x * blockDim.x)
    V[s] = make_float2(1.f, 0.f);
}

__global__ void amp_out_kernel(const double2* V, long long P, int ld, double2* out) {
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < P; s += (long long)gridDim.x * blockDim.x)
    out[s] = V[s * ld];
}

// one warp per sample; C2 = double2 (FP64 path) or float2 (mixed path),
// probabilities accumulated in FP64 either way
template <typename C2>
__global__ void sample_select_kernel(int S, int d, int Dm, const C2* __restrict__ W,
                                     const C2* __restrict__ Y, const double* __restrict__ u,
                                     int ustride, int site, uint64_t seed, uint64_t counter0,
                                     C2* __restrict__ vnew, uint8_t* __restrict__ out,
                                     int N, uint8_t* flags, double flag_tol) {
  const int lane = threadIdx.x & 31;
  const long long s = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  if (s >= S) return;
  const C2* w = W + (size_t)s * d * Dm;
  const C2* y = Y + (size_t)s * d * Dm;
  auto qof = [&](int p) {
    double part = 0.0;
    for (int b = lane; b < Dm; b += 32) {
      double2 yy = to_d(y[(size_t)p * Dm + b]), ww = to_d(w[(size_t)p * Dm + b]);
      part += yy.x * ww.x + yy.y * ww.y;
    }
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    return fmax(part, 0.0);
  };
  double Z = 0.0;
  double qs[8];
  for (int p = 0; p < d; ++p) {
    double q = qof(p);
    if (p < 8) qs[p] = q;
    Z += q;
  }
  double uu = u ? u[(size_t)s * ustride + site] : philox_uniform(seed, counter0 + s, (uint32_t)site);
  const double t = uu * Z;
  int pstar = -1, plast = 0;
  double C = 0.0, qsel = 0.0;
  bool flag = false;
  for (int p = 0; p < d; ++p) {
    double q = p < 8 ? qs[p] : qof(p);
    C += q;
    if (fabs(t - C) <= flag_tol * Z) flag = true;
    if (q > 0.0) plast = p;
    if (pstar < 0 && t < C) { pstar = p; qsel = q; }
  }
  if (pstar < 0) { pstar = plast; qsel = qof(pstar); }
  const double inv = qsel > 0.0 ? 1.0 / sqrt(qsel) : 0.0;
  for (int b = lane; b < Dm; b += 32) {
    double2 v = to_d(w[(size_t)pstar * Dm + b]);
    vnew[(size_t)s * Dm + b] = to_c<C2>(cscale(v, inv));
  }
  if (lane == 0) {
    out[(size_t)s * N + site] = (uint8_t)pstar;
    if (flags && flag) flags[s] = 1;
  }
}

}  // namespace

cudaError_t launch_zgemm(char opa, char opb, int M, int N, int K, double2 alpha,
                         const double2* A, int lda, long long sA, const double2* B, int ldb,
                         long long sB, double2 beta, double2* C, int ldc, long long sC,
                         int batch, cudaStream_t s) {
  if (M <= 0 || N <= 0 || batch <= 0) return cudaSuccess;
  dim3 grid((N + TN - 1) / TN, (M + TM - 1) / TM, batch);
  zgemm_kernel<<<grid, 256, 0, s>>>(opa, opb, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C,
                                    ldc, sC);
  return cudaGetLastError();
}

cudaError_t launch_zscale(double2* x, size_t n, const double2* factor, cudaStream_t s) {
  int blocks = (int)((n + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  zscale_kernel<<<blocks, 256, 0, s>>>(x, n, factor);
  return cudaGetLastError();
}

cudaError_t launch_norm_phase(const double2* R0, const double2* amp0, double2* factor,
                              int* status, cudaStream_t s) {
  norm_phase_kernel<<<1, 1, 0, s>>>(R0, amp0, factor, status);
  return cudaGetLastError();
}

cudaError_t launch_amplitudes(ChainView cv, long long P, const uint8_t* pats, double2* out,
                              double2* work, int maxD, cudaStream_t s) {
  double2* V = work;
  double2* Vn = work + (size_t)P * maxD;
  int blocks = (int)((P + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  amp_init_kernel<<<blocks, 256, 0, s>>>(V, P, maxD);
  for (int m = 0; m < cv.N; ++m) {
    int Dl = cv.D[m], Dr = cv.D[m + 1];
    long long n = P * Dr;
    if (n * 32 <= (1LL << 24) && Dl >= 32) {
      int bw = (int)((n * 32 + 255) / 256);
      amp_step_warp_kernel<<<bw, 256, 0, s>>>(cv.T + cv.toff[m], Dl, cv.d, Dr, pats, cv.N, m, P, V,
                                              Vn, maxD);
    } else {
      int b2 = (int)((n + 255) / 256);
      if (b2 > 8192) b2 = 8192;
      amp_step_kernel<<<b2, 256, 0, s>>>(cv.T + cv.toff[m], Dl, cv.d, Dr, pats, cv.N, m, P, V, Vn,
                                         maxD);
    }
    double2* t = V; V = Vn; Vn = t;
  }
  amp_out_kernel<<<blocks, 256, 0, s>>>(V, P, maxD, out);
  return cudaGetLastError();
}

cudaError_t launch_init_ones(double2* V, long long P, int ld, cudaStream_t s) {
  int blocks = (int)((P + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  amp_init_kernel<<<blocks, 256, 0, s>>>(V, P, ld);
  return cudaGetLastError();
}

cudaError_t launch_sample_select(int S, int d, int Dm, const double2* W, const double2* Y,
                                 const double* u, int ustride, int site, uint64_t seed,
                                 uint64_t counter0, double2* vnew, uint8_t* out, int N,
                                 uint8_t* flags, cudaStream_t s) {
  long long threads = (long long)S * 32;
  int blocks = (int)((threads + 255) / 256);
  sample_select_kernel<double2><<<blocks, 256, 0, s>>>(S, d, Dm, W, Y, u, ustride, site, seed,
                                                       counter0, vnew, out, N, flags, 1e-12);
  return cudaGetLastError();
}

cudaError_t launch_sample_select_mixed(int S, int d, int Dm, const float2* W, const float2* Y,
                                       const double* u, int ustride, int site, uint64_t seed,
                                       uint64_t counter0, float2* vnew, uint8_t* out, int N,
                                       uint8_t* flags, double flag_tol, cudaStream_t s) {
  long long threads = (long long)S * 32;
  int blocks = (int)((threads + 255) / 256);
  sample_select_kernel<float2><<<blocks, 256, 0, s>>>(S, d, Dm, W, Y, u, ustride, site, seed,
                                                      counter0, vnew, out, N, flags, flag_tol);
  return cudaGetLastError();
}

cudaError_t launch_init_ones_f(float2* V, long long P, cudaStream_t s) {
  int blocks = (int)((P + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  init_ones_f_kernel<<<blocks, 256, 0, s>>>(V, P);
  return cudaGetLastError();
}

cudaError_t launch_vac_norm_batch(const NormJob* jobs_dev, int count, int maxD, int* status,
                                  cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  const size_t smem = sizeof(double2) * 2 * (size_t)std::max(maxD, 1);
  cudaError_t e = cudaFuncSetAttribute(vac_norm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e) return e;
  vac_norm_kernel<<<count, 256, smem, s>>>(jobs_dev, maxD, status);
  COUNT_LAUNCH(1);
  return cudaGetLastError();
}
