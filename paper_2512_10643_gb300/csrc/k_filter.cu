// Mixed -> pure decomposition of Gaussian covariance matrices (Sec. III,
// Eq. (decompose); App. C, Eq. (loss) and (gradient)): the mixed covariance
// Gamma_th is split as Gamma_p + W, Gamma_p = S S^T / 2 pure (S symplectic),
// W >= 0 classical noise, by minimising L(S) = -lambda_min(Gamma_th - S S^T/2)
// with Riemannian gradient descent on Sp(2N) from S = I until L <= eps.
//
// One CTA per state: a batch of states of equal N is one launch, one state
// per SM, FP64 throughout (the loss is a smallest eigenvalue near zero).
//  * W = Gamma_th - S S^T / 2 lives in global memory (it stays in L2) and is
//    changed by the rank-2 term of each step; every `refresh` steps it is
//    recomputed from S, so rounding cannot drift.
//  * The lowest eigenpair of W: Householder tridiagonalisation of a copy in
//    shared memory; the smallest eigenvalue of the tridiagonal matrix by
//    multisection of Sturm counts (one warp, a lane per point of the current
//    interval, eleven rounds); its eigenvector by inverse iteration
//    (Gaussian elimination with partial pivoting on the tridiagonal); the
//    reflectors applied back.
//  * The gradient: with u = S^T v0, u^ = u / |u| and a^ = Omega^T u^ (a unit
//    vector orthogonal to u^), the unit element of sp(2N) = {Omega H, H = H^T}
//    (Frobenius norm) that maximises the rate (1/2) v0^T S (X + X^T) S^T v0
//    is G = (u^ u^T - a^ a^T) / sqrt 2, so exp(-alpha G) = 1 + (e^-b - 1)
//    u^ u^T + (e^b - 1) a^ a^T with b = alpha / sqrt 2, and
//      S <- S + (e^-b - 1) p u^T + (e^b - 1) q a^T,
//      W <- W - [(e^-2b - 1) p p^T + (e^2b - 1) q q^T] / 2,   p = S u^, q = S a^.
#include "internal.h"
#include <algorithm>
#include <math.h>

namespace {

constexpr int FT_THREADS = 512;
constexpr int FT_NW = FT_THREADS / 32;

struct FilterArgs {
  int n, count, max_iter, refresh;
  double alpha, eps;
  const double* gth;       // count x n x n
  double* S;               // count x n x n: the result (and the working S)
  double* W;               // count x n x n workspace
  int* iters;              // count
  double* loss;            // count
  int* status;
};

// block-wide sum in a fixed order (deterministic); red holds FT_NW doubles
__device__ double ft_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  for (int k = 0; k < FT_NW; ++k) t += red[k];
  return t;
}

// number of eigenvalues of the symmetric tridiagonal (d, e) below x
__device__ int sturm_count(const double* d, const double* e, int n, double x, double pivmin) {
  int c = 0;
  double q = d[0] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  c += q < 0.0;
  for (int i = 1; i < n; ++i) {
    q = d[i] - x - e[i - 1] * e[i - 1] / q;
    if (fabs(q) < pivmin) q = -pivmin;
    c += q < 0.0;
  }
  return c;
}

__global__ void __launch_bounds__(FT_THREADS, 1) filter_kernel(const FilterArgs a) {
  extern __shared__ __align__(16) double sh[];
  const int n = a.n, N = n / 2, tid = threadIdx.x;
  const int lane = tid & 31, wid = tid >> 5;
  double* A = sh;                     // n x n work copy, reflectors below the subdiagonal
  double* d = A + (size_t)n * n;
  double* e = d + n;
  double* tau = e + n;
  double* x = tau + n;                // eigenvector
  double* uh = x + n;
  double* ah = uh + n;
  double* p = ah + n;
  double* q = p + n;
  double* w = q + n;
  double* vv = w + n;                 // the current Householder vector, contiguous
  double* red = vv + n;               // FT_NW
  double* scal = red + FT_NW;         // 8 scalars
  const double* G = a.gth + (size_t)blockIdx.x * n * n;
  double* S = a.S + (size_t)blockIdx.x * n * n;
  double* W = a.W + (size_t)blockIdx.x * n * n;
  const double b = a.alpha / sqrt(2.0);
  const double cm = expm1(-b), cp = expm1(b), c2m = expm1(-2.0 * b), c2p = expm1(2.0 * b);

  for (int i = tid; i < n * n; i += FT_THREADS) S[i] = (i / n == i % n) ? 1.0 : 0.0;
  __syncthreads();
  int it = 0;
  double L = 0.0;
  for (;; ++it) {
    // ---- W (recomputed from S every `refresh` steps) and its copy in A ----
    if (it % a.refresh == 0) {
      for (int idx = tid; idx < n * n; idx += FT_THREADS) {
        const int i = idx / n, j = idx % n;
        if (j < i) continue;
        double s = 0.0;
        for (int k = 0; k < n; ++k) s = fma(S[(size_t)i * n + k], S[(size_t)j * n + k], s);
        const double v = 0.5 * (G[(size_t)i * n + j] + G[(size_t)j * n + i]) - 0.5 * s;
        W[(size_t)i * n + j] = v;
        W[(size_t)j * n + i] = v;
      }
      __syncthreads();
    }
    for (int idx = tid; idx < n * n; idx += FT_THREADS) A[idx] = W[idx];
    __syncthreads();
    // ---- Householder tridiagonalisation (lower part holds the reflectors) --
    for (int k = 0; k + 2 < n; ++k) {
      const int m = n - k - 1;
      double part = 0.0;
      for (int i = k + 2 + tid; i < n; i += FT_THREADS) part += A[(size_t)i * n + k] * A[(size_t)i * n + k];
      const double tail = ft_sum(part, red);
      const double x0 = A[(size_t)(k + 1) * n + k];
      if (tid == 0) d[k] = A[(size_t)k * n + k];
      if (tail == 0.0) {                          // already tridiagonal in this column
        if (tid == 0) { e[k] = x0; tau[k] = 0.0; }
        __syncthreads();
        continue;
      }
      const double nrm = sqrt(tail + x0 * x0);
      const double ah_ = x0 >= 0.0 ? -nrm : nrm;
      const double v0 = x0 - ah_;
      const double t = 2.0 / (tail + v0 * v0);
      // v (kept in column k for the back transformation, and contiguous in
      // vv: a column of A is one shared-memory bank)
      for (int r = tid; r < m; r += FT_THREADS) vv[r] = r == 0 ? v0 : A[(size_t)(k + 1 + r) * n + k];
      __syncthreads();                            // everyone read x0 before it is overwritten
      if (tid == 0) { e[k] = ah_; tau[k] = t; A[(size_t)(k + 1) * n + k] = v0; }
      // p = t A_sub v  (one warp per row of the trailing block)
      for (int r = wid; r < m; r += FT_NW) {
        const double* row = A + (size_t)(k + 1 + r) * n + k + 1;
        double s = 0.0;
        for (int c = lane; c < m; c += 32) s = fma(row[c], vv[c], s);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) p[r] = t * s;
      }
      __syncthreads();
      double kp = 0.0;
      for (int r = tid; r < m; r += FT_THREADS) kp += p[r] * vv[r];
      const double K = 0.5 * t * ft_sum(kp, red);
      for (int r = tid; r < m; r += FT_THREADS) w[r] = p[r] - K * vv[r];
      __syncthreads();
      for (int r = wid; r < m; r += FT_NW) {      // A_sub -= v w^T + w v^T, a warp per row
        double* row = A + (size_t)(k + 1 + r) * n + k + 1;
        const double vr = vv[r], wr = w[r];
        for (int c = lane; c < m; c += 32) row[c] = fma(-vr, w[c], fma(-wr, vv[c], row[c]));
      }
      __syncthreads();
    }
    if (tid == 0) {
      if (n >= 2) {
        d[n - 2] = A[(size_t)(n - 2) * n + n - 2];
        e[n - 2] = A[(size_t)(n - 1) * n + n - 2];
      }
      d[n - 1] = A[(size_t)(n - 1) * n + n - 1];
      // Gershgorin interval and the pivot floor of the Sturm counts
      double lo = d[0], hi = d[0], emax = 0.0;
      for (int i = 0; i < n; ++i) {
        const double r = (i > 0 ? fabs(e[i - 1]) : 0.0) + (i + 1 < n ? fabs(e[i]) : 0.0);
        lo = fmin(lo, d[i] - r);
        hi = fmax(hi, d[i] + r);
        if (i + 1 < n) emax = fmax(emax, e[i] * e[i]);
      }
      const double span = fmax(hi - lo, 1e-300);
      scal[0] = lo - 1e-15 * span;
      scal[1] = hi + 1e-15 * span;
      scal[2] = 1e-290 * fmax(1.0, emax);
    }
    __syncthreads();
    // ---- smallest eigenvalue: multisection of Sturm counts -----------------
    // one warp, 32 points a round (each count is n dependent FP64 divisions,
    // and GB300's FP64 pipe is narrow): 33^11 > 1e16 narrows the Gershgorin
    // interval to the rounding of the counts
    if (wid == 0) {
      double lo = scal[0], hi = scal[1];
      for (int round = 0; round < 11; ++round) {
        const double xt = lo + (hi - lo) * (double)(lane + 1) / 33.0;
        const unsigned hit = __ballot_sync(0xffffffffu, sturm_count(d, e, n, xt, scal[2]) >= 1);
        const int t0 = hit ? __ffs(hit) - 1 : 32;
        const double nlo = t0 == 0 ? lo : lo + (hi - lo) * (double)t0 / 33.0;
        const double nhi = t0 >= 32 ? hi : lo + (hi - lo) * (double)(t0 + 1) / 33.0;
        lo = nlo;
        hi = nhi;
      }
      if (lane == 0) { scal[0] = lo; scal[1] = hi; }
    }
    __syncthreads();
    const double lam = 0.5 * (scal[0] + scal[1]);
    L = -lam;
    if (L <= a.eps || it >= a.max_iter) break;
    // ---- its eigenvector: inverse iteration on T - lam I (thread 0) --------
    if (tid == 0) {
      // LU with partial pivoting of the tridiagonal: U has two superdiagonals
      // (kept in p = diag, q = first, w = second), the multipliers in uh, the
      // row swaps in ah (1.0 = swapped)
      double tnorm = 0.0;
      for (int i = 0; i < n; ++i) tnorm = fmax(tnorm, fabs(d[i]) + (i > 0 ? fabs(e[i - 1]) : 0.0) + (i + 1 < n ? fabs(e[i]) : 0.0));
      const double tiny = fmax(tnorm, 1e-300) * 1e-16;
      double cd = d[0] - lam, cs = n > 1 ? e[0] : 0.0;
      for (int i = 0; i + 1 < n; ++i) {
        const double sub = e[i], nd = d[i + 1] - lam, ns = i + 2 < n ? e[i + 1] : 0.0;
        if (fabs(cd) >= fabs(sub)) {
          const double piv = cd == 0.0 ? tiny : cd;
          const double l = sub / piv;
          p[i] = piv; q[i] = cs; w[i] = 0.0; uh[i] = l; ah[i] = 0.0;
          cd = nd - l * cs;
          cs = ns;
        } else {
          const double l = cd / sub;
          p[i] = sub; q[i] = nd; w[i] = ns; uh[i] = l; ah[i] = 1.0;
          cd = cs - l * nd;
          cs = -l * ns;
        }
      }
      p[n - 1] = cd == 0.0 ? tiny : cd;
      for (int i = 0; i < n; ++i) x[i] = 1.0;
      for (int sweep = 0; sweep < 3; ++sweep) {
        for (int i = 0; i + 1 < n; ++i) {                       // forward: row swaps, elimination
          if (ah[i] != 0.0) { const double tt = x[i]; x[i] = x[i + 1]; x[i + 1] = tt; }
          x[i + 1] -= uh[i] * x[i];
        }
        for (int i = n - 1; i >= 0; --i) {                      // back substitution
          double s = x[i];
          if (i + 1 < n) s -= q[i] * x[i + 1];
          if (i + 2 < n) s -= w[i] * x[i + 2];
          const double pv = fabs(p[i]) < tiny ? copysign(tiny, p[i]) : p[i];
          x[i] = s / pv;
        }
        double nr = 0.0;
        for (int i = 0; i < n; ++i) nr = fma(x[i], x[i], nr);
        nr = 1.0 / sqrt(nr);
        for (int i = 0; i < n; ++i) x[i] *= nr;
      }
    }
    __syncthreads();
    // ---- back to the eigenvector of W: x <- H_0 ... H_{n-3} x ---------------
    for (int k = n - 3; k >= 0; --k) {
      if (tau[k] == 0.0) continue;
      double part = 0.0;
      for (int r = k + 1 + tid; r < n; r += FT_THREADS) part += A[(size_t)r * n + k] * x[r];
      const double s = tau[k] * ft_sum(part, red);
      for (int r = k + 1 + tid; r < n; r += FT_THREADS) x[r] -= s * A[(size_t)r * n + k];
      __syncthreads();
    }
    // ---- gradient step ------------------------------------------------------
    for (int j = tid; j < n; j += FT_THREADS) {                   // u = S^T x
      double s = 0.0;
      for (int i = 0; i < n; ++i) s = fma(S[(size_t)i * n + j], x[i], s);
      uh[j] = s;
    }
    __syncthreads();
    double part = 0.0;
    for (int j = tid; j < n; j += FT_THREADS) part += uh[j] * uh[j];
    const double inv = 1.0 / sqrt(ft_sum(part, red));
    for (int j = tid; j < n; j += FT_THREADS) uh[j] *= inv;
    __syncthreads();
    for (int j = tid; j < n; j += FT_THREADS) ah[j] = j < N ? -uh[j + N] : uh[j - N];   // Omega^T u^
    __syncthreads();
    for (int r = wid; r < n; r += FT_NW) {                       // p = S u^, q = S a^
      double sp = 0.0, sq = 0.0;
      for (int c = lane; c < n; c += 32) {
        const double sv = S[(size_t)r * n + c];
        sp = fma(sv, uh[c], sp);
        sq = fma(sv, ah[c], sq);
      }
      for (int o = 16; o > 0; o >>= 1) {
        sp += __shfl_xor_sync(0xffffffffu, sp, o);
        sq += __shfl_xor_sync(0xffffffffu, sq, o);
      }
      if (lane == 0) { p[r] = sp; q[r] = sq; }
    }
    __syncthreads();
    for (int idx = tid; idx < n * n; idx += FT_THREADS) {
      const int i = idx / n, j = idx % n;
      S[idx] += cm * p[i] * uh[j] + cp * q[i] * ah[j];
      W[idx] -= 0.5 * (c2m * p[i] * p[j] + c2p * q[i] * q[j]);
    }
    __syncthreads();
  }
  if (tid == 0) {
    a.iters[blockIdx.x] = it;
    a.loss[blockIdx.x] = L;
  }
}

}  // namespace

size_t filter_smem_bytes(int n) {
  return sizeof(double) * ((size_t)n * n + 11 * (size_t)n + FT_NW + 8);
}

cudaError_t launch_filter(int count, int n, const double* gth, double* S, double* W, double alpha,
                          double eps, int max_iter, int refresh, int* iters, double* loss,
                          int* status, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  const size_t smem = filter_smem_bytes(n);
  cudaError_t e = cudaFuncSetAttribute(filter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e) return e;
  FilterArgs a{n, count, max_iter, refresh, alpha, eps, gth, S, W, iters, loss, status};
  filter_kernel<<<count, FT_THREADS, smem, s>>>(a);
  return cudaGetLastError();
}
