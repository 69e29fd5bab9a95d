// Gaussian SVD chain (Sec. II B) and input handling (Sec. II A, App. A), FP64.
//
// One CTA walks the cuts m = 1..N-1 of one state.  At cut m the residual
// state lives on (r_{m-1}, a_m, .., a_N); its reduced covariance on
// L_m = (r_{m-1}, a_m) is Williamson-diagonalised (Eq. (symDiag)), the
// Bogoliubov matrices U, V (Eq. (MUV)) give the regularised paired form of
// |A^m> = prod exp(b^dag l^dag)|0> (App. A), and the correlations of the
// active b modes with the rest are carried to the next cut (the b modes are
// renamed r_m, Eqs. (SVD3)-(bond)).  Because the brick-wall and Haar
// workloads have banded covariance (zero beyond a mode distance bw), only
// the bw modes to the right of the cut are carried.
//
// Williamson form: V = 2 Gamma_LL = L L^T (Cholesky); K = L^{-1} Omega L^{-T}
// is antisymmetric with eigenvalues +-i/D; the Hermitian i K is
// diagonalised by a parallel cyclic complex Jacobi method; for an eigenpair
// (1/D, w = (u + i v)/sqrt 2), the columns (v | u) give O with
// O^T K O = [[0, D^-1], [-D^-1, 0]] and S = L O diag(D, D)^{-1/2}.
#include "internal.h"
#include <math.h>

namespace {

constexpr int LD = N2M;
constexpr int CHAIN_THREADS = 256;
static_assert(CHAIN_THREADS == 256, "the spreads over sub-partitions, q = 8 lane + warp, assume 8 warps");
constexpr int MAX_SWEEPS = 40;

struct ChainSmem {
  double A[N2M * N2M];      // V = 2 Gamma_LL -> L -> S^{-1} active rows
  double B[N2M * N2M];      // L^{-1} -> S
  double2 H[N2M * N2M];     // i K -> (Jacobi) ; reused as work for inverses
  double2 W[N2M * N2M];     // eigenvectors
  double2 T[N2M * N2M];     // Jacobi scratch: FP32 copies of H, W; products
  double2 U[NLM * NLM];
  double2 V[NLM * NLM];
  double2 Ui[NLM * NLM];
  double Dprev[NEM];
  double ev[N2M];
  int perm[N2M];
  double Dq[NLM];
  double rsD[NLM];          // sqrt(2 / D_q)
  double2 pinv;             // Gauss-Jordan: inverse of the current pivot
  int rp[NLM], rq[NLM];
  double rcs[NLM], rsn[NLM];
  double2 rph[NLM];
  float fcs[NLM], fsn[NLM];  // FP32 stage: the same, kept in FP32 (no conversions)
  float2 fph[NLM];
  double2 fac[NLM];
  double red[CHAIN_THREADS];
  int ival[4];
  double dval[4];
};

__device__ double block_sum(double v, double* red) {
  const int t = threadIdx.x, nw = blockDim.x >> 5;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((t & 31) == 0) red[t >> 5] = v;
  __syncthreads();
  double r = 0.0;
  for (int w = 0; w < nw; ++w) r += red[w];
  __syncthreads();
  return r;
}

__device__ double block_max(double v, double* red) {
  const int t = threadIdx.x, nw = blockDim.x >> 5;
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((t & 31) == 0) red[t >> 5] = v;
  __syncthreads();
  double r = red[0];
  for (int w = 1; w < nw; ++w) r = fmax(r, red[w]);
  __syncthreads();
  return r;
}

// 1/sqrt(a) and 1/a in FP64 from the FP32 estimate and Newton steps (each
// doubles the correct bits: 3 steps from ~24 bits reach FP64 rounding); GB300
// runs FP64 division and square root as long FP64 instruction sequences on
// its slow FP64 pipe, these take a few FP64 multiply-adds
__device__ __forceinline__ double rsqrt_fp64(double a) {
  if (!(a > 1e-30 && a < 1e30)) return 1.0 / sqrt(a);
  double r = (double)rsqrtf((float)a);
  for (int it = 0; it < 3; ++it) r = r * (1.5 - 0.5 * a * r * r);
  return r;
}
__device__ __forceinline__ double rcp_fp64(double a) {
  if (!(fabs(a) > 1e-30 && fabs(a) < 1e30)) return 1.0 / a;
  double x = (double)(1.0f / (float)a);
  for (int it = 0; it < 3; ++it) x = x * (2.0 - a * x);
  return x;
}

// Sweeps of the cyclic complex Jacobi method on the n x n Hermitian H (ld LD,
// storage precision of T2), accumulating W <- W J.  Round-robin ordering:
// every round rotates n/2 disjoint index pairs at once.  Before each sweep
// the largest off-diagonal |Re| + |Im| is compared with conv; returns true
// once it is below, false after max_sweeps sweeps.
//
// The rotation for a pair is computed in FP32 from the current 2x2 block
// (angle accurate to ~1e-7 relative).  In the FP64 stage its (cos, sin) and
// phase are then brought to unit modulus by two Newton steps in FP64, so
// every applied J is unitary to FP64 rounding and the similarity is exact;
// an approximate angle only leaves ~1e-7 of the rotated element behind,
// which the next sweep removes.
template <typename T2, bool WARP>
__device__ bool jacobi_sweeps(ChainSmem& sm, T2* H, T2* W, int n, double conv, double skip,
                              int max_sweeps) {
  using R = decltype(T2{}.x);
  constexpr bool wide = sizeof(R) == 8;
  // WARP: warp 0 alone runs the sweeps; otherwise the whole block.  (The
  // block form is faster for both stages at these sizes: the phases are
  // latency-bound, and more threads means fewer dependent steps per thread.)
  const int tid = WARP ? (threadIdx.x & 31) : threadIdx.x;
  const int nt = WARP ? 32 : blockDim.x;
  const int half = n / 2;
  auto team_sync = [] { if (WARP) __syncwarp(); else __syncthreads(); };
  // rotation parameters live in FP64 for the FP64 stage and in FP32 for the
  // FP32 stage, so neither stage converts between the two in its loops
  auto rot = [&](int k, R& cs, R& sn, R& px, R& py) {
    if constexpr (wide) { cs = sm.rcs[k]; sn = sm.rsn[k]; px = sm.rph[k].x; py = sm.rph[k].y; }
    else { cs = sm.fcs[k]; sn = sm.fsn[k]; px = sm.fph[k].x; py = sm.fph[k].y; }
  };
  for (int sweep = 0;; ++sweep) {
    R loc = 0;
    for (int idx = tid; idx < n * n; idx += nt) {
      int i = idx / n, j = idx % n;
      if (i < j) {
        T2 v = H[i * LD + j];
        loc = fmax(loc, fabs(v.x) + fabs(v.y));
      }
    }
    double gmax;
    if (WARP) {
      double l = loc;
      for (int o = 16; o > 0; o >>= 1) l = fmax(l, __shfl_xor_sync(0xffffffffu, l, o));
      gmax = l;
    } else {
      gmax = block_max((double)loc, sm.red);
    }
    if (gmax <= conv) return true;
    if (sweep == max_sweeps) return false;
    for (int r = 0; r < n - 1; ++r) {
      // pair k is set up by lane k / 4 of warp k % 4 (block form): the
      // set-up's FP64 steps then run on all four SM sub-partitions
      const int k = WARP ? tid : (tid < 128 ? (((tid & 31) << 2) | (tid >> 5)) : half);
      if (k < half) {
        const int a = (r + k) % (n - 1);
        const int b = (k == 0) ? (n - 1) : (r - k + n - 1) % (n - 1);
        const int p = min(a, b), q = max(a, b);
        const T2 c = H[p * LD + q];
        const float fx = (float)c.x, fy = (float)c.y;
        const float mf = hypotf(fx, fy);
        float fc = 1.0f, fs = 0.0f, gx = 1.0f, gy = 0.0f;
        if (mf > (float)skip) {
          gx = fx / mf; gy = -fy / mf;                          // e^{-i phi}
          float tau = (float)(H[q * LD + q].x - H[p * LD + p].x) / (2.0f * mf);
          float t;
          if (fabsf(tau) > 1e18f) t = 0.5f / tau;
          else t = copysignf(1.0f, tau) / (fabsf(tau) + sqrtf(fmaf(tau, tau, 1.0f)));
          fc = rsqrtf(fmaf(t, t, 1.0f));
          fs = t * fc;
        }
        sm.rp[k] = p; sm.rq[k] = q;
        if constexpr (wide) {
          double cs = fc, sn = fs, phx = gx, phy = gy;
          if (fs != 0.0f) {
            for (int it = 0; it < 2; ++it) {
              double g = 1.5 - 0.5 * (cs * cs + sn * sn);
              cs *= g; sn *= g;
              double h = 1.5 - 0.5 * (phx * phx + phy * phy);
              phx *= h; phy *= h;
            }
          }
          sm.rcs[k] = cs; sm.rsn[k] = sn; sm.rph[k] = cmk(phx, phy);
        } else {
          sm.fcs[k] = fc; sm.fsn[k] = fs; sm.fph[k] = make_float2(gx, gy);
        }
      }
      team_sync();
      // columns: X = H J, W = W J with J = [[cs, sn], [-sn ph, cs ph]]
      for (int idx = tid; idx < half * n; idx += nt) {
        const int k = idx / n, i = idx % n;
        R cs, sn, px, py;
        rot(k, cs, sn, px, py);
        if (sn == (R)0) continue;
        const int p = sm.rp[k], q = sm.rq[k];
        T2 hp = H[i * LD + p], hq = H[i * LD + q];
        R qx = px * hq.x - py * hq.y, qy = px * hq.y + py * hq.x;
        H[i * LD + p] = T2{cs * hp.x - sn * qx, cs * hp.y - sn * qy};
        H[i * LD + q] = T2{sn * hp.x + cs * qx, sn * hp.y + cs * qy};
        T2 wp = W[i * LD + p], wq = W[i * LD + q];
        qx = px * wq.x - py * wq.y; qy = px * wq.y + py * wq.x;
        W[i * LD + p] = T2{cs * wp.x - sn * qx, cs * wp.y - sn * qy};
        W[i * LD + q] = T2{sn * wp.x + cs * qx, sn * wp.y + cs * qy};
      }
      team_sync();
      // rows: H = J^dag X
      for (int idx = tid; idx < half * n; idx += nt) {
        const int k = idx / n, j = idx % n;
        R cs, sn, px, py;
        rot(k, cs, sn, px, py);
        if (sn == (R)0) continue;
        py = -py;
        const int p = sm.rp[k], q = sm.rq[k];
        T2 xp = H[p * LD + j], xq = H[q * LD + j];
        R qx = px * xq.x - py * xq.y, qy = px * xq.y + py * xq.x;
        H[p * LD + j] = T2{cs * xp.x - sn * qx, cs * xp.y - sn * qy};
        H[q * LD + j] = T2{sn * xp.x + cs * qx, sn * xp.y + cs * qy};
      }
      team_sync();
    }
  }
}

// Eigen-decomposition of the n x n Hermitian H (FP64, ld LD).  On return H is
// diagonal (ev), W holds the eigenvectors as columns.  Stage 1: Jacobi in
// FP32 on a copy until the off-diagonal falls to ~4e-6 of ||H||_F (FP32
// updates run at the full FP32 rate).  Stage 2: the FP32 eigenvectors are
// made unitary in FP64 by two Newton-Schulz steps W <- W (3 - W^dag W) / 2,
// H is transformed to W^dag H W, and FP64 Jacobi sweeps (typically two)
// finish the diagonalisation with W accumulating.  Returns false if the
// FP64 stage does not reach 2.5e-16 n ||H||_F within MAX_SWEEPS.
__device__ bool jacobi_herm(ChainSmem& sm, int n) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  double2* H = sm.H;
  double2* W = sm.W;
  double2* T = sm.T;
  float2* H32 = reinterpret_cast<float2*>(sm.T);
  float2* W32 = H32 + N2M * N2M;
  double loc = 0.0;
  for (int idx = tid; idx < n * n; idx += nt) {
    const int i = idx / n, j = idx % n;
    const double2 h = H[i * LD + j];
    loc += cabs2(h);
    H32[i * LD + j] = make_float2((float)h.x, (float)h.y);
    W32[i * LD + j] = make_float2(i == j ? 1.0f : 0.0f, 0.0f);
  }
  const double normF = sqrt(block_sum(loc, sm.red));
  // threshold Jacobi: a pair whose element is already far below the stage's
  // stop criterion is left alone (no work), the check still covers it
  const double conv32 = 4e-6 * normF, conv64 = 2.5e-16 * n * normF;
  jacobi_sweeps<float2, false>(sm, H32, W32, n, conv32, 1e-300 + 0.025 * conv32, 12);
  for (int idx = tid; idx < n * n; idx += nt) {
    const int i = idx / n, j = idx % n;
    const float2 w = W32[i * LD + j];
    W[i * LD + j] = cmk(w.x, w.y);
  }
  __syncthreads();
  for (int it = 0; it < 2; ++it) {
    for (int idx = tid; idx < n * n; idx += nt) {          // T = W^dag W
      const int i = idx / n, j = idx % n;
      double2 s = cmk(0, 0);
      for (int k = 0; k < n; ++k) cfma(s, cconj(W[k * LD + i]), W[k * LD + j]);
      T[i * LD + j] = s;
    }
    __syncthreads();
    for (int row = warp; row < n; row += nw) {               // W <- W (3 - T) / 2, row-wise
      double2 o0 = cmk(0, 0), o1 = cmk(0, 0);
      const int j0 = lane, j1 = lane + 32;
      for (int k = 0; k < n; ++k) {
        const double2 w = W[row * LD + k];
        if (j0 < n) {
          double2 m = cscale(T[k * LD + j0], -0.5);
          if (k == j0) m.x += 1.5;
          cfma(o0, w, m);
        }
        if (j1 < n) {
          double2 m = cscale(T[k * LD + j1], -0.5);
          if (k == j1) m.x += 1.5;
          cfma(o1, w, m);
        }
      }
      __syncwarp();
      if (j0 < n) W[row * LD + j0] = o0;
      if (j1 < n) W[row * LD + j1] = o1;
    }
    __syncthreads();
  }
  for (int idx = tid; idx < n * n; idx += nt) {            // T = H W
    const int i = idx / n, j = idx % n;
    double2 s = cmk(0, 0);
    for (int k = 0; k < n; ++k) cfma(s, H[i * LD + k], W[k * LD + j]);
    T[i * LD + j] = s;
  }
  __syncthreads();
  for (int idx = tid; idx < n * n; idx += nt) {            // H = W^dag T (Hermitian: i <= j)
    const int i = idx / n, j = idx % n;
    if (i > j) continue;
    double2 s = cmk(0, 0);
    for (int k = 0; k < n; ++k) cfma(s, cconj(W[k * LD + i]), T[k * LD + j]);
    if (i == j) s.y = 0.0;
    H[i * LD + j] = s;
    H[j * LD + i] = cconj(s);
  }
  __syncthreads();
  // stop at a few units of the FP64 rounding floor of one sweep (~n eps ||H||_F)
  const bool ok = jacobi_sweeps<double2, false>(sm, H, W, n, conv64, 1e-300 + 0.25 * conv64,
                                                MAX_SWEEPS);
  // then one sweep more over every nonzero pair, with no stop test: the
  // criterion above leaves off-diagonal elements up to ~n eps ||H||_F, which
  // turn the eigenvectors of a nearly degenerate pair (gap g) by ~that / g
  // (1e-8 at g ~ 5e-7, a mode kept just above the freeze threshold); one
  // more sweep takes every element to the rounding floor of a single sweep,
  // where the eigenvectors are as well determined as FP64 allows
  jacobi_sweeps<double2, false>(sm, H, W, n, -1.0, 1e-300, 1);
  for (int i = tid; i < n; i += nt) sm.ev[i] = H[i * LD + i].x;
  __syncthreads();
  return ok;
}

// Inverse of the n x n complex matrix M (ld NLM) into Inv (ld NLM) by
// Gauss-Jordan elimination with partial pivoting; M is destroyed.  Returns
// log|det M| in sm.dval[0]; sets ival[0] = 1 on a zero pivot.
__device__ void cinv(ChainSmem& sm, double2* M, double2* Inv, int n) {
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int idx = tid; idx < n * n; idx += nt) {
    int i = idx / n, j = idx % n;
    Inv[i * NLM + j] = cmk(i == j ? 1.0 : 0.0, 0.0);
  }
  if (tid == 0) { sm.dval[0] = 0.0; sm.dval[1] = 1.0; sm.ival[0] = 0; }
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (tid == 0) {
      int pr = k;
      double best = cabs2(M[k * NLM + k]);
      for (int i = k + 1; i < n; ++i) {
        double v = cabs2(M[i * NLM + k]);
        if (v > best) { best = v; pr = i; }
      }
      if (best == 0.0) sm.ival[0] = 1;
      sm.ival[1] = pr;
      const double2 pv = M[pr * NLM + k];       // the pivot after the row swap
      const double pm = cabs2(pv);
      const double ipm = pm > 0.0 ? rcp_fp64(pm) : 0.0;
      sm.pinv = cmk(pv.x * ipm, -pv.y * ipm);
      sm.dval[1] *= (best > 0.0 ? best : 1e-300);    // |pivots|^2 of a near-unitary-scale U
      if (k == n - 1) sm.dval[0] = 0.5 * log(sm.dval[1]);
    }
    __syncthreads();
    int pr = sm.ival[1];
    if (pr != k) {
      for (int j = tid; j < n; j += nt) {
        double2 t = M[k * NLM + j]; M[k * NLM + j] = M[pr * NLM + j]; M[pr * NLM + j] = t;
        t = Inv[k * NLM + j]; Inv[k * NLM + j] = Inv[pr * NLM + j]; Inv[pr * NLM + j] = t;
      }
    }
    __syncthreads();
    const double2 pinv = sm.pinv;
    for (int j = tid; j < n; j += nt) {
      M[k * NLM + j] = cmul(M[k * NLM + j], pinv);
      Inv[k * NLM + j] = cmul(Inv[k * NLM + j], pinv);
    }
    for (int i = tid; i < n; i += nt) sm.fac[i] = M[i * NLM + k];
    __syncthreads();
    for (int idx = tid; idx < n * n; idx += nt) {
      int i = idx / n, j = idx % n;
      if (i == k) continue;
      double2 f = sm.fac[i];
      M[i * NLM + j] = csub(M[i * NLM + j], cmul(f, M[k * NLM + j]));
      Inv[i * NLM + j] = csub(Inv[i * NLM + j], cmul(f, Inv[k * NLM + j]));
    }
    __syncthreads();
  }
}

// Paired form of the pure state on L = (r, a) from its covariance in A
// (n2 x n2, ld LD): Q = M (1 + N)^{-1} (Eq. (paired-form)).
__device__ void last_site(ChainSmem& sm, int nL, double2* Qout, int* status) {
  const int tid = threadIdx.x, nt = blockDim.x;
  double2* Nm = sm.H;      // (1 + N), ld NLM
  double2* Mm = sm.W;      // M, ld NLM
  for (int idx = tid; idx < nL * nL; idx += nt) {
    int i = idx / nL, j = idx % nL;
    double gxx = sm.A[i * LD + j], gpp = sm.A[(nL + i) * LD + nL + j];
    double gxp = sm.A[i * LD + nL + j], gpx = sm.A[(nL + i) * LD + j];
    Nm[i * NLM + j] = cmk(0.5 * (gxx + gpp) + (i == j ? 0.5 : 0.0), 0.5 * (gxp - gpx));
    Mm[i * NLM + j] = cmk(0.5 * (gxx - gpp), 0.5 * (gxp + gpx));
  }
  __syncthreads();
  cinv(sm, Nm, sm.Ui, nL);
  if (tid == 0 && sm.ival[0]) set_status(status, ST_NUMERIC);
  // Q = M (1+N)^{-1}, symmetrised
  for (int idx = tid; idx < nL * nL; idx += nt) {
    int i = idx / nL, j = idx % nL;
    double2 a = cmk(0, 0), b = cmk(0, 0);
    for (int k = 0; k < nL; ++k) {
      cfma(a, Mm[i * NLM + k], sm.Ui[k * NLM + j]);
      cfma(b, Mm[j * NLM + k], sm.Ui[k * NLM + i]);
    }
    Qout[i * QS + j] = cscale(cadd(a, b), 0.5);
  }
  __syncthreads();
}

__device__ void chain_body(ChainSmem& sm, const double* __restrict__ gam, int N,
                           const int* __restrict__ bwp, double freeze, double* __restrict__ Gs,
                           BondArrays ba, double2* __restrict__ Qm, double* __restrict__ cm,
                           int* status) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const long long twoN = 2LL * N;
  const int bw = max(1, min(*bwp, N));
  const int ldg = 2 * bw;
  double* Gc = Gs;
  double* Gn = Gs + (size_t)2 * NEM * ldg;
  int nin = 0;
  if (tid == 0) { ba.ne[0] = 0; ba.ne[N] = 0; }
  for (int m = 0; m < N; ++m) {
    const int nL = nin + 1, n2 = 2 * nL;
    // ---- reduced covariance of L_m (xxpp: r_1..r_nin, a_m | p's) --------
    for (int idx = tid; idx < n2 * n2; idx += nt) sm.A[(idx / n2) * LD + idx % n2] = 0.0;
    __syncthreads();
    for (int i = tid; i < nin; i += nt) {
      sm.A[i * LD + i] = 0.5 * sm.Dprev[i];
      sm.A[(nL + i) * LD + nL + i] = 0.5 * sm.Dprev[i];
      double gxx = Gc[i * ldg], gxp = Gc[i * ldg + bw];
      double gpx = Gc[(nin + i) * ldg], gpp = Gc[(nin + i) * ldg + bw];
      sm.A[i * LD + nin] = gxx;           sm.A[nin * LD + i] = gxx;
      sm.A[(nL + i) * LD + nin] = gpx;    sm.A[nin * LD + nL + i] = gpx;
      sm.A[i * LD + nL + nin] = gxp;      sm.A[(nL + nin) * LD + i] = gxp;
      sm.A[(nL + i) * LD + nL + nin] = gpp; sm.A[(nL + nin) * LD + nL + i] = gpp;
    }
    if (tid == 0) {
      sm.A[nin * LD + nin] = gam[m * twoN + m];
      sm.A[nin * LD + nL + nin] = gam[m * twoN + N + m];
      sm.A[(nL + nin) * LD + nin] = gam[(N + m) * twoN + m];
      sm.A[(nL + nin) * LD + nL + nin] = gam[(N + m) * twoN + N + m];
    }
    __syncthreads();
    if (m == N - 1) {
      last_site(sm, nL, Qm + (size_t)m * QS * QS, status);
      if (tid == 0) cm[m] = 1.0;
      break;
    }
    // ---- Cholesky of V = 2 Gamma_LL (lower, in place) -------------------
    for (int idx = tid; idx < n2 * n2; idx += nt) sm.A[(idx / n2) * LD + idx % n2] *= 2.0;
    __syncthreads();
    for (int k = 0; k < n2; ++k) {
      if (tid == 0) {                  // one thread: 1/sqrt(akk) by Newton from FP32
        double akk = sm.A[k * LD + k];
        if (!(akk > 0.0)) { set_status(status, ST_NUMERIC); akk = 1e-300; }
        const double r = rsqrt_fp64(akk);
        sm.dval[2] = akk * r;
        sm.dval[3] = r;
      }
      __syncthreads();
      const double ilkk = sm.dval[3];
      for (int i = k + 1 + tid; i < n2; i += nt) sm.A[i * LD + k] *= ilkk;
      if (tid == 0) sm.A[k * LD + k] = sm.dval[2];
      __syncthreads();
      const int w = n2 - k - 1;
      for (int idx = tid; idx < w * w; idx += nt) {
        int i = k + 1 + idx / w, j = k + 1 + idx % w;
        if (j <= i) sm.A[i * LD + j] -= sm.A[i * LD + k] * sm.A[j * LD + k];
      }
      __syncthreads();
    }
    for (int idx = tid; idx < n2 * n2; idx += nt) {
      int i = idx / n2, j = idx % n2;
      if (j > i) sm.A[i * LD + j] = 0.0;
    }
    __syncthreads();
    // ---- L^{-1} by forward substitution, one column per thread ----------
    // (the diagonal's inverses first, one FP64 division each; column j runs
    // on lane j / 8 of warp j % 8, so the columns' FP64 work is spread over
    // the SM's four sub-partitions)
    for (int i = tid; i < n2; i += nt) sm.ev[i] = 1.0 / sm.A[i * LD + i];
    __syncthreads();
    {
      const int j = (tid >> 5) + 8 * (tid & 31);
      if (j < n2 && tid < 256) {
        for (int i = 0; i < n2; ++i) {
          double x;
          if (i < j) x = 0.0;
          else if (i == j) x = sm.ev[i];
          else {
            double acc = 0.0;
            for (int k = j; k < i; ++k) acc += sm.A[i * LD + k] * sm.B[k * LD + j];
            x = -acc * sm.ev[i];
          }
          sm.B[i * LD + j] = x;
        }
      }
    }
    __syncthreads();
    // ---- H = i K, K = L^{-1} Omega L^{-T} --------------------------------
    for (int idx = tid; idx < n2 * n2; idx += nt) {
      int i = idx / n2, j = idx % n2;
      double s = 0.0;
      for (int k = 0; k < nL; ++k)
        s += sm.B[i * LD + k] * sm.B[j * LD + nL + k] - sm.B[i * LD + nL + k] * sm.B[j * LD + k];
      sm.H[i * LD + j] = cmk(0.0, s);
    }
    __syncthreads();
    bool ok = jacobi_herm(sm, n2);
    if (!ok && tid == 0) set_status(status, ST_NOT_CONVERGED);
    // ---- order eigenvalues: positive half ascending = D descending ------
    // (a rank per eigenvalue, ties by index: the same order as a stable sort;
    // a NaN eigenvalue flags the cut and keeps every index in range)
    for (int i = tid; i < n2; i += nt) sm.perm[i] = i;
    __syncthreads();
    for (int i = tid; i < n2; i += nt) {
      const double e = sm.ev[i];
      if (e != e) { set_status(status, ST_NUMERIC); continue; }
      int rank = 0;
      for (int j = 0; j < n2; ++j) rank += (sm.ev[j] < e || (sm.ev[j] == e && j < i)) ? 1 : 0;
      sm.perm[rank] = i;
    }
    __syncthreads();
    {
      const int q = (tid & 31) * 8 + (tid >> 5);     // spread over the sub-partitions
      if (q < nL) {
        double e = sm.ev[sm.perm[nL + q]];
        if (!(e > 0.0)) { set_status(status, ST_NUMERIC); e = 1.0; }
        sm.Dq[q] = rcp_fp64(e);
        sm.rsD[q] = 1.4142135623730951 * e * rsqrt_fp64(e);   // sqrt(2) / sqrt(D_q)
      }
    }
    __syncthreads();
    // ---- S = L O diag(D, D)^{-1/2} into B --------------------------------
    for (int idx = tid; idx < n2 * n2; idx += nt) {
      int i = idx / n2, c = idx % n2;
      int q = c < nL ? c : c - nL;
      int col = sm.perm[nL + q];
      double s = 0.0;
      for (int k = 0; k <= i; ++k) {
        double2 w = sm.W[k * LD + col];
        s += sm.A[i * LD + k] * (c < nL ? w.y : w.x);
      }
      sm.B[i * LD + c] = s * sm.rsD[q];
    }
    __syncthreads();
    // ---- U, V (a = U b + V^* b^dag) --------------------------------------
    for (int idx = tid; idx < nL * nL; idx += nt) {
      int i = idx / nL, j = idx % nL;
      double s11 = sm.B[i * LD + j], s12 = sm.B[i * LD + nL + j];
      double s21 = sm.B[(nL + i) * LD + j], s22 = sm.B[(nL + i) * LD + nL + j];
      sm.U[i * NLM + j] = cmk(0.5 * (s11 + s22), 0.5 * (s21 - s12));
      sm.V[i * NLM + j] = cmk(0.5 * (s11 - s22), -0.5 * (s21 + s12));
    }
    __syncthreads();
    // ---- canonical gauge: largest |U_jq| of each column real positive ----
    for (int q = (tid & 31) * 8 + (tid >> 5); q < nL; q += nt) {   // spread over sub-partitions
      int jb = 0;
      double best = -1.0;
      for (int j = 0; j < nL; ++j) {
        double v = cabs2(sm.U[j * NLM + q]);
        if (v > best) { best = v; jb = j; }
      }
      double2 u = sm.U[jb * NLM + q];
      const double img = rsqrt_fp64(best);
      double2 ph = cmk(u.x * img, -u.y * img);
      for (int j = 0; j < nL; ++j) {
        sm.U[j * NLM + q] = cmul(sm.U[j * NLM + q], ph);
        sm.V[j * NLM + q] = cmul(sm.V[j * NLM + q], ph);
      }
    }
    if (tid == 0) {
      int na = 0;
      // Lambda^2 = (D - 1) / (D + 1) > freeze, without the division (D + 1 > 0)
      while (na < nL && sm.Dq[na] - 1.0 > freeze * (sm.Dq[na] + 1.0)) ++na;
      if (na > NEM) { set_status(status, ST_BOUNDS); na = NEM; }
      sm.ival[2] = na;
    }
    __syncthreads();
    const int na = sm.ival[2];
    // ---- U^{-1} and |det U| ----------------------------------------------
    for (int idx = tid; idx < nL * nL; idx += nt) {        // work copy, ld NLM
      int i = idx / nL, j = idx % nL;
      sm.H[i * NLM + j] = sm.U[i * NLM + j];
    }
    __syncthreads();
    cinv(sm, sm.H, sm.Ui, nL);
    if (tid == 0) {
      if (sm.ival[0]) set_status(status, ST_NUMERIC);
      cm[m] = exp(-0.5 * sm.dval[0]);
    }
    // ---- local paired form Q^m over (r_{m-1}, a_m, l_m), App. A ----------
    double2* Qo = Qm + (size_t)m * QS * QS;
    const int nq = nL + na;
    for (int idx = tid; idx < nq * nq; idx += nt) {
      int i = idx / nq, j = idx % nq;
      double2 v = cmk(0, 0);
      if (i < nL && j < nL) {            // U^-dag V^dag: sum_k conj(Ui_ki) conj(V_jk)
        for (int k = 0; k < nL; ++k) cfma(v, cconj(sm.Ui[k * NLM + i]), cconj(sm.V[j * NLM + k]));
        double2 w = cmk(0, 0);
        for (int k = 0; k < nL; ++k) cfma(w, cconj(sm.Ui[k * NLM + j]), cconj(sm.V[i * NLM + k]));
        v = cscale(cadd(v, w), 0.5);
      } else if (i < nL) {               // U^-dag restricted: conj(Ui_{q i})
        v = cconj(sm.Ui[(j - nL) * NLM + i]);
      } else if (j < nL) {               // U^-* : conj(Ui_{q j})
        v = cconj(sm.Ui[(i - nL) * NLM + j]);
      } else {                           // -V^T U^-dag: -sum_k V_kq conj(Ui_q'k)
        int q = i - nL, qp = j - nL;
        double2 w = cmk(0, 0);
        for (int k = 0; k < nL; ++k) {
          cfma(v, sm.V[k * NLM + q], cconj(sm.Ui[qp * NLM + k]));
          cfma(w, sm.V[k * NLM + qp], cconj(sm.Ui[q * NLM + k]));
        }
        v = cscale(cadd(v, w), -0.5);
      }
      Qo[i * QS + j] = v;
    }
    // ---- rows of S^{-1} for the active b modes (into A) -------------------
    for (int idx = tid; idx < na * nL; idx += nt) {
      int q = idx / nL, j = idx % nL;
      double2 u = sm.U[j * NLM + q], v = sm.V[j * NLM + q];
      sm.A[q * LD + j] = u.x - v.x;                 // x_b <- x
      sm.A[q * LD + nL + j] = u.y + v.y;            // x_b <- p
      sm.A[(na + q) * LD + j] = v.y - u.y;          // p_b <- x
      sm.A[(na + q) * LD + nL + j] = u.x + v.x;     // p_b <- p
    }
    if (tid < na) {
      double D = sm.Dq[tid];
      ba.lam2[(size_t)(m + 1) * NEM + tid] = (D - 1.0) / (D + 1.0);
    }
    if (tid == 0) ba.ne[m + 1] = na;
    __syncthreads();
    // ---- propagate: G_new = S^{-1}_act cov(L_m, a_{m+1 .. m+bw}) ---------
    for (int idx = tid; idx < 2 * na * ldg; idx += nt) {
      int rr = idx / ldg, c = idx % ldg;
      int isp = c >= bw;
      int cc = isp ? c - bw : c;         // mode m+1+cc
      int mode = m + 1 + cc;
      double s = 0.0;
      if (mode < N) {
        for (int k = 0; k < n2; ++k) {
          double g;
          bool kp = k >= nL;
          int kk = kp ? k - nL : k;
          if (kk < nin) {                // r row: carried G column cc+1
            g = (cc + 1 < bw) ? Gc[(kp ? nin + kk : kk) * ldg + (isp ? bw : 0) + cc + 1] : 0.0;
          } else {                       // a_m row
            long long row = kp ? (N + m) : m;
            long long col = isp ? (N + mode) : mode;
            g = gam[row * twoN + col];
          }
          s += sm.A[rr * LD + k] * g;
        }
      }
      Gn[rr * ldg + c] = s;
    }
    if (tid < na) sm.Dprev[tid] = sm.Dq[tid];
    __syncthreads();
    double* t = Gc; Gc = Gn; Gn = t;
    nin = na;
  }
}

__global__ void __launch_bounds__(CHAIN_THREADS)
gsvd_chain_kernel(const double* __restrict__ gam, int N, const int* __restrict__ bwp,
                  double freeze, double* __restrict__ Gs, BondArrays ba,
                  double2* __restrict__ Qm, double* __restrict__ cm, int* status) {
  extern __shared__ __align__(16) unsigned char smraw[];
  chain_body(*reinterpret_cast<ChainSmem*>(smraw), gam, N, bwp, freeze, Gs, ba, Qm, cm, status);
}

// many states at once: CTA b walks the chain of state b (the chains are
// independent, so a batch runs them side by side, one SM each)
__global__ void __launch_bounds__(CHAIN_THREADS)
gsvd_chain_batch_kernel(const ChainJob* __restrict__ jobs, int* status) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const ChainJob j = jobs[blockIdx.x];
  chain_body(*reinterpret_cast<ChainSmem*>(smraw), j.gamma, j.N, j.bw, j.freeze, j.G, j.ba, j.Qm,
             j.cm, status);
}

// ---- input checks -----------------------------------------------------------
// max |Gamma - Gamma^T| and max |(2 Gamma Omega)^2 + 1|, tiled 32 x 32.
__global__ void check_input_kernel(const double* __restrict__ g, int N,
                                   unsigned long long* maxes) {
  __shared__ double ta[32][33], tb[32][33];
  const int n = 2 * N;
  const int bi = blockIdx.y * 32, bj = blockIdx.x * 32;
  const int ty = threadIdx.y, tx = threadIdx.x;   // 32 x 8
  double acc[4] = {0, 0, 0, 0};
  double asym = 0.0;
  for (int k0 = 0; k0 < n; k0 += 32) {
    for (int r = ty; r < 32; r += 8) {
      int i = bi + r, k = k0 + tx;
      // X_ik = 2 (Gamma Omega)_ik : k < N -> -2 G[i][k+N]; k >= N -> 2 G[i][k-N]
      double x = 0.0;
      if (i < n && k < n) x = (k < N) ? -2.0 * g[(size_t)i * n + k + N] : 2.0 * g[(size_t)i * n + k - N];
      ta[r][tx] = x;
      int kk = k0 + r, j = bj + tx;
      double y = 0.0;
      if (kk < n && j < n) y = (j < N) ? -2.0 * g[(size_t)kk * n + j + N] : 2.0 * g[(size_t)kk * n + j - N];
      tb[r][tx] = y;
    }
    __syncthreads();
    for (int q = 0; q < 4; ++q) {
      int r = ty + 8 * q;
      double s = acc[q];
      for (int k = 0; k < 32; ++k) s += ta[r][k] * tb[k][tx];
      acc[q] = s;
    }
    __syncthreads();
  }
  double dev = 0.0;
  for (int q = 0; q < 4; ++q) {
    int i = bi + ty + 8 * q, j = bj + tx;
    if (i < n && j < n) {
      dev = fmax(dev, fabs(acc[q] + (i == j ? 1.0 : 0.0)));
      asym = fmax(asym, fabs(g[(size_t)i * n + j] - g[(size_t)j * n + i]));
    }
  }
  atomicMax(&maxes[0], __double_as_longlong(asym));
  atomicMax(&maxes[1], __double_as_longlong(dev));
}

__global__ void check_finish_kernel(const unsigned long long* maxes, double tol, int* status) {
  double asym = __longlong_as_double(maxes[0]);
  double dev = __longlong_as_double(maxes[1]);
  if (!(asym <= 1e-12)) set_status(status, ST_NOT_SYMMETRIC);
  if (!(dev <= tol)) set_status(status, ST_NOT_PURE);
}

__global__ void bandwidth_kernel(const double* __restrict__ g, int N, int* bw) {
  const int n = 2 * N;
  int best = 0;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < (size_t)n * n;
       idx += (size_t)gridDim.x * blockDim.x) {
    int i = idx / n, j = idx % n;
    if (g[idx] != 0.0) best = max(best, abs((i % N) - (j % N)));
  }
  for (int o = 16; o > 0; o >>= 1) best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
  if ((threadIdx.x & 31) == 0) atomicMax(bw, best);
}

// ---- Q -> Gamma: N = (1 - Q^* Q)^{-1} - 1, M = Q (1 + N) --------------------
__global__ void q_prep_kernel(const double2* __restrict__ Q, int N, double2* X) {
  // X = 1 - Q^* Q  (N x N)
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < (size_t)N * N;
       idx += (size_t)gridDim.x * blockDim.x) {
    int i = idx / N, j = idx % N;
    double2 s = cmk(i == j ? 1.0 : 0.0, 0.0);
    for (int k = 0; k < N; ++k) {
      double2 p = cmul(cconj(Q[(size_t)i * N + k]), Q[(size_t)k * N + j]);
      s = csub(s, p);
    }
    X[idx] = s;
  }
}

// in-place Gauss-Jordan step k on X (Hermitian positive definite: no pivoting)
__global__ void gj_save_kernel(const double2* X, int N, int k, double2* rowk, double2* colk) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < N; t += gridDim.x * blockDim.x) {
    rowk[t] = X[(size_t)k * N + t];
    colk[t] = X[(size_t)t * N + k];
  }
}
__global__ void gj_step_kernel(double2* X, int N, int k, const double2* rowk,
                               const double2* colk, int* status) {
  double2 piv = rowk[k];
  double pm = cabs2(piv);
  if (pm == 0.0) { if (blockIdx.x == 0 && threadIdx.x == 0) set_status(status, ST_NUMERIC); return; }
  double2 pinv = cmk(piv.x / pm, -piv.y / pm);
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < (size_t)N * N;
       idx += (size_t)gridDim.x * blockDim.x) {
    int i = idx / N, j = idx % N;
    double2 v;
    if (i == k && j == k) v = pinv;
    else if (i == k) v = cmul(rowk[j], pinv);
    else if (j == k) v = cmul(cscale(colk[i], -1.0), pinv);
    else v = csub(X[idx], cmul(cmul(colk[i], rowk[j]), pinv));
    X[idx] = v;
  }
}
__global__ void q_finish_kernel(const double2* __restrict__ Q, const double2* __restrict__ Xi,
                                int N, double* __restrict__ g) {
  // (1 + N) = Xi ; M = Q Xi
  const int n = 2 * N;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < (size_t)N * N;
       idx += (size_t)gridDim.x * blockDim.x) {
    int i = idx / N, j = idx % N;
    double2 nn = Xi[idx];
    nn.x -= (i == j) ? 1.0 : 0.0;
    double2 mm = cmk(0, 0);
    for (int k = 0; k < N; ++k) cfma(mm, Q[(size_t)i * N + k], Xi[(size_t)k * N + j]);
    double2 nt = Xi[(size_t)j * N + i];   // for symmetric averaging of N (Hermitian)
    nt.x -= (i == j) ? 1.0 : 0.0;
    double nre = 0.5 * (nn.x + nt.x), nim = 0.5 * (nn.y - nt.y);
    g[(size_t)i * n + j] = nre + mm.x + ((i == j) ? 0.5 : 0.0);            // xx
    g[(size_t)(N + i) * n + N + j] = nre - mm.x + ((i == j) ? 0.5 : 0.0);  // pp
    g[(size_t)i * n + N + j] = nim + mm.y;                                  // xp
    g[(size_t)(N + i) * n + j] = mm.y - nim;                                // px
  }
}

}  // namespace

cudaError_t launch_check_input(const double* gamma, int N, double purity_tol,
                               double* work, int* status, cudaStream_t s) {
  unsigned long long* maxes = reinterpret_cast<unsigned long long*>(work);
  cudaError_t e = cudaMemsetAsync(maxes, 0, 2 * sizeof(unsigned long long), s);
  if (e) return e;
  int nb = (2 * N + 31) / 32;
  check_input_kernel<<<dim3(nb, nb), dim3(32, 8), 0, s>>>(gamma, N, maxes);
  check_finish_kernel<<<1, 1, 0, s>>>(maxes, purity_tol, status);
  return cudaGetLastError();
}

cudaError_t launch_bandwidth(const double* gamma, int N, int* bw, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(bw, 0, sizeof(int), s);
  if (e) return e;
  size_t n = (size_t)4 * N * N;
  int blocks = (int)((n + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  bandwidth_kernel<<<blocks, 256, 0, s>>>(gamma, N, bw);
  return cudaGetLastError();
}

cudaError_t launch_q_to_gamma(const double2* Q, int N, double* gamma, double2* work,
                              int* status, cudaStream_t s) {
  double2* X = work;
  double2* rowk = work + (size_t)N * N;
  double2* colk = rowk + N;
  int blocks = (int)(((size_t)N * N + 255) / 256);
  if (blocks > 8192) blocks = 8192;
  q_prep_kernel<<<blocks, 256, 0, s>>>(Q, N, X);
  for (int k = 0; k < N; ++k) {
    gj_save_kernel<<<(N + 255) / 256, 256, 0, s>>>(X, N, k, rowk, colk);
    gj_step_kernel<<<blocks, 256, 0, s>>>(X, N, k, rowk, colk, status);
  }
  cudaError_t e = cudaMemsetAsync(gamma, 0, sizeof(double) * 4 * (size_t)N * N, s);
  if (e) return e;
  q_finish_kernel<<<blocks, 256, 0, s>>>(Q, X, N, gamma);
  return cudaGetLastError();
}

cudaError_t launch_gsvd_chain(const double* gamma, int N, const int* bw,
                              double lambda2_freeze, double* Gscratch, BondArrays ba,
                              double2* Qm, double* cm, int* status, cudaStream_t s) {
  size_t smem = sizeof(ChainSmem);
  cudaError_t e = cudaFuncSetAttribute(gsvd_chain_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e) return e;
  gsvd_chain_kernel<<<1, CHAIN_THREADS, smem, s>>>(gamma, N, bw, lambda2_freeze, Gscratch,
                                                   ba, Qm, cm, status);
  return cudaGetLastError();
}

cudaError_t launch_gsvd_chain_batch(const ChainJob* jobs_dev, int count, int* status,
                                    cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  size_t smem = sizeof(ChainSmem);
  cudaError_t e = cudaFuncSetAttribute(gsvd_chain_batch_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e) return e;
  gsvd_chain_batch_kernel<<<count, CHAIN_THREADS, smem, s>>>(jobs_dev, status);
  return cudaGetLastError();
}
