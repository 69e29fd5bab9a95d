// Projected-creation-operator (PCO) construction of local MPS tensors
// (Sec. II C, App. B), one CTA per tensor.
//
// The projected state P_V exp(1/2 d^dag Q d^dag)|0> is a product of commuting
// PCOs (Sec. II C); the closure identity P d^dag = P d^dag P lets the
// projector pass through any grouping of them.  The kernel groups them for
// the GPU:
//   1. left-only PCOs (r_q r_q' and r_q r_q) on a D_l vector u = P exp(X_LL)|0>,
//      right-only PCOs on a D_r vector w; C0 = u w^T is their product state;
//   2. cross PCOs exp(g r_q^dag l_q'^dag) on the D_l x D_r matrix C0;
//   3. the physical PCOs last: with l_L = sum_q Q_{r_q a} r_q^dag and
//      l_R = sum_q' Q_{a l_q'} l_q'^dag,
//        exp(a^dag (l_L + l_R) + g_aa a^dag^2 / 2) =
//        sum_p (a^dag)^p sum_k (g_aa/2)^k/k! sum_{i+j=p-2k} l_L^i l_R^j/(i! j!),
//      so A[., p, .] = c sqrt(p!) sum_k (g_aa/2)^k/k! sum_{i+j=p-2k}
//      (l_L^i C0 (l_R^T)^j)/(i! j!).
// Every PCO update is a pull along the lowering maps: the source of a target
// state with kappa quanta added to modes (q, q') is reached by kappa steps
// of low_q and low_q'; coefficients g^kappa/kappa! sqrt(n!/(n-kappa)!) are
// built as running products.  Each pass is out of place (double buffered);
// the paper's in-place reverse-ordered loop computes the same numbers.
#include "internal.h"
#include <math.h>

namespace {

constexpr int PCO_THREADS = 512;
constexpr int SQ_N = 260;

struct PcoSmem {
  double2 Q[QS * QS];
  double sq[SQ_N];
  int mol[NEM], mor[NEM];
  double2 coef[130];
};

__device__ inline int occ_of(const uint8_t* occ, int idx, int q) { return occ[(size_t)idx * NEM + q]; }

__global__ void __launch_bounds__(PCO_THREADS)
pco_kernel(const SiteTask* __restrict__ tasks, int d, double2* __restrict__ scratch,
           int* status) {
  __shared__ PcoSmem sm;
  const SiteTask t = tasks[blockIdx.x];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int nl = t.nl, nr = t.nr, Dl = t.Dl, Dr = t.Dr;
  const int nm = nl + 1 + nr;
  const int ia = nl;                         // index of a_m in c_m
  for (int idx = tid; idx < nm * nm; idx += nt)
    sm.Q[(idx / nm) * QS + idx % nm] = t.Q[(size_t)(idx / nm) * t.qs + idx % nm];
  for (int k = tid; k < SQ_N; k += nt) sm.sq[k] = sqrt((double)k);
  if (tid < NEM) { sm.mol[tid] = 0; sm.mor[tid] = 0; }
  __syncthreads();
  for (int idx = tid; idx < Dl * nl; idx += nt) atomicMax(&sm.mol[idx % nl], occ_of(t.occl, idx / nl, idx % nl));
  for (int idx = tid; idx < Dr * nr; idx += nt) atomicMax(&sm.mor[idx % nr], occ_of(t.occr, idx / nr, idx % nr));
  __syncthreads();
  for (int q = tid; q < nl; q += nt) if (sm.mol[q] >= SQ_N - 4) set_status(status, ST_BOUNDS);
  for (int q = tid; q < nr; q += nt) if (sm.mor[q] >= SQ_N - 4) set_status(status, ST_BOUNDS);

  const size_t DD = (size_t)Dl * Dr;
  double2* base = scratch + t.scratch_off;
  double2* u = base;
  double2* u2 = u + Dl;
  double2* w = u2 + Dl;
  double2* w2 = w + Dr;
  double2* Bf[4] = {w2 + Dr, w2 + Dr + DD, w2 + Dr + 2 * DD, w2 + Dr + 3 * DD};

  // ---- 1. one-sided PCOs on vectors --------------------------------------
  for (int side = 0; side < 2; ++side) {
    const int n = side == 0 ? nl : nr;
    const int D = side == 0 ? Dl : Dr;
    const uint8_t* occ = side == 0 ? t.occl : t.occr;
    const int* low = side == 0 ? t.lowl : t.lowr;
    const int cap = side == 0 ? t.capl : t.capr;
    const int* mo = side == 0 ? sm.mol : sm.mor;
    const int off = side == 0 ? 0 : nl + 1;
    double2* x = side == 0 ? u : w;
    double2* y = side == 0 ? u2 : w2;
    for (int i = tid; i < D; i += nt) x[i] = cmk(i == 0 ? 1.0 : 0.0, 0.0);
    __syncthreads();
    for (int q = 0; q < n; ++q) {
      for (int q2 = q; q2 < n; ++q2) {
        if (q == q2 ? mo[q] < 2 : (mo[q] == 0 || mo[q2] == 0)) continue;
        const double2 g = sm.Q[(off + q) * QS + off + q2];
        const int* lq = low + (size_t)q * cap;
        const int* lq2 = low + (size_t)q2 * cap;
        for (int mu = tid; mu < D; mu += nt) {
          double2 acc = x[mu];
          double2 tk = cmk(1.0, 0.0);
          int s = mu;
          const int a = occ_of(occ, mu, q);
          if (q != q2) {
            const int b = occ_of(occ, mu, q2);
            const int kmax = min(a, b);
            for (int k = 1; k <= kmax; ++k) {
              s = lq2[lq[s]];
              tk = cscale(cmul(tk, g), sm.sq[a - k + 1] * sm.sq[b - k + 1] / k);
              cfma(acc, tk, x[s]);
            }
          } else {
            const double2 gh = cscale(g, 0.5);
            for (int j = 1; 2 * j <= a; ++j) {
              s = lq[lq[s]];
              tk = cscale(cmul(tk, gh), sm.sq[a - 2 * j + 2] * sm.sq[a - 2 * j + 1] / j);
              cfma(acc, tk, x[s]);
            }
          }
          y[mu] = acc;
        }
        __syncthreads();
        double2* tt = x; x = y; y = tt;
      }
    }
    if (side == 0) { u = x; u2 = y; } else { w = x; w2 = y; }
  }
  // ---- C0 = u w^T ----------------------------------------------------------
  double2* cur = Bf[0];
  double2* nxt = Bf[1];
  for (size_t idx = tid; idx < DD; idx += nt) cur[idx] = cmul(u[idx / Dr], w[idx % Dr]);
  __syncthreads();
  // ---- 2. cross PCOs -------------------------------------------------------
  for (int q = 0; q < nl; ++q) {
    if (sm.mol[q] == 0) continue;
    const int* lq = t.lowl + (size_t)q * t.capl;
    for (int q2 = 0; q2 < nr; ++q2) {
      if (sm.mor[q2] == 0) continue;
      const double2 g = sm.Q[q * QS + nl + 1 + q2];
      const int* lr = t.lowr + (size_t)q2 * t.capr;
      for (size_t idx = tid; idx < DD; idx += nt) {
        const int mu = idx / Dr, nu = idx % Dr;
        const int a = occ_of(t.occl, mu, q), b = occ_of(t.occr, nu, q2);
        const int kmax = min(a, b);
        double2 acc = cur[idx];
        double2 tk = cmk(1.0, 0.0);
        int s = mu, r = nu;
        for (int k = 1; k <= kmax; ++k) {
          s = lq[s];
          r = lr[r];
          tk = cscale(cmul(tk, g), sm.sq[a - k + 1] * sm.sq[b - k + 1] / k);
          cfma(acc, tk, cur[(size_t)s * Dr + r]);
        }
        nxt[idx] = acc;
      }
      __syncthreads();
      double2* tt = cur; cur = nxt; nxt = tt;
    }
  }
  // ---- 3. physical PCOs: A[., p, .] ----------------------------------------
  double2* A = t.out;
  for (size_t idx = tid; idx < DD * d; idx += nt) A[idx] = cmk(0.0, 0.0);
  const double2 gaa2 = cscale(sm.Q[ia * QS + ia], 0.5);
  double2* P = cur;              // l_L^i C0
  double2* Pn = nxt;
  double2* Ya = Bf[2];
  double2* Yb = Bf[3];
  for (int i = 0; i < d; ++i) {
    if (i > 0) {
      if (nl == 0) break;
      __syncthreads();
      for (size_t idx = tid; idx < DD; idx += nt) {
        const int mu = idx / Dr, nu = idx % Dr;
        double2 acc = cmk(0.0, 0.0);
        for (int q = 0; q < nl; ++q) {
          const int a = occ_of(t.occl, mu, q);
          if (a == 0) continue;
          const int s = t.lowl[(size_t)q * t.capl + mu];
          cfma(acc, cscale(sm.Q[q * QS + ia], sm.sq[a]), P[(size_t)s * Dr + nu]);
        }
        Pn[idx] = acc;
      }
      __syncthreads();
      double2* tt = P; P = Pn; Pn = tt;
    }
    const double2* Ysrc = P;
    for (int j = 0; i + j < d; ++j) {
      // coefficients of this (i, j): c sqrt(p!) (g/2)^k / (k! i! j!), p = i + j + 2k
      const int kmx = (d - 1 - i - j) / 2;
      __syncthreads();
      if (tid == 0) {
        double2 gp = cmk(1.0, 0.0);
        for (int k = 0; k <= kmx && k < 130; ++k) {
          const int p = i + j + 2 * k;
          double lg = 0.5 * lgamma(p + 1.0) - lgamma(k + 1.0) - lgamma(i + 1.0) - lgamma(j + 1.0);
          sm.coef[k] = cscale(gp, t.c * exp(lg));
          gp = cmul(gp, gaa2);
        }
      }
      if (j > 0) {
        if (nr == 0) break;
        double2* Yn = (Ysrc == Ya) ? Yb : Ya;
        for (size_t idx = tid; idx < DD; idx += nt) {
          const int mu = idx / Dr, nu = idx % Dr;
          double2 acc = cmk(0.0, 0.0);
          for (int q = 0; q < nr; ++q) {
            const int b = occ_of(t.occr, nu, q);
            if (b == 0) continue;
            const int r = t.lowr[(size_t)q * t.capr + nu];
            cfma(acc, cscale(sm.Q[ia * QS + nl + 1 + q], sm.sq[b]), Ysrc[(size_t)mu * Dr + r]);
          }
          Yn[idx] = acc;
        }
        __syncthreads();
        Ysrc = Yn;
      } else {
        __syncthreads();
      }
      for (size_t idx = tid; idx < DD; idx += nt) {
        const int mu = idx / Dr, nu = idx % Dr;
        const double2 y = Ysrc[idx];
        for (int k = 0; k <= kmx; ++k) {
          const int p = i + j + 2 * k;
          double2* dst = A + ((size_t)mu * d + p) * Dr + nu;
          double2 v = *dst;
          cfma(v, sm.coef[k], y);
          *dst = v;
        }
      }
    }
  }
}

// lowering maps of an arbitrary down-closed basis (expert entry): brute search
__global__ void maps_brute_kernel(const uint8_t* __restrict__ occ, int D, int n, int* low,
                                  int cap, int* status) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < D * n; idx += gridDim.x * blockDim.x) {
    const int beta = idx / n, q = idx % n;
    const uint8_t* v = occ + (size_t)beta * NEM;
    int found = -1;
    if (v[q] > 0) {
      for (int i = 0; i < D && found < 0; ++i) {
        const uint8_t* u = occ + (size_t)i * NEM;
        bool eq = true;
        for (int k = 0; k < n && eq; ++k) eq = (u[k] == v[k] - (k == q ? 1 : 0));
        if (eq) found = i;
      }
      if (found < 0) set_status(status, ST_BOUNDS);
    }
    low[(size_t)q * cap + beta] = found;
  }
}

}  // namespace

size_t pco_scratch_elems(int Dl, int Dr) {
  return 2 * (size_t)Dl + 2 * (size_t)Dr + 4 * (size_t)Dl * Dr;
}

cudaError_t launch_pco(const SiteTask* tasks_dev, int ntasks, int d, int precision,
                       double2* scratch, int* status, cudaStream_t s) {
  (void)precision;
  pco_kernel<<<ntasks, PCO_THREADS, 0, s>>>(tasks_dev, d, scratch, status);
  return cudaGetLastError();
}

cudaError_t launch_maps_brute(const uint8_t* occ, int D, int n, int* low, int cap,
                              int* status, cudaStream_t s) {
  int blocks = (D * n + 255) / 256;
  if (blocks < 1) blocks = 1;
  maps_brute_kernel<<<blocks, 256, 0, s>>>(occ, D, n, low, cap, status);
  return cudaGetLastError();
}
