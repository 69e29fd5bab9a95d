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
// T = double is the FP64 path; T = float runs the same passes in FP32 (the
// mixed-precision build) and accumulates the output tensor in FP64.
#include "internal.h"
#include <algorithm>
#include <math.h>

namespace {

constexpr int PCO_THREADS = 512;
constexpr int SQ_N = 260;

struct PcoSmem {
  double2 Q[QS * QS];
  double sq[SQ_N];
  double ik[SQ_N];          // 1 / k: the loops multiply instead of dividing in FP64
  int mol[NEM], mor[NEM];
  double2 coef[130];
};

__device__ inline int occ_of(const uint8_t* occ, int idx, int q) { return occ[(size_t)idx * NEM + q]; }

template <typename T>
__device__ void pco_site(PcoSmem& sm, const SiteTask& t, int d, double2* __restrict__ scratch,
                         int* status) {
  using C2 = typename Cx<T>::type;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int nl = t.nl, nr = t.nr, Dl = t.Dl, Dr = t.Dr;
  const int nm = nl + 1 + nr;
  const int ia = nl;                         // index of a_m in c_m
  for (int idx = tid; idx < nm * nm; idx += nt)
    sm.Q[(idx / nm) * QS + idx % nm] = t.Q[(size_t)(idx / nm) * t.qs + idx % nm];
  for (int k = tid; k < SQ_N; k += nt) {
    sm.sq[k] = sqrt((double)k);
    sm.ik[k] = k > 0 ? 1.0 / k : 0.0;
  }
  if (tid < NEM) { sm.mol[tid] = 0; sm.mor[tid] = 0; }
  __syncthreads();
  for (int idx = tid; idx < Dl * nl; idx += nt) atomicMax(&sm.mol[idx % nl], occ_of(t.occl, idx / nl, idx % nl));
  for (int idx = tid; idx < Dr * nr; idx += nt) atomicMax(&sm.mor[idx % nr], occ_of(t.occr, idx / nr, idx % nr));
  __syncthreads();
  for (int q = tid; q < nl; q += nt) if (sm.mol[q] >= SQ_N - 4) set_status(status, ST_BOUNDS);
  for (int q = tid; q < nr; q += nt) if (sm.mor[q] >= SQ_N - 4) set_status(status, ST_BOUNDS);

  const size_t DD = (size_t)Dl * Dr;
  C2* base = reinterpret_cast<C2*>(scratch);
  C2* u = base;
  C2* u2 = u + Dl;
  C2* w = u2 + Dl;
  C2* w2 = w + Dr;
  C2* Bf[4] = {w2 + Dr, w2 + Dr + DD, w2 + Dr + 2 * DD, w2 + Dr + 3 * DD};
  const C2 zero = to_c<C2>(cmk(0.0, 0.0));
  const C2 one = to_c<C2>(cmk(1.0, 0.0));

  // ---- 1. one-sided PCOs on vectors --------------------------------------
  for (int side = 0; side < 2; ++side) {
    const int n = side == 0 ? nl : nr;
    const int D = side == 0 ? Dl : Dr;
    const uint8_t* occ = side == 0 ? t.occl : t.occr;
    const int* low = side == 0 ? t.lowl : t.lowr;
    const int cap = side == 0 ? t.capl : t.capr;
    const int* mo = side == 0 ? sm.mol : sm.mor;
    const int off = side == 0 ? 0 : nl + 1;
    C2* x = side == 0 ? u : w;
    C2* y = side == 0 ? u2 : w2;
    for (int i = tid; i < D; i += nt) x[i] = i == 0 ? one : zero;
    __syncthreads();
    for (int q = 0; q < n; ++q) {
      for (int q2 = q; q2 < n; ++q2) {
        if (q == q2 ? mo[q] < 2 : (mo[q] == 0 || mo[q2] == 0)) continue;
        const C2 g = to_c<C2>(sm.Q[(off + q) * QS + off + q2]);
        const int* lq = low + (size_t)q * cap;
        const int* lq2 = low + (size_t)q2 * cap;
        for (int mu = tid; mu < D; mu += nt) {
          C2 acc = x[mu];
          C2 tk = one;
          int s = mu;
          const int a = occ_of(occ, mu, q);
          if (q != q2) {
            const int b = occ_of(occ, mu, q2);
            const int kmax = min(a, b);
            for (int k = 1; k <= kmax; ++k) {
              s = lq2[lq[s]];
              tk = cscale(cmul(tk, g), (T)(sm.sq[a - k + 1] * sm.sq[b - k + 1] * sm.ik[k]));
              cfma(acc, tk, x[s]);
            }
          } else {
            const C2 gh = cscale(g, (T)0.5);
            for (int j = 1; 2 * j <= a; ++j) {
              s = lq[lq[s]];
              tk = cscale(cmul(tk, gh), (T)(sm.sq[a - 2 * j + 2] * sm.sq[a - 2 * j + 1] * sm.ik[j]));
              cfma(acc, tk, x[s]);
            }
          }
          y[mu] = acc;
        }
        __syncthreads();
        C2* tt = x; x = y; y = tt;
      }
    }
    if (side == 0) { u = x; u2 = y; } else { w = x; w2 = y; }
  }
  // ---- C0 = u w^T ----------------------------------------------------------
  C2* cur = Bf[0];
  C2* nxt = Bf[1];
  for (size_t idx = tid; idx < DD; idx += nt) cur[idx] = cmul(u[idx / Dr], w[idx % Dr]);
  __syncthreads();
  // ---- 2. cross PCOs -------------------------------------------------------
  for (int q = 0; q < nl; ++q) {
    if (sm.mol[q] == 0) continue;
    const int* lq = t.lowl + (size_t)q * t.capl;
    for (int q2 = 0; q2 < nr; ++q2) {
      if (sm.mor[q2] == 0) continue;
      const C2 g = to_c<C2>(sm.Q[q * QS + nl + 1 + q2]);
      const int* lr = t.lowr + (size_t)q2 * t.capr;
      for (size_t idx = tid; idx < DD; idx += nt) {
        const int mu = idx / Dr, nu = idx % Dr;
        const int a = occ_of(t.occl, mu, q), b = occ_of(t.occr, nu, q2);
        const int kmax = min(a, b);
        C2 acc = cur[idx];
        C2 tk = one;
        int s = mu, r = nu;
        for (int k = 1; k <= kmax; ++k) {
          s = lq[s];
          r = lr[r];
          tk = cscale(cmul(tk, g), (T)(sm.sq[a - k + 1] * sm.sq[b - k + 1] * sm.ik[k]));
          cfma(acc, tk, cur[(size_t)s * Dr + r]);
        }
        nxt[idx] = acc;
      }
      __syncthreads();
      C2* tt = cur; cur = nxt; nxt = tt;
    }
  }
  // ---- 3. physical PCOs: A[., p, .] ----------------------------------------
  double2* A = t.out;
  for (size_t idx = tid; idx < DD * d; idx += nt) A[idx] = cmk(0.0, 0.0);
  const double2 gaa2 = cscale(sm.Q[ia * QS + ia], 0.5);
  C2* P = cur;              // l_L^i C0
  C2* Pn = nxt;
  C2* Ya = Bf[2];
  C2* Yb = Bf[3];
  for (int i = 0; i < d; ++i) {
    if (i > 0) {
      if (nl == 0) break;
      __syncthreads();
      for (size_t idx = tid; idx < DD; idx += nt) {
        const int mu = idx / Dr, nu = idx % Dr;
        C2 acc = zero;
        for (int q = 0; q < nl; ++q) {
          const int a = occ_of(t.occl, mu, q);
          if (a == 0) continue;
          const int s = t.lowl[(size_t)q * t.capl + mu];
          cfma(acc, to_c<C2>(cscale(sm.Q[q * QS + ia], sm.sq[a])), P[(size_t)s * Dr + nu]);
        }
        Pn[idx] = acc;
      }
      __syncthreads();
      C2* tt = P; P = Pn; Pn = tt;
    }
    const C2* Ysrc = P;
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
        C2* Yn = (Ysrc == Ya) ? Yb : Ya;
        for (size_t idx = tid; idx < DD; idx += nt) {
          const int mu = idx / Dr, nu = idx % Dr;
          C2 acc = zero;
          for (int q = 0; q < nr; ++q) {
            const int b = occ_of(t.occr, nu, q);
            if (b == 0) continue;
            const int r = t.lowr[(size_t)q * t.capr + nu];
            cfma(acc, to_c<C2>(cscale(sm.Q[ia * QS + nl + 1 + q], sm.sq[b])), Ysrc[(size_t)mu * Dr + r]);
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
        const double2 y = to_d(Ysrc[idx]);
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

// one CTA per site, scratch at the task's own offset
template <typename T>
__global__ void __launch_bounds__(PCO_THREADS)
pco_kernel(const SiteTask* __restrict__ tasks, int d, double2* __restrict__ scratch_base,
           int* status) {
  __shared__ PcoSmem sm;
  const SiteTask t = tasks[blockIdx.x];
  pco_site<T>(sm, t, d, scratch_base + t.scratch_off, status);
}

// many sites of uneven size: persistent CTAs take the next task from a
// counter (the host orders tasks largest first), each with its own scratch slot
template <typename T>
__global__ void __launch_bounds__(PCO_THREADS)
pco_dynamic_kernel(const SiteTask* __restrict__ tasks, int ntasks, int d,
                   double2* __restrict__ scratch_base, size_t slot_elems, int* counter,
                   int* status) {
  __shared__ PcoSmem sm;
  __shared__ int next;
  double2* slot = scratch_base + (size_t)blockIdx.x * slot_elems;
  for (;;) {
    if (threadIdx.x == 0) next = atomicAdd(counter, 1);
    __syncthreads();
    const int k = next;
    if (k >= ntasks) break;
    const SiteTask t = tasks[k];
    pco_site<T>(sm, t, d, slot, status);
    __syncthreads();                 // shared memory and the slot are reused
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

// energy gauge of the mixed path: Ahat[a, p, b] = A[a, p, b] e^{-(E_b - E_a)/2}
// (the right environment of bond m is close to diag(e^{-E}), Eq. (SVD3), so
// this diagonal gauge makes the environments well conditioned in FP32)
__global__ void energy_gauge_kernel(const double2* __restrict__ A, int Dl, int d, int Dr,
                                    const double* __restrict__ El, const double* __restrict__ Er,
                                    double2* __restrict__ Ah) {
  size_t n = (size_t)Dl * d * Dr;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n;
       idx += (size_t)gridDim.x * blockDim.x) {
    int a = idx / ((size_t)d * Dr), b = idx % Dr;
    double el = Dl > 1 ? El[a] : 0.0, er = Dr > 1 ? Er[b] : 0.0;
    Ah[idx] = cscale(A[idx], exp(-0.5 * (er - el)));
  }
}

// the same over many sites (blockIdx.y = task) in one launch
__global__ void energy_gauge_batch_kernel(const GaugeTask* __restrict__ tasks, int d) {
  const GaugeTask t = tasks[blockIdx.y];
  const size_t n = (size_t)t.Dl * d * t.Dr;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int a = idx / ((size_t)d * t.Dr), b = idx % t.Dr;
    const double el = t.Dl > 1 ? t.El[a] : 0.0, er = t.Dr > 1 ? t.Er[b] : 0.0;
    t.Ah[idx] = cscale(t.A[idx], exp(-0.5 * (er - el)));
  }
}

}  // namespace

cudaError_t launch_energy_gauge_batch(const GaugeTask* tasks_dev, int ntasks, int d, int max_elems,
                                      cudaStream_t s) {
  if (ntasks <= 0) return cudaSuccess;
  int bx = (max_elems + 255) / 256;
  bx = std::max(1, std::min(bx, 64));
  for (int t0 = 0; t0 < ntasks; t0 += 65535) {
    dim3 grid(bx, std::min(65535, ntasks - t0));
    energy_gauge_batch_kernel<<<grid, 256, 0, s>>>(tasks_dev + t0, d);
  }
  return cudaGetLastError();
}

size_t pco_scratch_elems(int Dl, int Dr) {
  return 2 * (size_t)Dl + 2 * (size_t)Dr + 4 * (size_t)Dl * Dr;
}

cudaError_t launch_pco(const SiteTask* tasks_dev, int ntasks, int d, int precision,
                       double2* scratch, int* status, cudaStream_t s) {
  if (precision == GBSMPS_PREC_MIXED)
    pco_kernel<float><<<ntasks, PCO_THREADS, 0, s>>>(tasks_dev, d, scratch, status);
  else
    pco_kernel<double><<<ntasks, PCO_THREADS, 0, s>>>(tasks_dev, d, scratch, status);
  return cudaGetLastError();
}

int pco_dynamic_grid() {
  int dev = 0, nsm = 0, per = 0;
  if (cudaGetDevice(&dev) || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, pco_dynamic_kernel<double>, PCO_THREADS, 0))
    return 0;
  return nsm * std::max(per, 1);
}

cudaError_t launch_pco_dynamic(const SiteTask* tasks_dev, int ntasks, int d, double2* scratch,
                               size_t slot_elems, int grid, int* counter, int* status,
                               cudaStream_t s) {
  if (ntasks <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), s);
  if (e) return e;
  pco_dynamic_kernel<double><<<grid, PCO_THREADS, 0, s>>>(tasks_dev, ntasks, d, scratch, slot_elems,
                                                          counter, status);
  return cudaGetLastError();
}

cudaError_t launch_maps_brute(const uint8_t* occ, int D, int n, int* low, int cap,
                              int* status, cudaStream_t s) {
  int blocks = (D * n + 255) / 256;
  if (blocks < 1) blocks = 1;
  maps_brute_kernel<<<blocks, 256, 0, s>>>(occ, D, n, low, cap, status);
  return cudaGetLastError();
}

cudaError_t launch_energy_gauge(const double2* A, int Dl, int d, int Dr, const double* El,
                                const double* Er, double2* Ah, cudaStream_t s) {
  size_t n = (size_t)Dl * d * Dr;
  int blocks = (int)((n + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  energy_gauge_kernel<<<blocks, 256, 0, s>>>(A, Dl, d, Dr, El, Er, Ah);
  return cudaGetLastError();
}
