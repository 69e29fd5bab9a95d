// Projected-creation-operator (PCO) construction of local MPS tensors
// (Sec. II C, App. B), one CTA per tensor.
//
// The projected state P_V exp(1/2 d^dag Q d^dag)|0> is a product of commuting
// PCOs (Sec. II C); the closure identity P d^dag = P d^dag P lets the
// projector pass through any grouping of them.  The kernel groups them for
// the GPU:
//   1. left-only PCOs (r_q r_q' and r_q r_q) on a D_l vector u = P exp(X_LL)|0>,
//      right-only PCOs on a D_r vector w; C0 = u w^T is their product state;
//   2. cross PCOs exp(g r_q^dag l_q'^dag) on the D_l x D_r matrix C0, in place
//      and only on the entries they change (both modes occupied);
//   3. the physical PCOs last: with l_L = sum_q Q_{r_q a} r_q^dag and
//      l_R = sum_q' Q_{a l_q'} l_q'^dag (they commute),
//        exp(a^dag (l_L + l_R) + g_aa a^dag^2 / 2) =
//        sum_p (a^dag)^p sum_k (g_aa/2)^k/k! (l_L + l_R)^(p-2k) / (p-2k)!,
//      so A[., p, .] = c sqrt(p!) sum_k (g_aa/2)^k/k! W_{p-2k} with
//      W_s = (l_L + l_R)^s C0 / s!, built by d - 1 passes of l_L + l_R.
// Every PCO update is a pull along the lowering maps: the source of a target
// state with kappa quanta added to modes (q, q') is reached by kappa steps
// of low_q and low_q'; coefficients g^kappa/kappa! sqrt(n!/(n-kappa)!) are
// built as running products.  The one-sided passes are out of place (double
// buffered); the cross passes run in place, ordered by level, like the
// paper's in-place loop ordered from high occupation down.  GB300 runs FP64
// at about 2 fused multiply-adds per clock per SM, so the grouping is chosen
// for few FP64 operations: d - 1 passes of l_L + l_R instead of d(d+1)/2 - 1
// one-sided ones, term lists without empty modes, and the output written
// once per (s, k) instead of read and written per (i, j, k).
// T = double is the FP64 path; T = float runs the same passes in FP32 (the
// mixed-precision build) and accumulates the output tensor in FP64.
#include "internal.h"
#include <algorithm>
#include <math.h>

namespace {

constexpr int PCO_THREADS = 1024;   // one CTA per site: 512, 768, 1024 threads measured 5.0, 4.4, 4.1 ms (N = 144)
constexpr int SQ_N = 260;
constexpr int GE = 258;     // occupation-count table per mode: v = 0..257

struct PcoSmem {
  double2 Q[QS * QS];
  double sq[SQ_N];
  double ik[SQ_N];          // 1 / k: the loops multiply instead of dividing in FP64
  int mol[NEM], mor[NEM];
  double2 gk[SQ_N];         // cross phase: g^k / k!; physical phase: plane coefficients
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
  C2* W0 = w2 + Dr;                       // C0, then the cross PCOs in place
  C2* W1 = W0 + DD;
  C2* lc = W1 + DD;                       // physical-pass terms of each row / column
  C2* rc = lc + (size_t)Dl * NEM;
  int* ls = reinterpret_cast<int*>(rc + (size_t)Dr * NEM);
  int* rs = ls + (size_t)Dl * NEM;
  int* lcnt = rs + (size_t)Dr * NEM;
  int* rcnt = lcnt + Dl;
  int* listl = rcnt + Dr;                 // occupied rows per mode, occupation descending
  int* listr = listl + (size_t)NEM * Dl;
  int* gel = listr + (size_t)NEM * Dr;    // gel[q*GE + v] = rows with occupation >= v
  int* ger = gel + NEM * GE;
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
  // ---- C0 = u w^T; term lists for the passes below ----------------------
  for (size_t idx = tid; idx < DD; idx += nt) W0[idx] = cmul(u[idx / Dr], w[idx % Dr]);
  for (int side = 0; side < 2; ++side) {
    const int n = side == 0 ? nl : nr, D = side == 0 ? Dl : Dr;
    const uint8_t* occ = side == 0 ? t.occl : t.occr;
    const int* low = side == 0 ? t.lowl : t.lowr;
    const int cap = side == 0 ? t.capl : t.capr;
    const int off = side == 0 ? 0 : nl + 1;
    C2* cf = side == 0 ? lc : rc;
    int* src = side == 0 ? ls : rs;
    int* cnt = side == 0 ? lcnt : rcnt;
    // row mu of l_L (column nu of l_R): sum over occupied modes q of
    // Q_{q a} sqrt(n_q) times the entry one quantum lower in q
    for (int i = tid; i < D; i += nt) {
      int c = 0;
      for (int q = 0; q < n; ++q) {
        const int a = occ_of(occ, i, q);
        const double2 g = sm.Q[(off + q) * QS + ia];
        if (a == 0 || (g.x == 0.0 && g.y == 0.0)) continue;
        src[(size_t)i * NEM + c] = low[(size_t)q * cap + i];
        cf[(size_t)i * NEM + c] = to_c<C2>(cscale(g, sm.sq[a]));
        ++c;
      }
      cnt[i] = c;
    }
    // one warp per mode: the occupied entries by occupation, descending
    const int lane = tid & 31;
    for (int q = tid >> 5; q < n; q += nt >> 5) {
      const int mo = side == 0 ? sm.mol[q] : sm.mor[q];
      int* list = (side == 0 ? listl : listr) + (size_t)q * D;
      int* ge = (side == 0 ? gel : ger) + q * GE;
      int k = 0;
      for (int v = mo; v >= 1; --v) {
        for (int i0 = 0; i0 < D; i0 += 32) {
          const int i = i0 + lane;
          const bool hit = i < D && occ_of(occ, i, q) == v;
          const unsigned m = __ballot_sync(0xffffffffu, hit);
          if (hit) list[k + __popc(m & ((1u << lane) - 1u))] = i;
          k += __popc(m);
        }
        if (lane == 0) ge[v] = k;
      }
      if (lane == 0) ge[mo + 1] = 0;
    }
  }
  __syncthreads();
  // ---- 2. cross PCOs, in place ---------------------------------------------
  // exp(g r_q^dag l_q'^dag) adds to a target with occupations (a, b) the
  // entries (a - k, b - k), k = 1..min(a, b).  Only targets with both modes
  // occupied change.  Level m = min(a, b): a target of level m reads only
  // entries of lower levels, so taking the levels from the top down, with a
  // barrier between them, updates the buffer in place and gives the same
  // numbers as an out-of-place pass.
  for (int q = 0; q < nl; ++q) {
    if (sm.mol[q] == 0) continue;
    const int* lq = t.lowl + (size_t)q * t.capl;
    for (int q2 = 0; q2 < nr; ++q2) {
      const int mq = min(sm.mol[q], sm.mor[q2]);
      const double2 g = sm.Q[q * QS + nl + 1 + q2];
      if (mq == 0 || (g.x == 0.0 && g.y == 0.0)) continue;
      const int* lr = t.lowr + (size_t)q2 * t.capr;
      if (tid == 0) {                       // g^k / k!
        double2 gk = cmk(1.0, 0.0);
        sm.gk[0] = gk;
        for (int k = 1; k <= mq; ++k) { gk = cscale(cmul(gk, g), sm.ik[k]); sm.gk[k] = gk; }
      }
      __syncthreads();
      const int* la = listl + (size_t)q * Dl;
      const int* lb = listr + (size_t)q2 * Dr;
      for (int m = mq; m >= 1; --m) {
        const long long nA = gel[q * GE + m], nB = ger[q2 * GE + m];
        const long long nA1 = gel[q * GE + m + 1], nB1 = ger[q2 * GE + m + 1];
        for (long long e = tid; e < nA * nB; e += nt) {
          const long long i = e / nB, j = e - i * nB;
          if (i < nA1 && j < nB1) continue;            // a higher level
          const int mu = la[i], nu = lb[j];
          const int a = occ_of(t.occl, mu, q), b = occ_of(t.occr, nu, q2);
          C2 acc = W0[(size_t)mu * Dr + nu];
          double r = 1.0;
          int s = mu, rr = nu;
          for (int k = 1; k <= m; ++k) {
            s = lq[s];
            rr = lr[rr];
            r *= sm.sq[a - k + 1] * sm.sq[b - k + 1];
            cfma(acc, to_c<C2>(cscale(sm.gk[k], r)), W0[(size_t)s * Dr + rr]);
          }
          W0[(size_t)mu * Dr + nu] = acc;
        }
        __syncthreads();
      }
    }
  }
  // ---- 3. physical PCOs ----------------------------------------------------
  // l_L and l_R act on different bonds and commute, so the double sum over
  // l_L^i C0 (l_R^T)^j / (i! j!) with i + j = s is (l_L + l_R)^s C0 / s!:
  //   W_0 = C0,  W_s = (l_L W_{s-1} + W_{s-1} l_R^T) / s,
  //   A[., p, .] = c sqrt(p!) sum_k (g_aa/2)^k / k!  W_{p-2k}.
  // Each pass builds W_s and adds it to the planes p = s + 2k at once; plane
  // p is first reached at s = p mod 2, which writes it.
  double2* A = t.out;
  const double2 gaa2 = cscale(sm.Q[ia * QS + ia], 0.5);
  C2* Wp = W0;
  C2* Wn = W1;
  for (int s = 0; s < d; ++s) {
    const int kmx = (d - 1 - s) / 2;
    __syncthreads();
    if (tid == 0) {
      double2 gp = cmk(1.0, 0.0);
      for (int k = 0; k <= kmx; ++k) {
        const int p = s + 2 * k;
        sm.gk[k] = cscale(gp, t.c * exp(0.5 * lgamma(p + 1.0) - lgamma(k + 1.0)));
        gp = cmul(gp, gaa2);
      }
    }
    __syncthreads();
    const T inv_s = s > 0 ? (T)sm.ik[s] : (T)1;
    // from s = 2 on only the entries with n_mu + s + n_nu even are non-zero
    // in W_s (every PCO adds two quanta); every other entry of W_s, of the
    // planes p = s + 2k (written as zeros at s = p mod 2) and of the buffer
    // W_s overwrites (W_{s-2}) is zero already.  With the bonds' parity
    // lists the pass walks only those entries: rows of class c with the
    // columns of class c ^ (s & 1), a contiguous run of each list.
    const bool by_class = s >= 2 && t.pl != nullptr;
    const int sp = s & 1;
    const size_t n0 = (size_t)t.kl[0] * t.kr[sp], n1 = (size_t)t.kl[1] * t.kr[sp ^ 1];
    const size_t nent = by_class ? n0 + n1 : DD;
    for (size_t idx = tid; idx < nent; idx += nt) {
      int mu, nu;
      if (by_class) {
        const int c = idx < n0 ? 0 : 1;
        const size_t e = c ? idx - n0 : idx;
        const int cr = c ^ sp;
        const int kc = t.kr[cr];
        mu = t.pl[(c ? t.kl[0] : 0) + (int)(e / kc)];
        nu = t.pr[(cr ? t.kr[0] : 0) + (int)(e % kc)];
      } else {
        mu = idx / Dr;
        nu = idx % Dr;
      }
      const size_t ent = (size_t)mu * Dr + nu;
      C2 y;
      if (s == 0) {
        y = Wp[ent];
      } else {
        C2 acc = zero;
        const int cl = lcnt[mu], cr = rcnt[nu];
        for (int e = 0; e < cl; ++e)
          cfma(acc, lc[(size_t)mu * NEM + e], Wp[(size_t)ls[(size_t)mu * NEM + e] * Dr + nu]);
        for (int e = 0; e < cr; ++e)
          cfma(acc, rc[(size_t)nu * NEM + e], Wp[(size_t)mu * Dr + rs[(size_t)nu * NEM + e]]);
        y = cscale(acc, inv_s);
        if (s + 1 < d) Wn[ent] = y;
      }
      const double2 yd = to_d(y);
      for (int k = 0; k <= kmx; ++k) {
        double2* dst = A + ((size_t)mu * d + s + 2 * k) * Dr + nu;
        double2 v = s < 2 ? cmk(0.0, 0.0) : *dst;
        cfma(v, sm.gk[k], yd);
        *dst = v;
      }
    }
    if (s > 0) { C2* tt = Wp; Wp = Wn; Wn = tt; }
  }
}

// one CTA per site, scratch at the task's own offset
template <typename T>
__global__ void __launch_bounds__(PCO_THREADS, 1)
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
// energy gauge of one site into the parity-compact layout, as double-float
// pairs (df_pack):
// Ahat[c][a][(p, j)] = A[alpha, p, beta] e^{-(E_beta - E_alpha)/2}, alpha the
// a-th class-c state of the left bond, beta the j-th class-c^(p&1) state of
// the right bond (an end bond's energy is 0)
// (the factor e^{-(E_beta - E_alpha)/2} as e^{E_alpha/2} e^{-E_beta/2} from
// per-bond tables: an FP64 exponential per element would run on GB300's slow
// FP64 pipe)
__device__ inline void gauge_entry(const double2* __restrict__ A, int Dl, int d, int Dr,
                                   const double* __restrict__ Gup, const double* __restrict__ Gdn,
                                   const ParitySite& P, long long idx, double2* __restrict__ Ah) {
  int c, a, p, j, cr;
  pk_locate(P, d, idx, c, a, p, j, cr);
  const int al = P.pl[(c ? P.kl[0] : 0) + a], be = P.pr[(cr ? P.kr[0] : 0) + j];
  const double f = (Dl > 1 ? Gup[al] : 1.0) * (Dr > 1 ? Gdn[be] : 1.0);
  reinterpret_cast<float4*>(Ah)[idx] = df_pack(cscale(A[((long long)al * d + p) * Dr + be], f));
}

// per kept state of every bond: e^{+E/2} (first nb * cap entries), e^{-E/2} (next)
__global__ void gauge_scale_kernel(const double* __restrict__ E, long long n, double* __restrict__ G) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double h = 0.5 * E[i];
    G[i] = exp(h);
    G[n + i] = exp(-h);
  }
}

__global__ void energy_gauge_kernel(const double2* __restrict__ A, int Dl, int d, int Dr,
                                    const double* __restrict__ El, const double* __restrict__ Er,
                                    const ParitySite P, double2* __restrict__ Ah) {
  const long long n = pk_size(d, P.kl, P.kr);
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x)
    gauge_entry(A, Dl, d, Dr, El, Er, P, idx, Ah);
}

// the same over many sites (blockIdx.y = task) in one launch
__global__ void energy_gauge_batch_kernel(const GaugeTask* __restrict__ tasks, int d) {
  const GaugeTask t = tasks[blockIdx.y];
  const long long n = pk_size(d, t.P.kl, t.P.kr);
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x)
    gauge_entry(t.A, t.Dl, d, t.Dr, t.El, t.Er, t.P, idx, t.Ah);
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
  const size_t D = (size_t)Dl + Dr;
  const size_t ints = 2 * NEM * D + D + 2 * (size_t)NEM * GE;
  return 2 * D + 2 * (size_t)Dl * Dr + NEM * D + (ints * sizeof(int) + 15) / 16 + 1;
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

cudaError_t launch_pco_dynamic(const SiteTask* tasks_dev, int ntasks, int d, int precision,
                               double2* scratch, size_t slot_elems, int grid, int* counter,
                               int* status, cudaStream_t s) {
  if (ntasks <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), s);
  if (e) return e;
  if (precision == GBSMPS_PREC_MIXED)
    pco_dynamic_kernel<float><<<grid, PCO_THREADS, 0, s>>>(tasks_dev, ntasks, d, scratch, slot_elems,
                                                           counter, status);
  else
    pco_dynamic_kernel<double><<<grid, PCO_THREADS, 0, s>>>(tasks_dev, ntasks, d, scratch,
                                                            slot_elems, counter, status);
  return cudaGetLastError();
}

cudaError_t launch_maps_brute(const uint8_t* occ, int D, int n, int* low, int cap,
                              int* status, cudaStream_t s) {
  int blocks = (D * n + 255) / 256;
  if (blocks < 1) blocks = 1;
  maps_brute_kernel<<<blocks, 256, 0, s>>>(occ, D, n, low, cap, status);
  return cudaGetLastError();
}

cudaError_t launch_gauge_scale(const double* E, long long n, double* G, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int blocks = (int)std::min<long long>((n + 255) / 256, 1024);
  gauge_scale_kernel<<<blocks, 256, 0, s>>>(E, n, G);
  return cudaGetLastError();
}

cudaError_t launch_energy_gauge(const double2* A, int Dl, int d, int Dr, const double* El,
                                const double* Er, const ParitySite& P, double2* Ah, cudaStream_t s) {
  const long long n = pk_size(d, P.kl, P.kr);
  int blocks = (int)std::min<long long>((n + 255) / 256, 4096);
  if (blocks < 1) blocks = 1;
  energy_gauge_kernel<<<blocks, 256, 0, s>>>(A, Dl, d, Dr, El, Er, P, Ah);
  return cudaGetLastError();
}
