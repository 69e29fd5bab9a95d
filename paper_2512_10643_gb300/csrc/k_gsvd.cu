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
// the bw modes to the right of the cut are carried.  The chain keeps only
// what the next cut needs; each cut's U^{-1}, c_m and Q^m are formed after
// it, all cuts at once (qm_kernel), from the U, V it leaves in the site's
// Q^m slot.
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
static_assert(NLM <= 32, "the gauge and the active-mode count keep one mode per lane");
constexpr int MAX_SWEEPS = 40;
// final FP64 sweep: pairs whose rotation angle |h_pq| / |h_qq - h_pp| is below
// this are left alone.  The stop criterion of the FP64 sweeps already leaves
// angles up to ~1e-13 on pairs with gaps ~0.1; the final sweep is for nearly
// degenerate pairs (gap < 1e-3 at the residual |h_pq| ~ 1e-16), whose angle
// is far above it
constexpr double JAC_THETA = 1e-13;

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
  double rcs[2][NLM], rsn[2][NLM];   // Jacobi rotations of a round (two rounds' tables)
  double2 rph[2][NLM];
  float fcs[2][NLM], fsn[2][NLM];    // FP32 stage: the same, kept in FP32 (no conversions)
  float2 fph[2][NLM];
  unsigned short blk[NLM * (NLM + 1) / 2];   // upper 2 x 2 blocks (k << 8) | l, k <= l
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

// Rotation J of a Jacobi pair (p, q), p < q: columns (p, q) of X J are
// (cs x_p - sn ph x_q, sn x_p + cs ph x_q), i.e. J = [[cs, sn], [-sn ph, cs ph]]
// with |ph| = 1; sn == 0 is the identity.
template <typename R>
struct JRot {
  R cs, sn, px, py;
};

// one output of a pair rotation applied to the pair (v0, v1): s = 0 gives
// cs v0 - sn (ph v1), s = 1 gives sn v0 + cs (ph v1).  The column update of
// X J uses ph; the row update of J^dag X uses conj(ph).
template <typename T2, typename R>
__device__ __forceinline__ T2 jmix(T2 v0, T2 v1, int s, const JRot<R>& J) {
  const R wx = J.px * v1.x - J.py * v1.y, wy = J.px * v1.y + J.py * v1.x;
  if (s == 0) return T2{J.cs * v0.x - J.sn * wx, J.cs * v0.y - J.sn * wy};
  return T2{J.sn * v0.x + J.cs * wx, J.sn * v0.y + J.cs * wy};
}

template <typename T2>
__device__ __forceinline__ T2 cconj2(T2 v) { return T2{v.x, -v.y}; }

template <typename R>
__device__ __forceinline__ R rabs(R v) {
  if constexpr (sizeof(R) == 8) return fabs(v);
  else return fabsf(v);
}

// rotation tables, double-buffered by round parity: FP64 parameters for the
// FP64 stage, FP32 ones for the FP32 stage (neither stage converts in its loops)
template <typename R>
__device__ __forceinline__ JRot<R> jrot_load(const ChainSmem& sm, int b, int k) {
  if constexpr (sizeof(R) == 8) return JRot<R>{sm.rcs[b][k], sm.rsn[b][k], sm.rph[b][k].x, sm.rph[b][k].y};
  else return JRot<R>{sm.fcs[b][k], sm.fsn[b][k], sm.fph[b][k].x, sm.fph[b][k].y};
}

// The round-robin pairing: round r pairs (a, b) with a = (r + k) mod (n - 1)
// and b = n - 1 for k = 0, else (r - k) mod (n - 1); every pair of indices
// meets once in n - 1 rounds.  (p, q) = (min, max) of pair k.
__device__ __forceinline__ void jpair(int r, int k, int n, int& p, int& q) {
  const int nm1 = n - 1;
  int a = r + k;
  if (a >= nm1) a -= nm1;
  int b = nm1;
  if (k != 0) {
    b = r - k + nm1;
    if (b >= nm1) b -= nm1;
  }
  p = min(a, b);
  q = max(a, b);
}

// the inverse: index x is slot s (0: p, 1: q) of pair k in round r
__device__ __forceinline__ void jowner(int r, int x, int n, int& k, int& s) {
  const int nm1 = n - 1, half = n >> 1;
  if (x == nm1) { k = 0; s = 1; return; }
  int ka = x - r;
  if (ka < 0) ka += nm1;
  int partner;
  if (ka < half) {                     // x = a of pair ka
    k = ka;
    partner = nm1;
    if (ka != 0) { partner = r - ka; if (partner < 0) partner += nm1; }
  } else {                             // x = b of pair n - 1 - ka
    k = nm1 - ka;
    partner = r + k;
    if (partner >= nm1) partner -= nm1;
  }
  s = x < partner ? 0 : 1;
}

// Knuth's TwoSum in FP32: s + e = a + b exactly (round-to-nearest intrinsics,
// so that nothing is contracted or reassociated)
__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// (c0, s0) with c0^2 + s0^2 = 1 - e, |e| ~ 2^-23, scaled onto the unit circle
// in FP64: (c, s) = (c0, s0) (1 - e)^{-1/2} with (1 - e)^{-1/2} - 1 =
// e/2 + 3e^2/8 + O(e^3) formed in FP32 from error-free products and sums
// (Dekker's product by FMA, TwoSum), to ~1e-22 absolute; the only FP64
// operations are the conversions, one addition and the two FMAs
// c0 + c0 D, s0 + s0 D, each rounded once: c^2 + s^2 = 1 to FP64 rounding.
__device__ __forceinline__ void unit_fp64(float c0, float s0, double& c, double& s) {
  const float p1 = __fmul_rn(c0, c0), q1 = fmaf(c0, c0, -p1);
  const float p2 = __fmul_rn(s0, s0), q2 = fmaf(s0, s0, -p2);
  // e = 1 - p1 - p2 - q1 - q2 as eh + el: the large terms and the rounding
  // error of 1 - p1 (up to 2^-25 when p1 < 1/2) each enter a TwoSum, so only
  // errors of order 2^-48 are added in plain FP32
  float a, ea, b, eb, s1, t1, s2, t2, eh, t3;
  two_sum_f(1.0f, -p1, a, ea);
  two_sum_f(a, -p2, b, eb);
  two_sum_f(ea, -q1, s1, t1);
  two_sum_f(s1, -q2, s2, t2);
  two_sum_f(b, s2, eh, t3);
  const float el = __fadd_rn(__fadd_rn(t1, t2), __fadd_rn(t3, eb));
  float dh, dl;
  two_sum_f(__fmul_rn(0.5f, eh), __fmul_rn(0.375f, __fmul_rn(eh, eh)), dh, dl);
  dl = __fadd_rn(dl, __fmul_rn(0.5f, el));
  const double D = (double)dh + (double)dl;
  const double cd = (double)c0, sd = (double)s0;
  c = fma(cd, D, cd);
  s = fma(sd, D, sd);
}

// FP32 rotation angle of a pair with off-diagonal entry (fx, fy) and
// dd = h_qq - h_pp: J = [[fc, fs], [-fs g, fc g]] with g = e^{-i phi},
// h_pq = |h| e^{i phi}, t = fs / fc = tan of the angle that annihilates h_pq
// (the smaller root of t^2 + 2 tau t - 1 = 0, tau = dd / (2 |h|)).  Returns
// false (identity) when |Re| + |Im| <= skip or <= theta |dd|.  Accurate to
// ~1e-7 relative (fast reciprocal square roots and divisions): the next
// sweep removes what an approximate angle leaves behind.
__device__ __forceinline__ bool jangle(float fx, float fy, float dd, float skip, float theta,
                                       float& fc, float& fs, float& gx, float& gy) {
  const float mag = fabsf(fx) + fabsf(fy);
  if (!(mag > skip) || (theta > 0.0f && mag <= theta * fabsf(dd))) return false;
  if (mag < 0x1p-60f) { fx *= 0x1p100f; fy *= 0x1p100f; dd *= 0x1p100f; }   // keep |h|^2 normal
  const float im = rsqrtf(fmaf(fx, fx, fy * fy));   // 1 / |h|
  gx = fx * im;
  gy = -fy * im;
  const float tau = dd * (0.5f * im);
  const float at = fabsf(tau);
  float t;
  if (at > 1e18f) {
    t = __fdividef(0.5f, tau);
  } else {
    const float u = fmaf(tau, tau, 1.0f);
    t = copysignf(__fdividef(1.0f, at + u * rsqrtf(u)), tau);
  }
  fc = rsqrtf(fmaf(t, t, 1.0f));
  fs = t * fc;
  return true;
}

// Rotation of pair k (p, q) from the entries of the matrix it acts on
// (dd = h_qq - h_pp, h_pq = (hx, hy)), into table b.  The FP32 parameters
// are always stored; in the FP64 stage the FP32 (cos, sin) and phase are
// also put on the unit circle in FP64 (unit_fp64), so every applied J is
// unitary to FP64 rounding and the similarity is exact.
template <typename R>
__device__ __forceinline__ bool jrot_put(ChainSmem& sm, int b, int k, float dd, float hx, float hy,
                                         float skip, float theta) {
  float fc = 1.0f, fs = 0.0f, gx = 1.0f, gy = 0.0f;
  const bool go = jangle(hx, hy, dd, skip, theta, fc, fs, gx, gy);
  sm.fcs[b][k] = fc; sm.fsn[b][k] = fs; sm.fph[b][k] = make_float2(gx, gy);
  if constexpr (sizeof(R) == 8) {
    double cs = 1.0, sn = 0.0, phx = 1.0, phy = 0.0;
    if (go) {
      unit_fp64(fc, fs, cs, sn);
      unit_fp64(gx, gy, phx, phy);
    }
    sm.rcs[b][k] = cs; sm.rsn[b][k] = sn; sm.rph[b][k] = cmk(phx, phy);
  }
  return go;
}

// rotation of pair k of round r into table b, from the matrix H the round acts on
template <typename T2, typename R>
__device__ __forceinline__ bool jrot_direct(ChainSmem& sm, const T2* __restrict__ H, int b, int r,
                                            int k, int n, float skip, float theta) {
  int p, q;
  jpair(r, k, n, p, q);
  const T2 h = H[p * LD + q];
  return jrot_put<R>(sm, b, k, (float)(H[q * LD + q].x - H[p * LD + p].x), (float)h.x, (float)h.y,
                     skip, theta);
}

// Entry (x, y) of J^dag B J for the 2 x 2 block B = [[x0, y0], [x1, y1]]
// (rows pa, qa of a round's pair with rotation Ja, columns pb, qb of a pair
// with Jb; x is slot sa, y slot sb).  The same operations in the same order
// as the block update.
template <typename T2, typename R>
__device__ __forceinline__ T2 jelem4(T2 x0, T2 x1, T2 y0, T2 y1, JRot<R> Ja, int sa,
                                     const JRot<R>& Jb, int sb) {
  if (Jb.sn != (R)0) {
    x0 = jmix(x0, y0, sb, Jb);
    x1 = jmix(x1, y1, sb, Jb);
  } else if (sb) {
    x0 = y0;
    x1 = y1;
  }
  if (Ja.sn == (R)0) return sa ? x1 : x0;
  Ja.py = -Ja.py;
  return jmix(x0, x1, sa, Ja);
}

template <typename T2, typename R>
__device__ __forceinline__ T2 jelem(const T2* __restrict__ H, int pa, int qa, const JRot<R>& Ja,
                                    int sa, int pb, int qb, const JRot<R>& Jb, int sb) {
  return jelem4<T2, R>(H[pa * LD + pb], H[qa * LD + pb], H[pa * LD + qb], H[qa * LD + qb], Ja, sa,
                       Jb, sb);
}

__device__ __forceinline__ float2 tof2(double2 v) { return make_float2((float)v.x, (float)v.y); }

// change of the diagonal entry h_pp of a pair (p, q) under its rotation J:
// h'_pp = h_pp + d, h'_qq = h_qq - d, d = sn^2 (h_qq - h_pp) - 2 cs sn Re(ph h_pq)
__device__ __forceinline__ float jdiag_shift(const JRot<float>& J, float dlt, float2 h) {
  if (J.sn == 0.0f) return 0.0f;
  const float re = J.px * h.x - J.py * h.y;
  return J.sn * (J.sn * dlt - 2.0f * J.cs * re);
}

// The next round's rotation of pair k (by a set-up warp), from the matrix H that
// round r acts on and round r's rotations (table b).  FP32 stage: the three
// entries through the rotations, in FP32.  FP64 stage: FP64 only where
// cancellation needs it, so that the set-up ends within the round's FP64
// updates: the diagonal difference h'_qq - h'_pp is the FP64 difference of
// the current entries plus the FP32 shifts of both (jdiag_shift, from FP64
// differences), and h'_pq, an entry of the 2 x 2 block of two different
// pairs of round r (off-diagonal entries only: no cancellation), is formed
// in FP32.  The angle is an FP32 quantity in either stage.
template <typename T2, typename R>
__device__ __forceinline__ bool jsetup_next(ChainSmem& sm, const T2* __restrict__ H, int r, int b,
                                            int k, int n, float skip, float theta) {
  int p, q, k1, s1, k2, s2, pa, qa, pb, qb;
  jpair(r + 1, k, n, p, q);
  jowner(r, p, n, k1, s1);
  jowner(r, q, n, k2, s2);
  jpair(r, k1, n, pa, qa);
  jpair(r, k2, n, pb, qb);
  const JRot<float> Ja = jrot_load<float>(sm, b, k1), Jb = jrot_load<float>(sm, b, k2);
  if constexpr (sizeof(R) == 4) {
    const T2 hpp = jelem<T2, R>(H, pa, qa, Ja, s1, pa, qa, Ja, s1);
    const T2 hqq = jelem<T2, R>(H, pb, qb, Jb, s2, pb, qb, Jb, s2);
    const T2 hpq = jelem<T2, R>(H, pa, qa, Ja, s1, pb, qb, Jb, s2);
    return jrot_put<R>(sm, b ^ 1, k, hqq.x - hpp.x, hpq.x, hpq.y, skip, theta);
  } else {
    const float dA = jdiag_shift(Ja, (float)(H[qa * LD + qa].x - H[pa * LD + pa].x), tof2(H[pa * LD + qa]));
    const float dB = jdiag_shift(Jb, (float)(H[qb * LD + qb].x - H[pb * LD + pb].x), tof2(H[pb * LD + qb]));
    const float dp = s1 ? -dA : dA, dq = s2 ? -dB : dB;
    const float dd = (float)(H[q * LD + q].x - H[p * LD + p].x) + (dq - dp);
    const float2 hpq = jelem4<float2, float>(tof2(H[pa * LD + pb]), tof2(H[qa * LD + pb]),
                                             tof2(H[pa * LD + qb]), tof2(H[qa * LD + qb]), Ja, s1, Jb, s2);
    return jrot_put<R>(sm, b ^ 1, k, dd, hpq.x, hpq.y, skip, theta);
  }
}

// One item of round r's update from Hc into Hn with the rotations of table b:
// j < nb is the two-sided update J_k^dag B J_l of the upper 2 x 2 block
// sm.blk[j] = (k, l) of the round's pairs (the lower block mirrored), j >= nb
// is W <- W J in place on row i of W for the pairs g, g + G, ..
template <typename T2, typename R>
__device__ __forceinline__ void jround_item(const ChainSmem& sm, const T2* __restrict__ Hc,
                                            T2* __restrict__ Hn, T2* __restrict__ W, int r, int b,
                                            int j, int nb, int n, int half, int G, unsigned inv_n) {
  if (j < nb) {
    const int kl = sm.blk[j], k = kl >> 8, l = kl & 255;
    int pk, qk, pl, ql;
    jpair(r, k, n, pk, qk);
    jpair(r, l, n, pl, ql);
    JRot<R> Jk = jrot_load<R>(sm, b, k);
    const JRot<R> Jl = jrot_load<R>(sm, b, l);
    T2 h00 = Hc[pk * LD + pl], h01 = Hc[pk * LD + ql];
    T2 h10 = Hc[qk * LD + pl], h11 = Hc[qk * LD + ql];
    if (Jl.sn != (R)0) {                          // columns: X = B J_l
      const T2 a0 = jmix(h00, h01, 0, Jl), a1 = jmix(h00, h01, 1, Jl);
      const T2 c0 = jmix(h10, h11, 0, Jl), c1 = jmix(h10, h11, 1, Jl);
      h00 = a0; h01 = a1; h10 = c0; h11 = c1;
    }
    if (Jk.sn != (R)0) {                          // rows: J_k^dag X
      Jk.py = -Jk.py;
      const T2 a0 = jmix(h00, h10, 0, Jk), a1 = jmix(h00, h10, 1, Jk);
      const T2 c0 = jmix(h01, h11, 0, Jk), c1 = jmix(h01, h11, 1, Jk);
      h00 = a0; h10 = a1; h01 = c0; h11 = c1;
    }
    if (k == l) {                                 // Hermitian diagonal block
      h00.y = (R)0; h11.y = (R)0; h10 = cconj2(h01);
    }
    Hn[pk * LD + pl] = h00; Hn[pk * LD + ql] = h01;
    Hn[qk * LD + pl] = h10; Hn[qk * LD + ql] = h11;
    if (k != l) {
      Hn[pl * LD + pk] = cconj2(h00); Hn[ql * LD + pk] = cconj2(h01);
      Hn[pl * LD + qk] = cconj2(h10); Hn[ql * LD + qk] = cconj2(h11);
    }
  } else {
    const int jw = j - nb;
    const int g = (int)(((unsigned)jw * inv_n) >> 20), i = jw - g * n;   // jw / n, jw % n
    for (int l = g; l < half; l += G) {
      const JRot<R> Jl = jrot_load<R>(sm, b, l);
      if (Jl.sn == (R)0) continue;
      int pl, ql;
      jpair(r, l, n, pl, ql);
      const T2 wp = W[i * LD + pl], wq = W[i * LD + ql];
      W[i * LD + pl] = jmix(wp, wq, 0, Jl);
      W[i * LD + ql] = jmix(wp, wq, 1, Jl);
    }
  }
}

// Sweeps of the cyclic complex Jacobi method on the n x n Hermitian matrix in
// Hc (n even, ld LD, storage precision of T2; both triangles kept), with Hn
// as the second buffer of a ping-pong, accumulating W <- W J.  Every round
// rotates the n/2 disjoint pairs of the round-robin ordering at once, as one
// two-sided update J^dag H J of the 2 x 2 blocks of the round's pairs (the
// upper blocks computed, the lower ones mirrored) written to the other
// buffer, with the columns of W updated in place.
//
// Two warps set up the next round's rotations while the other six update,
// from the same pre-round matrix (the entries each pair needs, through this
// round's rotations: jsetup_next), so one barrier separates the rounds; a
// round whose rotations are all the identity is not applied (the barrier's
// OR-reduction says so).
//
// Before each sweep every off-diagonal entry is tested: |h_ij| <= conv, or
// |h_ij| <= theta |h_jj - h_ii|, for all i < j ends the sweeps (returns
// true); false after max_sweeps sweeps.  *Hout is the buffer that holds the
// result.  A pair is rotated only if |h_pq| > skip and > theta |h_qq - h_pp|
// (|h| = |Re| + |Im| in both tests).
template <typename T2>
__device__ bool jacobi_sweeps(ChainSmem& sm, T2* Hc, T2* Hn, T2* __restrict__ W, int n,
                              double conv_d, double skip_d, double theta_d, int max_sweeps,
                              T2** Hout) {
  using R = decltype(T2{}.x);
  const R conv = (R)conv_d, theta = (R)theta_d;
  const float skip = (float)skip_d, theta_f = (float)theta_d;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int half = n >> 1, nm1 = n - 1;
  const int nb = half * (half + 1) / 2;                  // upper 2 x 2 blocks (sm.blk)
  // warps 6 and 7 set up rotations (pair k on lane k / 2 of warp 6 + k % 2),
  // warps 0..5 update
  constexpr int NU = 192;
  const bool setter = warp >= 6;
  const int ks = setter ? (lane << 1) | (warp - 6) : NLM;
  const int G = max(1, min(half, (NU - nb) / n));       // pair groups per W row
  const int nitems = nb + n * G;
  const unsigned inv_n = ((1u << 20) + (unsigned)n - 1u) / (unsigned)n;   // jw / n for jw < 2048
  for (int sweep = 0;; ++sweep) {
    bool viol = false;
    for (int i = warp; i < n; i += 8) {
      const R di = Hc[i * LD + i].x;
      for (int j = lane; j < n; j += 32) {
        if (j <= i) continue;
        const T2 v = Hc[i * LD + j];
        const R mag = rabs(v.x) + rabs(v.y);
        if (mag > conv && !(theta > (R)0 && mag <= theta * rabs(Hc[j * LD + j].x - di))) viol = true;
      }
    }
    if (ks < half) jrot_direct<T2, R>(sm, Hc, 0, 0, ks, n, skip, theta_f);   // round 0
    const bool any = __syncthreads_or(viol) != 0;
    if (!any) { *Hout = Hc; return true; }
    if (sweep == max_sweeps) { *Hout = Hc; return false; }
    bool upd = true;                         // does the round rotate any pair
    for (int r = 0; r < nm1; ++r) {
      const int b = r & 1;
      bool go_next = false;
      if (setter) {
        if (ks < half && r + 1 < nm1) go_next = jsetup_next<T2, R>(sm, Hc, r, b, ks, n, skip, theta_f);
      } else if (upd) {
        for (int j = tid; j < nitems; j += NU)
          jround_item<T2, R>(sm, Hc, Hn, W, r, b, j, nb, n, half, G, inv_n);
      }
      const bool nxt = __syncthreads_or(go_next) != 0;   // a round of identities is skipped
      if (upd) { T2* t = Hc; Hc = Hn; Hn = t; }
      upd = nxt;
    }
  }
}

// Eigen-decomposition of the n x n Hermitian H = i K (K real, antisymmetric;
// FP64, ld LD, n even).  On return the eigenvalues are in sm.ev and W holds
// the eigenvectors as columns; H and T are overwritten.  Stage 1: Jacobi in
// FP32 on a copy until the off-diagonal falls to ~4e-6 of ||H||_F (FP32
// updates run at the full FP32 rate).  Stage 2: the FP32 eigenvectors are
// made unitary in FP64 by two Newton-Schulz steps W <- W (3 - W^dag W) / 2,
// H is transformed to W^dag H W, and FP64 Jacobi sweeps (two or three)
// finish the diagonalisation with W accumulating.  Returns false if the FP64
// stage does not reach 2.5e-16 n ||H||_F within MAX_SWEEPS.
__device__ bool jacobi_herm(ChainSmem& sm, int n) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  const int half = n >> 1;
  double2* H = sm.H;
  double2* W = sm.W;
  double2* T = sm.T;
  float2* H32 = reinterpret_cast<float2*>(sm.T);
  float2* W32 = H32 + N2M * N2M;
  float2* H32b = reinterpret_cast<float2*>(sm.B);       // L^{-1} is no longer needed here
  for (int k = tid; k < half; k += nt) {                  // the upper 2 x 2 blocks (k <= l)
    const int base = k * half - k * (k - 1) / 2;
    for (int l = k; l < half; ++l) sm.blk[base + l - k] = (unsigned short)((k << 8) | l);
  }
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
  float2* H32o;
  jacobi_sweeps<float2>(sm, H32, H32b, W32, n, conv32, 1e-300 + 0.025 * conv32, 0.0, 12, &H32o);
  for (int idx = tid; idx < n * n; idx += nt) {
    const int i = idx / n, j = idx % n;
    const float2 w = W32[i * LD + j];
    W[i * LD + j] = cmk(w.x, w.y);
  }
  __syncthreads();
  // Newton-Schulz, W <- W (3 - W^dag W) / 2 = W - W (W^dag W - 1) / 2, twice:
  // the residual R = W^dag W - 1 in FP64 (upper triangle, Hermitian), the
  // correction product W R in FP32 (R is ~1e-6, then ~1e-12: the FP32
  // rounding of the product, ~6e-8 of it, stays below the next residual and
  // then below FP64 rounding), applied in FP64
  float2* Rf = H32b;                                         // FP32 copy of R
  for (int it = 0; it < 2; ++it) {
    for (int idx = tid; idx < n * n; idx += nt) {
      const int i = idx / n, j = idx % n;
      if (i > j) continue;
      double2 s = cmk(i == j ? -1.0 : 0.0, 0.0);
      for (int k = 0; k < n; ++k) cfma(s, cconj(W[k * LD + i]), W[k * LD + j]);
      Rf[i * LD + j] = make_float2((float)s.x, (float)s.y);
      Rf[j * LD + i] = make_float2((float)s.x, -(float)s.y);
    }
    __syncthreads();
    for (int row = warp; row < n; row += nw) {               // row-wise: read, then write
      float2 o0 = make_float2(0.f, 0.f), o1 = make_float2(0.f, 0.f);
      const int j0 = lane, j1 = lane + 32;
      for (int k = 0; k < n; ++k) {
        const double2 wd = W[row * LD + k];
        const float wx = (float)wd.x, wy = (float)wd.y;
        if (j0 < n) {
          const float2 r = Rf[k * LD + j0];
          o0.x = fmaf(wx, r.x, fmaf(-wy, r.y, o0.x));
          o0.y = fmaf(wx, r.y, fmaf(wy, r.x, o0.y));
        }
        if (j1 < n) {
          const float2 r = Rf[k * LD + j1];
          o1.x = fmaf(wx, r.x, fmaf(-wy, r.y, o1.x));
          o1.y = fmaf(wx, r.y, fmaf(wy, r.x, o1.y));
        }
      }
      __syncwarp();
      if (j0 < n) {
        const double2 w = W[row * LD + j0];
        W[row * LD + j0] = cmk(w.x - 0.5 * (double)o0.x, w.y - 0.5 * (double)o0.y);
      }
      if (j1 < n) {
        const double2 w = W[row * LD + j1];
        W[row * LD + j1] = cmk(w.x - 0.5 * (double)o1.x, w.y - 0.5 * (double)o1.y);
      }
    }
    __syncthreads();
  }
  // T = H W with H = i K purely imaginary (K = L^{-1} Omega L^{-T} real):
  // T = i K W, two real multiply-adds per term
  for (int idx = tid; idx < n * n; idx += nt) {
    const int i = idx / n, j = idx % n;
    double sx = 0.0, sy = 0.0;
    for (int k = 0; k < n; ++k) {
      const double kk = H[i * LD + k].y;
      const double2 w = W[k * LD + j];
      sx = fma(-kk, w.y, sx);
      sy = fma(kk, w.x, sy);
    }
    T[i * LD + j] = cmk(sx, sy);
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
  double2* Hc;
  const bool ok = jacobi_sweeps<double2>(sm, H, T, W, n, conv64, 1e-300 + 0.25 * conv64, 0.0,
                                         MAX_SWEEPS, &Hc);
  // then one sweep more over every pair whose rotation angle is above
  // JAC_THETA, with no stop test: the criterion above leaves off-diagonal
  // elements up to ~n eps ||H||_F, which turn the eigenvectors of a nearly
  // degenerate pair (gap g) by ~that / g (1e-8 at g ~ 5e-7, a mode kept just
  // above the freeze threshold); one more sweep takes every such element to
  // the rounding floor of a single sweep, where the eigenvectors are as well
  // determined as FP64 allows (pairs whose angle is below JAC_THETA are left:
  // their rotation would change nothing above the sweep's own rounding)
  double2* Hf;
  jacobi_sweeps<double2>(sm, Hc, Hc == H ? T : H, W, n, 1e-300, 1e-300, JAC_THETA, 1, &Hf);
  for (int i = tid; i < n; i += nt) sm.ev[i] = Hf[i * LD + i].x;
  __syncthreads();
  return ok;
}

// Inverse of the n x n complex matrix M (ld NLM) into Inv (ld NLM) by
// Gauss-Jordan elimination with partial pivoting; M is destroyed.  Returns
// log|det M| in sm.dval[0]; sets ival[0] = 1 on a zero pivot.
template <typename Smem>
__device__ void cinv(Smem& sm, double2* M, double2* Inv, int n) {
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
    // ---- Cholesky of V = 2 Gamma_LL (lower, in place), right-looking ----
    // One barrier per column: step k updates the trailing matrix with the
    // raw column k times 1/a_kk (= r_k^2, r_k = a_kk^{-1/2} in sm.ev[k]) and
    // scales column k - 1 by r_{k-1} (nothing reads it in step k); thread 0,
    // which updates a_{k+1,k+1} first, then forms r_{k+1} for the next step.
    for (int idx = tid; idx < n2 * n2; idx += nt) sm.A[(idx / n2) * LD + idx % n2] *= 2.0;
    __syncthreads();
    if (tid == 0) {                    // 1/sqrt(a_00) by Newton from FP32
      double a = sm.A[0];
      if (!(a > 0.0)) { set_status(status, ST_NUMERIC); a = 1e-300; }
      sm.ev[0] = rsqrt_fp64(a);
    }
    __syncthreads();
    for (int k = 0; k < n2; ++k) {
      const double rk = sm.ev[k], ir2 = rk * rk;
      if (k > 0) {
        const double rp = sm.ev[k - 1];
        for (int i = k - 1 + tid; i < n2; i += nt) sm.A[i * LD + k - 1] *= rp;
      }
      const int w = n2 - k - 1;
      for (int idx = tid; idx < w * w; idx += nt) {   // idx 0 (thread 0): a_{k+1,k+1}
        const int i = k + 1 + idx / w, j = k + 1 + idx % w;
        if (j <= i) sm.A[i * LD + j] = fma(-sm.A[i * LD + k] * ir2, sm.A[j * LD + k], sm.A[i * LD + j]);
      }
      if (tid == 0 && w > 0) {
        double a = sm.A[(k + 1) * LD + k + 1];
        if (!(a > 0.0)) { set_status(status, ST_NUMERIC); a = 1e-300; }
        sm.ev[k + 1] = rsqrt_fp64(a);
      }
      __syncthreads();
    }
    for (int idx = tid; idx < n2 * n2; idx += nt) {
      const int i = idx / n2, j = idx % n2;
      if (j > i) sm.A[i * LD + j] = 0.0;
      else if (j == n2 - 1) sm.A[i * LD + j] *= sm.ev[n2 - 1];   // the last column
    }
    __syncthreads();
    // ---- L^{-1} into B, right-looking: B holds 1 - (eliminated rows); row
    // k is final once rows < k are eliminated from it, X_kj = B_kj / L_kk
    // (1/L_kk = r_k from the Cholesky).  Step k eliminates row k from the
    // rows below (B_ij -= L_ik r_k B_kj, j <= k) and scales row k - 1 by
    // r_{k-1} (nothing reads it in step k): one barrier per row.
    for (int idx = tid; idx < n2 * n2; idx += nt) {
      const int i = idx / n2, j = idx % n2;
      sm.B[i * LD + j] = (i == j) ? 1.0 : 0.0;
    }
    __syncthreads();
    for (int k = 0; k < n2; ++k) {
      const double rk = sm.ev[k];
      if (k > 0) {
        const double rp = sm.ev[k - 1];
        for (int j = tid; j < k; j += nt) sm.B[(k - 1) * LD + j] *= rp;
      }
      const int w = n2 - k - 1, h = k + 1;               // rows k+1 .., columns 0 .. k
      for (int idx = tid; idx < w * h; idx += nt) {
        const int i = k + 1 + idx / h, j = idx % h;
        sm.B[i * LD + j] = fma(-sm.A[i * LD + k] * rk, sm.B[k * LD + j], sm.B[i * LD + j]);
      }
      __syncthreads();
    }
    for (int j = tid; j < n2; j += nt) sm.B[(n2 - 1) * LD + j] *= sm.ev[n2 - 1];   // the last row
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
    // (warp w takes columns w, w + 8, ..; lane j holds |U_jq|^2 and a
    // butterfly keeps the largest, the first index among equal ones: the
    // choice of a serial scan with a strict comparison, in FP64)
    {
      const int lane = tid & 31, warp = tid >> 5;
      for (int q = warp; q < nL; q += (nt >> 5)) {
        double best = lane < nL ? cabs2(sm.U[lane * NLM + q]) : -1.0;
        int jb = lane;
        for (int o = 16; o > 0; o >>= 1) {
          const double v2 = __shfl_xor_sync(0xffffffffu, best, o);
          const int j2 = __shfl_xor_sync(0xffffffffu, jb, o);
          if (v2 > best || (v2 == best && j2 < jb)) { best = v2; jb = j2; }
        }
        const double2 u = sm.U[jb * NLM + q];
        const double img = rsqrt_fp64(best);
        const double2 ph = cmk(u.x * img, -u.y * img);
        __syncwarp();                        // every lane has read U_{jb q}
        if (lane < nL) {
          sm.U[lane * NLM + q] = cmul(sm.U[lane * NLM + q], ph);
          sm.V[lane * NLM + q] = cmul(sm.V[lane * NLM + q], ph);
        }
      }
    }
    if (tid < 32) {
      // active modes: the leading run of Lambda^2 = (D - 1) / (D + 1) > freeze
      // over D descending, without the division (D + 1 > 0)
      const bool act = tid < nL && sm.Dq[tid] - 1.0 > freeze * (sm.Dq[tid] + 1.0);
      const unsigned m = __ballot_sync(0xffffffffu, act);
      int na = __ffs(~m) - 1;
      if (tid == 0) {
        if (na > NEM) { set_status(status, ST_BOUNDS); na = NEM; }
        sm.ival[2] = na;
      }
    }
    __syncthreads();
    const int na = sm.ival[2];
    // ---- U, V to site m's Q^m slot: U^{-1}, c_m and Q^m (App. A) are not
    // needed by later cuts and are formed after the chain, all cuts at once
    // (qm_kernel); the first 2 NLM^2 entries of the slot hold U, then V
    {
      double2* Qo = Qm + (size_t)m * QS * QS;
      for (int idx = tid; idx < nL * nL; idx += nt) {
        const int i = idx / nL, j = idx % nL;
        Qo[i * NLM + j] = sm.U[i * NLM + j];
        Qo[NLM * NLM + i * NLM + j] = sm.V[i * NLM + j];
      }
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

// Shared memory of qm_kernel: the Bogoliubov matrices of one cut, the work
// copy and inverse of U, and cinv's scratch.
struct QmSmem {
  double2 H[NLM * NLM];
  double2 U[NLM * NLM];
  double2 V[NLM * NLM];
  double2 Ui[NLM * NLM];
  double2 fac[NLM];
  double2 pinv;
  int ival[4];
  double dval[4];
};

// Cut m's local paired form Q^m over (r_{m-1}, a_m, l_m) and c_m = |det U|^{-1/2}
// (App. A) from the gauge-fixed U, V that the chain left in the first
// 2 NLM^2 entries of the site's Q^m slot: U^{-1} by Gauss-Jordan with
// partial pivoting, then the four blocks of Q^m, written over the slot.
__device__ void qm_body(QmSmem& sm, int m, const int* __restrict__ ne, double2* __restrict__ Qm,
                        double* __restrict__ cm, int* status) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int nL = ne[m] + 1, na = ne[m + 1];
  double2* Qo = Qm + (size_t)m * QS * QS;
  for (int idx = tid; idx < nL * nL; idx += nt) {
    const int i = idx / nL, j = idx % nL;
    const double2 u = Qo[i * NLM + j];
    sm.U[i * NLM + j] = u;
    sm.H[i * NLM + j] = u;
    sm.V[i * NLM + j] = Qo[NLM * NLM + i * NLM + j];
  }
  __syncthreads();
  cinv(sm, sm.H, sm.Ui, nL);
  if (tid == 0) {
    if (sm.ival[0]) set_status(status, ST_NUMERIC);
    cm[m] = exp(-0.5 * sm.dval[0]);
  }
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
}

// all cuts of one state, one CTA each (the last site's Q is the chain's)
__global__ void __launch_bounds__(CHAIN_THREADS)
qm_kernel(const int* __restrict__ ne, double2* __restrict__ Qm, double* __restrict__ cm, int* status) {
  extern __shared__ __align__(16) unsigned char smraw[];
  qm_body(*reinterpret_cast<QmSmem*>(smraw), blockIdx.x, ne, Qm, cm, status);
}

// many states: CTA (m, b) takes cut m of state b, if the state has it
__global__ void __launch_bounds__(CHAIN_THREADS)
qm_batch_kernel(const ChainJob* __restrict__ jobs, int* status) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const ChainJob& j = jobs[blockIdx.y];
  if ((int)blockIdx.x >= j.N - 1) return;
  qm_body(*reinterpret_cast<QmSmem*>(smraw), blockIdx.x, j.ba.ne, j.Qm, j.cm, status);
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
  e = cudaGetLastError();
  if (e || N < 2) return e;
  qm_kernel<<<N - 1, CHAIN_THREADS, sizeof(QmSmem), s>>>(ba.ne, Qm, cm, status);
  COUNT_LAUNCH(1);
  return cudaGetLastError();
}

cudaError_t launch_gsvd_chain_batch(const ChainJob* jobs_dev, int count, int maxN, int* status,
                                    cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  size_t smem = sizeof(ChainSmem);
  cudaError_t e = cudaFuncSetAttribute(gsvd_chain_batch_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e) return e;
  gsvd_chain_batch_kernel<<<count, CHAIN_THREADS, smem, s>>>(jobs_dev, status);
  e = cudaGetLastError();
  if (e || maxN < 2) return e;
  if (count > 65535) return cudaErrorInvalidValue;
  qm_batch_kernel<<<dim3(maxN - 1, count), CHAIN_THREADS, sizeof(QmSmem), s>>>(jobs_dev, status);
  COUNT_LAUNCH(1);
  return cudaGetLastError();
}
