// Kept virtual subspace of every bond (Sec. II C) and its index maps (App. B).
//
// The kept basis is the D = min(chi, D(eps)) occupation vectors with the
// lowest entanglement energy E = sum_q n_q w_q, w_q = -log Lambda_q^2
// (Eq. (HE)).  One warp enumerates one bond by merging n_e sorted streams:
// stream q proposes "x + e_q" for the first listed x whose highest occupied
// mode is <= q; every vector is produced exactly once, by the stream of its
// highest occupied mode, and the merged list is non-decreasing in E.  Lane q
// owns stream q; the warp arg-min picks the next vector (O(D log 32) steps).
// Ties: energies within 1e-12 max(1, E) of the first member of a group are
// ordered lexicographically by occupation vector.
//
// Index maps: low[q][beta] is the index of |v_beta> with one quantum of mode q
// removed (-1 if n_q = 0); the set is down-closed, so the state is kept.  The
// paper's vector sets (Alg. 1) and compositions (Alg. 3) are walks along
// these lowering maps.
#include "internal.h"
#include <math.h>

namespace {

__device__ inline bool lex_less(const uint8_t* a, const uint8_t* b, int n) {
  for (int q = 0; q < n; ++q) {
    if (a[q] != b[q]) return a[q] < b[q];
  }
  return false;
}

__global__ void basis_kernel(BondArrays ba, int nbonds, int chi, double eps, int* status) {
  extern __shared__ unsigned char mm[];        // highest occupied mode per entry
  const int b = blockIdx.x;
  const int lane = threadIdx.x;
  const int n = ba.ne[b];
  const int cap = ba.cap;
  uint8_t* occ = ba.occ + (size_t)b * cap * NEM;
  double* E = ba.E + (size_t)b * cap;
  int* maxocc = ba.maxocc + (size_t)b * NEM;
  if (lane < NEM) maxocc[lane] = 0;
  if (n == 0) {
    if (lane == 0) { E[0] = 0.0; ba.D[b] = 1; ba.eps[b] = 0.0; }
    return;
  }
  const double l2 = lane < n ? ba.lam2[(size_t)b * NEM + lane] : 0.5;
  const double w = lane < n ? -log(l2) : INFINITY;
  double lz = lane < n ? -log1p(-l2) : 0.0;           // log Z = -sum log(1 - L^2), Eq. (Z)
  for (int o = 16; o > 0; o >>= 1) lz += __shfl_xor_sync(0xffffffffu, lz, o);
  const double logZ = lz;
  if (lane < NEM) occ[lane] = 0;
  if (lane == 0) { E[0] = 0.0; mm[0] = 0; }
  __syncwarp();
  int ptr = 0;
  int count = 1;
  double acc = exp(-logZ);
  int Dcut = -1;
  if (chi <= 1 || (eps > 0.0 && acc >= 1.0 - eps)) Dcut = 1;
  while (count < cap) {
    if (lane < n) {
      while (ptr < count && mm[ptr] > lane) ++ptr;
    }
    double ce = (lane < n && ptr < count) ? E[ptr] + w : INFINITY;
    double best = ce;
    int bl = lane;
    for (int o = 16; o > 0; o >>= 1) {
      double ob = __shfl_xor_sync(0xffffffffu, best, o);
      int ol = __shfl_xor_sync(0xffffffffu, bl, o);
      if (ob < best || (ob == best && ol < bl)) { best = ob; bl = ol; }
    }
    if (!(best < INFINITY)) break;
    if (Dcut >= 0) {
      double ed = E[Dcut - 1];
      if (best - ed > 4.0 * TIE_TOL * fmax(1.0, fabs(ed))) break;
    }
    const int src = __shfl_sync(0xffffffffu, ptr, bl);
    if (lane < n) occ[(size_t)count * NEM + lane] = occ[(size_t)src * NEM + lane] + (lane == bl ? 1 : 0);
    if (lane == 0) { E[count] = best; mm[count] = (unsigned char)bl; }
    if (lane == bl) ++ptr;
    ++count;
    __syncwarp();
    if (Dcut < 0) {
      acc += exp(-best - logZ);
      if (count >= chi || (eps > 0.0 && acc >= 1.0 - eps)) Dcut = count;
    }
  }
  if (Dcut < 0) { if (lane == 0) set_status(status, ST_BOUNDS); Dcut = count; }
  // tie groups, lexicographic inside (serial; groups are short)
  if (lane == 0) {
    int i = 0;
    while (i < count) {
      double e0 = E[i];
      int j = i + 1;
      while (j < count && E[j] - e0 <= TIE_TOL * fmax(1.0, fabs(e0))) ++j;
      for (int a = i + 1; a < j; ++a) {          // insertion sort of [i, j)
        int c = a;
        while (c > i && lex_less(occ + (size_t)c * NEM, occ + (size_t)(c - 1) * NEM, n)) {
          for (int q = 0; q < n; ++q) {
            uint8_t t = occ[(size_t)c * NEM + q];
            occ[(size_t)c * NEM + q] = occ[(size_t)(c - 1) * NEM + q];
            occ[(size_t)(c - 1) * NEM + q] = t;
          }
          double te = E[c]; E[c] = E[c - 1]; E[c - 1] = te;
          --c;
        }
      }
      i = j;
    }
  }
  __syncwarp();
  const int D = Dcut;
  double kept = 0.0;
  int mo = 0;
  for (int i = lane; i < D; i += 32) kept += exp(-E[i] - logZ);
  for (int o = 16; o > 0; o >>= 1) kept += __shfl_xor_sync(0xffffffffu, kept, o);
  if (lane < n) {
    for (int i = 0; i < D; ++i) mo = max(mo, (int)occ[(size_t)i * NEM + lane]);
    maxocc[lane] = mo;
  }
  if (lane == 0) { ba.D[b] = D; ba.eps[b] = 1.0 - kept; }
}

__global__ void maps_kernel(BondArrays ba, int nbonds, int* status) {
  const int b = blockIdx.y;
  const int n = ba.ne[b];
  const int D = ba.D[b];
  const int cap = ba.cap;
  const uint8_t* occ = ba.occ + (size_t)b * cap * NEM;
  const double* E = ba.E + (size_t)b * cap;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < D * n; idx += gridDim.x * blockDim.x) {
    const int beta = idx / n, q = idx % n;
    int* low = ba.low + ((size_t)b * NEM + q) * cap;
    const uint8_t* v = occ + (size_t)beta * NEM;
    if (v[q] == 0) { low[beta] = -1; continue; }
    const double wq = -log(ba.lam2[(size_t)b * NEM + q]);
    const double et = E[beta] - wq;
    const double tol = 1e-9 * fmax(1.0, E[beta]);
    int lo = 0, hi = beta;                       // the lowered state precedes beta
    while (lo < hi) {
      int mid = (lo + hi) >> 1;
      if (E[mid] < et - tol) lo = mid + 1; else hi = mid;
    }
    int found = -1;
    for (int i = lo; i < beta && E[i] <= et + tol; ++i) {
      const uint8_t* u = occ + (size_t)i * NEM;
      bool eq = true;
      for (int k = 0; k < n && eq; ++k) eq = (u[k] == v[k] - (k == q ? 1 : 0));
      if (eq) { found = i; break; }
    }
    if (found < 0) set_status(status, ST_BOUNDS);
    low[beta] = found;
  }
}

}  // namespace

cudaError_t launch_basis(BondArrays ba, int nbonds, int chi, double eps, int* status,
                         cudaStream_t s) {
  basis_kernel<<<nbonds, 32, ba.cap, s>>>(ba, nbonds, chi, eps, status);
  return cudaGetLastError();
}

cudaError_t launch_maps(BondArrays ba, int nbonds, int* status, cudaStream_t s) {
  maps_kernel<<<dim3(8, nbonds), 256, 0, s>>>(ba, nbonds, status);
  return cudaGetLastError();
}
