// gbsmps_build_site_noalloc: the single-site PCO build of gbsmps_build_site
// without any device allocation, for callers that must not allocate.
//
// All working memory (repacked occupation vectors, lowering maps, the task
// record and the PCO build buffers) lives in one file-scope device array of
// fixed size, created when the library is loaded on a device and held until
// the process exits.  Host code cannot use the array's name as a device
// address, so the first call on each device looks the address up with
// cudaGetSymbolAddress (with that device current) and caches it.
#include "internal.h"
#include <mutex>

#define NOALLOC_BYTES (1280 * 1024)
static_assert(NOALLOC_BYTES == GBSMPS_NOALLOC_SCRATCH_BYTES, "scratch size must match the header");

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

namespace {

struct DeviceScratch {
  bool ready = false;
  unsigned char* ptr = nullptr;
};
DeviceScratch g_scratch[64];
std::mutex g_scratch_mutex;

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// occupation vectors (D x n, packed) -> the NEM-strided layout of the kernels
__global__ void repack_occ_kernel(const uint8_t* __restrict__ src, int D, int n,
                                  uint8_t* __restrict__ dst) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < D * NEM; idx += gridDim.x * blockDim.x) {
    const int i = idx / NEM, q = idx % NEM;
    dst[idx] = q < n ? src[i * n + q] : 0;
  }
}

}  // namespace

// the body of gbsmps_build_site_noalloc (the C entry is in api.cu, which owns
// the context); on failure *detail names the reason
int noalloc_build_site(int device, cudaStream_t s, int* status_dev, int32_t nl, int32_t nr,
                       int32_t d, const double* Qm, double cscale, int32_t Dl,
                       const uint8_t* occ_l, int32_t Dr, const uint8_t* occ_r, int32_t precision,
                       double* out, const char** detail) {
  auto na_fail = [&](int code, const char* what) { *detail = what; return code; };
  if (!Qm || !out || !status_dev) return na_fail(GBSMPS_ERR_ARG, "NULL argument");
  if (nl < 0 || nr < 0 || nl > NEM || nr > NEM) return na_fail(GBSMPS_ERR_ARG, "nl/nr out of range");
  if ((nl > 0 && !occ_l) || (nr > 0 && !occ_r)) return na_fail(GBSMPS_ERR_ARG, "missing occupations");
  if (d < 1 || d > 255 || Dl < 1 || Dr < 1) return na_fail(GBSMPS_ERR_ARG, "sizes out of range");
  if (Dl > GBSMPS_NOALLOC_MAX_D || Dr > GBSMPS_NOALLOC_MAX_D)
    return na_fail(GBSMPS_ERR_BOUNDS, "Dl or Dr above GBSMPS_NOALLOC_MAX_D");
  if (device < 0 || device >= 64) return na_fail(GBSMPS_ERR_ARG, "bad device index");
  const size_t o_task = 0;
  const size_t o_occl = align256(o_task + sizeof(SiteTask));
  const size_t o_occr = align256(o_occl + (size_t)Dl * NEM);
  const size_t o_lowl = align256(o_occr + (size_t)Dr * NEM);
  const size_t o_lowr = align256(o_lowl + sizeof(int) * (size_t)NEM * Dl);
  const size_t o_pco = align256(o_lowr + sizeof(int) * (size_t)NEM * Dr);
  const size_t need = o_pco + sizeof(double2) * pco_scratch_elems(Dl, Dr);
  if (need > NOALLOC_BYTES) return na_fail(GBSMPS_ERR_BOUNDS, "problem needs more than the static scratch");
  cudaError_t e = cudaSetDevice(device);
  if (e) return na_fail(GBSMPS_ERR_CUDA, cudaGetErrorString(e));
  {
    std::lock_guard<std::mutex> lk(g_scratch_mutex);
    if (!g_scratch[device].ready) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) return na_fail(GBSMPS_ERR_CUDA, "cudaGetSymbolAddress failed");
      g_scratch[device].ptr = static_cast<unsigned char*>(p);
      g_scratch[device].ready = true;
    }
  }
  unsigned char* base = g_scratch[device].ptr;
  SiteTask t;
  t.nl = nl; t.nr = nr; t.Dl = Dl; t.Dr = Dr;
  t.Q = reinterpret_cast<const double2*>(Qm); t.qs = nl + 1 + nr; t.c = cscale;
  t.occl = base + o_occl; t.lowl = reinterpret_cast<const int*>(base + o_lowl); t.capl = Dl;
  t.occr = base + o_occr; t.lowr = reinterpret_cast<const int*>(base + o_lowr); t.capr = Dr;
  t.out = reinterpret_cast<double2*>(out);
  t.scratch_off = 0;
  e = cudaMemcpyAsync(base + o_task, &t, sizeof(SiteTask), cudaMemcpyHostToDevice, s);
  if (e) return na_fail(GBSMPS_ERR_CUDA, cudaGetErrorString(e));
  // every entry the kernels read is written here first: the array keeps the
  // previous call's contents
  if (nl) repack_occ_kernel<<<(Dl * NEM + 255) / 256, 256, 0, s>>>(occ_l, Dl, nl, base + o_occl);
  else e = cudaMemsetAsync(base + o_occl, 0, (size_t)Dl * NEM, s);
  if (!e) {
    if (nr) repack_occ_kernel<<<(Dr * NEM + 255) / 256, 256, 0, s>>>(occ_r, Dr, nr, base + o_occr);
    else e = cudaMemsetAsync(base + o_occr, 0, (size_t)Dr * NEM, s);
  }
  if (!e) e = cudaGetLastError();
  if (e) return na_fail(GBSMPS_ERR_CUDA, cudaGetErrorString(e));
  COUNT_LAUNCH((nl ? 1 : 0) + (nr ? 1 : 0));
  e = launch_maps_brute(base + o_occl, Dl, nl, reinterpret_cast<int*>(base + o_lowl), Dl, status_dev, s);
  if (!e) e = launch_maps_brute(base + o_occr, Dr, nr, reinterpret_cast<int*>(base + o_lowr), Dr, status_dev, s);
  COUNT_LAUNCH(2);
  if (e) return na_fail(GBSMPS_ERR_CUDA, cudaGetErrorString(e));
  // a basis that is not closed under lowering leaves -1 in the maps: stop here
  int st = 0;
  e = cudaMemcpyAsync(&st, status_dev, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (!e) e = cudaStreamSynchronize(s);
  if (e) return na_fail(GBSMPS_ERR_CUDA, cudaGetErrorString(e));
  if (st) {
    cudaMemsetAsync(status_dev, 0, sizeof(int), s);
    return na_fail(GBSMPS_ERR_BOUNDS, "a basis is not closed under removing one quantum");
  }
  e = launch_pco(reinterpret_cast<const SiteTask*>(base + o_task), 1, d, precision,
                 reinterpret_cast<double2*>(base + o_pco), status_dev, s);
  COUNT_LAUNCH(1);
  if (!e) e = cudaMemcpyAsync(&st, status_dev, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (!e) e = cudaStreamSynchronize(s);
  if (e) return na_fail(GBSMPS_ERR_CUDA, cudaGetErrorString(e));
  if (st) {
    cudaMemsetAsync(status_dev, 0, sizeof(int), s);
    return na_fail(GBSMPS_ERR_BOUNDS, "device status raised by the PCO build");
  }
  return GBSMPS_OK;
}
