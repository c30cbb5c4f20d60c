// nesa_matvec_noalloc: the NESA product for callers that must not allocate device
// memory.
//
// The ordinary product (nesa_matvec) keeps its per-level work vectors (the outgoing
// equivalent sources s and the incoming fields o of every box) in buffers that the
// context allocates with cudaMalloc the first time a given number of right-hand sides
// is used.  Some callers cannot let that happen: code running while a CUDA stream is
// being captured into a graph (cudaMalloc is not a stream operation and is not
// allowed to appear there), code that has a fixed device-memory budget decided up
// front, and real-time loops where an allocation (which may synchronise the device)
// would break the timing.  This entry point runs the same kernels but takes the work
// vectors from one fixed array in device memory that is part of the library image.
//
// The array is NESA_NOALLOC_SCRATCH_BYTES (32 MiB) on every GPU that loads the
// library, held until the process exits.  Its address is looked up once per device
// (cudaGetSymbolAddress, with that device current) by the first call made on that
// device; make that first call before starting any stream capture.  Call it with the
// context's device current: another current device is refused (NESA_ERR_INVALID_ARG),
// since its copy of the array is not the one the kernels should use.  All calls share
// the array and leave their data in it: two calls whose kernels overlap on the GPU
// (different streams, or different contexts used concurrently) race on it.  Nothing
// in the array needs to start at zero: every kernel writes each work-vector element
// it owns before any kernel reads it.
#include <mutex>
#include <new>
#include <string>

#include "nesa_device.cuh"

namespace nesa {

static __device__ __align__(256) unsigned char g_noalloc_scratch[NESA_NOALLOC_SCRATCH_BYTES];

static std::mutex g_noalloc_mutex;
static void *g_noalloc_ptr[256] = {nullptr};

// Device address of the scratch array on the current device (looked up once per device).
static int noalloc_scratch(void **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return NESA_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) return NESA_ERR_CUDA;
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return NESA_OK;
}

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace nesa

using namespace nesa;

extern "C" int nesa_matvec_noalloc(nesa_ctx *c, const nesa_c128 *x, nesa_c128 *y, int nrhs) {
  if (!c || !x || !y || nrhs < 1 || nrhs > 64) {
    set_last_error("nesa_matvec_noalloc: null pointer or nrhs outside 1..64");
    return NESA_ERR_INVALID_ARG;
  }
  // The scratch address is looked up on the current device; the kernels run on the
  // context's device.  They must be the same, or the kernels would reach into another
  // GPU's copy of the array.
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) {
    set_last_error("nesa_matvec_noalloc: cudaGetDevice failed");
    return NESA_ERR_CUDA;
  }
  if (cur != c->device) {
    set_last_error("nesa_matvec_noalloc: the current device (" + std::to_string(cur) +
                   ") is not the context's device (" + std::to_string(c->device) + "); make it current first");
    return NESA_ERR_INVALID_ARG;
  }
  // bytes of the work vectors s_l and o_l for l0..L
  size_t need = 0;
  for (int l = c->l0; l <= c->L; ++l)
    need += 2 * align256(sizeof(cplx) * (size_t)c->lev[l].nbox * 4 * nrhs * c->lev[l].q);
  if (need > (size_t)NESA_NOALLOC_SCRATCH_BYTES) {
    set_last_error("nesa_matvec_noalloc: the work vectors need " + std::to_string(need) +
                   " bytes, more than the fixed scratch of " + std::to_string((size_t)NESA_NOALLOC_SCRATCH_BYTES) +
                   " bytes; use nesa_matvec or fewer right-hand sides");
    return NESA_ERR_INVALID_ARG;
  }
  void *base = nullptr;
  int st = noalloc_scratch(&base);
  if (st != NESA_OK) {
    set_last_error("nesa_matvec_noalloc: cudaGetSymbolAddress of the scratch array failed");
    return st;
  }
  // point the levels at slices of the scratch array for this launch, then restore
  cplx *saved_s[NESA_MAX_LEVELS], *saved_o[NESA_MAX_LEVELS];
  unsigned char *p = (unsigned char *)base;
  for (int l = c->l0; l <= c->L; ++l) {
    DevLevel &d = c->lev[l];
    const size_t b = align256(sizeof(cplx) * (size_t)d.nbox * 4 * nrhs * d.q);
    saved_s[l] = d.s;
    saved_o[l] = d.o;
    d.s = (cplx *)p;
    p += b;
    d.o = (cplx *)p;
    p += b;
  }
  int status = NESA_OK;
  try {
    launch_matvec(c, (const cplx *)x, (cplx *)y, nrhs, NESA_PART_ALL);
    check_cuda(cudaGetLastError(), "matvec launch");
  } catch (const Error &e) {
    set_last_error(e.what);
    status = e.status;
  } catch (const std::bad_alloc &) {
    set_last_error("host allocation failed");
    status = NESA_ERR_OOM;
  }
  for (int l = c->l0; l <= c->L; ++l) {
    c->lev[l].s = saved_s[l];
    c->lev[l].o = saved_o[l];
  }
  return status;
}
