// noalloc.cu -- cg_solve_classic_f64_noalloc: the binary64 classic CG solve
// with its scratch memory in a fixed, file-scope device array instead of a
// caller-provided workspace, for callers that cannot allocate device memory.
//
// The array (control block + r, p, p', z) is a static __device__ object, so
// every GPU that loads this library holds it until the process exits.  Host
// code cannot use the symbol g_noalloc_scratch as a device address (on the
// host it names a stand-in object); the real address is looked up with
// cudaGetSymbolAddress, with the caller's device current, on every call.  The
// lookup allocates nothing and costs far less than the launch; not caching it
// keeps the address right after a device reset, which reloads the module and
// may move the array.
#include "launch.h"

namespace lap5 {

constexpr size_t kNoallocMaxPoints = LAP5CG_NOALLOC_MAX_POINTS;  // e.g. 512 x 512
constexpr size_t kNoallocBytes = kCtlBytes + 4 * kNoallocMaxPoints * sizeof(double);  // 256 KiB + 8 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

// Device address of g_noalloc_scratch on the current device.
static int noalloc_scratch(unsigned char** out) {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return LAP5CG_ERR_CUDA;
  *out = static_cast<unsigned char*>(p);
  return LAP5CG_OK;
}

}  // namespace lap5

using namespace lap5;

extern "C" LAP5CG_API int cg_solve_classic_f64_noalloc(int nx, int ny, int ld, const double* b, double* x,
                                                       double tol, int maxit, lap5cg_info* info, void* stream) {
  if (nx < 1 || ny < 1 || ld < nx || !b || !x || !info || maxit < 0 || tol != tol) return LAP5CG_ERR_INVALID_ARG;
  if ((size_t)ny * (size_t)ld > kNoallocMaxPoints) return LAP5CG_ERR_INVALID_ARG;  // beyond the fixed scratch
  if (ld % 2 != 0 || reinterpret_cast<uintptr_t>(b) % 16 || reinterpret_cast<uintptr_t>(x) % 16)
    return LAP5CG_ERR_INVALID_ARG;  // rows must be 16-byte aligned: there is no room for staging copies
  const uintptr_t b0 = reinterpret_cast<uintptr_t>(b), x0 = reinterpret_cast<uintptr_t>(x);
  const size_t bytes = (size_t)ny * (size_t)ld * sizeof(double);
  if (b0 < x0 + bytes && x0 < b0 + bytes) return LAP5CG_ERR_INVALID_ARG;
  unsigned char* ws = nullptr;
  int rc = noalloc_scratch(&ws);
  if (rc != LAP5CG_OK) return rc;
  SolvePlan p;
  p.nx = nx;
  p.ny = ny;
  p.ld = ld;
  p.ldw = ld;
  p.b = b;
  p.x = x;
  p.ws = ws;
  p.ws_bytes = kNoallocBytes;
  p.info = info;
  p.tol = tol;
  p.maxit = maxit;
  p.variant = LAP5CG_CLASSIC;
  p.precision = LAP5CG_PREC_F64;
  lap5cg_opts_default(&p.opts);
  return solve_f64(p, static_cast<cudaStream_t>(stream));
}
