// pp_noalloc.cu -- tsvdqII_noalloc: the *Q-SVDII entry point for callers that
// cannot allocate device memory.
//
// Who needs it: a caller whose device memory is owned entirely by some other
// allocator (for example a host framework's caching pool, where an extra
// cudaMalloc behind its back would break its accounting), a latency-critical
// loop that forbids allocation after start-up because cudaMalloc/cudaFree can
// synchronise the whole device, or a binding from another language that can
// only hand over pointers it already owns.  Such a caller can provide the
// inputs and the outputs but not the workspace that tsvdqII needs.
//
// This variant takes its workspace from one file-scope device array of fixed
// size (PP_NOALLOC_SCRATCH_BYTES).  Every GPU on which the library's module
// is loaded holds that array until the process exits.  The array is shared by
// every call on a device and keeps the previous call's contents; tsvdqII
// clears what has to start at zero (its status word) on every call, and writes
// every other scratch element before reading it.  Two calls whose work
// overlaps on the GPU (different streams, no ordering between them) use the
// same scratch and race: order them on one stream or with events.
//
// Host code cannot use the array's name as a device address (in host code it
// names a host-side stand-in).  Every call, with the target device current,
// asks the runtime for the array's device address with cudaGetSymbolAddress
// (cheap once the module is loaded; nothing is cached, so a context torn down
// and recreated, e.g. after cudaDeviceReset, gets the new address).  The first
// call on a device may load the module and should therefore come before any
// other work that must not be disturbed, in particular before any stream
// capture.  No call allocates or frees memory.
//
// Argument checks run in tsvdqII's own order (pointers, gamma, sizes, the
// longest slice side) before the size of the scratch is compared, so a bad
// argument gets the same status from both entry points.
#include "pp_internal.h"

namespace {

// The scratch.  256-byte aligned, as the workspace contract of pprod.h asks.
static __device__ __align__(256) unsigned char pp_noalloc_scratch[PP_NOALLOC_SCRATCH_BYTES];

// Device address of the scratch on the current device (nullptr on failure).
void *scratch_address() {
  void *ptr = nullptr;
  if (cudaGetSymbolAddress(&ptr, pp_noalloc_scratch) != cudaSuccess) return nullptr;
  return ptr;
}

}  // namespace

extern "C" pp_status tsvdqII_noalloc(const float *A, const float *Q, int64_t l, int64_t m,
                                     int64_t n, int64_t p, double gamma, int32_t *rho,
                                     int64_t *offs, float *Uh_pk, float *s_pk, float *Vh_pk,
                                     float *Ak, pp_report *rep, const pp_opts *opts,
                                     void *stream) {
  // tsvdqII without a workspace runs every one of its argument checks and then
  // stops at the workspace check (PP_EWORKSPACE), enqueuing nothing; any other
  // status is an argument error, reported as tsvdqII reports it.
  const pp_status pre = tsvdqII(A, Q, l, m, n, p, gamma, rho, offs, Uh_pk, s_pk, Vh_pk, Ak, rep,
                                opts, nullptr, 0, stream);
  if (pre != PP_EWORKSPACE) return pre;
  pp_shape sh{l, m, n, p, 0, 0};
  const size_t need = pp_workspace_bytes(PP_OP_TSVDQII, &sh);
  if (need > (size_t)PP_NOALLOC_SCRATCH_BYTES) return PP_EWORKSPACE;   // beyond the maximum
  void *ws = scratch_address();
  if (!ws) return PP_ECUDA;
  return tsvdqII(A, Q, l, m, n, p, gamma, rho, offs, Uh_pk, s_pk, Vh_pk, Ak, rep, opts, ws,
                 (size_t)PP_NOALLOC_SCRATCH_BYTES, stream);
}
