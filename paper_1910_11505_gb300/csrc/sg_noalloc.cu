// sg_precond_apply_noalloc: the field-split Gauss-Seidel preconditioner with its scratch in a
// fixed device array of this library instead of memory allocated for the handle.
//
// The Gauss-Seidel sweep keeps the right-hand sides of its P block solves as contiguous columns
// (stride ldN = N rounded up to a multiple of 4), from which it subtracts the coupling
// sum_{b<a} K_ab z_b.  Here they live in the file-scope array below, which every GPU that loads
// the library holds until the process exits.  Host code cannot use the array's name as a device
// address (it names a host-side stand-in), so every call looks the address up with
// cudaGetSymbolAddress on the current device.  The lookup allocates nothing, and since it is not
// cached a context torn down and created again (cudaDeviceReset) never leaves a stale address.
// The first lookup on a device loads the library's module there, so that first call should come
// before any stream capture.
#include "sg_internal.h"

static __device__ __align__(256) double g_noalloc_scratch[SG_NOALLOC_MAX_ENTRIES];

namespace {

int scratch_for_current_device(double** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || p == nullptr)
    return sg::fail(SG_ERR_CUDA, std::string("cudaGetSymbolAddress of the scratch array failed: ") +
                                     cudaGetErrorString(e));
  *out = static_cast<double*>(p);
  return SG_OK;
}

}  // namespace

extern "C" int sg_precond_apply_noalloc(sg_handle* h, int sys, const double* R, double* Z,
                                        void* stream) {
  if (!h || sys < 0 || sys >= (int)h->sys.size() || !R || !Z)
    return sg::fail(SG_ERR_ARG, "bad handle, system index or pointer");
  sg::System& s = *h->sys[sys];
  if (s.prm.precond != SG_PC_FS_GS || s.prm.outer_sweeps != 1)
    return sg::fail(SG_ERR_ARG, "sg_precond_apply_noalloc serves the field-split Gauss-Seidel "
                                "preconditioner with outer_sweeps = 1 only");
  const long long need = (long long)s.P * s.ldN;
  if (need > SG_NOALLOC_MAX_ENTRIES)
    return sg::fail(SG_ERR_ARG, "sg_precond_apply_noalloc: P x ldN = " + std::to_string(need) +
                                    " exceeds the fixed scratch of " +
                                    std::to_string(SG_NOALLOC_MAX_ENTRIES) + " doubles");
  int dev = -1;
  SG_CUDA(cudaGetDevice(&dev));
  if (dev != h->device)
    return sg::fail(SG_ERR_ARG, "the handle's device must be current");
  double* rhs_t = nullptr;
  SG_TRY(scratch_for_current_device(&rhs_t));
  return sg::fs_gs_apply_f64_with(s, R, Z, rhs_t, (cudaStream_t)stream);
}
