// sfhk_spectrum_noalloc.cu -- the spectrum entry point for callers that must
// not allocate device memory while they run (see sfhk_spectrum_noalloc in
// include/sfhk.h).  It launches the same kernels as sfhk_spectrum with
// device pointers; only the scratch comes from a fixed array below instead
// of a stream-ordered allocation.
#include <cuda_runtime.h>

#include <cstdio>

#include "sfhk_internal.h"

namespace sfhk {
namespace {

constexpr size_t kScratchPerPoint = sizeof(double2) + sizeof(double);   // twiddle + window

// Scratch of the no-allocation spectrum: the twiddle table (Nt double2)
// followed by the windowed samples (Nt doubles).  Every GPU that loads the
// library holds these SFHK_NOALLOC_MAX_NT * 24 bytes (768 KiB) until the
// process exits.  All calls on a device share it.
static __device__ __align__(256) unsigned char g_spectrum_scratch[SFHK_NOALLOC_MAX_NT *
                                                                  kScratchPerPoint];

// Device address of the scratch on the current device.  The array's name is
// only a host-side stand-in for the symbol, so host code has to ask the
// runtime for the address with the device current.  The lookup allocates
// nothing and is repeated on every call: an address kept from an earlier call
// would go stale once the device's primary context is reset or recreated
// (the module, and with it the array, is then loaded anew).
int scratch_address(void** out)
{
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_spectrum_scratch);
    if (e != cudaSuccess || p == nullptr) {
        std::fprintf(stderr, "sfhk: cudaGetSymbolAddress of the spectrum scratch failed: %s\n",
                     cudaGetErrorString(e));
        cudaGetLastError();
        return SFHK_E_CUDA;
    }
    *out = p;
    return SFHK_OK;
}

}  // namespace
}  // namespace sfhk

extern "C" int sfhk_spectrum_noalloc(const double* vz_dev, size_t nt, double dt, double t_origin,
                                     double tau_H, double* omega_dev, double* yield_dev,
                                     double* phase_dev, size_t n_out, void* stream)
{
    if (!vz_dev || nt < 2 || n_out == 0 || n_out > nt || !(dt > 0.0) || !(tau_H > 0.0))
        return SFHK_E_INVAL;
    if (nt > (size_t)SFHK_NOALLOC_MAX_NT) {
        std::fprintf(stderr, "sfhk_spectrum_noalloc: nt = %zu exceeds the fixed scratch size "
                             "(SFHK_NOALLOC_MAX_NT = %d)\n", nt, SFHK_NOALLOC_MAX_NT);
        return SFHK_E_INVAL;
    }
    void* scratch = nullptr;
    const int rc = sfhk::scratch_address(&scratch);
    if (rc) return rc;
    // launch_spectrum overwrites all Nt twiddle and windowed entries before
    // reading them, so nothing left by an earlier call needs clearing.
    return sfhk::launch_spectrum(vz_dev, (int)nt, dt, t_origin, tau_H, omega_dev, yield_dev,
                                 phase_dev, (int)n_out, reinterpret_cast<double2*>(scratch),
                                 reinterpret_cast<cudaStream_t>(stream));
}
