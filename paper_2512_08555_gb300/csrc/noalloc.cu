// Level-0 free-space solve that allocates no device memory.
//
// Some callers cannot call cudaMalloc at the point where they need the solve:
// code running while a stream is being captured into a CUDA graph (an
// allocation there fails or breaks the capture), hosts whose device memory is
// entirely handed out by their own pool allocator at start-up, and real-time
// loops where the implicit synchronisation of an allocation is not allowed.
// mrp_coarse_solve_noalloc gives them the level-0 FFT convolution with its
// spectral scratch in a fixed array that is part of the library image: every
// GPU that loads the library holds those bytes until the process exits.
#include "mrp_internal.h"

#include <mutex>

namespace mrp {

// Spectral scratch: Pz * Py * (Px/2 + 1) complex FP64 values at most.
constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(48) << 20;   // 48 MiB
static __device__ __align__(256) double2 g_noalloc_spec[NOALLOC_SCRATCH_BYTES / sizeof(double2)];

// Device addresses of the array, looked up once per device (host code cannot
// use the symbol itself as a device pointer).
static std::mutex g_noalloc_mu;
static void* g_noalloc_addr[256] = {nullptr};

static int noalloc_scratch(double2** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return MRP_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_spec) != cudaSuccess || !p) return MRP_ERR_CUDA;
        g_noalloc_addr[dev] = p;
    }
    *out = static_cast<double2*>(g_noalloc_addr[dev]);
    return MRP_OK;
}

}  // namespace mrp

extern "C" int mrp_coarse_solve_noalloc(mrp_handle* H, const double* f0, double* u0, void* stream) {
    using namespace mrp;
    if (!H || !f0 || !u0) return MRP_ERR_INVALID_ARG;
    if (H->g.size() != 1 || H->g[0]->nprob() != 1) return MRP_ERR_UNSUPPORTED;
    const Handle& h = *H->g[0];
    const Problem& p = h.pr[0];
    const size_t need = sizeof(double2) * (size_t)p.ax[2].P * p.ax[1].P * p.ax[0].K;
    if (need > NOALLOC_SCRATCH_BYTES) return MRP_ERR_TOO_LARGE;
    double2* spec = nullptr;
    const int rc = noalloc_scratch(&spec);
    if (rc != MRP_OK) return rc;
    launch_coarse_solve_ext(h, spec, f0, u0, (cudaStream_t)stream);
    // peek, not get: an error left by the caller's own earlier work stays
    // pending for the caller to see
    return cudaPeekAtLastError() == cudaSuccess ? MRP_OK : MRP_ERR_CUDA;
}
