// noalloc.cu -- rhosvd_c2t for callers that cannot allocate device memory.
//
// rhosvd_c2t needs a caller-provided device workspace.  Some callers cannot provide one:
// code embedded in a host application that owns every device allocation (its own pool, or
// allocation switched off), code that must not risk the device-wide synchronisation that
// cudaMalloc / cudaFree may cause, or a caller with no allocator at hand at all.  For them,
// rhosvd_c2t_noalloc runs the same reduction with its scratch space taken from one
// statically sized device array that lives in this file.
//
// Facts a user needs:
//   * The array holds RHOSVD_NOALLOC_SCRATCH_BYTES (64 MiB).  Every GPU that loads the library
//     keeps that much device memory until the process exits.
//   * Problems whose workspace (rhosvd_c2t_workspace_size) exceeds it are rejected with
//     RHOSVD_ERR_SCRATCH_LIMIT before anything is launched.
//   * The first call on a device looks up the array's device address (cudaGetSymbolAddress,
//     once per device, with that device current).  Make that first call before any stream
//     capture begins.
//   * The address is cached per device ordinal for the life of the process, so the entry point
//     assumes the runtime's primary context of each device: after cudaDeviceReset, or with
//     another context made current through the driver API, the cached address is stale and the
//     entry point must not be used.
//   * Every call on a device uses the same array, and the array keeps whatever the previous
//     call left in it.  The reduction clears what it needs cleared itself.  Calls whose work
//     overlaps on the GPU (other streams, other host threads) race on the array: serialise them.
//   * Nothing here calls cudaMalloc, cudaFree or an allocating library routine.
#include "internal.cuh"
#include <mutex>

namespace {

constexpr size_t SCRATCH_BYTES = (size_t)RHOSVD_NOALLOC_SCRATCH_BYTES;

// The scratch space.  Device code could name it directly; host code must not pass the
// symbol itself to a kernel (on the host it is only a stand-in), so the host looks up its
// device address below and passes that pointer.
static __device__ __align__(256) unsigned char g_scratch[SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
void* g_addr[MAX_DEVICES] = {};

// Device address of g_scratch on the current device (set up once per device).
int scratch_address(void** out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return RHOSVD_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return RHOSVD_ERR_CUDA;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return RHOSVD_OK;
}

}  // namespace

extern "C" int rhosvd_c2t_noalloc(const rhosvd_cp* cp, const rhosvd_opts* opts, const rhosvd_tucker* out,
                                  void* stream)
{
    const size_t need = rhosvd_c2t_workspace_size(cp, opts);
    if (need == 0) return RHOSVD_ERR_INVALID_ARG;
    if (need > SCRATCH_BYTES) return RHOSVD_ERR_SCRATCH_LIMIT;
    void* ws = nullptr;
    const int rc = scratch_address(&ws);
    if (rc != RHOSVD_OK) return rc;
    return rhosvd_c2t(cp, opts, out, ws, SCRATCH_BYTES, stream);
}
