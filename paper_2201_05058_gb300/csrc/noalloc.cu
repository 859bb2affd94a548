// Static-field build without any allocation and without a caller workspace.
//
// Some callers cannot allocate device memory at the moment they need a
// distance field: real-time planning loops that forbid allocation after
// start-up (an allocation can block or fail at an unpredictable moment), and
// hosts whose device memory is owned entirely by another runtime, so that
// they have no workspace to lend.  This entry point serves them: its scratch
// is a fixed array in the library's own device memory, sized for grids of up
// to PCDF_NOALLOC_MAX_VOXELS voxels.
//
// The array is a file-scope __device__ variable, so every GPU that loads the
// library holds it (about 12 MB) until the process exits.  CUDA loads modules
// lazily by default, so the array is allocated by the driver when the first
// call on a device loads this module: that first call can fail with an
// out-of-memory error (PCDF_ECUDA), and a caller that must not fail later
// makes it at start-up.  In host code the array's name is only a host-side
// stand-in; its device address is looked up with cudaGetSymbolAddress, with
// the call's device current, on every call whose stream is not being
// captured (so a device reset, which reloads the module, never leaves a stale
// address), and the last address found on the device is used while a stream
// is captured.  The first call on a device must therefore come before any
// capture.  All calls share the array: calls whose work overlaps on the GPU
// (different streams, or different host threads on the same device) race on
// it and must be serialised by the caller.  Nothing in it needs to start at
// zero: each call writes every scratch element before reading it.
#include <cuda_runtime.h>

#include <mutex>

#include "host.h"

using namespace pcdf::host;

namespace {

constexpr long long kMaxVoxels = PCDF_NOALLOC_MAX_VOXELS;
// int16 row distances and int32 partial distances of one grid, each section
// rounded up to the 256-byte alignment that the kernels' carving uses
constexpr size_t kScratchBytes = ((size_t)kMaxVoxels * 2 + 255) / 256 * 256 + ((size_t)kMaxVoxels * 4 + 255) / 256 * 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device: looked up again
// unless `stream` is being captured, when the last address found is used.
int scratch_address(cudaStream_t stream, void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices)
        return fail(PCDF_EINVAL, "device ordinal %d beyond %d", dev, kMaxDevices);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(stream, &cap);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaStreamIsCapturing");
    std::lock_guard<std::mutex> lock(g_mutex);
    if (cap == cudaStreamCaptureStatusNone || !g_scratch_ptr[dev]) {
        if (cap != cudaStreamCaptureStatusNone)
            return fail(PCDF_EINVAL, "the first allocation-free call on a device must not be captured");
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess)
            return cuda_fail(e, "cudaGetSymbolAddress of the scratch array");
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return PCDF_OK;
}

}  // namespace

extern "C" int pcdf_build_static_sdf_noalloc(const pcdf_grid *grid, const uint8_t *occ, int32_t *static_sq,
                                             float *static_sdf, void *stream)
{
    if (int rc = check_grid(grid))
        return rc;
    if (!occ || !static_sq)
        return fail(PCDF_EINVAL, "occ and static_sq must be non-NULL");
    const long long V = nvox(grid);
    if (V > kMaxVoxels)
        return fail(PCDF_EINVAL,
                    "grid of %lld voxels exceeds the %lld voxels of the allocation-free build; use "
                    "pcdf_build_static_sdf with a workspace",
                    V, kMaxVoxels);
    if (full_edt_ws(grid) > kScratchBytes)
        return fail(PCDF_EINVAL, "grid needs %zu scratch bytes, more than the %zu available", full_edt_ws(grid),
                    kScratchBytes);
    void *scratch = nullptr;
    if (int rc = scratch_address((cudaStream_t)stream, &scratch))
        return rc;
    static pcdf::CapBatch none;  // the occupancy-only row pass reads no capsules
    return run_full_edt(grid, 0, occ, &none, 0, static_sq, static_sdf, scratch, (cudaStream_t)stream);
}
