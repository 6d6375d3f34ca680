// check_trajectory_noalloc: the distance check for callers that must not allocate
// GPU memory during the call -- for example a fixed-period control loop in which
// an allocation's unbounded latency (or its implicit device synchronisation) would
// break the cycle deadline, or a host process whose memory was reserved up front
// and that is not allowed to grow it afterwards.
//
// Its scratch (sorted cloud, tile and super-tile spheres, counters)
// lives in one file-scope device array of fixed size instead of memory obtained
// from cudaMalloc.  Every GPU that loads this library holds the array until the
// process exits.  The kernels are the same ones check_trajectory launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "internal.h"

namespace {

constexpr int kNoAllocMaxPoints = 65536;
constexpr int kNoAllocMaxWaypoints = 4096;
constexpr size_t kSortedOff = 0;
constexpr size_t kTilesOff = kSortedOff + (size_t)kNoAllocMaxPoints * sizeof(float4);
constexpr size_t kSupersOff = kTilesOff + (size_t)(kNoAllocMaxPoints / 32) * sizeof(float4);
constexpr size_t kCountOff = kSupersOff + (size_t)(kNoAllocMaxPoints / 1024) * sizeof(float4);
constexpr size_t kStatusOff = kCountOff + 256;
constexpr size_t kScratchBytes = kStatusOff + 256;   // about 1.1 MiB

static_assert(SDF_NOALLOC_MAX_POINTS == kNoAllocMaxPoints, "header limit");
static_assert(SDF_NOALLOC_MAX_WAYPOINTS == kNoAllocMaxWaypoints, "header limit");

// The shared scratch.  In host code this name is only a stand-in for the device
// symbol; its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

struct PerDevice {
    std::once_flag once;
    cudaError_t err = cudaSuccess;
    unsigned char* base = nullptr;   // device address of g_noalloc_scratch on this device
};
constexpr int kMaxDevices = 64;
PerDevice g_per_device[kMaxDevices];

// Once per device, with that device current: look up the array's device address
// and set the kernels' shared-memory limit (neither allocates).
void setup_device(int dev, PerDevice* pd) {
    (void)dev;
    pd->err = cudaGetSymbolAddress((void**)&pd->base, g_noalloc_scratch);
    if (pd->err == cudaSuccess) pd->err = sdf::configure_kernels();
}

}  // namespace

extern "C" int check_trajectory_noalloc(const sdf_robot* R, void* cuda_stream, const float* q_dev, int32_t W,
                                        const float* points_dev, int32_t N, float* dist_dev,
                                        int32_t* argmin_link_dev, int32_t* argmin_point_dev,
                                        int32_t* status_dev) {
    if (!R || W < 0 || N < 0) return SDF_ERR_INVALID_ARG;
    if (W > kNoAllocMaxWaypoints || N > kNoAllocMaxPoints) return SDF_ERR_INVALID_ARG;
    if (W == 0) return SDF_OK;
    if (!dist_dev || !argmin_link_dev || !argmin_point_dev || (R->dof > 0 && !q_dev) || (N > 0 && !points_dev))
        return SDF_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(points_dev) & 3u) != 0) return SDF_ERR_INVALID_ARG;
    if (R->device < 0 || R->device >= kMaxDevices) return SDF_ERR_INVALID_ARG;

    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return SDF_ERR_CUDA;
    if (prev != R->device && cudaSetDevice(R->device) != cudaSuccess) return SDF_ERR_CUDA;
    PerDevice* pd = &g_per_device[R->device];
    std::call_once(pd->once, setup_device, R->device, pd);
    int rc = SDF_OK;
    if (pd->err != cudaSuccess) rc = SDF_ERR_CUDA;

    if (rc == SDF_OK) {
        const cudaStream_t stream = (cudaStream_t)cuda_stream;
        const int L = R->table.L;
        const int tw = 32 / L >= 2 ? 2 : 1;
        const int n_tiles = std::max(1, (N + 31) / 32);
        int* status = status_dev ? status_dev : reinterpret_cast<int*>(pd->base + kStatusOff);
        // the array keeps the previous call's contents: the prep kernel rewrites the
        // sorted cloud, spheres and count before the check reads them; the status
        // word must start cleared
        cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int), stream);

        sdf::PrepParams pp;
        pp.points = points_dev;
        pp.N = N;
        pp.stride = 3;
        pp.sorted = reinterpret_cast<float4*>(pd->base + kSortedOff);
        pp.tiles = reinterpret_cast<float4*>(pd->base + kTilesOff);
        pp.supers = reinterpret_cast<float4*>(pd->base + kSupersOff);
        pp.n_valid = reinterpret_cast<int*>(pd->base + kCountOff);
        pp.status = status;

        sdf::CheckParams p;
        p.T = R->table;
        p.q = q_dev;
        p.W = W;
        p.tw = tw;
        p.sorted = pp.sorted;
        p.tiles = pp.tiles;
        p.supers = pp.supers;
        p.n_valid = pp.n_valid;
        p.max_tiles = n_tiles;
        p.stage = n_tiles <= sdf::kMaxStagedTiles ? 1 : 0;
        p.cull = 1;
        p.dist = dist_dev;
        p.arg_link = argmin_link_dev;
        p.arg_point = argmin_point_dev;
        p.status = status;

        if (e == cudaSuccess) e = sdf::launch_prep(pp, stream);
        if (e == cudaSuccess) e = sdf::launch_check(p, stream);
        if (e != cudaSuccess) rc = SDF_ERR_CUDA;
    }
    if (prev >= 0 && prev != R->device) cudaSetDevice(prev);
    return rc;
}
