// check_trajectory_noalloc: the distance check for callers that must not allocate
// GPU memory during the call -- for example a fixed-period control loop in which
// an allocation's unbounded latency (or its implicit device synchronisation) would
// break the cycle deadline, or a host process whose memory was reserved up front
// and that is not allowed to grow it afterwards.
//
// Its scratch (sorted cloud, tile spheres, per-waypoint keys and tickets, counters)
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
constexpr size_t kKeysOff = kTilesOff + (size_t)(kNoAllocMaxPoints / 32) * sizeof(float4);
constexpr size_t kTicketsOff = kKeysOff + (size_t)kNoAllocMaxWaypoints * sizeof(unsigned long long);
constexpr size_t kCountOff = kTicketsOff + (size_t)kNoAllocMaxWaypoints * sizeof(unsigned);
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
    int num_sms = 0;
};
constexpr int kMaxDevices = 64;
PerDevice g_per_device[kMaxDevices];

// Once per device, with that device current: look up the array's device address
// and set the kernels' shared-memory limit (neither allocates).
void setup_device(int dev, PerDevice* pd) {
    pd->err = cudaGetSymbolAddress((void**)&pd->base, g_noalloc_scratch);
    if (pd->err == cudaSuccess) pd->err = cudaDeviceGetAttribute(&pd->num_sms, cudaDevAttrMultiProcessorCount, dev);
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
        const int tw = (4 * L <= 32) ? 4 : (2 * L <= 32 ? 2 : 1);
        const int wt = (W + tw - 1) / tw;
        const int n_tiles = std::max(1, (N + 31) / 32);
        int splits = std::min(std::max(1, (2 * pd->num_sms + wt - 1) / wt), n_tiles);
        const int per = (n_tiles + splits - 1) / splits;
        splits = (n_tiles + per - 1) / per;

        unsigned long long* keys = reinterpret_cast<unsigned long long*>(pd->base + kKeysOff);
        unsigned* tickets = reinterpret_cast<unsigned*>(pd->base + kTicketsOff);
        int* status = status_dev ? status_dev : reinterpret_cast<int*>(pd->base + kStatusOff);
        // the array keeps the previous call's contents: reset what must start cleared
        cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int), stream);
        if (e == cudaSuccess && splits > 1) e = cudaMemsetAsync(keys, 0xff, (size_t)W * sizeof(*keys), stream);
        if (e == cudaSuccess && splits > 1) e = cudaMemsetAsync(tickets, 0, (size_t)wt * sizeof(*tickets), stream);

        sdf::PrepParams pp;
        pp.points = points_dev;
        pp.N = N;
        pp.stride = 3;
        pp.sorted = reinterpret_cast<float4*>(pd->base + kSortedOff);
        pp.tiles = reinterpret_cast<float4*>(pd->base + kTilesOff);
        pp.n_valid = reinterpret_cast<int*>(pd->base + kCountOff);
        pp.status = status;

        sdf::CheckParams p;
        p.T = R->table;
        p.q = q_dev;
        p.W = W;
        p.sorted = pp.sorted;
        p.tiles = pp.tiles;
        p.n_valid = pp.n_valid;
        p.splits = splits;
        p.tiles_per_split = per;
        p.max_tiles = n_tiles;
        p.stage_tiles = n_tiles <= sdf::kMaxStagedTiles ? 1 : 0;
        p.cull = 1;
        p.dist = dist_dev;
        p.arg_link = argmin_link_dev;
        p.arg_point = argmin_point_dev;
        p.keys = splits > 1 ? keys : nullptr;
        p.tickets = splits > 1 ? tickets : nullptr;
        p.status = status;

        if (e == cudaSuccess) e = sdf::launch_prep(pp, stream);
        if (e == cudaSuccess) e = sdf::launch_check(p, tw, stream);
        if (e != cudaSuccess) rc = SDF_ERR_CUDA;
    }
    if (prev >= 0 && prev != R->device) cudaSetDevice(prev);
    return rc;
}
