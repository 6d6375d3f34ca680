// check_trajectory_noalloc: the distance check for callers that must not allocate
// GPU memory during the call -- for example a fixed-period control loop in which
// an allocation's unbounded latency (or its implicit device synchronisation) would
// break the cycle deadline, or a host process whose memory was reserved up front
// and that is not allowed to grow it afterwards.
//
// Its scratch (the sorted cloud, tile and super-tile spheres, counters) lives in
// one file-scope device array of fixed size instead of memory obtained
// from cudaMalloc.  Every GPU that loads this library holds the array until the
// process exits.  The kernels are the same ones check_trajectory launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <mutex>

#include "internal.h"

namespace {

constexpr int kNoAllocMaxPoints = 32768;
constexpr int kNoAllocMaxTiles = kNoAllocMaxPoints / 32;
constexpr int kNoAllocMaxSupers = kNoAllocMaxTiles / 32;
constexpr size_t kSortedOff = 0;
constexpr size_t kTilesOff = kSortedOff + (size_t)kNoAllocMaxPoints * sizeof(float4);
constexpr size_t kSupersOff = kTilesOff + (size_t)kNoAllocMaxTiles * sizeof(float4);
constexpr size_t kMiscOff = kSupersOff + (size_t)kNoAllocMaxSupers * sizeof(float4);
constexpr size_t kValidOff = kMiscOff;             // 1 x int
constexpr size_t kStatusOff = kMiscOff + 128;      // 1 x int
constexpr size_t kScratchBytes = kMiscOff + 256;   // about 0.5 MiB

static_assert(SDF_NOALLOC_MAX_POINTS == kNoAllocMaxPoints, "header limit");

// The shared scratch.  In host code this name is only a stand-in for the device
// symbol; its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

struct PerDevice {
    std::mutex mu;
    std::atomic<bool> ready{false};  // set-up done on this device
    unsigned char* base = nullptr;   // device address of g_noalloc_scratch on this device
    int num_sms = 0;
};
constexpr int kMaxDevices = 64;
PerDevice g_per_device[kMaxDevices];

// Once per device, with that device current: look up the array's device address
// and set the check kernel's shared-memory limit (neither allocates).  A set-up
// that failed (for instance inside a stream capture) is not remembered: the next
// call tries again.
cudaError_t setup_device(PerDevice* pd) {
    if (pd->ready.load(std::memory_order_acquire)) return cudaSuccess;
    std::lock_guard<std::mutex> lk(pd->mu);
    if (pd->ready.load(std::memory_order_relaxed)) return cudaSuccess;
    unsigned char* base = nullptr;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetSymbolAddress((void**)&base, g_noalloc_scratch);
    if (e == cudaSuccess) e = sdf::configure_kernels();
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        cudaGetLastError();   // do not leave the failure for the caller's next CUDA call
        return e;
    }
    pd->base = base;
    pd->num_sms = sms;
    pd->ready.store(true, std::memory_order_release);
    return cudaSuccess;
}

// The launch parameters are large (one kernel-parameter table); keep one per
// thread instead of on the stack.
thread_local sdf::BatchParams t_params;

}  // namespace

extern "C" int check_trajectory_noalloc(const sdf_robot* R, void* cuda_stream, const float* q_dev, int32_t W,
                                        const float* points_dev, int32_t N, float* dist_dev,
                                        int32_t* argmin_link_dev, int32_t* argmin_point_dev,
                                        int32_t* status_dev) {
    // W is an int32, so the block count ceil(W / tw) fits an int; it is still
    // computed in 64 bits below so that no W can wrap it
    if (!R || W < 0 || N < 0 || N > kNoAllocMaxPoints) return SDF_ERR_INVALID_ARG;
    if (W == 0) return SDF_OK;
    if (!dist_dev || !argmin_link_dev || !argmin_point_dev || (R->dof > 0 && !q_dev) || (N > 0 && !points_dev))
        return SDF_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(points_dev) & 3u) != 0) return SDF_ERR_INVALID_ARG;
    if (R->device < 0 || R->device >= kMaxDevices) return SDF_ERR_INVALID_ARG;

    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return SDF_ERR_CUDA;
    if (prev != R->device && cudaSetDevice(R->device) != cudaSuccess) return SDF_ERR_CUDA;
    PerDevice* pd = &g_per_device[R->device];
    int rc = setup_device(pd) == cudaSuccess ? SDF_OK : SDF_ERR_CUDA;

    if (rc == SDF_OK) {
        const cudaStream_t stream = (cudaStream_t)cuda_stream;
        unsigned char* base = pd->base;
        int* status = status_dev ? status_dev : reinterpret_cast<int*>(base + kStatusOff);
        // the array keeps the previous call's contents: the sort rewrites the points,
        // spheres and count before the check reads them; the status word must start
        // cleared
        cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int), stream);

        sdf::BatchParams& p = t_params;
        sdf::CloudDesc& C = p.cloud[0];
        C.points = points_dev;
        C.N = N;
        C.point_base = C.tile_base = C.super_base = 0;
        sdf::InstDesc& I = p.inst[0];
        I.robot = R->d_table;
        I.q = q_dev;
        I.dist = dist_dev;
        I.arg_link = argmin_link_dev;
        I.arg_point = argmin_point_dev;
        I.W = W;
        I.L = R->table.L;
        I.dof = R->dof;
        I.cloud = 0;
        I.tw = sdf::kCheckWarps / I.L > 0 ? sdf::kCheckWarps / I.L : 1;
        I.block_base = 0;
        I.mask = nullptr;
        I.warm = R->table.values;
        I.warm_bytes = (unsigned long long)I.L * R->table.n * R->table.n * R->table.n * sizeof(float);
        const int n_tiles = (N + 31) / 32;
        const long long n_blocks = ((long long)W + I.tw - 1) / I.tw;   // <= W < 2^31
        p.n_inst = 1;
        p.n_cloud = 1;
        p.n_blocks = (int)n_blocks;
        I.interleave = sdf::interleave_waypoints(p.n_blocks, I.tw, 16, pd->num_sms);
        p.stride = 3;
        p.cull = 1;
        p.stage_tiles = n_tiles < sdf::kMaxStagedTiles ? n_tiles : sdf::kMaxStagedTiles;
        p.skip_prep = 0;
        p.warm_l2 = 1;
        p.warps = 16;
        p.tex = 0;
        p.sorted = reinterpret_cast<float4*>(base + kSortedOff);
        p.tiles = reinterpret_cast<float4*>(base + kTilesOff);
        p.supers = reinterpret_cast<float4*>(base + kSupersOff);
        p.n_valid = reinterpret_cast<int*>(base + kValidOff);
        p.status = status;
        p.wait_polls = sdf::kDefaultWaitPolls;
        p.sort_ctas = 0;
        p.stats = nullptr;
        if (e == cudaSuccess) e = sdf::launch_batch(p, sdf::kDefaultTileBatch, stream, nullptr);
        if (e != cudaSuccess) rc = SDF_ERR_CUDA;
    }
    if (prev >= 0 && prev != R->device) cudaSetDevice(prev);
    return rc;
}
