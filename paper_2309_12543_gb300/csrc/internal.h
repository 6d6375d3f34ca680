// Internal definitions of the sdfcheck CUDA library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <utility>
#include <vector>

#include "sdfcheck.h"

namespace sdf {

constexpr int kMaxLinks = SDF_MAX_LINKS;
// Cull slack (metres): a sphere is skipped only when its lower bound exceeds the
// best distance found so far by more than this, which covers the FP32 rounding of
// the transform, the sphere centre and the interpolation (~1e-6 m).
constexpr float kCullSlack = 1e-4f;
constexpr int kMaxBatch = 128;            // trajectories per launch (kernel-parameter table)
constexpr int kCheckWarps = 16;           // warps per check block (the larger of the two shapes)
constexpr int kDefaultTileBatch = 1;      // list entries (tiles) per warp step (1, 2 or 4)
constexpr int kBlockList = 2048;          // (pair, tile) entries a block can queue in shared memory
constexpr int kMaxStagedTiles = 4096;     // tile spheres a block can stage in shared memory

// Robot + grids as the kernels see them.  The robot keeps a device copy.
struct LinkTable {
    int L;                    // links = dof + 1
    int dof;
    int n;                    // grid nodes per axis (same for every link)
    float base[12];           // world-from-base, row-major 3x4
    float dh_a[kMaxLinks], dh_d[kMaxLinks], dh_ca[kMaxLinks], dh_sa[kMaxLinks],
        dh_th[kMaxLinks];     // per joint: a, d, cos(alpha), sin(alpha), theta offset
    float4 sph_local[kMaxLinks];   // bounding sphere centre (link frame) + radius
    float4 cap_a[kMaxLinks];       // bounding capsule: segment start (link frame) + radius
    float4 cap_b[kMaxLinks];       // segment end (w unused)
    float4 grid_o[kMaxLinks];      // grid origin (link frame) + 1/h
    float grid_h[kMaxLinks];
    const float* values;           // L grids of n^3 floats, x fastest
};

// One obstacle cloud of a launch (requests that pass the same cloud share it).
struct CloudDesc {
    const float* points;      // N x stride
    int N;
    int point_base;           // sorted points (N)
    int tile_base;            // ceil(N / 32) tile spheres
    int super_base;           // ceil(N / 1024) super-tile spheres
};

// One trajectory check inside a launch.
struct InstDesc {
    const LinkTable* robot;   // device copy
    const float* q;           // W x dof
    float* dist;
    int32_t* arg_link;
    int32_t* arg_point;
    int W, L, dof;
    int cloud;                // index into BatchParams::cloud
    int tw;                   // waypoints per check block (tw * L <= kCheckWarps)
    int block_base;           // first check block of this trajectory
    const uint8_t* mask;      // optional: only waypoints with a non-zero byte are checked
    const float* warm;        // the robot's grids, for the first trajectory of each robot
                              // in the launch (null otherwise): its blocks prefetch them
                              // into L2 while the sort runs
    unsigned long long warm_bytes;
    int interleave;           // block b takes waypoints b, b + ceil(W / tw), ... instead of b * tw + j
};

struct BatchParams {
    int n_inst;
    int n_cloud;
    int n_blocks;             // check blocks over all trajectories
    int stride;               // floats per point: 3 or 4
    int cull;                 // 0: evaluate every pair
    int stage_tiles;          // tile spheres the dynamic shared memory holds (0: no staging)
    int skip_prep;            // the clouds are already sorted in the scratch: launch the check only
    int warps;                // warps per check block: 8 or 16
    int tex;                  // lookups by the texture unit (SDF_OPT_TEX3D)
    unsigned long long tex_h[kMaxLinks];  // texture objects of the launch's grids, by link
    int warm_l2;              // the check overlaps the sort (programmatic dependent launch):
                              // its blocks prefetch the grids meanwhile (InstDesc::warm)
    float4* sorted;           // finite points, spatially sorted: x, y, z, original index bits
    float4* tiles;            // sphere of each 32-point tile
    float4* supers;           // sphere of each 32-tile super-tile
    int* n_valid;             // finite points per cloud
    int* status;              // device status bits
    unsigned wait_polls;      // polls of the sphere-staging wait before it gives up
    int sort_ctas;            // CTAs of the sort's cluster: 8, 16 (allowed by the device), 0 = widest
    unsigned long long* stats;  // kStatCount counters, or null (statistics off)
    CloudDesc cloud[kMaxBatch];
    InstDesc inst[kMaxBatch];
};

enum StatusBits : int { kStatusNonFinite = 1, kStatusTimeout = 2 };

// Default poll limit of the bounded device waits (SDF_OPT_WAIT_POLLS); every wait
// that gave up is followed by a drain wait of this many polls, so that no copy or
// MMA issued by a block is still in flight when it releases its memory.
constexpr unsigned kDefaultWaitPolls = 1u << 22;

// Statistics counters (SDF_OPT_STATS); indices match SDF_STAT_* in sdfcheck.h.
constexpr int kStatCount = 32;

// Allocations (alloc.cu): every device and page-locked host allocation of the
// library goes through these, so that a test can make one fail on the host
// (sdf_debug_fail_alloc) and count what is live (sdf_debug_alloc_live).
cudaError_t dmalloc_raw(void** p, size_t bytes);
cudaError_t hmalloc_raw(void** p, size_t bytes);   // page-locked, cudaHostAllocDefault
template <typename T>
inline cudaError_t dmalloc(T** p, size_t bytes) { return dmalloc_raw(reinterpret_cast<void**>(p), bytes); }
template <typename T>
inline cudaError_t hmalloc(T** p, size_t bytes) { return hmalloc_raw(reinterpret_cast<void**>(p), bytes); }
void dfree(void* p);   // null is a no-op
void hfree(void* p);
cudaError_t amalloc3d(cudaArray_t* a, int n);   // n^3 FP32 texels (one channel)
void afree(cudaArray_t a);

// Launchers (check.cu / grid_build.cu).  Each returns the launch's cudaError_t.
cudaError_t configure_kernels();           // once per device, that device current
// The widest cluster the sort runs as on a device (16 where the device can place that
// non-portable size, else 8); known after configure_kernels ran for that device.
int max_sort_ctas(int device);
// One thread: moves the device status word to page-locked host memory (and clears
// it), then publishes ++(*d_seq) in *h_done behind a system-scope fence.
cudaError_t launch_finish(int* status, int* h_status, unsigned* d_seq, unsigned* h_done, cudaStream_t s);

// Whether a launch's blocks take interleaved waypoints (InstDesc::interleave): when
// a block holds several waypoints and every block is resident at once (one wave of
// 32 / nw blocks an SM at 64 registers a thread), the kernel ends with its slowest
// block, and pairing waypoints from distant parts of a trajectory evens the blocks
// out.  With more blocks than fit at once the block scheduler balances them.
inline int interleave_waypoints(long long n_blocks, int tw, int nw, int num_sms) {
    return tw > 1 && n_blocks <= (long long)num_sms * (32 / nw) ? 1 : 0;
}
// Enqueues the two kernels of one batch (spatial sort, check); ev_mid (may be null)
// is recorded between them.
cudaError_t launch_batch(const BatchParams& p, int tile_batch, cudaStream_t s, cudaEvent_t ev_mid);
cudaError_t launch_fk(const LinkTable& T, const float* q, int W, float* out, int* status, cudaStream_t s);
// Kinematics and the resets of a surrogate check (keys to ~0, re-check flags and the
// two work counters to 0), overlapping the sort launched just before it on s; completes only
// after that sort.
cudaError_t launch_fk_reset(const LinkTable& T, const float* q, int W, float* out, int* status,
                            unsigned long long* keys, uint8_t* recheck, int* counter, cudaStream_t s);
// Sorts one cloud into the scratch of p (prep kernel only).
cudaError_t launch_prep(const BatchParams& p, cudaStream_t s);
cudaError_t launch_grid_build(const float* tris9, const int* comp_off, int n_comp, int n_tris, float ox,
                              float oy, float oz, float h, int n, float* out, cudaStream_t s);

}  // namespace sdf

struct sdf_ctx;
namespace sdf {
// api.cu: sort one cloud into ctx's scratch and fill p's cloud/scratch fields.
int sort_cloud(sdf_ctx* ctx, const float* points_dev, int N, BatchParams* p);
// surrogate.cu: the grids a surrogate was built on.
const sdf_grids* surrogate_grids(const sdf_surrogate* s);
}  // namespace sdf

struct sdf_grids {
    int device = 0;
    int n_links = 0;
    int n = 0;
    float* values = nullptr;  // device, n_links * n^3
    sdf_grid_meta meta[SDF_MAX_LINKS];
    bool capsules = false;    // cap_a / cap_b computed (on first use)
    float4 cap_a[SDF_MAX_LINKS], cap_b[SDF_MAX_LINKS];
    // hardware-filtered copy (SDF_OPT_TEX3D), made by the first check that asks for it:
    // one 3-D array and linear-filtering texture object per link
    cudaArray_t tex_arr[SDF_MAX_LINKS] = {};
    cudaTextureObject_t tex[SDF_MAX_LINKS] = {};
    bool tex_ready = false;
};

struct sdf_robot {
    int device = 0;
    int dof = 0;
    uint64_t id = 0;                       // unique per created robot (cache keys)
    const sdf_grids* grids = nullptr;
    sdf::LinkTable table;                  // host copy
    sdf::LinkTable* d_table = nullptr;     // device copy read by the kernels
};

struct sdf_ctx {
    int device = 0;
    int num_sms = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    // options
    int cull = 1;
    int point_stride = 3;
    int time_kernels = 0;
    int stats = 0;
    unsigned long long* d_stats = nullptr;  // kStatCount counters on the device
    int tw = 0;                            // waypoints per check block (0: tuned or as many as fit)
    int tile_batch = 0;                    // list entries per warp step (0: tuned or 4)
    int reuse_sort = 0;                    // internal: the next check reuses the scratch's sorted cloud
    int block_warps = 0;                   // warps per check block (0: tuned or 16)
    int tex3d = 0;                         // lookups by the texture unit's trilinear filter
    int sort_ctas = 0;                     // CTAs of the sort's cluster (SDF_OPT_SORT_CTAS)
    unsigned wait_polls = sdf::kDefaultWaitPolls;  // polls of a bounded device wait (SDF_OPT_WAIT_POLLS)
    struct Shape { int tw, tb, nw, sort; };
    std::map<uint64_t, Shape> tuned;       // launch shape key -> (waypoints per block, tile batch, warps,
                                           // CTAs of the sort's cluster)
    // scratch owned by the context (grown on demand, or up front by sdf_ctx_reserve)
    float4* sorted = nullptr;
    size_t sorted_cap = 0;
    float4* tiles = nullptr;
    size_t tiles_cap = 0;
    float4* supers = nullptr;
    size_t supers_cap = 0;
    int* n_valid = nullptr;
    size_t n_valid_cap = 0;
    int* status = nullptr;
    int* h_status = nullptr;               // page-locked copy of the status word
    // completion word of the host-buffer path: finish_kernel bumps d_seq and writes it
    // to page-locked h_done after the status, and the host waits for the value it
    // expects (seq) by polling instead of a stream synchronisation
    unsigned* d_seq = nullptr;
    unsigned* h_done = nullptr;
    unsigned seq = 0;
    // staging for check_trajectory_host
    float* st_q = nullptr;
    size_t st_q_cap = 0;
    float* st_pts = nullptr;
    size_t st_pts_cap = 0;
    float* st_dist = nullptr;
    int32_t* st_link = nullptr;
    int32_t* st_point = nullptr;
    size_t st_out_cap = 0;
    // Robot-SDF workspace (grown on demand)
    unsigned* rs_sdf = nullptr;
    size_t rs_sdf_cap = 0;
    unsigned* rs_bits = nullptr;
    size_t rs_bits_cap = 0;
    int* rs_list = nullptr;
    size_t rs_list_cap = 0;
    float* rs_poses = nullptr;
    size_t rs_poses_cap = 0;
    // surrogate check workspace (grown on demand)
    float* sur_poses = nullptr;
    unsigned long long* sur_keys = nullptr;
    uint8_t* sur_mask = nullptr;
    size_t sur_w_cap = 0;
    int* sur_count = nullptr;              // work-item counter of the fused surrogate check
    uint8_t* sur_wimg = nullptr;           // the networks' weights as the fused check holds them
    size_t sur_wimg_cap = 0;
    uint64_t sur_wimg_id = 0, sur_wimg_version = 0;   // the surrogate (id, version) the image holds
    // timing
    cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev2 = nullptr;
    bool timed_valid = false;
    // check_trajectory_host: one CUDA graph per argument set (copies in, sort, check,
    // copies out), dropped whenever scratch or staging moves or an option changes
    struct HostGraph {
        uint64_t robot;
        const void* ptr[5];
        int W, N;
        bool zero_copy;
        cudaGraphExec_t exec;
    };
    std::vector<HostGraph> host_graphs;
    cudaStream_t capture_stream = nullptr;
};
