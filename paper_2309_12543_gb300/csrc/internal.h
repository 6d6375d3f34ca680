// Internal definitions of the sdfcheck CUDA library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "sdfcheck.h"

namespace sdf {

constexpr int kMaxLinks = SDF_MAX_LINKS;
constexpr int kMaxWaypointsPerBlock = 32;  // one warp per (waypoint, link): TW * L <= 32
// Cull slack (metres): a pair is skipped only when its bounding-sphere lower bound
// exceeds the best distance found so far by more than this, which covers the FP32
// rounding of the transform, the sphere centre and the interpolation (~1e-6 m).
constexpr float kCullSlack = 1e-4f;

// Robot + grids as the kernels see them (passed by value as a kernel parameter).
struct LinkTable {
    int L;                    // links = dof + 1
    int dof;
    int n;                    // grid nodes per axis (same for every link)
    float base[12];           // world-from-base, row-major 3x4
    float dh_a[kMaxLinks], dh_d[kMaxLinks], dh_ca[kMaxLinks], dh_sa[kMaxLinks],
        dh_th[kMaxLinks];     // per joint: a, d, cos(alpha), sin(alpha), theta offset
    float4 sph_local[kMaxLinks];   // bounding sphere centre (link frame) + radius
    float4 grid_o[kMaxLinks];      // grid origin (link frame) + 1/h
    float grid_h[kMaxLinks];
    const float* values;           // L grids of n^3 floats, x fastest
};

constexpr int kCells = 32768;             // 32^3 Morton cells for the cloud sort
constexpr int kMaxStagedTiles = 4096;     // tile spheres staged in shared memory (64 KiB)
constexpr int kTileBatch = 4;             // tiles per warp step in the sweep

// Spatial sort of the obstacle points (cloud_prep_kernel).
struct PrepParams {
    const float* points;      // N x stride, caller's layout
    int N;
    int stride;               // 3 or 4
    float4* sorted;           // N: x, y, z, original index (int bits); finite points only
    float4* tiles;            // ceil(N / 32): bounding sphere of each 32-point tile
    float4* supers;           // ceil(N / 1024): bounding sphere of each 32-tile super-tile
    int* n_valid;             // number of finite points written to `sorted`
    int* status;
};

struct CheckParams {
    LinkTable T;
    const float* q;           // W x dof
    int W;
    int tw;                   // waypoints per block (block = 32 * tw * L threads)
    const float4* sorted;     // from PrepParams
    const float4* tiles;
    const float4* supers;
    const int* n_valid;
    int max_tiles;            // ceil(N / 32): tiles the scratch can hold
    int stage;                // 1: copy tile and super-tile spheres to shared memory
    int cull;                 // 0: evaluate every pair
    float* dist;
    int32_t* arg_link;
    int32_t* arg_point;
    int* status;              // device status bits
};

enum StatusBits : int { kStatusNonFinite = 1, kStatusTimeout = 2 };

// Launchers (check.cu / grid_build.cu).  Return a cudaError_t of the launch.
cudaError_t configure_kernels();           // once per device, that device current
cudaError_t launch_prep(const PrepParams& p, cudaStream_t s);
cudaError_t launch_check(const CheckParams& p, cudaStream_t s);
cudaError_t launch_fk(const LinkTable& T, const float* q, int W, float* out, int* status,
                      cudaStream_t s);
cudaError_t launch_grid_build(const float* tris9, const int* comp_off, int n_comp, int n_tris,
                              float ox, float oy, float oz, float h, int n, float* out,
                              cudaStream_t s);

}  // namespace sdf

struct sdf_grids {
    int device = 0;
    int n_links = 0;
    int n = 0;
    float* values = nullptr;  // device, n_links * n^3
    sdf_grid_meta meta[SDF_MAX_LINKS];
};

struct sdf_robot {
    int device = 0;
    int dof = 0;
    const sdf_grids* grids = nullptr;
    sdf::LinkTable table;
};

struct sdf_ctx {
    int device = 0;
    int num_sms = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    // options
    int cull = 1;
    int point_stride = 3;
    int tw = 0;
    int time_kernels = 0;
    // scratch owned by the context
    float4* sorted = nullptr;
    size_t sorted_cap = 0;
    float4* tiles = nullptr;
    size_t tiles_cap = 0;
    float4* supers = nullptr;
    size_t supers_cap = 0;
    int* n_valid = nullptr;
    int* status = nullptr;
    // staging for check_trajectory_host
    float* st_q = nullptr;
    size_t st_q_cap = 0;
    float* st_pts = nullptr;
    size_t st_pts_cap = 0;
    float* st_dist = nullptr;
    int32_t* st_link = nullptr;
    int32_t* st_point = nullptr;
    size_t st_out_cap = 0;
    // timing
    cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev2 = nullptr;
    bool timed_valid = false;
};
