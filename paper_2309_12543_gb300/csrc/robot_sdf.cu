// The paper's own formulation of the check (Sec. III-A), kept beside the per-point
// path for comparison: per-configuration Robot SDFs on an environment voxel grid,
// read at the voxelised obstacles.
//
// Transforming a Link SDF so that its samples fall on environment voxel centres
// (the Euclidean transformation of Eq. (4) with the alignment shift of Eq. (1)-(3))
// is the same as evaluating the link SDF at each voxel centre mapped into the link
// frame, which is what robot_sdf_kernel does for the voxels of each link's block
// (the "grids in sphere" of Sec. III-B: radius R_link + reach + sqrt(3) r_e / 2
// around the link's bounding-sphere centre).  The Robot SDF of a configuration is
// the minimum over links per voxel (an atomicMin on order-preserving bits); the
// distance is its minimum over the occupied voxels.  Memory: W x voxels x 4 bytes,
// the cost of the formulation the paper reports (Sec. V).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <string>

#include "internal.h"
#include "lookup.cuh"

namespace sdf {
namespace {

using namespace dev;

constexpr unsigned kUnset = 0xffffffffu;   // a voxel no block wrote (above every ordered value)

struct EnvArgs {
    float ox, oy, oz;   // grid origin (lower corner)
    float r, inv_r;     // voxel edge and fl32(1 / r)
    int nx, ny, nz;
    long long nv;       // voxels
    float reach;        // distance range the blocks cover beyond a link's bounding sphere
};

// Voxel index of a point, taken in single precision without contraction:
// floor((p - o) * fl32(1 / r)) per axis; -1 outside the grid or non-finite.
__device__ __forceinline__ long long voxel_of(const EnvArgs& E, float x, float y, float z) {
    const float fx = __fmul_rn(__fsub_rn(x, E.ox), E.inv_r);
    const float fy = __fmul_rn(__fsub_rn(y, E.oy), E.inv_r);
    const float fz = __fmul_rn(__fsub_rn(z, E.oz), E.inv_r);
    if (!(fx >= 0.f && fx < (float)E.nx && fy >= 0.f && fy < (float)E.ny && fz >= 0.f && fz < (float)E.nz))
        return -1;
    const long long i = (long long)floorf(fx), j = (long long)floorf(fy), k = (long long)floorf(fz);
    if (i >= E.nx || j >= E.ny || k >= E.nz) return -1;
    return i + (long long)E.nx * (j + (long long)E.ny * k);
}

// Voxelise the cloud: one bit per voxel; the point that sets a voxel's bit appends
// the voxel to the occupied list.
__global__ void voxelize_kernel(const float* __restrict__ pts, int N, int stride, EnvArgs E,
                                unsigned* __restrict__ bits, int* __restrict__ list, int* __restrict__ count) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const float* p = pts + (size_t)i * stride;
    const long long v = voxel_of(E, p[0], p[1], p[2]);
    if (v < 0) return;
    const unsigned bit = 1u << (unsigned)(v & 31);
    const unsigned old = atomicOr(&bits[v >> 5], bit);
    if (!(old & bit)) list[atomicAdd(count, 1)] = (int)v;
}

__device__ __forceinline__ int clamp_index(float f, int lo, int hi) {
    if (!(f >= (float)lo)) return lo;   // also NaN
    if (f > (float)hi) return hi;
    return (int)f;
}

// One CTA per (configuration, link): every voxel of the link's block gets the link
// SDF at its centre (trilinear, out-of-box rule), folded into the configuration's
// Robot SDF.
__global__ void __launch_bounds__(256) robot_sdf_kernel(const float* __restrict__ poses, int L,
                                                        const LinkTable* __restrict__ T, EnvArgs E,
                                                        unsigned* __restrict__ robot_sdf) {
    const int w = blockIdx.x / L, l = blockIdx.x % L;
    const float4* P = reinterpret_cast<const float4*>(poses + ((size_t)w * L + l) * 16);
    const float4 r0 = P[0], r1 = P[1], r2 = P[2], sph = P[3];
    if (!(isfinite(sph.x) && isfinite(sph.y) && isfinite(sph.z))) return;   // flagged by the FK
    const float rho = sph.w + E.reach + 0.8660254f * E.r;
    const float rho2 = rho * rho;
    // the block's bounding cube in voxel indices, clamped to the grid before any
    // conversion to int (a far-away link gives an empty range)
    const int i0 = clamp_index(floorf((sph.x - rho - E.ox) * E.inv_r), 0, E.nx);
    const int j0 = clamp_index(floorf((sph.y - rho - E.oy) * E.inv_r), 0, E.ny);
    const int k0 = clamp_index(floorf((sph.z - rho - E.oz) * E.inv_r), 0, E.nz);
    const int i1 = clamp_index(floorf((sph.x + rho - E.ox) * E.inv_r), -1, E.nx - 1);
    const int j1 = clamp_index(floorf((sph.y + rho - E.oy) * E.inv_r), -1, E.ny - 1);
    const int k1 = clamp_index(floorf((sph.z + rho - E.oz) * E.inv_r), -1, E.nz - 1);
    if (i0 > i1 || j0 > j1 || k0 > k1) return;
    const int ni = i1 - i0 + 1, nj = j1 - j0 + 1;
    const long long cube = (long long)ni * nj * (k1 - k0 + 1);
    const int n = T->n;
    const float* G = T->values + (size_t)l * n * n * n;
    const float4 go = T->grid_o[l];
    const float gh = T->grid_h[l];
    unsigned* R = robot_sdf + (size_t)w * E.nv;
    for (long long t = threadIdx.x; t < cube; t += blockDim.x) {
        const int i = i0 + (int)(t % ni);
        const int j = j0 + (int)((t / ni) % nj);
        const int k = k0 + (int)(t / ((long long)ni * nj));
        const float x = fmaf((float)i + 0.5f, E.r, E.ox);
        const float y = fmaf((float)j + 0.5f, E.r, E.oy);
        const float z = fmaf((float)k + 0.5f, E.r, E.oz);
        const float dx = x - sph.x, dy = y - sph.y, dz = z - sph.z;
        if (fmaf(dx, dx, fmaf(dy, dy, dz * dz)) > rho2) continue;
        const float lx = fmaf(r0.x, x, fmaf(r0.y, y, fmaf(r0.z, z, r0.w)));
        const float ly = fmaf(r1.x, x, fmaf(r1.y, y, fmaf(r1.z, z, r1.w)));
        const float lz = fmaf(r2.x, x, fmaf(r2.y, y, fmaf(r2.z, z, r2.w)));
        const float g = grid_lookup(G, n, go, gh, lx, ly, lz);
        if (isnan(g)) continue;
        atomicMin(&R[i + (long long)E.nx * (j + (long long)E.ny * k)], ordered_bits(g));
    }
}

// One CTA per configuration: the minimum of its Robot SDF over the occupied voxels,
// with the voxel attaining it (smallest index on ties).
__global__ void __launch_bounds__(256) rs_gather_kernel(const unsigned* __restrict__ robot_sdf, long long nv,
                                                        const int* __restrict__ list, const int* __restrict__ count,
                                                        float* __restrict__ dist, int32_t* __restrict__ arg_voxel) {
    __shared__ unsigned long long s_min[8];
    const int w = blockIdx.x;
    const int n = *count;
    const unsigned* R = robot_sdf + (size_t)w * nv;
    unsigned long long best = ~0ull;
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        const int v = list[t];
        const unsigned u = R[v];
        if (u == kUnset) continue;
        const unsigned long long key = ((unsigned long long)u << 32) | (unsigned)v;
        best = key < best ? key : best;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long other = __shfl_xor_sync(0xffffffffu, best, o);
        best = other < best ? other : best;
    }
    if ((threadIdx.x & 31) == 0) s_min[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) best = s_min[k] < best ? s_min[k] : best;
        best = s_min[0] < best ? s_min[0] : best;
        if (best == ~0ull) {
            dist[w] = __int_as_float(0x7f800000);
            arg_voxel[w] = -1;
        } else {
            dist[w] = from_ordered((unsigned)(best >> 32));
            arg_voxel[w] = (int32_t)(best & 0xffffffffu);
        }
    }
}

}  // namespace
}  // namespace sdf

namespace {

int rfail(sdf_ctx* ctx, int code, const std::string& msg) {
    if (ctx) ctx->err = msg;
    return code;
}

struct DevGuard {
    int prev = -1;
    explicit DevGuard(int d) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != d) cudaSetDevice(d);
    }
    ~DevGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

template <typename T>
cudaError_t grow_buf(cudaStream_t st, T** buf, size_t* cap, size_t need) {
    if (need <= *cap) return cudaSuccess;
    cudaStreamSynchronize(st);
    sdf::dfree(*buf);
    *buf = nullptr;
    *cap = 0;
    const cudaError_t e = sdf::dmalloc(buf, need * sizeof(T));
    if (e == cudaSuccess) *cap = need;
    return e;
}

}  // namespace

extern "C" int check_trajectory_robot_sdf(sdf_ctx* ctx, const sdf_robot* R, const sdf_env_grid* env,
                                          const float* q_dev, int32_t W, const float* points_dev, int32_t N,
                                          float* dist_dev, int32_t* argmin_voxel_dev) {
    if (!ctx || !R || !env) return rfail(ctx, SDF_ERR_INVALID_ARG, "check_trajectory_robot_sdf: null");
    if (W < 0 || N < 0 || N > SDF_MAX_POINTS || !(env->voxel > 0.f) || env->dims[0] < 1 || env->dims[1] < 1 ||
        env->dims[2] < 1 || !(env->reach >= 0.f) || !std::isfinite(env->origin[0]) ||
        !std::isfinite(env->origin[1]) || !std::isfinite(env->origin[2]))
        return rfail(ctx, SDF_ERR_INVALID_ARG, "check_trajectory_robot_sdf: invalid grid or sizes");
    const long long nv = (long long)env->dims[0] * env->dims[1] * env->dims[2];
    if (nv > (1ll << 31) - 1) return rfail(ctx, SDF_ERR_INVALID_ARG, "check_trajectory_robot_sdf: too many voxels");
    if (W == 0) return SDF_OK;
    if (!dist_dev || !argmin_voxel_dev || (R->dof > 0 && !q_dev) || (N > 0 && !points_dev))
        return rfail(ctx, SDF_ERR_INVALID_ARG, "check_trajectory_robot_sdf: null buffer");
    if (R->device != ctx->device) return rfail(ctx, SDF_ERR_INVALID_ARG, "check_trajectory_robot_sdf: other device");
    DevGuard guard(ctx->device);
    cudaStream_t st = ctx->stream;
    const int L = R->table.L;
    const size_t words = (size_t)((nv + 31) / 32);
    const size_t list_cap = (size_t)std::max<long long>(1, std::min<long long>(N, nv));
    cudaError_t e = grow_buf(st, &ctx->rs_sdf, &ctx->rs_sdf_cap, (size_t)W * nv);
    if (e == cudaSuccess) e = grow_buf(st, &ctx->rs_bits, &ctx->rs_bits_cap, words);
    if (e == cudaSuccess) e = grow_buf(st, &ctx->rs_list, &ctx->rs_list_cap, list_cap + 1);   // + the count
    if (e == cudaSuccess) e = grow_buf(st, &ctx->rs_poses, &ctx->rs_poses_cap, (size_t)W * L * 16);
    if (e != cudaSuccess)
        return rfail(ctx, e == cudaErrorMemoryAllocation ? SDF_ERR_OOM : SDF_ERR_CUDA,
                     std::string("check_trajectory_robot_sdf: workspace: ") + cudaGetErrorString(e));
    int* count = ctx->rs_list + list_cap;
    sdf::EnvArgs E;
    E.ox = env->origin[0];
    E.oy = env->origin[1];
    E.oz = env->origin[2];
    E.r = env->voxel;
    E.inv_r = (float)(1.0 / (double)env->voxel);
    E.nx = env->dims[0];
    E.ny = env->dims[1];
    E.nz = env->dims[2];
    E.nv = nv;
    E.reach = env->reach;
    e = cudaMemsetAsync(ctx->rs_sdf, 0xff, (size_t)W * nv * sizeof(unsigned), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->rs_bits, 0, words * sizeof(unsigned), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(count, 0, sizeof(int), st);
    if (e == cudaSuccess) e = sdf::launch_fk(R->table, q_dev, W, ctx->rs_poses, ctx->status, st);
    if (e == cudaSuccess && N > 0) {
        sdf::voxelize_kernel<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(points_dev, N, ctx->point_stride, E,
                                                                         ctx->rs_bits, ctx->rs_list, count);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        sdf::robot_sdf_kernel<<<(unsigned)(W * L), 256, 0, st>>>(ctx->rs_poses, L, R->d_table, E, ctx->rs_sdf);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        sdf::rs_gather_kernel<<<(unsigned)W, 256, 0, st>>>(ctx->rs_sdf, nv, ctx->rs_list, count, dist_dev,
                                                          argmin_voxel_dev);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess)
        return rfail(ctx, e == cudaErrorMemoryAllocation ? SDF_ERR_OOM : SDF_ERR_CUDA,
                     std::string("check_trajectory_robot_sdf: ") + cudaGetErrorString(e));
    return SDF_OK;
}
