// Runtime distance check for sm_103a: a spatial sort of the obstacle cloud, then
// one fused kernel for forward kinematics, culling, transform, lookup and the
// per-waypoint min.
//
// cloud_prep_kernel (one cluster of 8 CTAs x 1024 threads) orders the points in
// space: bounding box, 32^3-cell Morton key per point, counting sort of the keys
// in distributed shared memory, scatter into a float4 array (x, y, z, original
// index), then a bounding sphere per tile of 32 consecutive sorted points and per
// super-tile of 32 consecutive tiles.  Non-finite points are dropped from the
// sorted cloud (and flagged), so they can never be a minimum.
//
// check_kernel: one warp per (waypoint, link) pair; a block holds the pairs of TW
// waypoints.  Each warp, with no block-wide barrier after set-up:
//   1. forward kinematics (Sec. III-A "parallel forward kinematics"): lanes build
//      one DH joint transform each and a warp scan composes them; the warp keeps
//      its link's link-from-world transform and world bounding-sphere centre in
//      registers;
//   2. seed: evaluates the tile whose farthest point is nearest to its link's
//      sphere centre, which makes the waypoint's best value (shared by the
//      waypoint's warps through a shared-memory atomic) a tight upper bound;
//   3. walks super-tiles -> tiles -> points, lanes over the children, skipping
//      every sphere with ||c - c_link|| - r - R_link > best + slack (the analogue
//      of the paper's "grids in sphere", Sec. III-B).  Surviving points are
//      compacted into a per-warp queue and evaluated 32 at a time: transform into
//      the link frame (the per-point form of Sec. II-B / Fig. 2), trilinear lookup
//      in the FP32 link grid (the grid-sample interpolation of Sec. III-A),
//      distance to the grid box outside it;
//   4. reduction with min per waypoint (Sec. III-A): each value is packed with its
//      original point index and link into one 64-bit key whose unsigned order is
//      (distance, point, link); warp shuffles, a shared-memory atomicMin, and the
//      waypoint's last warp writes the decoded result.
// The tile and super-tile spheres reach shared memory by one TMA bulk copy that
// completes on an mbarrier (with a bounded wait).
//
// The culls are exact: a skipped pair's interpolated distance exceeds the best
// value already found by more than the FP32 rounding of the bound, so culled and
// unculled runs give bit-identical results.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace cg = cooperative_groups;

namespace sdf {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr unsigned kOrderedInf = 0xff800000u;   // ordered_bits(+inf): "no value yet"
constexpr int kPrepThreads = 1024;
constexpr int kPrepCtas = 8;                        // one portable-size cluster
constexpr int kBinsPerCta = kCells / kPrepCtas;
constexpr int kPrepCached = 4;                      // points per thread kept in registers

__device__ __forceinline__ unsigned ordered_bits(float f) {
    unsigned u = __float_as_uint(f + 0.0f);  // -0 -> +0
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float from_ordered(unsigned o) {
    return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o);
}

// Affine 3x4 composition C = X * Y (row-major, implicit last row 0 0 0 1).
__device__ __forceinline__ void affine_mul(const float* X, const float* Y, float* C) {
    float t[12];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
#pragma unroll
        for (int c = 0; c < 3; ++c)
            t[4 * r + c] = fmaf(X[4 * r + 0], Y[c], fmaf(X[4 * r + 1], Y[4 + c], X[4 * r + 2] * Y[8 + c]));
        t[4 * r + 3] = fmaf(X[4 * r + 0], Y[3], fmaf(X[4 * r + 1], Y[7], fmaf(X[4 * r + 2], Y[11], X[4 * r + 3])));
    }
#pragma unroll
    for (int k = 0; k < 12; ++k) C[k] = t[k];
}

// Warp-cooperative forward kinematics of one waypoint.  Lane j (< dof) ends with
// the world-from-link transform of link j+1 (base * A_1 ... A_{j+1}) in M.
__device__ __forceinline__ void fk_warp(const LinkTable& T, const float* qw, int lane, float* M) {
    // local joint transform Rz(theta) Tz(d) Tx(a) Rx(alpha), closed form
    if (lane < T.dof) {
        float s, c;
        sincosf(T.dh_th[lane] + qw[lane], &s, &c);
        const float ca = T.dh_ca[lane], sa = T.dh_sa[lane], a = T.dh_a[lane], d = T.dh_d[lane];
        M[0] = c;  M[1] = -s * ca; M[2] = s * sa;  M[3] = a * c;
        M[4] = s;  M[5] = c * ca;  M[6] = -c * sa; M[7] = a * s;
        M[8] = 0.f; M[9] = sa;     M[10] = ca;     M[11] = d;
    } else {
#pragma unroll
        for (int k = 0; k < 12; ++k) M[k] = (k == 0 || k == 5 || k == 10) ? 1.f : 0.f;
    }
    // inclusive scan: after the step with offset o, lane j holds A_{j-2o+1} ... A_j
#pragma unroll
    for (int o = 1; o < 16; o <<= 1) {
        float X[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) X[k] = __shfl_up_sync(kFull, M[k], o);
        if (lane >= o) affine_mul(X, M, M);
    }
    affine_mul(T.base, M, M);
}

// Write the link-from-world rows [R^T | -R^T t] and the world sphere centre.
__device__ __forceinline__ void store_link(const float* M, float4 sph_local, float4* xf_rows,
                                           float4* sph_out) {
    const float tx = M[3], ty = M[7], tz = M[11];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        // row r of R^T is column r of R
        const float a = M[r], b = M[4 + r], c = M[8 + r];
        xf_rows[r] = make_float4(a, b, c, -fmaf(a, tx, fmaf(b, ty, c * tz)));
    }
    const float cx = fmaf(M[0], sph_local.x, fmaf(M[1], sph_local.y, fmaf(M[2], sph_local.z, tx)));
    const float cy = fmaf(M[4], sph_local.x, fmaf(M[5], sph_local.y, fmaf(M[6], sph_local.z, ty)));
    const float cz = fmaf(M[8], sph_local.x, fmaf(M[9], sph_local.y, fmaf(M[10], sph_local.z, tz)));
    *sph_out = make_float4(cx, cy, cz, sph_local.w);
}

// FK of one waypoint by one warp into (xf, sph) arrays indexed by link.
__device__ __forceinline__ void fk_links(const LinkTable& T, const float* qw, int lane,
                                         float4 (*xf)[3], float4* sph) {
    float M[12];
    fk_warp(T, qw, lane, M);
    if (lane < T.dof) store_link(M, T.sph_local[lane + 1], xf[lane + 1], &sph[lane + 1]);
    if (lane == 0) store_link(T.base, T.sph_local[0], xf[0], &sph[0]);
}

// Interpolated link SDF at a link-frame point (trilinear inside the grid box,
// distance to the box + boundary value outside).  Branch-free: the point is
// clamped in index space and the clamp distance is added.
__device__ __forceinline__ float grid_lookup(const float* __restrict__ G, int n, float4 o_ih,
                                             float h, float px, float py, float pz) {
    const float top = (float)(n - 1);
    const float ux = (px - o_ih.x) * o_ih.w;
    const float uy = (py - o_ih.y) * o_ih.w;
    const float uz = (pz - o_ih.z) * o_ih.w;
    const float cx = fminf(fmaxf(ux, 0.f), top);
    const float cy = fminf(fmaxf(uy, 0.f), top);
    const float cz = fminf(fmaxf(uz, 0.f), top);
    const float ex = ux - cx, ey = uy - cy, ez = uz - cz;
    const float dout = h * sqrtf(fmaf(ex, ex, fmaf(ey, ey, ez * ez)));
    const int ix = min((int)cx, n - 2), iy = min((int)cy, n - 2), iz = min((int)cz, n - 2);
    const float fx = cx - (float)ix, fy = cy - (float)iy, fz = cz - (float)iz;
    const size_t nn = (size_t)n * n;
    const float* b = G + (size_t)ix + (size_t)n * iy + nn * iz;
    const float v000 = __ldg(b), v100 = __ldg(b + 1);
    const float v010 = __ldg(b + n), v110 = __ldg(b + n + 1);
    const float v001 = __ldg(b + nn), v101 = __ldg(b + nn + 1);
    const float v011 = __ldg(b + nn + n), v111 = __ldg(b + nn + n + 1);
    const float c00 = fmaf(fx, v100 - v000, v000), c10 = fmaf(fx, v110 - v010, v010);
    const float c01 = fmaf(fx, v101 - v001, v001), c11 = fmaf(fx, v111 - v011, v011);
    const float c0 = fmaf(fy, c10 - c00, c00), c1 = fmaf(fy, c11 - c01, c01);
    return dout + fmaf(fz, c1 - c0, c0);
}

__device__ __forceinline__ float3 load_point(const float* __restrict__ pts, int stride, int i) {
    if (stride == 4) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(pts) + i);
        return make_float3(v.x, v.y, v.z);
    }
    const float* p = pts + 3 * (size_t)i;
    return make_float3(__ldg(p), __ldg(p + 1), __ldg(p + 2));
}

__device__ __forceinline__ bool finite3(float3 p) {
    return isfinite(p.x) && isfinite(p.y) && isfinite(p.z);
}

__device__ __forceinline__ unsigned long long pack_key(float g, int point, int link) {
    return ((unsigned long long)ordered_bits(g) << 32) | ((unsigned)point << 4) | (unsigned)link;
}

__device__ __forceinline__ void write_result(const CheckParams& P, int w, unsigned long long key) {
    if (key == ~0ull) {
        P.dist[w] = __int_as_float(0x7f800000);
        P.arg_link[w] = -1;
        P.arg_point[w] = -1;
    } else {
        P.dist[w] = from_ordered((unsigned)(key >> 32));
        P.arg_link[w] = (int)(key & 15u);
        P.arg_point[w] = (int)((key & 0xffffffffu) >> 4);
    }
}

__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long other = __shfl_xor_sync(kFull, k, o);
        k = other < k ? other : k;
    }
    return k;
}

// (score, index) arg-min across the warp; ties go to the smaller index.
__device__ __forceinline__ int warp_argmin(float s, int idx) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float so = __shfl_xor_sync(kFull, s, o);
        const int io = __shfl_xor_sync(kFull, idx, o);
        if (so < s || (so == s && io < idx)) { s = so; idx = io; }
    }
    return idx;
}

// 5-bit spread for a 15-bit Morton key.
__device__ __forceinline__ unsigned spread5(unsigned v) {
    v &= 31u;
    v = (v | (v << 8)) & 0x0300Fu;
    v = (v | (v << 4)) & 0x030C3u;
    v = (v | (v << 2)) & 0x09249u;
    return v;
}

__device__ __forceinline__ unsigned cell_key(float3 p, float3 lo, float3 inv) {
    const int ix = min(max((int)((p.x - lo.x) * inv.x), 0), 31);
    const int iy = min(max((int)((p.y - lo.y) * inv.y), 0), 31);
    const int iz = min(max((int)((p.z - lo.z) * inv.z), 0), 31);
    return spread5((unsigned)ix) | (spread5((unsigned)iy) << 1) | (spread5((unsigned)iz) << 2);
}

template <typename Op>
__device__ __forceinline__ float block_reduce(float v, float* s_tmp, Op op) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = op(v, __shfl_xor_sync(kFull, v, o));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) s_tmp[warp] = v;
    __syncthreads();
    v = s_tmp[lane];   // kPrepThreads / 32 == 32 partials
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = op(v, __shfl_xor_sync(kFull, v, o));
    return v;
}

struct FMin { __device__ float operator()(float a, float b) const { return fminf(a, b); } };
struct FMax { __device__ float operator()(float a, float b) const { return fmaxf(a, b); } };

// Spatial sort of the cloud by one thread-block cluster: the 32^3 cell counters
// are spread over the CTAs' shared memory (distributed shared memory), so every
// phase is one pass over the points with cluster barriers in between.  Up to
// kPrepCached points per thread stay in registers between the passes.
__global__ void __cluster_dims__(kPrepCtas, 1, 1) __launch_bounds__(kPrepThreads, 1)
    cloud_prep_kernel(const __grid_constant__ PrepParams P) {
    cg::cluster_group cluster = cg::this_cluster();
    const unsigned rank = cluster.block_rank();
    __shared__ unsigned s_bins[kBinsPerCta];     // counters, then cursors, of this CTA's cells
    __shared__ float s_tmp[32];
    __shared__ float s_box[6];
    __shared__ unsigned s_tot[32];
    __shared__ unsigned s_cta_total;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int gtid = (int)rank * kPrepThreads + tid;
    constexpr int kStride = kPrepCtas * kPrepThreads;
    const float kInf = __int_as_float(0x7f800000);
    const bool cached = P.N <= kStride * kPrepCached;

    float3 pc[kPrepCached];
#pragma unroll
    for (int k = 0; k < kPrepCached; ++k) {
        const int i = gtid + k * kStride;
        pc[k] = (cached && i < P.N) ? load_point(P.points, P.stride, i) : make_float3(0.f, 0.f, 0.f);
    }
    auto point_at = [&](int k, int i) -> float3 { return cached ? pc[k] : load_point(P.points, P.stride, i); };
    // visits every point index of this thread: f(point, index)
    auto for_each_point = [&](auto&& f) {
        if (cached) {
#pragma unroll
            for (int k = 0; k < kPrepCached; ++k) {
                const int i = gtid + k * kStride;
                if (i < P.N) f(point_at(k, i), i);
            }
        } else {
            for (int i = gtid; i < P.N; i += kStride) f(load_point(P.points, P.stride, i), i);
        }
    };

    // 1. bounding box of the finite points (per CTA, then across the cluster)
    float lo[3] = {kInf, kInf, kInf}, hi[3] = {-kInf, -kInf, -kInf};
    bool bad = false;
    for_each_point([&](float3 p, int) {
        if (finite3(p)) {
            lo[0] = fminf(lo[0], p.x); lo[1] = fminf(lo[1], p.y); lo[2] = fminf(lo[2], p.z);
            hi[0] = fmaxf(hi[0], p.x); hi[1] = fmaxf(hi[1], p.y); hi[2] = fmaxf(hi[2], p.z);
        } else {
            bad = true;
        }
    });
    if (__syncthreads_or(bad) && tid == 0) atomicOr(P.status, kStatusNonFinite);
    const float r0 = block_reduce(lo[0], s_tmp, FMin()), r1 = block_reduce(lo[1], s_tmp, FMin());
    const float r2 = block_reduce(lo[2], s_tmp, FMin()), r3 = block_reduce(hi[0], s_tmp, FMax());
    const float r4 = block_reduce(hi[1], s_tmp, FMax()), r5 = block_reduce(hi[2], s_tmp, FMax());
    if (tid == 0) {
        s_box[0] = r0; s_box[1] = r1; s_box[2] = r2; s_box[3] = r3; s_box[4] = r4; s_box[5] = r5;
    }
    for (int b = tid; b < kBinsPerCta; b += kPrepThreads) s_bins[b] = 0u;
    cluster.sync();
    float3 blo = make_float3(kInf, kInf, kInf), bhi = make_float3(-kInf, -kInf, -kInf);
#pragma unroll
    for (int r = 0; r < kPrepCtas; ++r) {
        const float* b = cluster.map_shared_rank(s_box, r);
        blo.x = fminf(blo.x, b[0]); blo.y = fminf(blo.y, b[1]); blo.z = fminf(blo.z, b[2]);
        bhi.x = fmaxf(bhi.x, b[3]); bhi.y = fmaxf(bhi.y, b[4]); bhi.z = fmaxf(bhi.z, b[5]);
    }
    const float3 inv = make_float3(32.f / fmaxf(bhi.x - blo.x, 1e-6f), 32.f / fmaxf(bhi.y - blo.y, 1e-6f),
                                   32.f / fmaxf(bhi.z - blo.z, 1e-6f));

    // 2. histogram: cell c is counted in CTA c / kBinsPerCta
    for_each_point([&](float3 p, int) {
        if (finite3(p)) {
            const unsigned c = cell_key(p, blo, inv);
            atomicAdd(cluster.map_shared_rank(&s_bins[c % kBinsPerCta], (int)(c / kBinsPerCta)), 1u);
        }
    });
    cluster.sync();

    // 3. exclusive scan of this CTA's cells (warp w owns a contiguous run), then
    //    the CTA totals of lower ranks give the CTA's global offset
    constexpr int kPerWarp = kBinsPerCta / (kPrepThreads / 32);
    unsigned running = 0;
    for (int k = 0; k < kPerWarp; k += 32) {
        const int idx = warp * kPerWarp + k + lane;
        const unsigned c = s_bins[idx];
        unsigned incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned v = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += v;
        }
        s_bins[idx] = running + incl - c;
        running += __shfl_sync(kFull, incl, 31);
    }
    if (lane == 0) s_tot[warp] = running;
    __syncthreads();
    if (warp == 0) {
        const unsigned t = s_tot[lane];
        unsigned ti = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned v = __shfl_up_sync(kFull, ti, o);
            if (lane >= o) ti += v;
        }
        s_tot[lane] = ti - t;
        if (lane == 31) s_cta_total = ti;
    }
    cluster.sync();
    unsigned prefix = 0, total = 0;
#pragma unroll
    for (int r = 0; r < kPrepCtas; ++r) {
        const unsigned t = *cluster.map_shared_rank(&s_cta_total, r);
        prefix += (r < (int)rank) ? t : 0u;
        total += t;
    }
    const unsigned off = prefix + s_tot[warp];
    for (int k = 0; k < kPerWarp; k += 32) s_bins[warp * kPerWarp + k + lane] += off;
    const int n_valid = (int)total;
    cluster.sync();

    // 4. scatter (order inside a cell is arbitrary; keys carry the original index)
    for_each_point([&](float3 p, int i) {
        if (finite3(p)) {
            const unsigned c = cell_key(p, blo, inv);
            const unsigned pos = atomicAdd(cluster.map_shared_rank(&s_bins[c % kBinsPerCta], (int)(c / kBinsPerCta)), 1u);
            P.sorted[pos] = make_float4(p.x, p.y, p.z, __int_as_float(i));
        }
    });
    // the cluster barrier orders these writes before the reads below (cluster scope)
    cluster.sync();

    // 5. tile spheres: centre of the tile's box, radius to its farthest point
    const int n_tiles = (n_valid + 31) >> 5;
    constexpr int kClusterWarps = kPrepCtas * (kPrepThreads / 32);
    for (int t = (int)rank * (kPrepThreads / 32) + warp; t < n_tiles; t += kClusterWarps) {
        const int i = t * 32 + lane;
        const bool v = i < n_valid;
        const float4 p = v ? __ldcg(&P.sorted[i]) : make_float4(0.f, 0.f, 0.f, 0.f);
        float mn[3] = {v ? p.x : kInf, v ? p.y : kInf, v ? p.z : kInf};
        float mx[3] = {v ? p.x : -kInf, v ? p.y : -kInf, v ? p.z : -kInf};
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                mn[a] = fminf(mn[a], __shfl_xor_sync(kFull, mn[a], o));
                mx[a] = fmaxf(mx[a], __shfl_xor_sync(kFull, mx[a], o));
            }
        const float cx = 0.5f * (mn[0] + mx[0]), cy = 0.5f * (mn[1] + mx[1]), cz = 0.5f * (mn[2] + mx[2]);
        float r2 = v ? (p.x - cx) * (p.x - cx) + (p.y - cy) * (p.y - cy) + (p.z - cz) * (p.z - cz) : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r2 = fmaxf(r2, __shfl_xor_sync(kFull, r2, o));
        if (lane == 0) P.tiles[t] = make_float4(cx, cy, cz, sqrtf(r2) * (1.f + 1e-6f) + 1e-7f);
    }
    cluster.sync();

    // 6. super-tile spheres over 32 consecutive tiles: box of the tile spheres,
    //    radius to the farthest tile sphere
    const int n_super = (n_tiles + 31) >> 5;
    for (int s = (int)rank * (kPrepThreads / 32) + warp; s < n_super; s += kClusterWarps) {
        const int t = s * 32 + lane;
        const bool v = t < n_tiles;
        const float4 c = v ? __ldcg(&P.tiles[t]) : make_float4(0.f, 0.f, 0.f, 0.f);
        float mn[3] = {v ? c.x - c.w : kInf, v ? c.y - c.w : kInf, v ? c.z - c.w : kInf};
        float mx[3] = {v ? c.x + c.w : -kInf, v ? c.y + c.w : -kInf, v ? c.z + c.w : -kInf};
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                mn[a] = fminf(mn[a], __shfl_xor_sync(kFull, mn[a], o));
                mx[a] = fmaxf(mx[a], __shfl_xor_sync(kFull, mx[a], o));
            }
        const float cx = 0.5f * (mn[0] + mx[0]), cy = 0.5f * (mn[1] + mx[1]), cz = 0.5f * (mn[2] + mx[2]);
        float r = v ? sqrtf((c.x - cx) * (c.x - cx) + (c.y - cy) * (c.y - cy) + (c.z - cz) * (c.z - cz)) + c.w : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r = fmaxf(r, __shfl_xor_sync(kFull, r, o));
        if (lane == 0) P.supers[s] = make_float4(cx, cy, cz, r * (1.f + 1e-6f) + 1e-7f);
    }
    if (rank == 0 && tid == 0) *P.n_valid = n_valid;
}

// ---- TMA bulk copy (global -> shared) completing on an mbarrier ----------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: gives up after kMaxWaitPolls polls (each poll may itself block
// for a short, hardware-defined time) instead of spinning forever.
constexpr int kMaxWaitPolls = 1 << 22;
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity) {
    for (int i = 0; i < kMaxWaitPolls; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// The link-from-world rows and world sphere of link l for waypoint w, computed by
// the whole warp (every lane ends with the same values).
__device__ __forceinline__ void warp_link_pose(const LinkTable& T, const float* qw, int lane, int l,
                                               float4* rows, float4* sph) {
    float M[12];
    fk_warp(T, qw, lane, M);
    const int src = l > 0 ? l - 1 : 0;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        const float v = __shfl_sync(kFull, M[k], src);
        M[k] = l > 0 ? v : T.base[k];
    }
    store_link(M, T.sph_local[l], rows, sph);
}

// One warp per (waypoint, link) pair; blockDim.x = 32 * TW * L.
__global__ void __launch_bounds__(1024, 1) check_kernel(const __grid_constant__ CheckParams P) {
    extern __shared__ float4 s_spheres[];        // tiles, then super-tiles (one bulk copy)
    __shared__ unsigned s_best[kMaxWaypointsPerBlock];
    __shared__ unsigned long long s_key[kMaxWaypointsPerBlock];
    __shared__ unsigned s_done[kMaxWaypointsPerBlock];
    __shared__ unsigned s_queue[32][64];
    __shared__ __align__(8) uint64_t s_mbar;

    const LinkTable& T = P.T;
    const int L = T.L;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int tw = P.tw;
    const int wl = warp / L, l = warp - wl * L;
    const int w = blockIdx.x * tw + wl;
    const int nw = min(tw, P.W - (int)blockIdx.x * tw);
    const int n_valid = *P.n_valid;
    const int n_tiles = (n_valid + 31) >> 5;
    const int n_super = (n_tiles + 31) >> 5;
    const bool staged = P.stage && n_tiles > 0;

    // 0. one thread starts the copy of all tile and super-tile spheres
    if (staged && threadIdx.x == 0) {
        mbar_init(&s_mbar, 1);
        const unsigned tb = (unsigned)n_tiles * (unsigned)sizeof(float4);
        const unsigned sb = (unsigned)n_super * (unsigned)sizeof(float4);
        mbar_expect_tx(&s_mbar, tb + sb);
        bulk_copy_g2s(s_spheres, P.tiles, tb, &s_mbar);
        bulk_copy_g2s(s_spheres + P.max_tiles, P.supers, sb, &s_mbar);
    }
    if (threadIdx.x < kMaxWaypointsPerBlock) {
        s_best[threadIdx.x] = kOrderedInf;
        s_key[threadIdx.x] = ~0ull;
        s_done[threadIdx.x] = 0u;
    }
    __syncthreads();   // the only block-wide barrier
    if (wl >= nw) return;

    // 1. forward kinematics; this warp keeps link l's pose in registers
    const float* qw = P.q + (size_t)w * T.dof;
    if (l == 0 && lane < T.dof && !isfinite(qw[lane])) atomicOr(P.status, kStatusNonFinite);
    float4 rows[3], sph;
    warp_link_pose(T, qw, lane, l, rows, &sph);
    const float* G = T.values + (size_t)l * T.n * T.n * T.n;
    const float4 g_o = T.grid_o[l];
    const float g_h = T.grid_h[l];

    if (staged && !mbar_wait_bounded(&s_mbar, 0)) {
        // the copy did not complete in time: report, then leave this warp (the block
        // stays resident until every warp has waited the same bounded time)
        if (lane == 0) atomicOr(P.status, kStatusTimeout);
        return;
    }
    const float4* tiles = staged ? s_spheres : P.tiles;
    const float4* supers = staged ? s_spheres + P.max_tiles : P.supers;

    unsigned long long lk = ~0ull;
    auto evaluate = [&](int pos) {
        const float4 p = __ldg(&P.sorted[pos]);
        const float lx = fmaf(rows[0].x, p.x, fmaf(rows[0].y, p.y, fmaf(rows[0].z, p.z, rows[0].w)));
        const float ly = fmaf(rows[1].x, p.x, fmaf(rows[1].y, p.y, fmaf(rows[1].z, p.z, rows[1].w)));
        const float lz = fmaf(rows[2].x, p.x, fmaf(rows[2].y, p.y, fmaf(rows[2].z, p.z, rows[2].w)));
        const float g = grid_lookup(G, T.n, g_o, g_h, lx, ly, lz);
        const unsigned long long key = pack_key(g, __float_as_int(p.w), l);
        if (key < lk) lk = key;
        const unsigned ob = (unsigned)(key >> 32);
        if (ob < s_best[wl]) atomicMin(&s_best[wl], ob);
    };
    const float kInf = __int_as_float(0x7f800000);
    auto threshold = [&]() -> float {   // best + R + slack: a distance from the sphere centre
        if (!P.cull) return kInf;
        const float t = from_ordered(s_best[wl]) + sph.w + kCullSlack;
        return (t == t) ? t : kInf;
    };
    auto reach = [&](float4 c, float thr) -> bool {   // sphere c may hold a pair below the bound
        const float dx = c.x - sph.x, dy = c.y - sph.y, dz = c.z - sph.z;
        const float base = thr + c.w;
        return base >= 0.f && fmaf(dx, dx, fmaf(dy, dy, dz * dz)) <= base * base;
    };

    // 2. seed: nearest super-tile, nearest tile in it, all its points
    if (P.cull && n_tiles > 0) {
        float bs = kInf;
        int bi = 0x7fffffff;
        for (int s0 = 0; s0 < n_super; s0 += 32) {
            const int s = s0 + lane;
            if (s < n_super) {
                const float4 c = supers[s];
                const float dx = c.x - sph.x, dy = c.y - sph.y, dz = c.z - sph.z;
                const float sc = sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz))) + c.w;
                if (sc < bs) { bs = sc; bi = s; }
            }
        }
        const int s_seed = warp_argmin(bs, bi);   // n_super..INT_MAX when every score is NaN
        if (s_seed < n_super) {
            const int t = s_seed * 32 + lane;
            float ts = kInf;
            if (t < n_tiles) {
                const float4 c = tiles[t];
                const float dx = c.x - sph.x, dy = c.y - sph.y, dz = c.z - sph.z;
                ts = sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz))) + c.w;
            }
            const int t_seed = warp_argmin(ts, t < n_tiles ? t : 0x7fffffff);
            if (t_seed < n_tiles && t_seed * 32 + lane < n_valid) evaluate(t_seed * 32 + lane);
        }
    }

    // 3. hierarchical sweep with survivor compaction
    unsigned* q = s_queue[warp];
    int qn = 0;
    const unsigned lt_mask = (1u << lane) - 1u;
    auto push_points = [&](const float4 (&pk)[kTileBatch], const int (&tk)[kTileBatch], int cnt, float thr) {
#pragma unroll
        for (int k = 0; k < kTileBatch; ++k) {
            if (k >= cnt) break;
            const int pos = tk[k] * 32 + lane;
            const float dx = pk[k].x - sph.x, dy = pk[k].y - sph.y, dz = pk[k].z - sph.z;
            const bool surv = pos < n_valid && thr >= 0.f && fmaf(dx, dx, fmaf(dy, dy, dz * dz)) <= thr * thr;
            const unsigned m = __ballot_sync(kFull, surv);
            if (m) {
                if (surv) q[qn + __popc(m & lt_mask)] = (unsigned)pos;
                qn += __popc(m);
                if (qn >= 32) {   // qn < 64: evaluate the top 32 entries with all lanes
                    __syncwarp();
                    const unsigned ent = q[qn - 32 + lane];
                    __syncwarp();
                    qn -= 32;
                    evaluate((int)ent);
                }
            }
        }
    };
    for (int s0 = 0; s0 < n_super; s0 += 32) {
        float thr = threshold();
        const int s = s0 + lane;
        unsigned ms = __ballot_sync(kFull, s < n_super && reach(supers[min(s, n_super - 1)], thr));
        while (ms) {
            const int sidx = s0 + __ffs(ms) - 1;
            ms &= ms - 1;
            thr = threshold();
            const int t = sidx * 32 + lane;
            unsigned mt = __ballot_sync(kFull, t < n_tiles && reach(tiles[min(t, n_tiles - 1)], thr));
            while (mt) {
                // up to kTileBatch surviving tiles: issue their point loads together
                int tk[kTileBatch];
                float4 pk[kTileBatch];
                int cnt = 0;
#pragma unroll
                for (int k = 0; k < kTileBatch; ++k) {
                    tk[k] = 0;
                    if (mt) {
                        tk[k] = sidx * 32 + __ffs(mt) - 1;
                        mt &= mt - 1;
                        cnt = k + 1;
                    }
                }
#pragma unroll
                for (int k = 0; k < kTileBatch; ++k) {
                    const int pos = tk[k] * 32 + lane;
                    pk[k] = (k < cnt && pos < n_valid) ? __ldg(&P.sorted[pos]) : make_float4(0.f, 0.f, 0.f, 0.f);
                }
                push_points(pk, tk, cnt, threshold());
            }
        }
    }
    __syncwarp();
    if (lane < qn) evaluate((int)q[lane]);

    // 4. reduce: warp min, shared atomicMin, last warp of the waypoint writes
    lk = warp_min_u64(lk);
    if (lane == 0) {
        if (lk != ~0ull) atomicMin(&s_key[wl], lk);
        __threadfence_block();
        if (atomicAdd(&s_done[wl], 1u) == (unsigned)L - 1u) {
            __threadfence_block();
            write_result(P, w, atomicAdd(&s_key[wl], 0ull));
        }
    }
}

__global__ void __launch_bounds__(128) fk_kernel(const __grid_constant__ LinkTable T,
                                                 const float* __restrict__ q, int W,
                                                 float* __restrict__ out, int* status) {
    __shared__ float4 s_xf[4][kMaxLinks][3];
    __shared__ float4 s_sph[4][kMaxLinks];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int w = blockIdx.x * 4 + warp;
    if (w >= W) return;   // whole warp leaves together
    const float* qw = q + (size_t)w * T.dof;
    if (lane < T.dof && !isfinite(qw[lane])) atomicOr(status, kStatusNonFinite);
    fk_links(T, qw, lane, s_xf[warp], s_sph[warp]);
    __syncwarp();
    for (int l = lane; l < T.L; l += 32) {
        float4* o = reinterpret_cast<float4*>(out + ((size_t)w * T.L + l) * 16);
        o[0] = s_xf[warp][l][0];
        o[1] = s_xf[warp][l][1];
        o[2] = s_xf[warp][l][2];
        o[3] = s_sph[warp][l];
    }
}

}  // namespace

cudaError_t launch_prep(const PrepParams& p, cudaStream_t s) {
    cloud_prep_kernel<<<kPrepCtas, kPrepThreads, 0, s>>>(p);
    return cudaGetLastError();
}

size_t staged_bytes(int max_tiles) {
    return (size_t)(max_tiles + (max_tiles + 31) / 32) * sizeof(float4);
}

cudaError_t configure_kernels() {
    return cudaFuncSetAttribute(check_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)staged_bytes(kMaxStagedTiles));
}

cudaError_t launch_check(const CheckParams& p, cudaStream_t s) {
    const dim3 block((unsigned)(32 * p.tw * p.T.L));
    const dim3 grid((unsigned)((p.W + p.tw - 1) / p.tw));
    const size_t smem = p.stage ? staged_bytes(p.max_tiles) : 0;
    check_kernel<<<grid, block, smem, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_fk(const LinkTable& T, const float* q, int W, float* out, int* status,
                      cudaStream_t s) {
    fk_kernel<<<(unsigned)((W + 3) / 4), 128, 0, s>>>(T, q, W, out, status);
    return cudaGetLastError();
}

}  // namespace sdf
