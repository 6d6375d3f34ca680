// Runtime distance check for sm_103a, for one trajectory or a batch of them.
// Two kernels per launch:
//
// prep_kernel -- one thread-block cluster (16 CTAs x 1024 threads where the device
//   allows that non-portable size, else 8) per cloud sorts
//   its obstacle points in space: bounding box (shared through distributed shared
//   memory), 16^3-cell Morton key, a counting sort whose partial histograms are
//   merged slice by slice through distributed shared memory, each CTA scattering
//   its own points into float4 (x, y, z, original index); then a bounding sphere
//   per tile of 32 sorted points and per super-tile of 32 tiles.  Non-finite
//   points are dropped (and flagged).
// check_kernel -- one block per (trajectory, group of waypoints), started while
//   the sort runs (programmatic dependent launch).  Before it waits for the sort,
//   the block runs forward kinematics (Sec. III-A "parallel forward kinematics":
//   lanes build the DH joint transforms and a warp scan composes them; each pair's
//   link-from-world transform and world bounding capsule go to shared memory) and
//   prefetches its share of the robot's grids into L2.  A block of two waypoints
//   takes two from distant parts of the trajectory when the launch is one wave.
//   The trajectory's tile and super-tile spheres then reach shared memory by one
//   TMA bulk copy that completes on an mbarrier (bounded wait).
//   Phase A, one warp per (waypoint, link) pair:
//   * seed: the tile nearest to the link's capsule is evaluated in full, which
//     makes the waypoint's best value (a shared-memory atomic shared by the
//     waypoint's warps) a tight upper bound early;
//   * culls super-tiles, then tiles, against the capsule with best + slack (the
//     analogue of the paper's "grids in sphere", Sec. III-B); every surviving
//     (pair, tile) sets the pair's bit in the tile's mask in shared memory (when the
//     tile spheres are staged; otherwise it goes to a block-wide list of (pair, tile)
//     entries).
//   Phase B, all warps of the block: the tiles with a mask are compacted into the
//   block list and taken a few at a time (loads issued together); a tile's points
//   are loaded once and tested against the capsule of every pair in its mask (or,
//   with the flat list, against the entry's pair); survivors are compacted into a
//   per-warp queue and evaluated 32 at a
//   time: transform into the link frame (the per-point form of Sec. II-B / Fig.
//   2), trilinear lookup in the FP32 link grid (the grid-sample interpolation of
//   Sec. III-A), distance to the grid box outside it.  Each value is folded into
//   the waypoint's minimum (Sec. III-A) as a 64-bit key whose unsigned order is
//   (distance, point, link), so atomicMin gives a deterministic arg-min.
//
// The culls are exact: a skipped pair's interpolated distance exceeds a value
// already found by more than the FP32 rounding of the bound, so culled and
// unculled runs give bit-identical results.
#include <atomic>
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"
#include "lookup.cuh"

namespace cg = cooperative_groups;

namespace sdf {
namespace {

using namespace dev;

constexpr unsigned kFull = 0xffffffffu;
constexpr unsigned kOrderedInf = 0xff800000u;   // ordered_bits(+inf): "no value yet"
constexpr int kCellsPerAxis = 16;
constexpr int kCells = kCellsPerAxis * kCellsPerAxis * kCellsPerAxis;   // Morton cells of the cloud sort
constexpr int kPrepThreads = 1024;
constexpr int kPrepCtas = 8;                        // the portable cluster size (16 where allowed)
constexpr int kPrepChunk = 4;                       // points a thread loads before using them

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
    const int ix = min(max((int)((p.x - lo.x) * inv.x), 0), kCellsPerAxis - 1);
    const int iy = min(max((int)((p.y - lo.y) * inv.y), 0), kCellsPerAxis - 1);
    const int iz = min(max((int)((p.z - lo.z) * inv.z), 0), kCellsPerAxis - 1);
    return spread5((unsigned)ix) | (spread5((unsigned)iy) << 1) | (spread5((unsigned)iz) << 2);
}



// ------------------------------------------------------------------ prep kernel

// Warp-wide minimum / maximum of a float in one redux.sync on its order-preserving
// unsigned encoding (exact; -0 and +0 compare equal).
__device__ __forceinline__ float warp_min(float x) {
    return from_ordered(__reduce_min_sync(kFull, ordered_bits(x)));
}
__device__ __forceinline__ float warp_max(float x) {
    return from_ordered(__reduce_max_sync(kFull, ordered_bits(x)));
}
// ... of a float known to be >= 0 (its bits already order as unsigned)
__device__ __forceinline__ float warp_max_nonneg(float x) {
    return __uint_as_float(__reduce_max_sync(kFull, __float_as_uint(x)));
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// One cluster of CT CTAs (8, or 16 where the device allows that non-portable size) per
// cloud sorts it by 16^3-cell Morton key, a
// counting sort without remote atomics: each CTA histograms its share of the points
// in its own shared memory; every CTA then reads the CT partial histograms
// through distributed shared memory, which gives each cell's start and this CTA's
// first slot in it; each CTA scatters its own points with local atomics.
template <int CT>
__global__ void __launch_bounds__(kPrepThreads, 1) prep_kernel(const __grid_constant__ BatchParams P) {
    cg::cluster_group cluster = cg::this_cluster();
    const unsigned rank = cluster.block_rank();
    const int cidx = blockIdx.x / CT;
    const CloudDesc& C = P.cloud[cidx];
    // the check grid may start now: its set-up reads nothing this kernel writes
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    // this CTA's histogram of its share of the points, then its scatter cursors
    __shared__ __align__(16) unsigned bins[kCells];
    __shared__ float s_box6[32][6];
    __shared__ __align__(16) float s_box[8];
    __shared__ float s_gbox[6];
    __shared__ unsigned s_warp_total[32];
    __shared__ unsigned s_cloud_total, s_slice_off;
    __shared__ __align__(16) unsigned s_slice_cnt[CT];   // this CTA's points in each slice
    __shared__ unsigned s_cnt[CT][kCells / CT];   // the slice's counts, by rank
    __shared__ float4 s_tile[4][32];                             // tile spheres of four super-tiles
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int gtid = (int)rank * kPrepThreads + tid;
    constexpr int kStride = CT * kPrepThreads;
    const float kInf = __int_as_float(0x7f800000);
    const int N = C.N;
    const float* pts = C.points;
    // phase timestamps of the first CTA (SDF_OPT_STATS)
    const bool clock = P.stats != nullptr && rank == 0 && tid == 0;
    unsigned long long t_mark = clock ? global_ns() : 0ull;
    auto mark = [&](int slot) {
        if (clock) {
            const unsigned long long t = global_ns();
            atomicAdd(&P.stats[slot], t - t_mark);
            t_mark = t;
        }
    };

    // 1. bounding box of the finite points: this CTA's share, then across the cluster.
    //    A share of at most kPrepChunk points a thread is loaded once and kept in
    //    registers for the histogram and the scatter.
    float lo[3] = {kInf, kInf, kInf}, hi[3] = {-kInf, -kInf, -kInf};
    bool bad = false;
    const bool in_regs = N <= kStride * kPrepChunk;
    float3 pv[kPrepChunk];
    auto extend_box = [&](float3 p) {
        if (finite3(p)) {
            lo[0] = fminf(lo[0], p.x); lo[1] = fminf(lo[1], p.y); lo[2] = fminf(lo[2], p.z);
            hi[0] = fmaxf(hi[0], p.x); hi[1] = fmaxf(hi[1], p.y); hi[2] = fmaxf(hi[2], p.z);
        } else {
            bad = true;
        }
    };
    if (in_regs) {
#pragma unroll
        for (int k = 0; k < kPrepChunk; ++k) {   // all loads in flight before the first use
            const int i = gtid + k * kStride;
            pv[k] = i < N ? load_point(pts, P.stride, i) : make_float3(0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int k = 0; k < kPrepChunk; ++k)
            if (gtid + k * kStride < N) extend_box(pv[k]);
    } else {
        for (int i = gtid; i < N; i += kStride) extend_box(load_point(pts, P.stride, i));
    }
    // the six extremes at once: maxima as negated minima, warp then CTA
    float e6[6] = {lo[0], lo[1], lo[2], -hi[0], -hi[1], -hi[2]};
#pragma unroll
    for (int a = 0; a < 6; ++a) e6[a] = warp_min(e6[a]);
    if (lane == 0)
#pragma unroll
        for (int a = 0; a < 6; ++a) s_box6[warp][a] = e6[a];
    for (int b = tid; b < kCells; b += kPrepThreads) bins[b] = 0u;
    if (tid < CT) s_slice_cnt[tid] = 0u;
    if (__syncthreads_or(bad) && tid == 0) atomicOr(P.status, kStatusNonFinite);
    if (warp == 0) {
#pragma unroll
        for (int a = 0; a < 6; ++a) {
            const float v = warp_min(s_box6[lane][a]);   // kPrepThreads / 32 == 32 partials
            if (lane == 0) s_box[a] = a < 3 ? v : -v;
        }
    }
    cluster.sync();
    // lane r < CT of warp 0 reads rank r's box; the cluster's box goes to all
    // threads through this CTA's shared memory
    if (warp == 0) {
        float g[6] = {kInf, kInf, kInf, kInf, kInf, kInf};   // minima and negated maxima
        if (lane < CT) {
            const float4* b = reinterpret_cast<const float4*>(cluster.map_shared_rank(s_box, lane));
            const float4 b0 = b[0], b1 = b[1];
            g[0] = b0.x; g[1] = b0.y; g[2] = b0.z; g[3] = -b0.w; g[4] = -b1.x; g[5] = -b1.y;
        }
#pragma unroll
        for (int a = 0; a < 6; ++a) g[a] = warp_min(g[a]);
        if (lane == 0)
#pragma unroll
            for (int a = 0; a < 6; ++a) s_gbox[a] = a < 3 ? g[a] : -g[a];
    }
    __syncthreads();
    const float3 blo = make_float3(s_gbox[0], s_gbox[1], s_gbox[2]);
    const float3 bhi = make_float3(s_gbox[3], s_gbox[4], s_gbox[5]);
    constexpr float kAxis = (float)kCellsPerAxis;
    const float3 inv = make_float3(kAxis / fmaxf(bhi.x - blo.x, 1e-6f), kAxis / fmaxf(bhi.y - blo.y, 1e-6f),
                                   kAxis / fmaxf(bhi.z - blo.z, 1e-6f));
    mark(20);

    // 2. each CTA counts its own share of the points (shared-memory atomics); the
    //    share's cell keys stay in registers for the scatter
    unsigned kc[kPrepChunk];
    auto count_chunk = [&](int i0, bool load) {
        if (load) {
#pragma unroll
            for (int k = 0; k < kPrepChunk; ++k) {   // all loads of the chunk in flight before the first use
                const int i = i0 + k * kStride;
                pv[k] = i < N ? load_point(pts, P.stride, i) : make_float3(0.f, 0.f, 0.f);
            }
        }
#pragma unroll
        for (int k = 0; k < kPrepChunk; ++k) {
            const int i = i0 + k * kStride;
            kc[k] = 0xffffffffu;
            if (i < N && finite3(pv[k])) {
                kc[k] = cell_key(pv[k], blo, inv);
                atomicAdd(&bins[kc[k]], 1u);
            }
        }
    };
    if (in_regs) {
        count_chunk(gtid, false);   // the points loaded for the box
    } else {
        for (int i0 = gtid; i0 < N; i0 += kStride * kPrepChunk) count_chunk(i0, true);
    }
    // this CTA's count in each slice of kSlice cells: warp w sums cells 128 w .. 128 w + 127
    constexpr int kSlice = kCells / CT;
    static_assert(kCells == 4 * kPrepThreads && kSlice % 128 == 0, "four cells a thread, whole warps a slice");
    __syncthreads();
    {
        const uint4 c = reinterpret_cast<const uint4*>(bins)[tid];
        const unsigned sum = __reduce_add_sync(kFull, c.x + c.y + c.z + c.w);
        if (lane == 0 && sum) atomicAdd(&s_slice_cnt[(warp * 128) / kSlice], sum);
    }
    cluster.sync();
    mark(21);

    // 3. merge of the partial histograms, one slice of kSlice cells per CTA: CTA r
    //    reads the counts of its slice from every rank and scans the slice; warp 1
    //    reads every rank's slice totals, which give the lower slices' total; CTA r
    //    then writes into every rank's histogram that rank's first slot in each cell
    //    of the slice (the histogram becomes its cursors).  The cells of slice r are
    //    read and written by CTA r alone, so no barrier separates the reads from the
    //    writes.  Thread t serves cell t mod kSlice and ranks 4 (t / kSlice) + 0..3.
    static_assert(kSlice * (CT / 4) == kPrepThreads, "CT / 4 threads per slice cell, four ranks each");
    const int cl = tid & (kSlice - 1), half = tid / kSlice;   // half: the thread's group of four ranks
    const int cell = (int)rank * kSlice + cl;
    if (warp == 1) {
        unsigned below = 0, total = 0;
        if (lane < CT) {
            const uint4* c = reinterpret_cast<const uint4*>(cluster.map_shared_rank(s_slice_cnt, lane));
#pragma unroll
            for (int q = 0; q < CT / 4; ++q) {
                const uint4 cq = c[q];
                const unsigned v[4] = {cq.x, cq.y, cq.z, cq.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    total += v[e];
                    below += 4 * q + e < (int)rank ? v[e] : 0u;
                }
            }
        }
        below = __reduce_add_sync(kFull, below);
        total = __reduce_add_sync(kFull, total);
        if (lane == 0) {
            s_slice_off = below;
            s_cloud_total = total;
        }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) s_cnt[4 * half + k][cl] = cluster.map_shared_rank(bins, 4 * half + k)[cell];
    __syncthreads();
    unsigned total_c = 0;
#pragma unroll
    for (int r = 0; r < CT; ++r) total_c += s_cnt[r][cl];
    unsigned incl = total_c;   // inclusive scan over the slice's cells (threads 0 .. kSlice-1)
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned v = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31 && half == 0) s_warp_total[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        constexpr int kSliceWarps = kSlice / 32;
        const unsigned t = lane < kSliceWarps ? s_warp_total[lane] : 0u;
        unsigned ti = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned v = __shfl_up_sync(kFull, ti, o);
            if (lane >= o) ti += v;
        }
        s_warp_total[lane] = ti - t;
    }
    __syncthreads();
    {
        const unsigned start = s_slice_off + s_warp_total[warp % (kSlice / 32)] + incl - total_c;
        unsigned pre = 0;
        for (int r = 0; r < 4 * half; ++r) pre += s_cnt[r][cl];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int r = 4 * half + k;
            cluster.map_shared_rank(bins, r)[cell] = start + pre;
            pre += s_cnt[r][cl];
        }
    }
    const unsigned running = s_cloud_total;
    cluster.sync();   // every rank's cursors are written before any scatter
    const int n_valid = (int)running;
    mark(22);

    // 4. scatter this CTA's points (order inside a cell is arbitrary; the w
    //    component carries the original index)
    float4* sorted = P.sorted + C.point_base;
    if (in_regs) {
        unsigned pos[kPrepChunk];
#pragma unroll
        for (int k = 0; k < kPrepChunk; ++k) pos[k] = kc[k] != 0xffffffffu ? atomicAdd(&bins[kc[k]], 1u) : 0u;
#pragma unroll
        for (int k = 0; k < kPrepChunk; ++k)
            if (kc[k] != 0xffffffffu)
                sorted[pos[k]] = make_float4(pv[k].x, pv[k].y, pv[k].z, __int_as_float(gtid + k * kStride));
    } else {
        for (int i = gtid; i < N; i += kStride) {
            const float3 p = load_point(pts, P.stride, i);
            if (!finite3(p)) continue;
            const unsigned pos = atomicAdd(&bins[cell_key(p, blo, inv)], 1u);
            sorted[pos] = make_float4(p.x, p.y, p.z, __int_as_float(i));
        }
    }
    cluster.sync();   // orders every CTA's scatter before the reads below (cluster scope)
    mark(23);

    // 5. tile and super-tile spheres.  CTA r builds super-tiles r, r + CT, ...,
    //    kRounds of them at a time: warp w loads tile 32 s + w of each (all loads in
    //    flight before the first use) and computes its sphere (centre of the tile's
    //    box, radius to its farthest point); warp k then forms super-tile k of the
    //    group (box of the tile spheres, radius to the farthest one) from shared
    //    memory -- no cluster barrier needed
    const int n_tiles = (n_valid + 31) >> 5;
    const int n_super = (n_tiles + 31) >> 5;
    float4* tiles = P.tiles + C.tile_base;
    float4* supers = P.supers + C.super_base;
    static_assert(kPrepThreads / 32 == 32, "one warp per tile of a super-tile");
    constexpr int kRounds = 4;
    for (int s0 = (int)rank; s0 < n_super; s0 += kRounds * CT) {
        float4 p[kRounds];
        bool v[kRounds];
#pragma unroll
        for (int k = 0; k < kRounds; ++k) {
            const int t = (s0 + k * CT) * 32 + warp;
            v[k] = t * 32 + lane < n_valid;
            p[k] = v[k] ? __ldcg(&sorted[t * 32 + lane]) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int k = 0; k < kRounds; ++k) {
            const int t = (s0 + k * CT) * 32 + warp;
            if (t < n_tiles) {   // uniform across the warp
                const float mn[3] = {warp_min(v[k] ? p[k].x : kInf), warp_min(v[k] ? p[k].y : kInf),
                                     warp_min(v[k] ? p[k].z : kInf)};
                const float mx[3] = {warp_max(v[k] ? p[k].x : -kInf), warp_max(v[k] ? p[k].y : -kInf),
                                     warp_max(v[k] ? p[k].z : -kInf)};
                const float cx = 0.5f * (mn[0] + mx[0]), cy = 0.5f * (mn[1] + mx[1]), cz = 0.5f * (mn[2] + mx[2]);
                float r2 = v[k] ? (p[k].x - cx) * (p[k].x - cx) + (p[k].y - cy) * (p[k].y - cy) +
                                      (p[k].z - cz) * (p[k].z - cz)
                                : 0.f;
                r2 = warp_max_nonneg(r2);
                if (lane == 0) {
                    const float4 sph = make_float4(cx, cy, cz, sqrtf(r2) * (1.f + 1e-6f) + 1e-7f);
                    tiles[t] = sph;
                    s_tile[k][warp] = sph;
                }
            }
        }
        __syncthreads();
        const int s = s0 + warp * CT;
        if (warp < kRounds && s < n_super) {
            const bool vt = s * 32 + lane < n_tiles;
            const float4 c = vt ? s_tile[warp][lane] : make_float4(0.f, 0.f, 0.f, 0.f);
            const float mn[3] = {warp_min(vt ? c.x - c.w : kInf), warp_min(vt ? c.y - c.w : kInf),
                                 warp_min(vt ? c.z - c.w : kInf)};
            const float mx[3] = {warp_max(vt ? c.x + c.w : -kInf), warp_max(vt ? c.y + c.w : -kInf),
                                 warp_max(vt ? c.z + c.w : -kInf)};
            const float cx = 0.5f * (mn[0] + mx[0]), cy = 0.5f * (mn[1] + mx[1]), cz = 0.5f * (mn[2] + mx[2]);
            float r = vt ? sqrtf((c.x - cx) * (c.x - cx) + (c.y - cy) * (c.y - cy) + (c.z - cz) * (c.z - cz)) + c.w
                         : 0.f;
            r = warp_max_nonneg(r);
            if (lane == 0) supers[s] = make_float4(cx, cy, cz, r * (1.f + 1e-6f) + 1e-7f);
        }
        __syncthreads();   // s_tile is rewritten by the next group
    }
    mark(24);
    if (rank == 0 && tid == 0) P.n_valid[cidx] = n_valid;
    mark(25);
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
// Bounded wait: gives up after `limit` polls (each poll may itself block for a
// short, hardware-defined time) instead of spinning forever.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity, unsigned limit) {
    for (unsigned i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// L2 prefetch of a global range (bulk, no completion to wait for).  The start must
// be 16-byte aligned; the size is a multiple of 16.
__device__ __forceinline__ void prefetch_l2(const void* src, unsigned bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// ------------------------------------------------------------------ check kernel

// per-warp statistics rows (SDF_OPT_STATS), written by lane 0 of their warp
enum WarpStat { kWsSeed, kWsSuperT, kWsSuperP, kWsTileT, kWsTileP, kWsPointT, kWsLookups, kWsOver, kWsCount };
enum WarpNs { kWnSeed, kWnCull, kWnPoints, kWnCount };

constexpr unsigned kTileMask = (1u << 28) - 1u;     // tile index of a list entry

struct BlockState {
    const float4* sorted;      // this trajectory's sorted points
    const float* values;       // this robot's grids
    int n, n3, L, n_valid;
    float4 (*pose)[6];         // per pair: rows[3], sphere, capsule start (+radius), capsule axis (+1/len^2)
    const uchar2* pair_wl;     // per pair: (waypoint of the block, link), no division in the hot loops
    const float4* grid_o;      // per link (shared memory)
    const float* grid_h;
    unsigned* best;            // per waypoint of the block
    unsigned long long* key;
    int cull;
    unsigned* stat;            // this warp's statistics row, or null
};

__device__ __forceinline__ void stat_add(const BlockState& B, int idx, unsigned v, int lane) {
    if (B.stat && lane == 0) B.stat[idx] += v;
}

__device__ __forceinline__ float pair_threshold(const BlockState& B, int pair) {
    if (!B.cull) return __int_as_float(0x7f800000);
    const float t = from_ordered(B.best[B.pair_wl[pair].x]) + B.pose[pair][4].w + kCullSlack;
    return (t == t) ? t : __int_as_float(0x7f800000);
}

// Squared distance from (x, y, z) to the segment A + t D, t in [0, 1] (D.w = 1/|D|^2,
// 0 for a point).
__device__ __forceinline__ float seg_dist2(float x, float y, float z, float4 A, float4 D) {
    const float px = x - A.x, py = y - A.y, pz = z - A.z;
    const float t = fminf(fmaxf(fmaf(px, D.x, fmaf(py, D.y, pz * D.z)) * D.w, 0.f), 1.f);
    const float qx = fmaf(-t, D.x, px), qy = fmaf(-t, D.y, py), qz = fmaf(-t, D.z, pz);
    return fmaf(qx, qx, fmaf(qy, qy, qz * qz));
}

// Can a sphere c (centre, radius) hold a point within thr of the link's capsule
// surface?  thr already includes the capsule radius.
__device__ __forceinline__ bool capsule_reaches(float4 c, float4 A, float4 D, float thr) {
    const float base = thr + c.w;
    return base >= 0.f && seg_dist2(c.x, c.y, c.z, A, D) <= base * base;
}

// Interpolated distance of sorted point `pos` for block pair `pair`, folded into
// the waypoint's best value and key when it can still be the minimum.
__device__ __forceinline__ void evaluate(const BlockState& B, int pos, int pair) {
    const float4 p = __ldg(&B.sorted[pos]);
    const float4 r0 = B.pose[pair][0], r1 = B.pose[pair][1], r2 = B.pose[pair][2];
    const uchar2 pw = B.pair_wl[pair];
    const int wl = pw.x, l = pw.y;
    const float lx = fmaf(r0.x, p.x, fmaf(r0.y, p.y, fmaf(r0.z, p.z, r0.w)));
    const float ly = fmaf(r1.x, p.x, fmaf(r1.y, p.y, fmaf(r1.z, p.z, r1.w)));
    const float lz = fmaf(r2.x, p.x, fmaf(r2.y, p.y, fmaf(r2.z, p.z, r2.w)));
    const float g = grid_lookup(B.values + (size_t)(l * B.n3), B.n, B.grid_o[l], B.grid_h[l], lx, ly, lz);
    const unsigned long long key = pack_key(g, __float_as_int(p.w), l);
    const unsigned ob = (unsigned)(key >> 32);
    if (ob <= B.best[wl]) {
        atomicMin(&B.best[wl], ob);
        atomicMin(&B.key[wl], key);
    }
}

// The same through the texture unit's filter (SDF_OPT_TEX3D), called by the whole warp
// (lanes with `valid` false take part without a point).  A texture fetch is given a
// handle that is the same in every lane and comes from the kernel parameters: the
// warp fetches link by link, the link of the first pending lane each round (a
// handle that differs between lanes is not used).
__device__ __forceinline__ void evaluate_tex(const BatchParams& P, const BlockState& B, int pos, int pair,
                                             bool valid) {
    const float4 p = valid ? __ldg(&B.sorted[pos]) : make_float4(0.f, 0.f, 0.f, 0.f);
    const int pr = valid ? pair : 0;
    const float4 r0 = B.pose[pr][0], r1 = B.pose[pr][1], r2 = B.pose[pr][2];
    const uchar2 pw = B.pair_wl[pr];
    const int wl = pw.x, l = valid ? (int)pw.y : -1;
    const int ll = valid ? l : 0;
    const float lx = fmaf(r0.x, p.x, fmaf(r0.y, p.y, fmaf(r0.z, p.z, r0.w)));
    const float ly = fmaf(r1.x, p.x, fmaf(r1.y, p.y, fmaf(r1.z, p.z, r1.w)));
    const float lz = fmaf(r2.x, p.x, fmaf(r2.y, p.y, fmaf(r2.z, p.z, r2.w)));
    TexCoord c = tex_coord(B.n, B.grid_o[ll], B.grid_h[ll], lx, ly, lz);
    float v = 0.f;
    unsigned pending = __ballot_sync(kFull, valid);
    while (pending) {
        const int k = __shfl_sync(kFull, l, __ffs(pending) - 1);
        unsigned long long h = 0;
        switch (k) {
#define SDF_TEX_CASE(i) case i: h = P.tex_h[i]; break;
            SDF_TEX_CASE(0) SDF_TEX_CASE(1) SDF_TEX_CASE(2) SDF_TEX_CASE(3) SDF_TEX_CASE(4) SDF_TEX_CASE(5)
            SDF_TEX_CASE(6) SDF_TEX_CASE(7) SDF_TEX_CASE(8) SDF_TEX_CASE(9) SDF_TEX_CASE(10) SDF_TEX_CASE(11)
            SDF_TEX_CASE(12) SDF_TEX_CASE(13) SDF_TEX_CASE(14) SDF_TEX_CASE(15)
#undef SDF_TEX_CASE
            default: break;
        }
        const float t = tex3d_fetch(h, c.x, c.y, c.z);
        if (l == k) v = t;
        pending &= ~__ballot_sync(kFull, l == k);
    }
    if (!valid) return;
    const float g = c.dout + v;
    const unsigned long long key = pack_key(g, __float_as_int(p.w), l);
    const unsigned ob = (unsigned)(key >> 32);
    if (ob <= B.best[wl]) {
        atomicMin(&B.best[wl], ob);
        atomicMin(&B.key[wl], key);
    }
}

template <bool TEX>
__device__ __forceinline__ void evaluate_lane(const BatchParams& P, const BlockState& B, int pos, int pair,
                                              bool valid) {
    if constexpr (TEX)
        evaluate_tex(P, B, pos, pair, valid);
    else if (valid)
        evaluate(B, pos, pair);
}

// Per-warp queue of (sorted point, pair) entries; 32 entries are evaluated at once.
struct WarpQueue {
    uint2* q;      // 64 slots in shared memory
    int n;
};

template <bool TEX>
__device__ __forceinline__ void queue_push(const BatchParams& P, const BlockState& B, WarpQueue& Q, bool surv,
                                           int pos, int pair,
                                           int lane) {
    const unsigned m = __ballot_sync(kFull, surv);
    if (!m) return;
    stat_add(B, kWsLookups, (unsigned)__popc(m), lane);
    if (surv) Q.q[Q.n + __popc(m & ((1u << lane) - 1u))] = make_uint2((unsigned)pos, (unsigned)pair);
    Q.n += __popc(m);
    if (Q.n >= 32) {   // Q.n < 64: evaluate the top 32 entries with all lanes
        __syncwarp();
        const uint2 e = Q.q[Q.n - 32 + lane];
        __syncwarp();
        Q.n -= 32;
        evaluate_lane<TEX>(P, B, (int)e.x, (int)e.y, true);
    }
}

template <bool TEX>
__device__ __forceinline__ void queue_flush(const BatchParams& P, const BlockState& B, WarpQueue& Q, int lane) {
    __syncwarp();
    if constexpr (TEX) {
        const uint2 e = lane < Q.n ? Q.q[lane] : make_uint2(0u, 0u);
        evaluate_tex(P, B, (int)e.x, (int)e.y, lane < Q.n);
    } else if (lane < Q.n) {
        const uint2 e = Q.q[lane];
        evaluate(B, (int)e.x, (int)e.y);
    }
    __syncwarp();
    Q.n = 0;
}

// Point tests of up to TB (pair, tile) entries, the point loads issued together.
template <int TB, bool TEX>
__device__ __forceinline__ void test_tiles(const BatchParams& P, const BlockState& B, WarpQueue& Q,
                                           const unsigned (&ent)[TB],
                                           int cnt, int lane) {
    float4 pt[TB];
    int pos[TB];
#pragma unroll
    for (int k = 0; k < TB; ++k) {
        pos[k] = (int)(ent[k] & kTileMask) * 32 + lane;
        pt[k] = (k < cnt && pos[k] < B.n_valid) ? __ldg(&B.sorted[pos[k]]) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    // every entry's test first (independent shared-memory reads), then the pushes
    // (whose evaluations may lower the thresholds of later groups)
    bool surv[TB];
#pragma unroll
    for (int k = 0; k < TB; ++k) {
        const int pair = (int)(ent[k] >> 28);
        const float thr = pair_threshold(B, pair);
        surv[k] = k < cnt && pos[k] < B.n_valid && thr >= 0.f &&
                  seg_dist2(pt[k].x, pt[k].y, pt[k].z, B.pose[pair][4], B.pose[pair][5]) <= thr * thr;
    }
#pragma unroll
    for (int k = 0; k < TB; ++k) {
        if (k >= cnt) break;
        if (B.stat) stat_add(B, kWsPointT, (unsigned)__popc(__ballot_sync(kFull, pos[k] < B.n_valid)), lane);
        queue_push<TEX>(P, B, Q, surv[k], pos[k], (int)(ent[k] >> 28), lane);
    }
}

// Point tests of up to TB listed tiles against every pair whose capsule reached them
// (mask[t]: one bit per pair of the block), each tile's points loaded once and the
// TB loads issued together.  The masks are read by every lane alike, so the loop
// over a tile's pairs is uniform across the warp.
template <int TB, bool TEX>
__device__ __forceinline__ void test_tile_groups(const BatchParams& P, const BlockState& B, WarpQueue& Q,
                                                 const unsigned (&ent)[TB], int cnt, const unsigned* mask,
                                                 int lane) {
    float4 pt[TB];
    int pos[TB];
    unsigned mk[TB];
#pragma unroll
    for (int k = 0; k < TB; ++k) {
        pos[k] = (int)ent[k] * 32 + lane;
        pt[k] = (k < cnt && pos[k] < B.n_valid) ? __ldg(&B.sorted[pos[k]]) : make_float4(0.f, 0.f, 0.f, 0.f);
        mk[k] = k < cnt ? mask[ent[k]] : 0u;
    }
#pragma unroll
    for (int k = 0; k < TB; ++k) {
        unsigned m = mk[k];
        while (m) {
            const int pair = __ffs(m) - 1;
            m &= m - 1;
            const float thr = pair_threshold(B, pair);
            const bool surv = pos[k] < B.n_valid && thr >= 0.f &&
                              seg_dist2(pt[k].x, pt[k].y, pt[k].z, B.pose[pair][4], B.pose[pair][5]) <= thr * thr;
            if (B.stat) stat_add(B, kWsPointT, (unsigned)__popc(__ballot_sync(kFull, pos[k] < B.n_valid)), lane);
            queue_push<TEX>(P, B, Q, surv, pos[k], pair, lane);
        }
    }
}

// TB: list entries a warp takes per step in phase B (their point loads go out together).
// NW: warps per block (8 or 16); at 64 registers a thread, 32 / NW blocks fit an SM.
// TEX: lookups by the texture unit's trilinear filter (SDF_OPT_TEX3D).
template <int TB, int NW, bool TEX>
__global__ void __launch_bounds__(NW * 32, 32 / NW) check_kernel(const __grid_constant__ BatchParams P) {
    extern __shared__ float4 s_spheres[];            // tiles [stage_tiles], then super-tiles, then pair masks
    __shared__ float4 s_pose[NW][6];
    __shared__ uchar2 s_pair_wl[NW];
    __shared__ float4 s_grid_o[kMaxLinks];
    __shared__ float s_grid_h[kMaxLinks];
    __shared__ unsigned s_best[NW];
    __shared__ unsigned long long s_key[NW];
    __shared__ unsigned s_list[kBlockList];
    __shared__ unsigned s_list_n, s_list_next;
    __shared__ uint2 s_queue[NW][64];
    __shared__ __align__(8) uint64_t s_mbar;
    __shared__ unsigned s_stat[NW][kWsCount];
    __shared__ unsigned long long s_stat_ns[NW][kWnCount];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool stats = P.stats != nullptr;
    unsigned long long t_block0 = 0;
    if (stats) {
        if (tid == 0) t_block0 = global_ns();
        if (lane < kWsCount) s_stat[warp][lane] = 0u;
        if (lane < kWnCount) s_stat_ns[warp][lane] = 0ull;
    }
    // block -> trajectory (block_base is increasing)
    int lo = 0, hi = P.n_inst - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (P.inst[mid].block_base <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
    }
    const InstDesc& I = P.inst[lo];
    const CloudDesc& C = P.cloud[I.cloud];
    const LinkTable& T = *I.robot;
    const int L = I.L;
    // waypoint j of this block: b + j * n_blk (interleaved: a block's waypoints come
    // from distant parts of the trajectory, which evens out the blocks' work), else b * tw + j
    const int b_loc = (int)blockIdx.x - I.block_base;
    const int n_blk = (int)(((long long)I.W + I.tw - 1) / I.tw);   // no int overflow for W near 2^31
    const int w0 = I.interleave ? b_loc : b_loc * I.tw;             // < W
    const int w_step = I.interleave ? n_blk : 1;
    const int nw = I.interleave ? (int)min((long long)I.tw, ((long long)I.W - b_loc + n_blk - 1) / n_blk)
                                : min(I.tw, I.W - w0);
    const int n_pair = nw * L;
    if (I.mask) {   // a masked re-check: blocks without a selected waypoint leave at once
        const bool any = tid < nw && I.mask[w0 + tid * w_step] != 0;
        if (!__syncthreads_or(any)) return;
    }
    if (tid < NW) {
        s_best[tid] = kOrderedInf;
        s_key[tid] = ~0ull;
    }
    if (tid < L) {
        s_grid_o[tid] = T.grid_o[tid];
        s_grid_h[tid] = T.grid_h[tid];
    }
    if (tid < n_pair) s_pair_wl[tid] = make_uchar2((unsigned char)(tid / L), (unsigned char)(tid % L));
    if (tid == 0) {
        s_list_n = 0u;
        s_list_next = 0u;
    }
    // staged launches: per tile, the bits of the pairs whose capsule reaches it
    unsigned* s_mask = reinterpret_cast<unsigned*>(s_spheres + P.stage_tiles + P.stage_tiles / 32 + 1);
    for (int i = tid; i < P.stage_tiles; i += NW * 32) s_mask[i] = 0u;

    // phase A.1: forward kinematics, one warp per waypoint (before the sort is
    // waited for); lane j writes link j's pose
    if (warp < nw) {
        const float* qw = I.q + (size_t)(w0 + warp * w_step) * I.dof;
        if (lane < I.dof && !isfinite(qw[lane])) atomicOr(P.status, kStatusNonFinite);
        float M[12];
        fk_warp(T, qw, lane, M);
        float Mj[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            const float v = __shfl_up_sync(kFull, M[k], 1);
            Mj[k] = lane == 0 ? T.base[k] : v;
        }
        if (lane < L) {
            float4 rows[3], sp;
            store_link(Mj, T.sph_local[lane], rows, &sp);
            float4* dst = s_pose[warp * L + lane];
            dst[0] = rows[0];
            dst[1] = rows[1];
            dst[2] = rows[2];
            dst[3] = sp;
            // the link's bounding capsule in the world frame
            const float4 a = T.cap_a[lane], b = T.cap_b[lane];
            float A[3], Bw[3];
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                A[r] = fmaf(Mj[4 * r], a.x, fmaf(Mj[4 * r + 1], a.y, fmaf(Mj[4 * r + 2], a.z, Mj[4 * r + 3])));
                Bw[r] = fmaf(Mj[4 * r], b.x, fmaf(Mj[4 * r + 1], b.y, fmaf(Mj[4 * r + 2], b.z, Mj[4 * r + 3])));
            }
            const float dx = Bw[0] - A[0], dy = Bw[1] - A[1], dz = Bw[2] - A[2];
            const float dd = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            // under the texture lookup the capsule grows by the filter's point shift
            dst[4] = make_float4(A[0], A[1], A[2], TEX ? a.w + tex_cull_pad(T.grid_h[lane]) : a.w);
            dst[5] = make_float4(dx, dy, dz, dd > 0.f ? 1.f / dd : 0.f);
        }
    }
    const bool pair_warp = warp < n_pair;
    // the trajectory's blocks split the robot's grids and prefetch them into L2
    // while the sort runs (the lookups then miss only to L2); not when nothing
    // overlaps the prefetch
    if (P.warm_l2 && I.warm && warp == NW - 1 && lane == 0) {
        const unsigned long long chunks = I.warm_bytes >> 4;   // whole 16-byte units
        const unsigned long long nb = (unsigned long long)n_blk;
        const unsigned long long per = (chunks + nb - 1) / nb;
        unsigned long long c = (unsigned long long)((int)blockIdx.x - I.block_base) * per;
        const unsigned long long end = min(c + per, chunks);
        constexpr unsigned long long kPiece = 1u << 12;        // 64 KB per prefetch
        for (; c < end; c += kPiece)
            prefetch_l2(reinterpret_cast<const char*>(I.warm) + (c << 4), (unsigned)(min(kPiece, end - c) << 4));
    }

    // wait for the sort (a no-op without programmatic dependent launch), then stage
    // this trajectory's tile and super-tile spheres
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int n_valid = P.n_valid[I.cloud];
    const int n_tiles = (n_valid + 31) >> 5;
    const int n_super = (n_tiles + 31) >> 5;
    const bool staged = n_tiles > 0 && n_tiles <= P.stage_tiles;
    if (staged && tid == 0) {
        mbar_init(&s_mbar, 1);
        const unsigned tb = (unsigned)n_tiles * (unsigned)sizeof(float4);
        const unsigned sb = (unsigned)n_super * (unsigned)sizeof(float4);
        mbar_expect_tx(&s_mbar, tb + sb);
        bulk_copy_g2s(s_spheres, P.tiles + C.tile_base, tb, &s_mbar);
        bulk_copy_g2s(s_spheres + P.stage_tiles, P.supers + C.super_base, sb, &s_mbar);
    }
    __syncthreads();
    if (staged) {
        const bool ok = mbar_wait_bounded(&s_mbar, 0, P.wait_polls);
        if (!__syncthreads_and(ok)) {
            // the copy did not complete in time: report it and leave.  A drain wait of
            // the default length first, so that the copy has landed before the block's
            // shared memory is released; should that wait give up too, the status
            // already says that every output of this launch is invalid.
            if (tid == 0) {
                atomicOr(P.status, kStatusTimeout);
                mbar_wait_bounded(&s_mbar, 0, kDefaultWaitPolls);
            }
            __syncthreads();
            return;
        }
    }
    const float4* tiles = staged ? s_spheres : P.tiles + C.tile_base;
    const float4* supers = staged ? s_spheres + P.stage_tiles : P.supers + C.super_base;
    const unsigned long long t_fk = (stats && tid == 0) ? global_ns() : 0ull;
    const float4 capA = s_pose[pair_warp ? warp : 0][4];
    const float4 capD = s_pose[pair_warp ? warp : 0][5];

    BlockState B;
    B.sorted = P.sorted + C.point_base;
    B.values = T.values;
    B.n = T.n;
    B.n3 = T.n * T.n * T.n;
    B.L = L;
    B.pair_wl = s_pair_wl;
    B.n_valid = n_valid;
    B.pose = s_pose;
    B.grid_o = s_grid_o;
    B.grid_h = s_grid_h;
    B.best = s_best;
    B.key = s_key;
    B.cull = P.cull;
    B.stat = stats ? s_stat[warp] : nullptr;
    WarpQueue Q{s_queue[warp], 0};
    const float kInf = __int_as_float(0x7f800000);

    if (pair_warp) {
        unsigned long long t_a = stats ? global_ns() : 0ull;
        // phase A.2: seed -- nearest super-tile, nearest tile in it, all its points
        int seed_tile = -1;   // every point of it evaluated for this pair
        if (P.cull && n_tiles > 0) {
            float bs = kInf;
            int bi = 0x7fffffff;
            for (int s0 = 0; s0 < n_super; s0 += 32) {
                const int s = s0 + lane;
                if (s < n_super) {
                    const float4 c = supers[s];
                    const float sc = sqrtf(seg_dist2(c.x, c.y, c.z, capA, capD)) + c.w;
                    if (sc < bs) { bs = sc; bi = s; }
                }
            }
            const int s_seed = warp_argmin(bs, bi);   // >= n_super when every score is NaN
            if (s_seed < n_super) {
                const int t = s_seed * 32 + lane;
                float ts = kInf;
                if (t < n_tiles) {
                    const float4 c = tiles[t];
                    ts = sqrtf(seg_dist2(c.x, c.y, c.z, capA, capD)) + c.w;
                }
                const int t_seed = warp_argmin(ts, t < n_tiles ? t : 0x7fffffff);
                if (t_seed < n_tiles) seed_tile = t_seed;
                const bool ev = t_seed < n_tiles && t_seed * 32 + lane < n_valid;
                if (stats) stat_add(B, kWsSeed, (unsigned)__popc(__ballot_sync(kFull, ev)), lane);
                evaluate_lane<TEX>(P, B, t_seed * 32 + lane, warp, ev);
            }
        }
        if (stats) {
            const unsigned long long t_b = global_ns();
            if (lane == 0) s_stat_ns[warp][kWnSeed] += t_b - t_a;
            t_a = t_b;
        }
        // phase A.3: cull super-tiles, then tiles; survivors go to the block list,
        // or are tested here when the list is full
        unsigned over_ent[TB];
        int over_n = 0;
        for (int s0 = 0; s0 < n_super; s0 += 32) {
            const int s = s0 + lane;
            float thr = pair_threshold(B, warp);
            unsigned ms = __ballot_sync(kFull, s < n_super && capsule_reaches(supers[min(s, n_super - 1)], capA, capD, thr));
            if (stats) {
                stat_add(B, kWsSuperT, (unsigned)min(32, n_super - s0), lane);
                stat_add(B, kWsSuperP, (unsigned)__popc(ms), lane);
            }
            // two surviving super-tiles per round: their tile tests and ballots are
            // independent, and one list reservation covers both
            while (ms) {
                const int sa = s0 + __ffs(ms) - 1;
                ms &= ms - 1;
                const int sb = ms ? s0 + __ffs(ms) - 1 : -1;
                if (ms) ms &= ms - 1;
                thr = pair_threshold(B, warp);
                const int ta = sa * 32 + lane, tb = sb * 32 + lane;
                const bool ra = ta < n_tiles && capsule_reaches(tiles[min(ta, n_tiles - 1)], capA, capD, thr);
                const bool rb = sb >= 0 && tb < n_tiles && capsule_reaches(tiles[min(tb, n_tiles - 1)], capA, capD, thr);
                const unsigned mta = __ballot_sync(kFull, ra), mtb = __ballot_sync(kFull, rb);
                if (stats) {
                    stat_add(B, kWsTileT, (unsigned)min(32, n_tiles - sa * 32), lane);
                    stat_add(B, kWsTileP, (unsigned)__popc(mta), lane);
                    if (sb >= 0) {
                        stat_add(B, kWsTileT, (unsigned)min(32, n_tiles - sb * 32), lane);
                        stat_add(B, kWsTileP, (unsigned)__popc(mtb), lane);
                    }
                }
                const unsigned na = (unsigned)__popc(mta);
                if (!(mta | mtb)) continue;
                if (staged) {   // the pair's bit in each reached tile's mask (no list, no overflow),
                                // except its seed tile, whose points it has evaluated already
                    if (ra && ta != seed_tile) atomicOr(&s_mask[ta], 1u << warp);
                    if (rb && tb != seed_tile) atomicOr(&s_mask[tb], 1u << warp);
                    continue;
                }
                unsigned base = 0;
                if (lane == 0) base = atomicAdd(&s_list_n, na + (unsigned)__popc(mtb));
                base = __shfl_sync(kFull, base, 0);
                const unsigned lt = (1u << lane) - 1u;
                const unsigned slot_a = base + __popc(mta & lt), slot_b = base + na + __popc(mtb & lt);
                if (ra && slot_a < (unsigned)kBlockList) s_list[slot_a] = ((unsigned)warp << 28) | (unsigned)ta;
                if (rb && slot_b < (unsigned)kBlockList) s_list[slot_b] = ((unsigned)warp << 28) | (unsigned)tb;
#pragma unroll
                for (int h = 0; h < 2; ++h) {   // the list is full: test the rest here
                    const int sidx = h ? sb : sa;
                    unsigned over = __ballot_sync(kFull, h ? (rb && slot_b >= (unsigned)kBlockList)
                                                           : (ra && slot_a >= (unsigned)kBlockList));
                    if (stats) stat_add(B, kWsOver, (unsigned)__popc(over), lane);
                    while (over) {
                        over_ent[over_n] = ((unsigned)warp << 28) | (unsigned)(sidx * 32 + __ffs(over) - 1);
                        over &= over - 1;
                        if (++over_n == TB) {
                            test_tiles<TB, TEX>(P, B, Q, over_ent, over_n, lane);
                            over_n = 0;
                        }
                    }
                }
            }
        }
        if (over_n) test_tiles<TB, TEX>(P, B, Q, over_ent, over_n, lane);
        if (stats && lane == 0) s_stat_ns[warp][kWnCull] += global_ns() - t_a;
    }
    __syncthreads();
    const unsigned long long t_b0 = stats ? global_ns() : 0ull;

    // phase B: every warp takes list entries a few at a time
    auto take = [&](unsigned n_list, auto&& test) {
        for (;;) {
            unsigned k0 = 0;
            if (lane == 0) k0 = atomicAdd(&s_list_next, (unsigned)TB);
            k0 = __shfl_sync(kFull, k0, 0);
            if (k0 >= n_list) break;
            unsigned ent[TB];
            int cnt = 0;
#pragma unroll
            for (int k = 0; k < TB; ++k) {
                ent[k] = 0u;
                if (k0 + k < n_list) {
                    ent[k] = s_list[k0 + k];
                    cnt = k + 1;
                }
            }
            test(ent, cnt);
        }
    };
    if (staged) {
        // the reached tiles, grouped: each tile's points are loaded once for every pair
        // that reached it (in the paper scene about four pairs a tile).  The tiles with
        // a mask are compacted into the block list kBlockList at a time.
        for (int base = 0; base < n_tiles; base += kBlockList) {
            if (base > 0) __syncthreads();   // the previous round's tiles are taken
            if (tid == 0) {
                s_list_n = 0u;
                s_list_next = 0u;
            }
            __syncthreads();
            const int end = min(n_tiles, base + kBlockList);
            for (int t0 = base + warp * 32; t0 < end; t0 += NW * 32) {
                const int t = t0 + lane;
                const unsigned m = t < end ? s_mask[t] : 0u;
                const unsigned b = __ballot_sync(kFull, m != 0u);
                if (b) {
                    unsigned off = 0;
                    if (lane == 0) off = atomicAdd(&s_list_n, (unsigned)__popc(b));
                    off = __shfl_sync(kFull, off, 0);
                    if (m) s_list[off + __popc(b & ((1u << lane) - 1u))] = (unsigned)t;
                }
            }
            __syncthreads();
            take(s_list_n, [&](const unsigned (&ent)[TB], int cnt) {
                test_tile_groups<TB, TEX>(P, B, Q, ent, cnt, s_mask, lane);
            });
        }
    } else {
        take(min(s_list_n, (unsigned)kBlockList),
             [&](const unsigned (&ent)[TB], int cnt) { test_tiles<TB, TEX>(P, B, Q, ent, cnt, lane); });
    }
    queue_flush<TEX>(P, B, Q, lane);
    if (stats && lane == 0) s_stat_ns[warp][kWnPoints] += global_ns() - t_b0;
    __syncthreads();
    if (stats) {
        // block sums of the warp rows, one global atomic per counter
        if (tid < kWsCount) {
            unsigned long long v = 0;
            for (int k = 0; k < NW; ++k) v += s_stat[k][tid];
            const int dst[kWsCount] = {1, 2, 3, 4, 5, 6, 7, 8};
            atomicAdd(&P.stats[dst[tid]], v);
        } else if (tid >= 32 && tid < 32 + kWnCount) {
            unsigned long long v = 0;
            for (int k = 0; k < NW; ++k) v += s_stat_ns[k][tid - 32];
            atomicAdd(&P.stats[11 + (tid - 32)], v);
        } else if (tid == 64) {
            const unsigned long long t_end = global_ns();
            atomicAdd(&P.stats[0], (unsigned long long)n_pair);
            atomicAdd(&P.stats[9], 1ull);
        }
        if (tid == 0) {
            const unsigned long long t_end = global_ns();
            atomicAdd(&P.stats[10], t_fk - t_block0);
            atomicAdd(&P.stats[14], t_end - t_block0);
            atomicMax(&P.stats[15], t_end - t_block0);
            atomicMin(&P.stats[17], t_block0);
            atomicMax(&P.stats[18], t_end);
        }
    }

    // results of the block's waypoints
    if (tid < nw && (!I.mask || I.mask[w0 + tid * w_step] != 0)) {
        const int w = w0 + tid * w_step;
        const unsigned long long key = s_key[tid];
        if (key == ~0ull) {
            I.dist[w] = kInf;
            I.arg_link[w] = -1;
            I.arg_point[w] = -1;
        } else {
            I.dist[w] = from_ordered((unsigned)(key >> 32));
            I.arg_link[w] = (int)(key & 15u);
            I.arg_point[w] = (int)((key & 0xffffffffu) >> 4);
        }
    }
}

// End of a host-buffer check: the status word reaches host memory, then the
// completion count (the results were written to host memory by the check kernel,
// which precedes this kernel in stream order).
__global__ void finish_kernel(int* status, int* h_status, unsigned* d_seq, unsigned* h_done) {
    const int st = *status;
    *status = 0;
    *reinterpret_cast<volatile int*>(h_status) = st;
    const unsigned s = *d_seq + 1u;
    *d_seq = s;
    __threadfence_system();
    *reinterpret_cast<volatile unsigned*>(h_done) = s;
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

// Kinematics as fk_kernel, plus the resets of a surrogate check's keys (~0), re-check
// flags (0) and two work counters (0), launched right after the sort and overlapping it
// (programmatic dependent launch: the sort lets its dependents start at once).  Every
// thread waits for the sort before it exits, so that this kernel completes only after
// the sort: a kernel behind it in the stream sees both.  It writes nothing the sort
// reads.
__global__ void __launch_bounds__(128) fk_reset_kernel(const __grid_constant__ LinkTable T,
                                                       const float* __restrict__ q, int W,
                                                       float* __restrict__ out, int* status,
                                                       unsigned long long* keys, uint8_t* recheck, int* counter) {
    __shared__ float4 s_xf[4][kMaxLinks][3];
    __shared__ float4 s_sph[4][kMaxLinks];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int w = blockIdx.x * 4 + warp;
    if (w < W) {   // whole warps
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
    const int gt = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
    for (int i = gt; i < W; i += stride) {
        keys[i] = ~0ull;
        recheck[i] = 0;
    }
    if (gt == 0) {
        counter[0] = 0;
        counter[1] = 0;
    }
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

}  // namespace

// Dynamic shared memory of a check block: the staged tile spheres [stage_tiles], the
// super-tile spheres [stage_tiles / 32 + 1], then one pair mask per staged tile.
size_t staged_bytes(int stage_tiles) {
    return stage_tiles > 0 ? (size_t)(stage_tiles + stage_tiles / 32 + 1) * sizeof(float4) +
                                 (size_t)stage_tiles * sizeof(unsigned)
                           : 0;
}

namespace {
// Whether each device can run the sort as one 16-CTA cluster (a non-portable cluster
// size) instead of 8 CTAs: decided once per device by configure_kernels.
constexpr int kMaxDevices = 64;
std::atomic<int> g_prep_ctas[kMaxDevices] = {};
}  // namespace

int max_sort_ctas(int device) {
    return device >= 0 && device < kMaxDevices && g_prep_ctas[device].load(std::memory_order_relaxed) == 16 ? 16 : kPrepCtas;
}

namespace {

template <int CT>
cudaError_t launch_prep_ct(const BatchParams& p, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(CT * p.n_cloud));
    cfg.blockDim = dim3(kPrepThreads);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CT;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, prep_kernel<CT>, p);
}

cudaError_t launch_prep_kernel(const BatchParams& p, cudaStream_t s) {
    int dev = 0;
    if (!p.sort_ctas && cudaGetDevice(&dev) != cudaSuccess) dev = -1;
    const int ctas = p.sort_ctas ? p.sort_ctas : max_sort_ctas(dev);
    return ctas == 16 ? launch_prep_ct<16>(p, s) : launch_prep_ct<kPrepCtas>(p, s);
}

}  // namespace

cudaError_t configure_kernels() {
    {   // a 16-CTA cluster for the sort, where the device can place one
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        int ctas = kPrepCtas;
        if (cudaFuncSetAttribute(prep_kernel<16>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(16);
            cfg.blockDim = dim3(kPrepThreads);
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = 16;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            int clusters = 0;
            if (cudaOccupancyMaxActiveClusters(&clusters, prep_kernel<16>, &cfg) == cudaSuccess && clusters > 0) ctas = 16;
        }
        cudaGetLastError();   // a refused attribute or query is not an error here
        if (dev >= 0 && dev < kMaxDevices) g_prep_ctas[dev].store(ctas, std::memory_order_relaxed);
    }
    const int smem = (int)staged_bytes(kMaxStagedTiles);
    const void* fns[8] = {(const void*)check_kernel<1, 16, false>, (const void*)check_kernel<2, 16, false>,
                          (const void*)check_kernel<4, 16, false>, (const void*)check_kernel<1, 8, false>,
                          (const void*)check_kernel<2, 8, false>,  (const void*)check_kernel<4, 8, false>,
                          (const void*)check_kernel<1, 16, true>,  (const void*)check_kernel<1, 8, true>};
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 8 && e == cudaSuccess; ++k)
        e = cudaFuncSetAttribute(fns[k], cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    return e;
}

cudaError_t launch_batch(const BatchParams& p, int tile_batch, cudaStream_t s, cudaEvent_t ev_mid) {
    if (p.n_inst <= 0 || p.n_blocks <= 0) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    if (!p.skip_prep) {
        e = launch_prep_kernel(p, s);
        if (e != cudaSuccess) return e;
    }
    if (ev_mid) {   // a timing event between the kernels; the check then starts after the sort ends
        e = cudaEventRecord(ev_mid, s);
        if (e != cudaSuccess) return e;
    }
    // programmatic dependent launch: the check grid starts while the sort finishes,
    // runs its forward kinematics, then waits (griddepcontrol.wait) for the sort
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)p.n_blocks);
    const int nw = p.warps == 8 ? 8 : 16;
    cfg.blockDim = dim3(nw * 32);
    cfg.dynamicSmemBytes = staged_bytes(p.stage_tiles);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = (ev_mid || p.skip_prep) ? 0 : 1;
    if (p.tex)   // the texture form: one list batch (1), either block width
        return nw == 16 ? cudaLaunchKernelEx(&cfg, check_kernel<1, 16, true>, p)
                        : cudaLaunchKernelEx(&cfg, check_kernel<1, 8, true>, p);
    switch (tile_batch * 100 + nw) {
        case 116: return cudaLaunchKernelEx(&cfg, check_kernel<1, 16, false>, p);
        case 216: return cudaLaunchKernelEx(&cfg, check_kernel<2, 16, false>, p);
        case 416: return cudaLaunchKernelEx(&cfg, check_kernel<4, 16, false>, p);
        case 108: return cudaLaunchKernelEx(&cfg, check_kernel<1, 8, false>, p);
        case 208: return cudaLaunchKernelEx(&cfg, check_kernel<2, 8, false>, p);
        case 408: return cudaLaunchKernelEx(&cfg, check_kernel<4, 8, false>, p);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_prep(const BatchParams& p, cudaStream_t s) {
    if (p.n_cloud <= 0) return cudaSuccess;
    return launch_prep_kernel(p, s);
}

cudaError_t launch_finish(int* status, int* h_status, unsigned* d_seq, unsigned* h_done, cudaStream_t s) {
    finish_kernel<<<1, 1, 0, s>>>(status, h_status, d_seq, h_done);
    return cudaGetLastError();
}

cudaError_t launch_fk(const LinkTable& T, const float* q, int W, float* out, int* status, cudaStream_t s) {
    fk_kernel<<<(unsigned)((W + 3) / 4), 128, 0, s>>>(T, q, W, out, status);
    return cudaGetLastError();
}

cudaError_t launch_fk_reset(const LinkTable& T, const float* q, int W, float* out, int* status,
                            unsigned long long* keys, uint8_t* recheck, int* counter, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(W > 0 ? (W + 3) / 4 : 1));
    cfg.blockDim = dim3(128);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, fk_reset_kernel, T, q, W, out, status, keys, recheck, counter);
}

}  // namespace sdf
