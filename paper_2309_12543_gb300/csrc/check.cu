// Fused runtime distance check for sm_103a.
//
// Two kernels per call.
//
// cloud_prep_kernel (one cluster of 8 CTAs x 1024 threads) orders the obstacle
// points in space: bounding box, 32^3-cell Morton key per point, counting sort of
// the keys in distributed shared memory, scatter into a float4 array (x, y, z,
// original index), and a bounding sphere per tile of 32 consecutive sorted points.  Non-finite points are
// dropped from the sorted cloud (and flagged), so they can never be a minimum.
//
// check_kernel: one block owns TW consecutive waypoints and one chunk of tiles.
//   1. forward kinematics, one warp per waypoint (Sec. III-A "parallel forward
//      kinematics"): each lane builds one DH joint transform, a warp scan composes
//      them, the link-from-world transforms land in shared memory;
//   2. seed: for every (waypoint, link) pair the tile whose farthest point is
//      nearest to the link's bounding-sphere centre is evaluated in full, so the
//      per-waypoint best starts as a tight upper bound;
//   3. sweep: each warp walks tiles; the lanes test the tile's sphere against all
//      (waypoint, link) spheres at once (||c_t - c_l|| - r_t - R_l > best + slack
//      => skip, the analogue of the paper's "grids in sphere", Sec. III-B), then for
//      each surviving pair the 32 lanes test the tile's points.  Surviving (point,
//      pair) entries are compacted into a per-warp queue and evaluated 32 at a time:
//      transform into the link frame (the per-point form of Sec. II-B / Fig. 2),
//      trilinear lookup in the FP32 link grid (the grid-sample interpolation of
//      Sec. III-A), distance-to-box outside the grid;
//   4. reduction with min per waypoint (Sec. III-A): each value is packed with its
//      original point index and link into one 64-bit key whose unsigned order is
//      (distance, point, link), so atomicMin yields a deterministic arg-min.
// With several tile chunks per waypoint tile the blocks combine their keys with a
// global atomicMin; the last block of a waypoint tile (ticket counter) decodes the
// keys and returns the scratch to its idle state.
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
// phase is one pass over the points with cluster barriers in between.
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

    // 1. bounding box of the finite points (per CTA, then across the cluster)
    float lo[3] = {kInf, kInf, kInf}, hi[3] = {-kInf, -kInf, -kInf};
    bool bad = false;
    for (int i = gtid; i < P.N; i += kStride) {
        const float3 p = load_point(P.points, P.stride, i);
        if (finite3(p)) {
            lo[0] = fminf(lo[0], p.x); lo[1] = fminf(lo[1], p.y); lo[2] = fminf(lo[2], p.z);
            hi[0] = fmaxf(hi[0], p.x); hi[1] = fmaxf(hi[1], p.y); hi[2] = fmaxf(hi[2], p.z);
        } else {
            bad = true;
        }
    }
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
    for (int i = gtid; i < P.N; i += kStride) {
        const float3 p = load_point(P.points, P.stride, i);
        if (finite3(p)) {
            const unsigned c = cell_key(p, blo, inv);
            atomicAdd(cluster.map_shared_rank(&s_bins[c % kBinsPerCta], (int)(c / kBinsPerCta)), 1u);
        }
    }
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
    for (int i = gtid; i < P.N; i += kStride) {
        const float3 p = load_point(P.points, P.stride, i);
        if (finite3(p)) {
            const unsigned c = cell_key(p, blo, inv);
            const unsigned pos = atomicAdd(cluster.map_shared_rank(&s_bins[c % kBinsPerCta], (int)(c / kBinsPerCta)), 1u);
            P.sorted[pos] = make_float4(p.x, p.y, p.z, __int_as_float(i));
        }
    }
    __threadfence();
    cluster.sync();   // every CTA's writes of `sorted` are visible; no remote smem use after this

    // 5. tile spheres: centre of the tile's box, radius to its farthest point
    const int n_tiles = (n_valid + 31) >> 5;
    for (int t = (int)rank * (kPrepThreads / 32) + warp; t < n_tiles; t += kPrepCtas * (kPrepThreads / 32)) {
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

template <int TW>
__global__ void __launch_bounds__(kBlock, 2) check_kernel(const __grid_constant__ CheckParams P) {
    extern __shared__ float4 s_tiles[];        // tile spheres, staged by one bulk copy
    __shared__ float4 s_xf[TW][kMaxLinks][3];
    __shared__ float4 s_sph[TW][kMaxLinks];
    __shared__ unsigned s_best[TW];
    __shared__ unsigned long long s_key[TW];
    __shared__ float s_seed_s[kWarps][32];
    __shared__ int s_seed_t[kWarps][32];
    __shared__ unsigned s_queue[kWarps][64];
    __shared__ __align__(8) uint64_t s_mbar;
    __shared__ bool s_last;

    const LinkTable& T = P.T;
    const int L = T.L;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int w0 = blockIdx.x * TW;
    const int nw = min(TW, P.W - w0);
    const int pairs = nw * L;                  // <= 32 by construction of TW
    const int n_valid = *P.n_valid;
    const int n_tiles = (n_valid + 31) >> 5;
    const int t_begin = min(n_tiles, (int)blockIdx.y * P.tiles_per_split);
    const int t_end = min(n_tiles, t_begin + P.tiles_per_split);
    const bool staged = P.stage_tiles && n_tiles > 0;

    // 0. start the copy of all tile spheres into shared memory
    if (staged && threadIdx.x == 0) {
        mbar_init(&s_mbar, 1);
        const unsigned bytes = (unsigned)n_tiles * (unsigned)sizeof(float4);
        mbar_expect_tx(&s_mbar, bytes);
        bulk_copy_g2s(s_tiles, P.tiles, bytes, &s_mbar);
    }

    // 1. forward kinematics, one warp per waypoint (overlaps the copy)
    if (warp < nw) {
        const float* qw = P.q + (size_t)(w0 + warp) * T.dof;
        if (lane < T.dof && !isfinite(qw[lane])) atomicOr(P.status, kStatusNonFinite);
        fk_links(T, qw, lane, s_xf[warp], s_sph[warp]);
    }
    if (threadIdx.x < TW) {
        s_best[threadIdx.x] = kOrderedInf;
        s_key[threadIdx.x] = ~0ull;
    }
    __syncthreads();
    if (staged) {
        const bool ok = mbar_wait_bounded(&s_mbar, 0);
        if (!__syncthreads_and(ok)) {
            // the copy did not complete: report it, give it one more bounded wait so
            // no transfer into this block's shared memory is left in flight, leave
            if (threadIdx.x == 0) {
                atomicOr(P.status, kStatusTimeout);
                mbar_wait_bounded(&s_mbar, 0);
            }
            return;
        }
    }
    const float4* tiles = staged ? s_tiles : P.tiles;

    unsigned long long lk[TW];
#pragma unroll
    for (int i = 0; i < TW; ++i) lk[i] = ~0ull;

    auto evaluate = [&](int pos, int wl, int l) {
        const float4 p = __ldg(&P.sorted[pos]);
        const float4 r0 = s_xf[wl][l][0], r1 = s_xf[wl][l][1], r2 = s_xf[wl][l][2];
        const float lx = fmaf(r0.x, p.x, fmaf(r0.y, p.y, fmaf(r0.z, p.z, r0.w)));
        const float ly = fmaf(r1.x, p.x, fmaf(r1.y, p.y, fmaf(r1.z, p.z, r1.w)));
        const float lz = fmaf(r2.x, p.x, fmaf(r2.y, p.y, fmaf(r2.z, p.z, r2.w)));
        const float g = grid_lookup(T.values + (size_t)l * T.n * T.n * T.n, T.n, T.grid_o[l],
                                    T.grid_h[l], lx, ly, lz);
        const unsigned long long key = pack_key(g, __float_as_int(p.w), l);
        const unsigned ob = (unsigned)(key >> 32);
#pragma unroll
        for (int i = 0; i < TW; ++i)
            if (i == wl && key < lk[i]) lk[i] = key;
        if (ob < s_best[wl]) atomicMin(&s_best[wl], ob);
    };

    // this lane's (waypoint, link) pair for the lane-parallel tile tests
    const bool has_pair = lane < pairs;
    const int my_wl = has_pair ? lane / L : 0;
    const int my_l = has_pair ? lane - my_wl * L : 0;
    const float4 my_sph = s_sph[my_wl][my_l];

    // 2. seed: per pair, the tile (over the whole cloud) whose farthest point is
    //    nearest to the link's sphere centre is evaluated in full
    if (P.cull) {
        float best_s = __int_as_float(0x7f800000);
        int best_t = -1;
        for (int t = warp; t < n_tiles; t += kWarps) {
            const float4 tc = tiles[t];
            const float dx = tc.x - my_sph.x, dy = tc.y - my_sph.y, dz = tc.z - my_sph.z;
            const float s = sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz))) + tc.w;
            if (s < best_s) { best_s = s; best_t = t; }
        }
        s_seed_s[warp][lane] = best_s;
        s_seed_t[warp][lane] = best_t;
        __syncthreads();
        if (threadIdx.x < pairs) {
            float bs = s_seed_s[0][threadIdx.x];
            int bt = s_seed_t[0][threadIdx.x];
            for (int k = 1; k < kWarps; ++k)
                if (s_seed_s[k][threadIdx.x] < bs) { bs = s_seed_s[k][threadIdx.x]; bt = s_seed_t[k][threadIdx.x]; }
            s_seed_t[0][threadIdx.x] = bt;
        }
        __syncthreads();
        for (int e = warp; e < pairs; e += kWarps) {
            const int t = s_seed_t[0][e];
            if (t >= 0 && t * 32 + lane < n_valid) evaluate(t * 32 + lane, e / L, e % L);
        }
        __syncthreads();
    }

    // 3. sweep, kTileBatch consecutive tiles per warp step: tile tests across pairs
    //    (lanes), point loads for all surviving tiles together, then point tests
    //    across lanes with survivor compaction
    unsigned* q = s_queue[warp];
    int qn = 0;
    const unsigned lt_mask = (1u << lane) - 1u;
    const float kInf = __int_as_float(0x7f800000);
    for (int t0 = t_begin + warp * kTileBatch; t0 < t_end; t0 += kWarps * kTileBatch) {
        // this lane's pair threshold: best + R + slack (a distance from the centre)
        float thr = kInf;
        if (P.cull && has_pair) {
            unsigned ob = s_best[my_wl];
            if (P.splits > 1) {
                const unsigned long long gk = *reinterpret_cast<volatile unsigned long long*>(&P.keys[w0 + my_wl]);
                ob = min(ob, (unsigned)(gk >> 32));
            }
            thr = from_ordered(ob) + my_sph.w + kCullSlack;
            if (!(thr == thr)) thr = kInf;
        }
        unsigned tm[kTileBatch];
        float4 pt[kTileBatch];
#pragma unroll
        for (int k = 0; k < kTileBatch; ++k) {
            const int t = t0 + k;
            bool ts = false;
            if (has_pair && t < t_end) {
                const float4 tc = tiles[t];
                const float dx = tc.x - my_sph.x, dy = tc.y - my_sph.y, dz = tc.z - my_sph.z;
                const float base = thr + tc.w;
                ts = base >= 0.f && fmaf(dx, dx, fmaf(dy, dy, dz * dz)) <= base * base;
            }
            tm[k] = __ballot_sync(kFull, ts);
        }
#pragma unroll
        for (int k = 0; k < kTileBatch; ++k) {
            const int pos = (t0 + k) * 32 + lane;
            pt[k] = (tm[k] && pos < n_valid) ? __ldg(&P.sorted[pos]) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int k = 0; k < kTileBatch; ++k) {
            const int pos = (t0 + k) * 32 + lane;
            const bool valid = pos < n_valid;
            unsigned m_t = tm[k];
            while (m_t) {
                const int e = __ffs(m_t) - 1;
                m_t &= m_t - 1;
                const float te = __shfl_sync(kFull, thr, e);
                const float4 s = s_sph[e / L][e % L];
                const float dx = pt[k].x - s.x, dy = pt[k].y - s.y, dz = pt[k].z - s.z;
                const bool surv = valid && te >= 0.f && fmaf(dx, dx, fmaf(dy, dy, dz * dz)) <= te * te;
                const unsigned m = __ballot_sync(kFull, surv);
                if (m) {
                    if (surv) q[qn + __popc(m & lt_mask)] = ((unsigned)pos << 8) | (unsigned)e;
                    qn += __popc(m);
                    if (qn >= 32) {
                        __syncwarp();
                        const unsigned ent = q[qn - 32 + lane];
                        __syncwarp();
                        qn -= 32;
                        const int ee = (int)(ent & 255u);
                        evaluate((int)(ent >> 8), ee / L, ee % L);
                    }
                }
            }
        }
    }
    __syncwarp();
    if (lane < qn) {
        const unsigned ent = q[lane];
        const int ee = (int)(ent & 255u);
        evaluate((int)(ent >> 8), ee / L, ee % L);
    }

    // 4. reduce keys: warp shuffle, then shared atomics
#pragma unroll
    for (int i = 0; i < TW; ++i) {
        unsigned long long k = lk[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long other = __shfl_xor_sync(kFull, k, o);
            k = other < k ? other : k;
        }
        if (lane == 0 && i < nw && k != ~0ull) atomicMin(&s_key[i], k);
    }
    __syncthreads();

    if (P.splits == 1) {
        if (threadIdx.x < nw) write_result(P, w0 + threadIdx.x, s_key[threadIdx.x]);
        return;
    }
    if (threadIdx.x < nw && s_key[threadIdx.x] != ~0ull) atomicMin(&P.keys[w0 + threadIdx.x], s_key[threadIdx.x]);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned ticket = atomicAdd(&P.tickets[blockIdx.x], 1u);
        s_last = (ticket == (unsigned)P.splits - 1u);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (threadIdx.x < nw) {
        const int w = w0 + threadIdx.x;
        const unsigned long long key = atomicExch(&P.keys[w], ~0ull);   // read and reset
        write_result(P, w, key);
    }
    if (threadIdx.x == 0) P.tickets[blockIdx.x] = 0u;
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

cudaError_t configure_kernels() {
    const int smem = kMaxStagedTiles * (int)sizeof(float4);
    cudaError_t e = cudaFuncSetAttribute(check_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(check_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(check_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    return e;
}

cudaError_t launch_check(const CheckParams& p, int tw, cudaStream_t s) {
    const dim3 block(kBlock);
    const dim3 grid((unsigned)((p.W + tw - 1) / tw), (unsigned)p.splits);
    const size_t smem = p.stage_tiles ? (size_t)p.max_tiles * sizeof(float4) : 0;
    switch (tw) {
        case 1: check_kernel<1><<<grid, block, smem, s>>>(p); break;
        case 2: check_kernel<2><<<grid, block, smem, s>>>(p); break;
        case 4: check_kernel<4><<<grid, block, smem, s>>>(p); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_fk(const LinkTable& T, const float* q, int W, float* out, int* status,
                      cudaStream_t s) {
    fk_kernel<<<(unsigned)((W + 3) / 4), 128, 0, s>>>(T, q, W, out, status);
    return cudaGetLastError();
}

}  // namespace sdf
