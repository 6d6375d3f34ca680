// Link SDF pre-processing on the GPU (Sec. III-A, "Link SDFs"): one thread per
// grid node computes the signed distance to the link mesh by brute force over its
// triangles, which are staged through shared memory in chunks.
//
// Unsigned distance: project the node onto the triangle's plane; if the projection
// lies inside the triangle (same-side tests against the three edges) the distance
// is the plane distance, otherwise it is the distance to the nearest of the three
// edge segments.  Sign: generalised winding number, the sum of the triangles'
// signed solid angles (Van Oosterom & Strackee) over 4 pi, inside when >= 1/2.
// Components of a union mesh are contiguous triangle ranges; the node value is the
// minimum over components.
#include <cuda_runtime.h>

#include "internal.h"

namespace sdf {
namespace {

constexpr int kTriChunk = 128;
constexpr int kBuildBlock = 128;

__device__ __forceinline__ float3 sub(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float dot(float3 a, float3 b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }
__device__ __forceinline__ float3 cross(float3 a, float3 b) {
    return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

__device__ __forceinline__ float segment_dist2(float3 p, float3 a, float3 ab) {
    const float3 ap = sub(p, a);
    const float den = dot(ab, ab);
    float t = den > 0.f ? dot(ap, ab) / den : 0.f;
    t = fminf(fmaxf(t, 0.f), 1.f);
    const float3 d = make_float3(ap.x - t * ab.x, ap.y - t * ab.y, ap.z - t * ab.z);
    return dot(d, d);
}

__device__ __forceinline__ float tri_dist2(float3 p, float3 a, float3 b, float3 c) {
    const float3 ab = sub(b, a), bc = sub(c, b), ca = sub(a, c);
    const float3 n = cross(ab, sub(c, a));
    const float nn = dot(n, n);
    const float3 ap = sub(p, a), bp = sub(p, b), cp = sub(p, c);
    // projection inside <=> p lies on the inner side of all three edge planes
    const bool inside = nn > 0.f && dot(cross(ab, ap), n) >= 0.f && dot(cross(bc, bp), n) >= 0.f &&
                        dot(cross(ca, cp), n) >= 0.f;
    if (inside) {
        const float h = dot(ap, n);
        return h * h / nn;
    }
    const float e0 = segment_dist2(p, a, ab), e1 = segment_dist2(p, b, bc), e2 = segment_dist2(p, c, ca);
    return fminf(e0, fminf(e1, e2));
}

__device__ __forceinline__ float solid_angle(float3 p, float3 a, float3 b, float3 c) {
    const float3 ra = sub(a, p), rb = sub(b, p), rc = sub(c, p);
    const float la = sqrtf(dot(ra, ra)), lb = sqrtf(dot(rb, rb)), lc = sqrtf(dot(rc, rc));
    const float num = dot(ra, cross(rb, rc));
    const float den = la * lb * lc + dot(ra, rb) * lc + dot(ra, rc) * lb + dot(rb, rc) * la;
    return 2.f * atan2f(num, den);
}

__global__ void __launch_bounds__(kBuildBlock) grid_build_kernel(
    const float* __restrict__ tris9, const int* __restrict__ comp_off, int n_comp, int n_tris,
    float ox, float oy, float oz, float h, int n, float* __restrict__ out) {
    __shared__ float s_tri[kTriChunk * 9];
    const long long total = (long long)n * n * n;
    const long long idx = (long long)blockIdx.x * kBuildBlock + threadIdx.x;
    const bool active = idx < total;
    const int i = (int)(idx % n), j = (int)((idx / n) % n), k = (int)(idx / ((long long)n * n));
    const float3 p = make_float3(ox + (float)i * h, oy + (float)j * h, oz + (float)k * h);

    const float kInf = __int_as_float(0x7f800000);
    float result = kInf, best2 = kInf, omega = 0.f;
    int comp = 0, comp_end = comp_off[1];
    for (int t0 = 0; t0 < n_tris; t0 += kTriChunk) {
        const int cnt = min(kTriChunk, n_tris - t0);
        __syncthreads();
        for (int e = threadIdx.x; e < cnt * 9; e += kBuildBlock) s_tri[e] = tris9[(size_t)t0 * 9 + e];
        __syncthreads();
        for (int t = 0; t < cnt; ++t) {
            if (t0 + t == comp_end) {   // uniform across the block: close a component
                const float d = sqrtf(best2);
                result = fminf(result, omega >= 2.f * 3.14159265358979f ? -d : d);
                best2 = kInf;
                omega = 0.f;
                ++comp;
                comp_end = comp < n_comp ? comp_off[comp + 1] : n_tris;
            }
            const float* tr = s_tri + 9 * t;
            const float3 a = make_float3(tr[0], tr[1], tr[2]);
            const float3 b = make_float3(tr[3], tr[4], tr[5]);
            const float3 c = make_float3(tr[6], tr[7], tr[8]);
            best2 = fminf(best2, tri_dist2(p, a, b, c));
            omega += solid_angle(p, a, b, c);
        }
    }
    const float d = sqrtf(best2);
    result = fminf(result, omega >= 2.f * 3.14159265358979f ? -d : d);
    if (active) out[idx] = result;
}

}  // namespace

cudaError_t launch_grid_build(const float* tris9, const int* comp_off, int n_comp, int n_tris,
                              float ox, float oy, float oz, float h, int n, float* out,
                              cudaStream_t s) {
    const long long total = (long long)n * n * n;
    const unsigned blocks = (unsigned)((total + kBuildBlock - 1) / kBuildBlock);
    grid_build_kernel<<<blocks, kBuildBlock, 0, s>>>(tris9, comp_off, n_comp, n_tris, ox, oy, oz, h,
                                                     n, out);
    return cudaGetLastError();
}

}  // namespace sdf
