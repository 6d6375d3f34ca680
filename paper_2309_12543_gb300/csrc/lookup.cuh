// Device helpers shared by the grid check and the surrogate kernels: the
// order-preserving encoding of FP32 distances, the packed arg-min key, and the
// link-grid lookup (trilinear interpolation, Sec. III-A, with the out-of-box rule).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sdf {
namespace dev {

// FP32 -> unsigned with the same order (-0 and +0 map to the same value).
__device__ __forceinline__ unsigned ordered_bits(float f) {
    unsigned u = __float_as_uint(f + 0.0f);  // -0 -> +0
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float from_ordered(unsigned o) {
    return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o);
}

// 64-bit key whose unsigned order is (distance, point, link): atomicMin of keys
// gives the minimum distance with a deterministic arg-min.
__device__ __forceinline__ unsigned long long pack_key(float g, int point, int link) {
    return ((unsigned long long)ordered_bits(g) << 32) | ((unsigned)point << 4) | (unsigned)link;
}

// Grid value at a link-frame point: trilinear interpolation in the n^3 FP32 grid G
// (x fastest) with origin o_ih.xyz and 1/h in o_ih.w; outside the grid box, the
// distance to the box plus the interpolated value at the nearest box point.
// Branch-free: the point is clamped in index space and the clamp distance added.
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
    const int nn = n * n;   // grids hold at most 512^3 < 2^31 values: 32-bit offsets
    const float* b = G + (ix + n * iy + nn * iz);
    const float v000 = __ldg(b), v100 = __ldg(b + 1);
    const float v010 = __ldg(b + n), v110 = __ldg(b + n + 1);
    const float v001 = __ldg(b + nn), v101 = __ldg(b + nn + 1);
    const float v011 = __ldg(b + nn + n), v111 = __ldg(b + nn + n + 1);
    const float c00 = fmaf(fx, v100 - v000, v000), c10 = fmaf(fx, v110 - v010, v010);
    const float c01 = fmaf(fx, v101 - v001, v001), c11 = fmaf(fx, v111 - v011, v011);
    const float c0 = fmaf(fy, c10 - c00, c00), c1 = fmaf(fy, c11 - c01, c01);
    return dout + fmaf(fz, c1 - c0, c0);
}

// The texture unit's form of the lookup (SDF_OPT_TEX3D): the hardware trilinear
// filter of a linear-filtering texture object over the link's grid (unnormalised
// coordinates, node (i,j,k) at texel centre (i,j,k) + 1/2, clamped addressing).  The
// out-of-box rule stays in software: tex_coord gives the texel coordinates of the
// clamped point and the distance to the box; the value is dout + tex3D(x, y, z).
// The filter holds each axis's interpolation weight in fixed point with 8 fractional
// bits, so the value is the exact trilinear value at a point moved by at most h/256
// per axis from the query point.
struct TexCoord {
    float x, y, z, dout;
};
__device__ __forceinline__ TexCoord tex_coord(int n, float4 o_ih, float h, float px, float py, float pz) {
    const float top = (float)(n - 1);
    const float ux = (px - o_ih.x) * o_ih.w;
    const float uy = (py - o_ih.y) * o_ih.w;
    const float uz = (pz - o_ih.z) * o_ih.w;
    const float cx = fminf(fmaxf(ux, 0.f), top);
    const float cy = fminf(fmaxf(uy, 0.f), top);
    const float cz = fminf(fmaxf(uz, 0.f), top);
    const float ex = ux - cx, ey = uy - cy, ez = uz - cz;
    TexCoord c;
    c.x = cx + 0.5f;
    c.y = cy + 0.5f;
    c.z = cz + 0.5f;
    c.dout = h * sqrtf(fmaf(ex, ex, fmaf(ey, ey, ez * ez)));
    return c;
}

// Filtered fetch of texture object `tex` at texel coordinates (x, y, z), issued as
// explicit PTX.  (Inlined into the check kernel, the tex3D intrinsic returned a valid
// value only for the warp's first lane; this form is exact there.)
__device__ __forceinline__ float tex3d_fetch(unsigned long long tex, float x, float y, float z) {
    float v[4];
    asm volatile("tex.3d.v4.f32.f32 {%0, %1, %2, %3}, [%4, {%5, %6, %7, %8}];"
                 : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3])
                 : "l"(tex), "f"(x), "f"(y), "f"(z), "f"(0.f));
    return v[0];   // a one-channel texture: the value is the first component
}

// Extra radius for the bounding-volume culls under the texture lookup: the filtered
// value is the exact interpolant at a point within sqrt(3) h / 256 of the query,
// so the link's lower bound holds after growing its bounding volume by that much.
__device__ __forceinline__ float tex_cull_pad(float h) { return 1.7320509f * h * (1.0f / 256.0f) * 1.001f; }

}  // namespace dev
}  // namespace sdf
