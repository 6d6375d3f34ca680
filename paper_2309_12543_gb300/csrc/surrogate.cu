// Learned link-SDF surrogate on the fifth-generation tensor cores (tcgen05).
//
// No counterpart in the paper, whose only network approximates its grid transform
// (Eq. (5)).  Here one small network per link stands in for the link's grid lookup
// (Sec. III-A): f(x) = w4 . s(W3 s(W2 s(W1 x + b1) + b2) + b3) + b4, s = SiLU,
// hidden width 128, x = (p_loc - m) / a the link-frame point normalised to the
// grid box (centre m, half-span a), distance = a f(x), and outside the box the
// grid path's rule (distance to the box + value at the nearest box point).
//
// The two 128 x 128 layers run as tcgen05 MMAs (bf16 operands from shared memory,
// f32 accumulators in tensor memory); the 3-wide input layer and the 1-wide output
// layer run on the FP32 cores.  Training (mean absolute error, Adam) runs one CTA
// per link, one 128-sample batch per step; every product of the backward pass is a
// tcgen05 MMA as well:
//   dH2 = dZ3 W3,  dW3 = dZ3^T H2,  db3 = dZ3^T 1,  dw4 = H3^T g
//   dH1 = dZ2 W2,  dW2 = dZ2^T H1,  db2 = dZ2^T 1,  [dW1 db1] = dZ1^T [x 1]
// with all operands bf16.  Tensor memory (512 columns of 128 lanes) holds
//   [0,128)   Z2, then dH1           [128,256) Z3, then dH2, then dW2
//   [256,384) dW3                     [384,448) four 16-column small products
// Master weights, Adam moments and step counts stay in FP32 in device memory; the
// 128 x 128 blocks are stored transposed there ([in][out]) so that the thread of
// output unit o reads them coalesced.
//
// The training samples come from a counter-based generator (Philox4x32-10,
// Salmon et al., SC'11) and are labelled by the link's grid.
#include <atomic>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"
#include "lookup.cuh"
#include "tc.cuh"

namespace sdf {
namespace {

using namespace dev;

constexpr int kH = SDF_MLP_HIDDEN;
constexpr int kPar = SDF_MLP_PARAMS;
constexpr int kOW1 = 0, kOB1 = 384, kOW2 = 512, kOB2 = kOW2 + kH * kH, kOW3 = kOB2 + kH, kOB3 = kOW3 + kH * kH,
              kOW4 = kOB3 + kH, kOB4 = kOW4 + kH;
static_assert(kOB4 + 1 == kPar, "parameter layout");
// Floats between consecutive links' parameters (and Adam moments) in device memory:
// kPar rounded up to 16, so that every link's block starts 64-byte aligned.
constexpr int kParStride = (kPar + 15) & ~15;

constexpr int kTileBytes = kH * kH * 2;        // one 128 x 128 bf16 operand tile
constexpr int kAuxCols = 16;                    // [x0 x1 x2 1 g 0 ...] per sample
constexpr int kAuxBytes = kH * kAuxCols * 2;
constexpr uint32_t kWaitPolls = 1u << 22;   // drain wait after a timeout (MMAs in flight end)

// training kernel shared memory (dynamic part)
constexpr int kSW2 = 0, kSW3 = kTileBytes, kSH1 = 2 * kTileBytes, kSH2 = 3 * kTileBytes, kSDZ = 4 * kTileBytes,
              kSH3 = 5 * kTileBytes, kSAux = 6 * kTileBytes, kSSmall = kSAux + kAuxBytes;
constexpr int kSmallFloats = 384 + 4 * kH + 4;  // W1, b1, b2, b3, w4, b4 (+pad)
constexpr int kTrainSmem = kSSmall + kSmallFloats * 4;
// evaluation kernel shared memory: W2 and W3 of the current link, then one activation
// tile per warpgroup pipeline (H1 and H2 of its tile in turn), then the small parameters
constexpr int kEvalPipes = 4;   // warpgroups of an evaluation CTA, each on its own 128-query tile
constexpr int kEW2 = 0, kEW3 = kTileBytes, kEH = 2 * kTileBytes, kESmall = kEH + kEvalPipes * kTileBytes;
constexpr int kEvalSmem = kESmall + kSmallFloats * 4;

// tensor-memory columns
constexpr uint32_t kTZ2 = 0, kTZ3 = 128, kTDW3 = 256, kTS3 = 384, kTS2 = 400, kTS1 = 416, kTS4 = 432;

// K-major operand of a 128-column tile: K-direction stride 128 B, row groups 2048 B,
// 16 K-elements per MMA = 256 B.  MN-major: K-direction stride = row groups.
constexpr uint32_t kRowGroup = 2048, kAuxRowGroup = 256;

// Logistic function with the fast exponential and division intrinsics (a few ulp;
// the results are rounded to bfloat16 or compared at ~1e-3 anyway).  For z below
// about -88 the exponential overflows and the quotient is 0.
__device__ __forceinline__ float silu_sigma(float z) { return __fdividef(1.0f, 1.0f + __expf(-z)); }

// SiLU for the evaluation kernels, from sigma(z) = (1 + tanh(z / 2)) / 2:
//   SiLU(z) = z sigma(z) = u (1 + tanh u) = u + u tanh u,   u = z / 2,
// one tanh.approx on the transcendental (XU) pipe and one FMA, where the exponential
// and reciprocal form takes about eleven issue slots.  The evaluation layout of the
// small parameters holds W1, b1, b2 and b3 halved (exact: a power of two), so that u
// comes out of the same FMAs that formed z.  tanh.approx.f32 is documented with a
// maximum relative error near 2^-11, so |error| <= |u| 2^-11 = |z| 2^-12: below half
// a bfloat16 unit of the result for z > 0, and at most 2.5e-4 |z| in absolute terms
// for z < 0, where the result tends to 0.  (Large negative u gives tanh = -1 and a
// result of exactly 0.)
__device__ __forceinline__ float tanh_xu(float x) {
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float silu_half(float u) { return fmaf(u, tanh_xu(u), u); }

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}
// 8 consecutive columns (one 16-byte core-matrix row) of a tile row.
__device__ __forceinline__ void store_bf16x8(uint8_t* tile, int row, int col0, int cols, const float* v) {
    uint4 u;
    u.x = pack_bf16x2(v[0], v[1]);
    u.y = pack_bf16x2(v[2], v[3]);
    u.z = pack_bf16x2(v[4], v[5]);
    u.w = pack_bf16x2(v[6], v[7]);
    *reinterpret_cast<uint4*>(tile + tc::tile_offset(row, col0, cols)) = u;
}

// All threads' shared-memory writes become visible to the tensor core, and the
// tensor-memory reads before this point are ordered before the next MMA.
__device__ __forceinline__ void sync_for_mma() {
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
}

// Wait for the MMA batch just committed, at most `limit` polls (SDF_OPT_WAIT_POLLS);
// the block agrees on the outcome.
__device__ __forceinline__ bool wait_mma(uint64_t* mbar, uint32_t& phase, uint32_t limit) {
    const bool ok = tc::mbar_wait(mbar, phase, limit);
    phase ^= 1u;
    tc::fence_after_sync();
    return __syncthreads_and(ok) != 0;
}

// One K=128 product: 8 MMAs of K = 16.
__device__ __forceinline__ void mma_k128(uint32_t d, uint32_t a_addr, uint32_t a_lbo, uint32_t a_sbo, uint32_t a_step,
                                         uint32_t b_addr, uint32_t b_lbo, uint32_t b_sbo, uint32_t b_step,
                                         uint32_t idesc) {
#pragma unroll
    for (int k = 0; k < 8; ++k)
        tc::mma_bf16(d, tc::smem_desc(a_addr + k * a_step, a_lbo, a_sbo), tc::smem_desc(b_addr + k * b_step, b_lbo, b_sbo),
                     idesc, k > 0);
}

// Operand roles of a 128-column tile T (rows r, 8-element chunks along columns):
//   K-major, M/N = rows, K = columns:  lbo 128, sbo 2048, step 256
//   MN-major, K = rows, M/N = columns: lbo 2048, sbo 128, step 4096
#define KMAJ(addr) (addr), 128u, kRowGroup, 256u
#define MNMAJ(addr) (addr), kRowGroup, 128u, 2u * kRowGroup
#define AUXMN(addr) (addr), kAuxRowGroup, 128u, 2u * kAuxRowGroup

// Load one link's weights: the W2/W3 blocks (stored [in][out]) into K-major bf16
// tiles [out][in], the small parameters into FP32.  All `nthreads` threads help;
// consecutive threads read consecutive output units (coalesced).
// Small parameters in the evaluation kernels' layout: (W1 row j, b1 j) as one float4
// per unit, then b2, b3, w4 and b4, so that each is read with 16-byte loads.  W1, b1,
// b2 and b3 are halved (the evaluation forms z / 2; see silu_half).
constexpr int kEWB = 0, kEB2 = 4 * kH, kEB3 = 5 * kH, kEW4 = 6 * kH, kEB4 = 7 * kH;
static_assert(kEB4 + 1 <= kSmallFloats, "evaluation layout of the small parameters");

template <bool kEvalLayout = false>
__device__ __forceinline__ void load_weights(const float* __restrict__ P, uint8_t* w2, uint8_t* w3, float* small,
                                             int t, int nthreads) {
    constexpr int kChunks = kH * (kH / 8);   // 8-element row chunks per block
    for (int idx = t; idx < 2 * kChunks; idx += nthreads) {
        const int blk = idx / kChunks, rem = idx % kChunks;
        const int o = rem % kH, i0 = (rem / kH) * 8;
        const float* src = P + (blk == 0 ? kOW2 : kOW3);
        float v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = src[(i0 + k) * kH + o];
        store_bf16x8(blk == 0 ? w2 : w3, o, i0, kH, v);
    }
    if constexpr (kEvalLayout) {
        for (int i = t; i < kH; i += nthreads) {
            reinterpret_cast<float4*>(small + kEWB)[i] = make_float4(0.5f * P[kOW1 + 3 * i], 0.5f * P[kOW1 + 3 * i + 1],
                                                                     0.5f * P[kOW1 + 3 * i + 2], 0.5f * P[kOB1 + i]);
            small[kEB2 + i] = 0.5f * P[kOB2 + i];
            small[kEB3 + i] = 0.5f * P[kOB3 + i];
            small[kEW4 + i] = P[kOW4 + i];
        }
        if (t == 0) small[kEB4] = P[kOB4];
    } else {
        for (int i = t; i < 384; i += nthreads) small[i] = P[kOW1 + i];
        for (int i = t; i < kH; i += nthreads) {
            small[384 + i] = P[kOB1 + i];
            small[384 + kH + i] = P[kOB2 + i];
            small[384 + 2 * kH + i] = P[kOB3 + i];
            small[384 + 3 * kH + i] = P[kOW4 + i];
        }
        if (t == 0) small[384 + 4 * kH] = P[kOB4];
    }
}

// The training kernel's CTA: four warpgroups over one 128-sample batch.  Thread
// (g, r) = (t / 128, t % 128) holds sample r (tensor-memory lane r) in the forward and
// backward passes and output unit r in the update, and takes the 32 columns
// [32 g, 32 g + 32) of every 128-column product: its layer-1 units, its share of
// each epilogue, and the inputs of unit r whose W2/W3 weights it updates.  Four warps
// per SM sub-partition instead of one hide the latency of each other's dependent
// instructions; the batch and the order of the step are those of one 128-thread CTA.
constexpr int kTrainGroups = 4;
constexpr int kTrainThreads = 128 * kTrainGroups;
constexpr int kTrainCols = kH / kTrainGroups;   // 32
static_assert(kTrainCols == 32, "one 32-column tensor-memory load per epilogue share");

// Layer 1 of sample `row`, units [c0, c0 + 32), into the H1 tile (bf16).
__device__ __forceinline__ void layer1(const float* small, float x0, float x1, float x2, uint8_t* h1, int row,
                                       int c0) {
    const float* W1 = small;
    const float* b1 = small + 384;
#pragma unroll 1
    for (int j0 = c0; j0 < c0 + kTrainCols; j0 += 8) {
        float h[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int j = j0 + k;
            const float z = fmaf(W1[3 * j], x0, fmaf(W1[3 * j + 1], x1, fmaf(W1[3 * j + 2], x2, b1[j])));
            h[k] = z * silu_sigma(z);
        }
        store_bf16x8(h1, row, j0, kH, h);
    }
}

// Hidden layer epilogue: s(D + b) of columns [c0, c0 + 32) of this thread's lane into
// row `row` of tile out.
__device__ __forceinline__ void hidden_epilogue(uint32_t taddr, const float* b, uint8_t* out, int row, int c0) {
    float v[32];
    tc::tmem_ld32(taddr + c0, v);
#pragma unroll
    for (int k = 0; k < 32; k += 8) {
        float h[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const float z = v[k + e] + b[c0 + k + e];
            h[e] = z * silu_sigma(z);
        }
        store_bf16x8(out, row, c0 + k, kH, h);
    }
}

// ------------------------------------------------------------------ training

struct TrainArgs {
    float* master;            // [L][kParStride], W2/W3 blocks [in][out]
    float* adam_m;
    float* adam_v;
    int* step;                // [L] Adam steps taken
    const float* x;           // [L][n][3] normalised inputs
    const float* y;           // [L][n] normalised labels
    long long n;
    long long batch0;         // step s uses samples ((batch0 + s) * 128 + j) mod n
    int steps;
    int link0;
    float lr, beta1, beta2, eps;
    float* grad_out;          // gradient mode: [kPar] in the public layout (no update)
    float* loss_out;          // [L]: sum over the steps of the batch loss
    int* status;
    uint32_t wait_polls;      // polls of an MMA completion wait before it gives up
};

__global__ void __launch_bounds__(kTrainThreads, 1) mlp_train_kernel(const __grid_constant__ TrainArgs A) {
    extern __shared__ __align__(1024) uint8_t sm[];
    __shared__ uint64_t mbar;
    __shared__ uint32_t tmem_slot;
    __shared__ float red[2][4];
    __shared__ float red_f[kTrainGroups][kH];   // each warpgroup's share of the output sums
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int grp = t >> 7, r = t & 127, c0 = grp * kTrainCols;
    const int link = A.link0 + blockIdx.x;
    float* P = A.master + (size_t)link * kParStride;
    uint8_t* sW2 = sm + kSW2;
    uint8_t* sW3 = sm + kSW3;
    uint8_t* sH1 = sm + kSH1;
    uint8_t* sH2 = sm + kSH2;
    uint8_t* sDZ = sm + kSDZ;
    uint8_t* sH3 = sm + kSH3;
    uint8_t* sAux = sm + kSAux;
    float* small = reinterpret_cast<float*>(sm + kSSmall);
    const float* W1 = small;
    const float* b1 = small + 384;
    const float* b2 = small + 384 + kH;
    const float* b3 = small + 384 + 2 * kH;
    const float* w4 = small + 384 + 3 * kH;

    load_weights(P, sW2, sW3, small, t, kTrainThreads);
    if (warp == 0) tc::tmem_alloc(&tmem_slot, 512);
    if (t == 0) tc::mbar_init(&mbar, 1);
    sync_for_mma();
    const uint32_t tm = tmem_slot;
    const uint32_t lane_addr = tm + ((uint32_t)((warp & 3) * 32) << 16);
    const uint32_t aW2 = tc::smem_u32(sW2), aW3 = tc::smem_u32(sW3), aH1 = tc::smem_u32(sH1),
                   aH2 = tc::smem_u32(sH2), aDZ = tc::smem_u32(sDZ), aH3 = tc::smem_u32(sH3),
                   aAux = tc::smem_u32(sAux);
    constexpr uint32_t kN128KK = tc::idesc_bf16(128, 128, 0, 0);   // A K-major, B K-major
    constexpr uint32_t kN128KM = tc::idesc_bf16(128, 128, 0, 1);   // A K-major, B MN-major
    constexpr uint32_t kN128MM = tc::idesc_bf16(128, 128, 1, 1);
    constexpr uint32_t kN16MM = tc::idesc_bf16(128, 16, 1, 1);
    uint32_t phase = 0;
    bool ok = true;
    float loss_sum = 0.f;
    // sample r of step s, loaded one step ahead
    auto load_sample = [&](int step, float& a0, float& a1, float& a2, float& ay) {
        const long long idx = ((A.batch0 + step) * 128 + r) % A.n;
        const float* xs = A.x + ((size_t)link * A.n + idx) * 3;
        a0 = xs[0];
        a1 = xs[1];
        a2 = xs[2];
        ay = A.y[(size_t)link * A.n + idx];
    };
    float nx0 = 0.f, nx1 = 0.f, nx2 = 0.f, ny = 0.f;
    if (A.steps > 0) load_sample(0, nx0, nx1, nx2, ny);
    // Adam (Kingma & Ba, Algorithm 1) on the FP32 master weights
    const float b1c = A.beta1, b2c = A.beta2, lr = A.lr, eps = A.eps;
    float* M = A.adam_m + (size_t)link * kParStride;
    float* V = A.adam_v + (size_t)link * kParStride;
    // one 128 x 128 block (gradient in tensor-memory columns `col`, lane = output unit
    // o = r): this thread's inputs [c0, c0 + 32), 16 at a time with their loads issued
    // together (consecutive threads, consecutive outputs: coalesced in the [in][out]
    // master layout); the new weights go to the bf16 operand tile
    auto adam_block = [&](uint32_t col, int base, uint8_t* tile, int step) {
        const int o = r;
        const int ts = A.step[link] + step + 1;
        const float c1 = 1.f - powf(b1c, (float)ts), c2 = 1.f - powf(b2c, (float)ts);
        float* __restrict__ Pr = P;
        float* __restrict__ Mr = M;
        float* __restrict__ Vr = V;
#pragma unroll 1
        for (int cc = c0; cc < c0 + kTrainCols; cc += 16) {
            float gr[16], pm[16], pv[16], pp[16];
            tc::tmem_ld16(lane_addr + col + cc, gr);
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                const int i = base + (cc + e) * kH + o;
                pm[e] = Mr[i];
                pv[e] = Vr[i];
                pp[e] = Pr[i];
            }
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                const int i = base + (cc + e) * kH + o;
                const float m = fmaf(b1c, pm[e], (1.f - b1c) * gr[e]);
                const float v = fmaf(b2c, pv[e], (1.f - b2c) * gr[e] * gr[e]);
                const float p = pp[e] - lr * (m / c1) / (sqrtf(v / c2) + eps);
                Mr[i] = m;
                Vr[i] = v;
                Pr[i] = p;
                pp[e] = p;
            }
            store_bf16x8(tile, o, cc, kH, pp);
            store_bf16x8(tile, o, cc + 8, kH, pp + 8);
        }
    };

    for (int s = 0; s < A.steps && ok; ++s) {
        // ---- the batch: sample r of this step
        const float x0 = nx0, x1 = nx1, x2 = nx2, yv = ny;
        if (s + 1 < A.steps) load_sample(s + 1, nx0, nx1, nx2, ny);
        if (grp == 0) {
            const float aux[8] = {x0, x1, x2, 1.f, 0.f, 0.f, 0.f, 0.f};
            const float zero[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            store_bf16x8(sAux, r, 0, kAuxCols, aux);
            store_bf16x8(sAux, r, 8, kAuxCols, zero);
        }
        // ---- forward
        layer1(small, x0, x1, x2, sH1, r, c0);
        sync_for_mma();
        if (t == 0) {
            mma_k128(tm + kTZ2, KMAJ(aH1), KMAJ(aW2), kN128KK);
            tc::mma_commit(&mbar);
        }
        if (!(ok = wait_mma(&mbar, phase, A.wait_polls))) break;
        hidden_epilogue(lane_addr + kTZ2, b2, sH2, r, c0);
        sync_for_mma();
        if (t == 0) {
            mma_k128(tm + kTZ3, KMAJ(aH2), KMAJ(aW3), kN128KK);
            tc::mma_commit(&mbar);
        }
        if (!(ok = wait_mma(&mbar, phase, A.wait_polls))) break;
        // output layer: this warpgroup's share of f, then f and the loss gradient
        // g = sign(f - y) / 128
        {
            float v[32];
            float fp = 0.f;
            tc::tmem_ld32(lane_addr + kTZ3 + c0, v);
#pragma unroll
            for (int k = 0; k < 32; k += 8) {
                float h[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const float z = v[k + e] + b3[c0 + k + e];
                    h[e] = z * silu_sigma(z);
                    fp = fmaf(w4[c0 + k + e], h[e], fp);
                }
                store_bf16x8(sH3, r, c0 + k, kH, h);
            }
            red_f[grp][r] = fp;
        }
        __syncthreads();
        float f = small[384 + 4 * kH];
#pragma unroll
        for (int q = 0; q < kTrainGroups; ++q) f += red_f[q][r];
        const float res = f - yv;
        const float g = res > 0.f ? (1.f / 128.f) : (res < 0.f ? -(1.f / 128.f) : 0.f);
        if (grp == 0) {
            const float aux[8] = {x0, x1, x2, 1.f, g, 0.f, 0.f, 0.f};
            store_bf16x8(sAux, r, 0, kAuxCols, aux);
        }
        // dz3 = g w4 s'(z3)
        {
            float v[32];
            tc::tmem_ld32(lane_addr + kTZ3 + c0, v);
#pragma unroll
            for (int k = 0; k < 32; k += 8) {
                float d[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const float z = v[k + e] + b3[c0 + k + e];
                    const float sg = silu_sigma(z);
                    d[e] = g * w4[c0 + k + e] * (sg * fmaf(z, 1.f - sg, 1.f));
                }
                store_bf16x8(sDZ, r, c0 + k, kH, d);
            }
        }
        // batch loss and db4 = sum g (warpgroup 0 holds one copy of each sample)
        if (grp == 0) {
            float la = fabsf(res), lg = g;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                la += __shfl_xor_sync(0xffffffffu, la, o);
                lg += __shfl_xor_sync(0xffffffffu, lg, o);
            }
            if (lane == 0) {
                red[0][warp] = la;
                red[1][warp] = lg;
            }
        }
        sync_for_mma();
        if (t == 0) {
            mma_k128(tm + kTZ3, KMAJ(aDZ), MNMAJ(aW3), kN128KM);     // dH2 = dZ3 W3
            mma_k128(tm + kTDW3, MNMAJ(aDZ), MNMAJ(aH2), kN128MM);   // dW3 = dZ3^T H2
            mma_k128(tm + kTS3, MNMAJ(aDZ), AUXMN(aAux), kN16MM);    // db3 (column 3)
            mma_k128(tm + kTS4, MNMAJ(aH3), AUXMN(aAux), kN16MM);    // dw4 (column 4)
            tc::mma_commit(&mbar);
        }
        if (!(ok = wait_mma(&mbar, phase, A.wait_polls))) break;
        // dz2 = dH2 s'(z2)
        {
            float dh[32], zz[32];
            tc::tmem_ld32(lane_addr + kTZ3 + c0, dh);
            tc::tmem_ld32(lane_addr + kTZ2 + c0, zz);
#pragma unroll
            for (int k = 0; k < 32; k += 8) {
                float d[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const float z = zz[k + e] + b2[c0 + k + e];
                    const float sg = silu_sigma(z);
                    d[e] = dh[k + e] * (sg * fmaf(z, 1.f - sg, 1.f));
                }
                store_bf16x8(sDZ, r, c0 + k, kH, d);
            }
        }
        sync_for_mma();
        if (t == 0) {
            mma_k128(tm + kTZ2, KMAJ(aDZ), MNMAJ(aW2), kN128KM);     // dH1 = dZ2 W2
            mma_k128(tm + kTZ3, MNMAJ(aDZ), MNMAJ(aH1), kN128MM);    // dW2 = dZ2^T H1
            mma_k128(tm + kTS2, MNMAJ(aDZ), AUXMN(aAux), kN16MM);    // db2 (column 3)
            tc::mma_commit(&mbar);
        }
        // W3's update while these products run (they read neither W3 nor dW3)
        if (!A.grad_out) adam_block(kTDW3, kOW3, sW3, s);
        if (!(ok = wait_mma(&mbar, phase, A.wait_polls))) break;
        // dz1 = dH1 s'(z1), z1 recomputed
        {
            float dh[32];
            tc::tmem_ld32(lane_addr + kTZ2 + c0, dh);
#pragma unroll
            for (int k = 0; k < 32; k += 8) {
                float d[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const int j = c0 + k + e;
                    const float z = fmaf(W1[3 * j], x0, fmaf(W1[3 * j + 1], x1, fmaf(W1[3 * j + 2], x2, b1[j])));
                    const float sg = silu_sigma(z);
                    d[e] = dh[k + e] * (sg * fmaf(z, 1.f - sg, 1.f));
                }
                store_bf16x8(sDZ, r, c0 + k, kH, d);
            }
        }
        sync_for_mma();
        if (t == 0) {
            mma_k128(tm + kTS1, MNMAJ(aDZ), AUXMN(aAux), kN16MM);    // [dW1 db1] (columns 0..3)
            tc::mma_commit(&mbar);
        }
        // W2's update while this product runs (it reads neither W2 nor dW2)
        if (!A.grad_out) adam_block(kTZ3, kOW2, sW2, s);
        if (!(ok = wait_mma(&mbar, phase, A.wait_polls))) break;
        const float batch_loss = (red[0][0] + red[0][1] + red[0][2] + red[0][3]) * (1.f / 128.f);
        const float db4 = red[1][0] + red[1][1] + red[1][2] + red[1][3];
        loss_sum += batch_loss;

        // ---- gradients of output unit o = r (W2/W3 inputs [c0, c0 + 32) here; the
        // small parameters by warpgroup 0), then the update
        const int o = r;
        float s1[16], s2[16], s3[16], s4[16];   // the small parameters' gradient columns
        auto load_small_grads = [&]() {
            tc::tmem_ld16(lane_addr + kTS1, s1);
            tc::tmem_ld16(lane_addr + kTS2, s2);
            tc::tmem_ld16(lane_addr + kTS3, s3);
            tc::tmem_ld16(lane_addr + kTS4, s4);
        };
        if (A.grad_out) {
            float* G = A.grad_out;
            float v[32];
            tc::tmem_ld32(lane_addr + kTZ3 + c0, v);
            for (int k = 0; k < 32; ++k) G[kOW2 + o * kH + c0 + k] = v[k];
            tc::tmem_ld32(lane_addr + kTDW3 + c0, v);
            for (int k = 0; k < 32; ++k) G[kOW3 + o * kH + c0 + k] = v[k];
            if (grp == 0) {
                load_small_grads();
                G[kOW1 + 3 * o] = s1[0];
                G[kOW1 + 3 * o + 1] = s1[1];
                G[kOW1 + 3 * o + 2] = s1[2];
                G[kOB1 + o] = s1[3];
                G[kOB2 + o] = s2[3];
                G[kOB3 + o] = s3[3];
                G[kOW4 + o] = s4[4];
                if (o == 0) G[kOB4] = db4;
            }
            break;   // gradient mode: one batch, no update
        }
        // Adam on the small parameters
        const int tstep = A.step[link] + s + 1;
        const float bc1 = 1.f - powf(A.beta1, (float)tstep), bc2 = 1.f - powf(A.beta2, (float)tstep);
        auto adam = [&](int i, float gr) -> float {
            const float m = fmaf(b1c, M[i], (1.f - b1c) * gr);
            const float v = fmaf(b2c, V[i], (1.f - b2c) * gr * gr);
            M[i] = m;
            V[i] = v;
            const float p = P[i] - lr * (m / bc1) / (sqrtf(v / bc2) + eps);
            P[i] = p;
            return p;
        };
        float nw[7];
        float nb4 = 0.f;
        if (grp == 0) {
            load_small_grads();
            nw[0] = adam(kOW1 + 3 * o, s1[0]);
            nw[1] = adam(kOW1 + 3 * o + 1, s1[1]);
            nw[2] = adam(kOW1 + 3 * o + 2, s1[2]);
            nw[3] = adam(kOB1 + o, s1[3]);
            nw[4] = adam(kOB2 + o, s2[3]);
            nw[5] = adam(kOB3 + o, s3[3]);
            nw[6] = adam(kOW4 + o, s4[4]);
            if (o == 0) nb4 = adam(kOB4, db4);
        }
        __syncthreads();   // every thread is done reading the small parameters of this step
        if (grp == 0) {
            small[3 * o] = nw[0];
            small[3 * o + 1] = nw[1];
            small[3 * o + 2] = nw[2];
            small[384 + o] = nw[3];
            small[384 + kH + o] = nw[4];
            small[384 + 2 * kH + o] = nw[5];
            small[384 + 3 * kH + o] = nw[6];
            if (o == 0) small[384 + 4 * kH] = nb4;
        }
        // the next step reads the new small parameters; its first MMA is preceded by
        // sync_for_mma, which publishes the rewritten weight tiles to the tensor core
        __syncthreads();
    }
    if (!ok) {
        if (t == 0) atomicOr(A.status, kStatusTimeout);
        tc::mbar_wait(&mbar, phase ^ 1u, kWaitPolls);   // give an MMA still in flight time to end
    }
    if (t == 0) {
        if (A.loss_out) A.loss_out[link] = (A.grad_out ? 0.f : A.loss_out[link]) + loss_sum;
        if (!A.grad_out && ok) A.step[link] += A.steps;
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_free(tm, 512);
}

// ------------------------------------------------------------------ evaluation

struct EvalArgs {
    const float* master;               // [L][kParStride]
    const float* x3;                   // n x 3 normalised points
    int L;
    int n;                             // queries of link `link0`
    int link0;
    float* f_out;                      // f(x) (normalised)
    int* status;
    uint32_t wait_polls;               // polls of an MMA completion wait before it gives up
};

constexpr int kEvalThreads = 128 * kEvalPipes;

// Named barrier of one warpgroup (ids 1..4; id 0 is __syncthreads).
__device__ __forceinline__ void pipe_sync(int pipe) {
    asm volatile("bar.sync %0, 128;" ::"r"(pipe + 1) : "memory");
}
// Warpgroup-wide AND of a flag.
__device__ __forceinline__ bool pipe_all(int pipe, bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.and.pred q, %2, 128, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}\n"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(pipe + 1)
        : "memory");
    return r != 0;
}
// Shared-memory writes of the warpgroup become visible to the tensor core, and its
// tensor-memory reads are ordered before the next MMA.
__device__ __forceinline__ void pipe_sync_for_mma(int pipe) {
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    pipe_sync(pipe);
    tc::fence_after_sync();
}

// One hidden layer's epilogue on this thread's tensor-memory lane: s(D + b) of the
// 128 units into row r of the activation tile H (bf16).  bh = b / 2, 16-byte aligned.
__device__ __forceinline__ void pipe_hidden(uint32_t taddr, const float* bh, uint8_t* H, int r) {
#pragma unroll 1
    for (int c0 = 0; c0 < kH; c0 += 32) {
        float v[32];
        tc::tmem_ld32(taddr + c0, v);
#pragma unroll
        for (int k = 0; k < 32; k += 8) {
            const float4 b0 = *reinterpret_cast<const float4*>(bh + c0 + k);
            const float4 b1 = *reinterpret_cast<const float4*>(bh + c0 + k + 4);
            float h[8];
            h[0] = silu_half(fmaf(0.5f, v[k + 0], b0.x));
            h[1] = silu_half(fmaf(0.5f, v[k + 1], b0.y));
            h[2] = silu_half(fmaf(0.5f, v[k + 2], b0.z));
            h[3] = silu_half(fmaf(0.5f, v[k + 3], b0.w));
            h[4] = silu_half(fmaf(0.5f, v[k + 4], b1.x));
            h[5] = silu_half(fmaf(0.5f, v[k + 5], b1.y));
            h[6] = silu_half(fmaf(0.5f, v[k + 6], b1.z));
            h[7] = silu_half(fmaf(0.5f, v[k + 7], b1.w));
            store_bf16x8(H, r, c0 + k, kH, h);
        }
    }
}

// The network at one query per thread of a warpgroup (thread r = query row r =
// tensor-memory lane r): layer 1 and the epilogues on the FP32 cores, the two
// 128 x 128 layers as tcgen05 MMAs into this pipeline's 128 tensor-memory columns
// (Z2, then Z3 in the same columns).  H holds H1, then H2 (each MMA has finished
// reading its operand before the next write).  `small` is in the evaluation layout.
// Returns false if an MMA wait gave up (the pipeline agrees on it); f is valid
// otherwise.
__device__ __forceinline__ bool pipe_network(int pipe, int r, const float* small, uint8_t* H, uint32_t aH,
                                             uint32_t aW2, uint32_t aW3, uint32_t d_tmem, uint32_t taddr,
                                             uint64_t* mbar, uint32_t& phase, uint32_t limit, float4 x, float& f) {
    const float4* wb = reinterpret_cast<const float4*>(small + kEWB);
    const float* b3 = small + kEB3;
    const float* w4 = small + kEW4;
    constexpr uint32_t kN128KK = tc::idesc_bf16(128, 128, 0, 0);
#pragma unroll 1
    for (int j0 = 0; j0 < kH; j0 += 8) {
        float h[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const float4 w = wb[j0 + e];
            const float u = fmaf(w.x, x.x, fmaf(w.y, x.y, fmaf(w.z, x.z, w.w)));   // z / 2
            h[e] = silu_half(u);
        }
        store_bf16x8(H, r, j0, kH, h);
    }
    pipe_sync_for_mma(pipe);
    if (r == 0) {
        mma_k128(d_tmem, KMAJ(aH), KMAJ(aW2), kN128KK);
        tc::mma_commit(mbar);
    }
    bool ok = tc::mbar_wait(mbar, phase, limit);
    phase ^= 1u;
    tc::fence_after_sync();
    if (!pipe_all(pipe, ok)) return false;
    pipe_hidden(taddr, small + kEB2, H, r);
    pipe_sync_for_mma(pipe);
    if (r == 0) {
        mma_k128(d_tmem, KMAJ(aH), KMAJ(aW3), kN128KK);
        tc::mma_commit(mbar);
    }
    ok = tc::mbar_wait(mbar, phase, limit);
    phase ^= 1u;
    tc::fence_after_sync();
    if (!pipe_all(pipe, ok)) return false;
    float acc = small[kEB4];
#pragma unroll 1
    for (int c0 = 0; c0 < kH; c0 += 32) {
        float v[32];
        tc::tmem_ld32(taddr + c0, v);
#pragma unroll
        for (int k = 0; k < 32; k += 4) {
            const float4 b = *reinterpret_cast<const float4*>(b3 + c0 + k);
            const float4 w = *reinterpret_cast<const float4*>(w4 + c0 + k);
            acc = fmaf(w.x, silu_half(fmaf(0.5f, v[k + 0], b.x)), acc);
            acc = fmaf(w.y, silu_half(fmaf(0.5f, v[k + 1], b.y)), acc);
            acc = fmaf(w.z, silu_half(fmaf(0.5f, v[k + 2], b.z)), acc);
            acc = fmaf(w.w, silu_half(fmaf(0.5f, v[k + 3], b.w)), acc);
        }
    }
    f = acc;
    // the tensor-memory reads above come before the next tile's first MMA
    tc::fence_before_sync();
    return true;
}

// Shared-memory writes of the whole block become visible to the tensor core, and its
// tensor-memory reads are ordered before the next MMA.
__device__ __forceinline__ void block_sync_for_mma() {
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
}

// The network at one 128-query tile with all four pipelines on it: thread (p, r) takes
// row r (tensor-memory lane r) and the 32 units [32p, 32p + 32) of every layer, so that
// a lone tile runs on four warps per SM sub-partition instead of one.  The tile's
// accumulator is pipeline 0's tensor-memory columns (d_tmem0; taddr0 = this warp's lane
// quarter of them), its activations pipeline 0's tile H0; `part` (4 x 128 floats) holds
// the per-row partial sums of the output layer.  Thread 0 issues the MMAs and commits to
// `mbar`, which every thread waits on.  Returns false if an MMA wait gave up (the block
// agrees on it); f is valid in pipeline 0 otherwise.
__device__ __forceinline__ bool block_network(int pipe, int r, int t, const float* small, uint8_t* H0, uint32_t aH0,
                                              uint32_t aW2, uint32_t aW3, uint32_t d_tmem0, uint32_t taddr0,
                                              uint64_t* mbar, uint32_t& phase, uint32_t limit, float4 x,
                                              float* part, float& f) {
    const float4* wb = reinterpret_cast<const float4*>(small + kEWB);
    const int c0 = 32 * pipe;
    constexpr uint32_t kN128KK = tc::idesc_bf16(128, 128, 0, 0);
#pragma unroll 1
    for (int j0 = c0; j0 < c0 + 32; j0 += 8) {
        float h[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const float4 w = wb[j0 + e];
            h[e] = silu_half(fmaf(w.x, x.x, fmaf(w.y, x.y, fmaf(w.z, x.z, w.w))));   // z / 2
        }
        store_bf16x8(H0, r, j0, kH, h);
    }
    block_sync_for_mma();
    if (t == 0) {
        mma_k128(d_tmem0, KMAJ(aH0), KMAJ(aW2), kN128KK);
        tc::mma_commit(mbar);
    }
    bool ok = tc::mbar_wait(mbar, phase, limit);
    phase ^= 1u;
    tc::fence_after_sync();
    if (!__syncthreads_and(ok)) return false;
    {
        const float* bh = small + kEB2;
        float v[32];
        tc::tmem_ld32(taddr0 + c0, v);
#pragma unroll
        for (int k = 0; k < 32; k += 8) {
            float h[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) h[e] = silu_half(fmaf(0.5f, v[k + e], bh[c0 + k + e]));
            store_bf16x8(H0, r, c0 + k, kH, h);
        }
    }
    block_sync_for_mma();
    if (t == 0) {
        mma_k128(d_tmem0, KMAJ(aH0), KMAJ(aW3), kN128KK);
        tc::mma_commit(mbar);
    }
    ok = tc::mbar_wait(mbar, phase, limit);
    phase ^= 1u;
    tc::fence_after_sync();
    if (!__syncthreads_and(ok)) return false;
    {
        const float* b3 = small + kEB3;
        const float* w4 = small + kEW4;
        float v[32];
        tc::tmem_ld32(taddr0 + c0, v);
        float acc = 0.f;
#pragma unroll
        for (int k = 0; k < 32; ++k) acc = fmaf(w4[c0 + k], silu_half(fmaf(0.5f, v[k], b3[c0 + k])), acc);
        part[pipe * 128 + r] = acc;
    }
    // the tensor-memory reads above come before the next MMA; the partial sums are in
    tc::fence_before_sync();
    __syncthreads();
    if (pipe == 0) f = small[kEB4] + ((part[r] + part[128 + r]) + (part[256 + r] + part[384 + r]));
    return true;
}

// f(x) of one link at n points: four warpgroup pipelines per CTA, each evaluating its
// own 128-query tiles, so that one pipeline's MMA and waits overlap the others' FP32
// epilogues; the pipelines share the link's W2/W3 in shared memory.
__global__ void __launch_bounds__(kEvalThreads, 1) mlp_eval_kernel(const __grid_constant__ EvalArgs A) {
    extern __shared__ __align__(1024) uint8_t sm[];
    __shared__ uint64_t mbar[kEvalPipes];
    __shared__ uint32_t tmem_slot;
    const int t = threadIdx.x, warp = t >> 5;
    const int pipe = warp >> 2, r = t & 127;
    uint8_t* sW2 = sm + kEW2;
    uint8_t* sW3 = sm + kEW3;
    uint8_t* sH = sm + kEH + pipe * kTileBytes;
    float* small = reinterpret_cast<float*>(sm + kESmall);

    // this CTA's range of 128-query tiles
    const int total = (A.n + 127) / 128;
    const int first = (int)((long long)total * blockIdx.x / gridDim.x);
    const int last = (int)((long long)total * (blockIdx.x + 1) / gridDim.x);
    if (first >= last) return;

    if (warp == 0) tc::tmem_alloc(&tmem_slot, 512);
    if (t < kEvalPipes) tc::mbar_init(&mbar[t], 1);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tm = tmem_slot;
    const uint32_t d_tmem = tm + (uint32_t)(128 * pipe);
    const uint32_t taddr = d_tmem + ((uint32_t)((warp & 3) * 32) << 16);
    const uint32_t aW2 = tc::smem_u32(sW2), aW3 = tc::smem_u32(sW3), aH = tc::smem_u32(sH);
    uint32_t phase = 0;
    bool ok = true;
    load_weights<true>(A.master + (size_t)A.link0 * kParStride, sW2, sW3, small, t, kEvalThreads);
    tc::fence_smem_to_async();   // the weights are MMA operands
    __syncthreads();
    for (int tl = first + pipe; tl < last; tl += kEvalPipes) {
        const int k = tl * 128 + r;
        const bool valid = k < A.n;
        const float4 xq = valid ? make_float4(A.x3[3 * (size_t)k], A.x3[3 * (size_t)k + 1], A.x3[3 * (size_t)k + 2], 0.f)
                                : make_float4(0.f, 0.f, 0.f, 0.f);
        float f = 0.f;
        ok = pipe_network(pipe, r, small, sH, aH, aW2, aW3, d_tmem, taddr, &mbar[pipe], phase, A.wait_polls, xq, f);
        if (!ok) break;
        if (valid) A.f_out[k] = f;
    }
    if (!ok) {
        // a wait gave up: report it, then let the MMA still in flight end before the
        // tensor memory is released
        if (r == 0) atomicOr(A.status, kStatusTimeout);
        tc::mbar_wait(&mbar[pipe], phase ^ 1u, kWaitPolls);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_free(tm, 512);
}

// ------------------------------------------------------------------ sampler

// Philox4x32-10: 10 rounds of the multiply-xor round function with a Weyl key schedule.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

struct SampleArgs {
    const float* grid;        // the link's n^3 values
    int n;
    float4 o_ih;              // grid origin, 1/h
    float h;
    float lo[3], span[3];     // box
    float m[3], inv_a;        // centre, 1/half-span
    uint2 key;                // seed
    float band;               // near: |value| <= band (metres)
    int near10;               // samples j with j % 10 < near10 are near samples
    long long n_samples;
    long long n_near;
    float* x;                 // [n_samples][3]
    float* y;                 // [n_samples]
    long long* source;        // [n_samples] (stream << 40 | counter), may be null
    long long start;          // near stream: first candidate of this chunk
    int count;                // near stream: candidates in this chunk
    int* block_count;         // per-block accepted counts
    long long* found;         // near samples found before this chunk (device)
};

__device__ __forceinline__ void candidate(const SampleArgs& A, uint32_t stream, unsigned long long i, float* p) {
    const uint4 r = philox4x32_10(make_uint4((uint32_t)i, stream, 0u, 0u), A.key);
    const float u0 = (float)(r.x >> 8) * (1.0f / 16777216.0f);
    const float u1 = (float)(r.y >> 8) * (1.0f / 16777216.0f);
    const float u2 = (float)(r.z >> 8) * (1.0f / 16777216.0f);
    p[0] = fmaf(u0, A.span[0], A.lo[0]);
    p[1] = fmaf(u1, A.span[1], A.lo[1]);
    p[2] = fmaf(u2, A.span[2], A.lo[2]);
}

__device__ __forceinline__ void emit(const SampleArgs& A, long long j, const float* p, float g, long long src) {
    A.x[3 * j] = (p[0] - A.m[0]) * A.inv_a;
    A.x[3 * j + 1] = (p[1] - A.m[1]) * A.inv_a;
    A.x[3 * j + 2] = (p[2] - A.m[2]) * A.inv_a;
    A.y[j] = g * A.inv_a;
    if (A.source) A.source[j] = src;
}

// Uniform samples: sample j with j % 10 >= near10 is uniform candidate u of stream 1.
__global__ void sample_uniform_kernel(const __grid_constant__ SampleArgs A) {
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= A.n_samples || (int)(j % 10) < A.near10) return;
    const long long u = (j / 10) * (10 - A.near10) + (j % 10 - A.near10);
    float p[3];
    candidate(A, 1u, (unsigned long long)u, p);
    const float g = grid_lookup(A.grid, A.n, A.o_ih, A.h, p[0], p[1], p[2]);
    emit(A, j, p, g, (1ll << 40) | u);
}

__device__ __forceinline__ bool near_ok(const SampleArgs& A, long long i, float* p, float* g) {
    candidate(A, 0u, (unsigned long long)i, p);
    *g = grid_lookup(A.grid, A.n, A.o_ih, A.h, p[0], p[1], p[2]);
    return fabsf(*g) <= A.band;
}

// Near candidates: per-block counts of accepted candidates of this chunk.
__global__ void __launch_bounds__(1024) sample_count_kernel(const __grid_constant__ SampleArgs A) {
    __shared__ int cnt;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    const int i = blockIdx.x * 1024 + threadIdx.x;
    float p[3], g;
    const bool acc = i < A.count && near_ok(A, A.start + i, p, &g);
    const unsigned b = __ballot_sync(0xffffffffu, acc);
    if ((threadIdx.x & 31) == 0 && b) atomicAdd(&cnt, __popc(b));
    __syncthreads();
    if (threadIdx.x == 0) A.block_count[blockIdx.x] = cnt;
}

// Exclusive scan of the block counts (one block); the chunk's total is added to *found
// after the scatter has used the old value (scatter reads found_before).
__global__ void __launch_bounds__(1024) sample_scan_kernel(int* counts, int nb, long long* found,
                                                           long long* found_before) {
    __shared__ int part[1024];
    const int t = threadIdx.x;
    const int per = (nb + 1023) / 1024;
    int s = 0;
    for (int k = 0; k < per; ++k) {
        const int i = t * per + k;
        if (i < nb) s += counts[i];
    }
    part[t] = s;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const int v = t >= o ? part[t - o] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int run = part[t] - s;   // exclusive prefix of this thread's range
    for (int k = 0; k < per; ++k) {
        const int i = t * per + k;
        if (i < nb) {
            const int c = counts[i];
            counts[i] = run;
            run += c;
        }
    }
    if (t == 1023) {
        *found_before = *found;
        *found += part[1023];
    }
}

// Scatter accepted candidates in counter order: near sample k goes to position
// j = (k / near10) * 10 + k % near10.
__global__ void __launch_bounds__(1024) sample_scatter_kernel(const __grid_constant__ SampleArgs A,
                                                              const long long* found_before) {
    __shared__ int warp_off[32];
    const int i = blockIdx.x * 1024 + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float p[3], g = 0.f;
    const bool acc = i < A.count && near_ok(A, A.start + i, p, &g);
    const unsigned b = __ballot_sync(0xffffffffu, acc);
    if (lane == 0) warp_off[warp] = __popc(b);
    __syncthreads();
    if (warp == 0) {
        const int v = warp_off[lane];
        int incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        warp_off[lane] = incl - v;
    }
    __syncthreads();
    if (!acc) return;
    const long long k = *found_before + A.block_count[blockIdx.x] + warp_off[warp] + __popc(b & ((1u << lane) - 1u));
    if (k >= A.n_near) return;
    const long long j = (k / A.near10) * 10 + k % A.near10;
    if (j < A.n_samples) emit(A, j, p, g, A.start + i);
}

// ------------------------------------------------------------------ error measurement

__global__ void error_reduce_kernel(const float* f, const float* y, int n, float a, unsigned* max_bits,
                                    double* sum) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    float e = 0.f;
    if (i < n) e = fabsf(f[i] - y[i]) * a;
    float m = e, s = e;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(max_bits, __float_as_uint(m));   // non-negative floats order as their bits
        atomicAdd(sum, (double)s);
    }
}


// ------------------------------------------------------------------ surrogate check

// The weights of each link as the evaluation kernels hold them in shared memory: W2
// and W3 as bf16 core-matrix tiles, then the small parameters in FP32.  Made once per
// check, so that a CTA switching links copies 69 KB with 16-byte loads instead of
// converting the FP32 master weights again.
constexpr int kImgBytes = 2 * kTileBytes + kSmallFloats * 4;
static_assert(kImgBytes % 16 == 0, "16-byte copies");


__global__ void __launch_bounds__(512) weight_image_kernel(const float* __restrict__ master, uint8_t* image) {
    uint8_t* img = image + (size_t)blockIdx.x * kImgBytes;
    load_weights<true>(master + (size_t)blockIdx.x * kParStride, img, img + kTileBytes,
                 reinterpret_cast<float*>(img + 2 * kTileBytes), threadIdx.x, blockDim.x);
}

// Copy one link's image to shared memory (all threads of the CTA).
__device__ __forceinline__ void load_image(const uint8_t* __restrict__ img, uint8_t* sm_w, int t, int nthreads) {
    const uint4* src = reinterpret_cast<const uint4*>(img);
    uint4* dst = reinterpret_cast<uint4*>(sm_w);
    constexpr int kVec = kImgBytes / 16;
    for (int i = t; i < kVec; i += nthreads) dst[i] = __ldg(src + i);
}

// The check with the network in place of the grid lookup, in one persistent kernel.
// Work items, taken in order from a counter: first a seed item per (link, group of
// kSurGroup waypoints), then a cull item per (link, group), link-major, so that a CTA
// reloads its weights only when the link changes and the cull items find every
// link's seed minimum already published.
//   seed: one warp per waypoint picks the tile nearest to the link's bounding capsule
//     (nearest super-tile first), and the kSeedPts of its 32 points nearest to the
//     capsule become queries (a seed only sets the first threshold, and the 8
//     nearest points set it about as low as all 32, at a quarter of the queries);
//     the item's one tile is evaluated by all four pipelines together (block_network),
//     as is every evaluation round of one tile;
//   cull: with the waypoint's minimum so far (over all links) plus the surrogate's
//     error bound as the threshold, one warp per waypoint culls super-tiles and tiles
//     against the capsule into a (waypoint, tile) list in shared memory; then every
//     warp takes list entries, tests the tile's points against the capsule and
//     appends the survivors to a query ring in shared memory.
// Whenever the ring holds 3 tiles of 128 queries (or the list is done) the four
// warpgroup pipelines evaluate its whole tiles on the tensor cores, fold each value into the
// waypoint's packed key (ordered distance, point, link) and tighten the thresholds.
// A waypoint whose list overflowed is marked for the grid re-check, which decides it
// exactly.  Cull items take interleaved waypoints (g, g + n, ...); a waypoint already
// below margin + error bound stops being refined when its surrogate minimum is not
// wanted; each item copies the sphere tables into the idle activation tiles before its
// seed scan or culls; the last CTA to finish writes the results and re-check flags.
constexpr int kSurGroup = 16;      // waypoints per work item: one warp each in the culls
constexpr int kSurTake = 2;        // list entries a warp takes per step of the production
constexpr int kSurFill = 3 * 128;  // the production stops once the ring holds this many queries
constexpr int kSurRing = kSurFill + 16 * 32 * kSurTake;   // + what 16 warps may add past it
constexpr int kSurList = 384;      // (waypoint, tile) entries of one cull item
constexpr int kSeedPts = 8;        // seed queries per (waypoint, link): a tile's points nearest the capsule
// shared memory of the fused kernel: the link's image (W2, W3, small parameters), the
// pipelines' activation tiles, the query ring (points, tags) and the entry list
constexpr int kSurImg = 0;
constexpr int kSurH = kImgBytes;
constexpr int kSurQ = kSurH + kEvalPipes * kTileBytes;
constexpr int kSurTag = kSurQ + kSurRing * 16;
constexpr int kSurLst = kSurTag + kSurRing * 4;
constexpr int kSurSmem = kSurLst + kSurList * 4;
static_assert(kSeedPts * kSurGroup <= 128, "a seed item is one tile");
static_assert(kSurSmem + 2048 <= 232448, "dynamic + static shared memory of the fused check within 227 KB");
constexpr uint32_t kNoTag = 0xffffffffu;

struct SurFusedArgs {
    const float* poses;               // [W][L][16]: link-from-world 3x4, sphere centre (world), radius
    int W, L, group, n_groups;        // waypoints per work item (<= kSurGroup), ceil(W / group)
    const float4* sorted;             // the sorted cloud (x, y, z, original index bits)
    const float4* tiles;              // sphere per 32 sorted points
    const float4* supers;             // sphere per 32 tiles
    const int* n_valid;
    float lo[kMaxLinks][3], hi[kMaxLinks][3], m[kMaxLinks][3], inv_a[kMaxLinks], scale[kMaxLinks];
    float4 cap_a[kMaxLinks], cap_b[kMaxLinks];   // bounding capsules (link frame), radius in cap_a.w
    const uint8_t* image;             // [L][kImgBytes] weights as held in shared memory
    int seed_group;                   // waypoints per seed item (16: one tile of kSeedPts each)
    unsigned long long* keys;         // [W] packed keys, ~0 = none (set before the launch)
    uint8_t* recheck;                 // [W] 1 where a list overflowed (zeroed before the launch)
    int* work;                        // [0] item counter, [1] CTAs done (zeroed before the launch)
    float limit;                      // margin + error bound: below it the grid re-checks
    float* dist;                      // [W] results (the grid re-check overwrites its waypoints)
    int32_t* arg_link;
    int32_t* arg_point;
    float* sur_dist;                  // [W] surrogate minima, or null
    uint8_t* recheck_out;             // [W] re-check flags for the caller, or null
    float slack;                      // error bound of the surrogate + rounding slack
    float decided_below;              // a waypoint whose minimum so far is below this (margin +
                                      // error bound) is decided by the grid re-check, whatever
                                      // its final surrogate minimum: its culls stop (-inf: never,
                                      // when the caller wants the surrogate minimum itself)
    int* status;
    uint32_t wait_polls;
    unsigned long long* stats;        // statistics counters or null
};

// Distance from sphere s (centre, radius) to the segment A + t D (D.w = 1/|D|^2),
// minus the sphere's radius.
__device__ __forceinline__ float capsule_gap(float4 s, float4 A, float4 D) {
    const float px = s.x - A.x, py = s.y - A.y, pz = s.z - A.z;
    const float t = fminf(fmaxf(fmaf(px, D.x, fmaf(py, D.y, pz * D.z)) * D.w, 0.f), 1.f);
    const float qx = fmaf(-t, D.x, px), qy = fmaf(-t, D.y, py), qz = fmaf(-t, D.z, pz);
    return sqrtf(fmaf(qx, qx, fmaf(qy, qy, qz * qz))) - s.w;
}

// The network's input for sorted point p of waypoint slot j: the link-frame point
// clamped to the grid box and normalised to it (xyz), and the distance to the box
// added outside it (w).
__device__ __forceinline__ float4 make_query(const SurFusedArgs& A, int l, const float4* M, float4 p) {
    const float lx = fmaf(M[0].x, p.x, fmaf(M[0].y, p.y, fmaf(M[0].z, p.z, M[0].w)));
    const float ly = fmaf(M[1].x, p.x, fmaf(M[1].y, p.y, fmaf(M[1].z, p.z, M[1].w)));
    const float lz = fmaf(M[2].x, p.x, fmaf(M[2].y, p.y, fmaf(M[2].z, p.z, M[2].w)));
    const float cx = fminf(fmaxf(lx, A.lo[l][0]), A.hi[l][0]);
    const float cy = fminf(fmaxf(ly, A.lo[l][1]), A.hi[l][1]);
    const float cz = fminf(fmaxf(lz, A.lo[l][2]), A.hi[l][2]);
    const float ex = lx - cx, ey = ly - cy, ez = lz - cz;
    const float ia = A.inv_a[l];
    return make_float4((cx - A.m[l][0]) * ia, (cy - A.m[l][1]) * ia, (cz - A.m[l][2]) * ia,
                       sqrtf(fmaf(ex, ex, fmaf(ey, ey, ez * ez))));
}

__device__ __forceinline__ unsigned long long sur_ns() {
    unsigned long long v;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(v));
    return v;
}

__global__ void __launch_bounds__(kEvalThreads, 1) sur_check_kernel(const __grid_constant__ SurFusedArgs A) {
    extern __shared__ __align__(1024) uint8_t sm[];
    __shared__ uint64_t mbar[kEvalPipes + 1];   // one per pipeline, one for the whole block
    __shared__ uint32_t tmem_slot;
    __shared__ float4 s_M[kSurGroup][3];           // link-from-world rows of each waypoint's link pose
    __shared__ float4 s_cA[kSurGroup], s_cD[kSurGroup];   // world capsule: start (+radius), axis (+1/len^2)
    __shared__ unsigned long long s_key[kSurGroup];
    __shared__ float s_thr[kSurGroup];
    __shared__ int s_item, s_qn, s_ln, s_lnext, s_fail;
    __shared__ unsigned s_over;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int pipe = warp >> 2, r = t & 127;
    uint8_t* sW2 = sm + kSurImg;
    uint8_t* sW3 = sm + kSurImg + kTileBytes;
    float* small = reinterpret_cast<float*>(sm + kSurImg + 2 * kTileBytes);
    uint8_t* sH = sm + kSurH + pipe * kTileBytes;
    float4* s_q = reinterpret_cast<float4*>(sm + kSurQ);
    uint32_t* s_tag = reinterpret_cast<uint32_t*>(sm + kSurTag);
    uint32_t* s_list = reinterpret_cast<uint32_t*>(sm + kSurLst);

    if (warp == 0) tc::tmem_alloc(&tmem_slot, 512);
    if (t <= kEvalPipes) tc::mbar_init(&mbar[t], 1);
    if (t == 0) s_fail = 0;
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tm = tmem_slot;
    const uint32_t d_tmem = tm + (uint32_t)(128 * pipe);
    const uint32_t taddr = d_tmem + ((uint32_t)((warp & 3) * 32) << 16);
    const uint32_t aW2 = tc::smem_u32(sW2), aW3 = tc::smem_u32(sW3), aH = tc::smem_u32(sH);
    // the whole block on one tile (seed items): pipeline 0's columns and activation tile,
    // the partial output sums in pipeline 1's activation tile
    uint8_t* sH0 = sm + kSurH;
    const uint32_t aH0 = tc::smem_u32(sH0);
    const uint32_t taddr0 = tm + ((uint32_t)((warp & 3) * 32) << 16);
    float* s_part = reinterpret_cast<float*>(sm + kSurH + kTileBytes);
    uint32_t phase = 0, phase_b = 0;
    bool ok = true;
    const int nv = *A.n_valid;
    const int n_tiles = (nv + 31) >> 5, n_sup = (n_tiles + 31) >> 5;
    // The pipelines' activation tiles are idle from an item's start to its first
    // evaluation round, which is after every read of the sphere tables (the seed scan,
    // the cull lists): each item copies the tables there when they fit, and the
    // evaluation then overwrites them.
    float4* s_sph = reinterpret_cast<float4*>(sm + kSurH);
    const bool staged = n_tiles + n_sup <= kEvalPipes * kTileBytes / 16;
    const float4* tiles = staged ? s_sph : A.tiles;
    const float4* supers = staged ? s_sph + n_tiles : A.supers;
    const int n_seed_groups = (A.W + A.seed_group - 1) / A.seed_group;
    const int n_seed_items = A.L * n_seed_groups;
    const int n_items = n_seed_items + A.L * A.n_groups;
    unsigned long long n_seed_q = 0, n_cull_q = 0;
    int loaded = -1;
    // phase times (SDF_OPT_STATS): thread 0 stamps the block-wide phase boundaries,
    // each taken just after the barrier that closes a phase
    const bool timed = A.stats != nullptr && t == 0;
    const unsigned long long t_cta0 = timed ? sur_ns() : 0ull;
    unsigned long long t_mark = t_cta0, ns_prod = 0, ns_eval = 0, ns_list = 0;
    auto stamp = [&](unsigned long long* acc) {
        if (timed) {
            const unsigned long long n = sur_ns();
            if (acc) *acc += n - t_mark;
            t_mark = n;
        }
    };

    // Evaluate queries [0, nq) of the ring, a tile of 128 per pipeline at a time, and
    // fold them into s_key (warps of one pipeline combine the lanes of a waypoint
    // first).  Link l's weights are loaded.
    auto evaluate_ring = [&](int l, int nq) {
        const int nt = (nq + 127) >> 7;
        for (int tl = pipe; tl < nt && ok; tl += kEvalPipes) {
            const int qi = tl * 128 + r;
            const uint32_t tag = qi < nq ? s_tag[qi] : kNoTag;
            const float4 x = tag != kNoTag ? s_q[qi] : make_float4(0.f, 0.f, 0.f, 0.f);
            float f = 0.f;
            ok = pipe_network(pipe, r, small, sH, aH, aW2, aW3, d_tmem, taddr, &mbar[pipe], phase, A.wait_polls,
                              x, f);
            if (!ok) {
                if (r == 0) s_fail = 1;
                break;
            }
            const float d = fmaf(A.scale[l], f, x.w);
            const bool use = tag != kNoTag && !isnan(d);
            const unsigned j = use ? tag >> 24 : kNoTag;
            const unsigned hi = use ? ordered_bits(d) : 0xffffffffu;
            const unsigned lo = use ? (((tag & 0xffffffu) << 4) | (unsigned)l) : 0xffffffffu;
            const unsigned peers = __match_any_sync(0xffffffffu, j);
            const unsigned hmin = __reduce_min_sync(peers, hi);
            const unsigned lmin = __reduce_min_sync(peers, hi == hmin ? lo : 0xffffffffu);
            if (use && lane == __ffs(peers) - 1) atomicMin(&s_key[j], ((unsigned long long)hmin << 32) | lmin);
        }
    };

    // Evaluate queries [0, nq) of the ring, nq <= 128, as one tile with the whole block
    // (a seed item's tile, and a cull round of one tile), and fold them into s_key as
    // evaluate_ring does.
    auto evaluate_block = [&](int l, int nq) {
        const uint32_t tag = r < nq ? s_tag[r] : kNoTag;
        const float4 x = tag != kNoTag ? s_q[r] : make_float4(0.f, 0.f, 0.f, 0.f);
        float f = 0.f;
        ok = block_network(pipe, r, t, small, sH0, aH0, aW2, aW3, tm, taddr0, &mbar[kEvalPipes], phase_b,
                           A.wait_polls, x, s_part, f);
        if (!ok) {
            if (t == 0) s_fail = 1;
            return;
        }
        if (pipe == 0) {
            const float d = fmaf(A.scale[l], f, x.w);
            const bool use = tag != kNoTag && !isnan(d);
            const unsigned j = use ? tag >> 24 : kNoTag;
            const unsigned hi = use ? ordered_bits(d) : 0xffffffffu;
            const unsigned lo = use ? (((tag & 0xffffffu) << 4) | (unsigned)l) : 0xffffffffu;
            const unsigned peers = __match_any_sync(0xffffffffu, j);
            const unsigned hmin = __reduce_min_sync(peers, hi);
            const unsigned lmin = __reduce_min_sync(peers, hi == hmin ? lo : 0xffffffffu);
            if (use && lane == __ffs(peers) - 1) atomicMin(&s_key[j], ((unsigned long long)hmin << 32) | lmin);
        }
    };

    for (;;) {
        __syncthreads();
        if (t == 0) s_item = atomicAdd(A.work, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= n_items || s_fail) break;
        stamp(nullptr);
        const bool seed = item < n_seed_items;
        const int rem = seed ? item : item - n_seed_items;
        const int ng = seed ? n_seed_groups : A.n_groups;
        const int gsz = seed ? A.seed_group : A.group;
        const int l = rem / ng, g = rem % ng;
        // a seed item takes gsz consecutive waypoints; a cull item takes waypoints g,
        // g + ng, g + 2 ng, ...: heavy waypoints come in runs along a trajectory, and
        // spreading each run over many items evens out the items' work
        const int w0 = seed ? g * gsz : g;
        const int w_step = seed ? 1 : ng;
        const int nw = seed ? min(gsz, A.W - w0) : (A.W - g + ng - 1) / ng;
        if (!seed && A.decided_below > -INFINITY) {
            // a cull item whose waypoints are all decided by the grid re-check adds nothing
            bool open = false;
            if (t < nw) {
                const unsigned long long k = __ldcg(&A.keys[w0 + t * w_step]);
                open = !(k != ~0ull && from_ordered((unsigned)(k >> 32)) < A.decided_below);
            }
            if (!__syncthreads_or(open)) continue;
        }
        if (l != loaded) {
            load_image(A.image + (size_t)l * kImgBytes, sm + kSurImg, t, kEvalThreads);
            tc::fence_smem_to_async();   // the weights are MMA operands
            loaded = l;
        }
        // the group's poses and world capsules of link l
        if (warp < nw) {
            const float4* P =
                reinterpret_cast<const float4*>(A.poses + ((size_t)(w0 + warp * w_step) * A.L + l) * 16);
            const float4 M0 = P[0], M1 = P[1], M2 = P[2];
            if (lane == 0) {
                s_M[warp][0] = M0;
                s_M[warp][1] = M1;
                s_M[warp][2] = M2;
                const float4 a = A.cap_a[l], b = A.cap_b[l];
                const float ax = a.x - M0.w, ay = a.y - M1.w, az = a.z - M2.w;
                const float bx = b.x - M0.w, by = b.y - M1.w, bz = b.z - M2.w;
                const float Ax = fmaf(M0.x, ax, fmaf(M1.x, ay, M2.x * az));
                const float Ay = fmaf(M0.y, ax, fmaf(M1.y, ay, M2.y * az));
                const float Az = fmaf(M0.z, ax, fmaf(M1.z, ay, M2.z * az));
                const float Bx = fmaf(M0.x, bx, fmaf(M1.x, by, M2.x * bz));
                const float By = fmaf(M0.y, bx, fmaf(M1.y, by, M2.y * bz));
                const float Bz = fmaf(M0.z, bx, fmaf(M1.z, by, M2.z * bz));
                const float dx = Bx - Ax, dy = By - Ay, dz = Bz - Az;
                const float dd = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                s_cA[warp] = make_float4(Ax, Ay, Az, a.w);
                s_cD[warp] = make_float4(dx, dy, dz, dd > 0.f ? 1.f / dd : 0.f);
                // cull items start from the minimum over every link published so far
                s_key[warp] = seed ? ~0ull : A.keys[w0 + warp * w_step];
            }
        }
        if (t == 0) {
            s_qn = 0;
            s_ln = 0;
            s_lnext = 0;
            s_over = 0u;
        }
        if (staged) {   // the evaluation rounds of the previous item are over (barrier above)
            for (int i = t; i < n_tiles; i += kEvalThreads) s_sph[i] = __ldg(&A.tiles[i]);
            for (int i = t; i < n_sup; i += kEvalThreads) s_sph[n_tiles + i] = __ldg(&A.supers[i]);
        }
        __syncthreads();
        stamp(&ns_prod);

        if (seed) {
            // the 32 points of the tile nearest to the capsule (nearest super-tile first)
            uint32_t tag = kNoTag;
            float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
            float gq = INFINITY;
            if (warp < nw && nv > 0) {
                const float4 cA = s_cA[warp], cD = s_cD[warp];
                float best = INFINITY;
                int bi = 0x7fffffff;
                for (int s = lane; s < n_sup; s += 32) {
                    const float gp = capsule_gap(supers[s], cA, cD);
                    if (gp < best) { best = gp; bi = s; }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const float ob = __shfl_xor_sync(0xffffffffu, best, o);
                    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                    if (ob < best || (ob == best && oi < bi)) { best = ob; bi = oi; }
                }
                if (bi < n_sup) {
                    const int tt = bi * 32 + lane;
                    float tb = INFINITY;
                    int ti = 0x7fffffff;
                    if (tt < n_tiles) { tb = capsule_gap(tiles[tt], cA, cD); ti = tt; }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        const float ob = __shfl_xor_sync(0xffffffffu, tb, o);
                        const int oi = __shfl_xor_sync(0xffffffffu, ti, o);
                        if (ob < tb || (ob == tb && oi < ti)) { tb = ob; ti = oi; }
                    }
                    const int k = ti * 32 + lane;
                    if (ti < n_tiles && k < nv) {
                        const float4 p = __ldg(&A.sorted[k]);
                        q = make_query(A, l, s_M[warp], p);
                        tag = ((unsigned)warp << 24) | (unsigned)__float_as_int(p.w);
                        gq = capsule_gap(make_float4(p.x, p.y, p.z, 0.f), cA, cD);
                    }
                }
            }
            if (warp < gsz) {
                // the kSeedPts points of the tile nearest to the capsule (ties by lane)
                int rank = 0;
#pragma unroll 8
                for (int j = 0; j < 32; ++j) {
                    const float gj = __shfl_sync(0xffffffffu, gq, j);
                    rank += (gj < gq || (gj == gq && j < lane)) ? 1 : 0;
                }
                if (rank < kSeedPts) {
                    s_q[warp * kSeedPts + rank] = q;
                    s_tag[warp * kSeedPts + rank] = tag;
                }
                if (A.stats) n_seed_q += (unsigned)__popc(__ballot_sync(0xffffffffu, tag != kNoTag && rank < kSeedPts));
            }
            __syncthreads();
            stamp(&ns_prod);
            evaluate_block(l, gsz * kSeedPts);
            __syncthreads();
            stamp(&ns_eval);
        } else {
            if (t < nw) {
                const unsigned long long k = s_key[t];
                const float best = k == ~0ull ? INFINITY : from_ordered((unsigned)(k >> 32));
                s_thr[t] = best < A.decided_below ? -INFINITY : best + A.slack + s_cA[t].w;
            }
            __syncthreads();
            // list: (waypoint slot, tile) entries whose tile sphere reaches the threshold
            if (warp < nw) {
                const float4 cA = s_cA[warp], cD = s_cD[warp];
                const float thr = s_thr[warp];
                for (int s0 = 0; s0 < n_sup; s0 += 32) {
                    const int sidx = s0 + lane;
                    unsigned bs = __ballot_sync(0xffffffffu,
                                                sidx < n_sup && capsule_gap(supers[sidx], cA, cD) <= thr);
                    while (bs) {
                        const int sv = s0 + __ffs(bs) - 1;
                        bs &= bs - 1;
                        const int tt = sv * 32 + lane;
                        const bool reach = tt < n_tiles && capsule_gap(tiles[tt], cA, cD) <= thr;
                        const unsigned bt = __ballot_sync(0xffffffffu, reach);
                        if (!bt) continue;
                        int base = 0;
                        if (lane == 0) base = atomicAdd(&s_ln, __popc(bt));
                        base = __shfl_sync(0xffffffffu, base, 0);
                        const int slot = base + __popc(bt & ((1u << lane) - 1u));
                        if (reach && slot < kSurList) s_list[slot] = ((unsigned)warp << 24) | (unsigned)tt;
                        if (base + __popc(bt) > kSurList && lane == 0) atomicOr(&s_over, 1u << warp);
                    }
                }
            }
            __syncthreads();
            if (timed) {
                const unsigned long long m = t_mark;
                stamp(&ns_prod);
                ns_list += t_mark - m;
            }
            const int n_list = min(s_ln, kSurList);
            for (;;) {
                // produce: kSurTake entries per warp step (their point loads go out
                // together) until the ring holds kSurFill queries
                for (;;) {
                    int e0 = 0x7fffffff;
                    if (lane == 0 && *reinterpret_cast<volatile int*>(&s_qn) < kSurFill)
                        e0 = atomicAdd(&s_lnext, kSurTake);
                    e0 = __shfl_sync(0xffffffffu, e0, 0);
                    if (e0 >= n_list) break;
                    float4 p[kSurTake];
                    int jj[kSurTake];
#pragma unroll
                    for (int u = 0; u < kSurTake; ++u) {
                        const bool ve = e0 + u < n_list;
                        const uint32_t ent = ve ? s_list[e0 + u] : 0u;
                        jj[u] = ve ? (int)(ent >> 24) : -1;
                        const int k = (int)(ent & 0xffffffu) * 32 + lane;
                        p[u] = (ve && k < nv) ? __ldg(&A.sorted[k]) : make_float4(0.f, 0.f, 0.f, 0.f);
                        if (!(ve && k < nv)) jj[u] = -1;
                    }
                    bool take[kSurTake];
                    unsigned b[kSurTake];
                    int cnt = 0;
#pragma unroll
                    for (int u = 0; u < kSurTake; ++u) {
                        const int j = max(jj[u], 0);
                        take[u] = jj[u] >= 0 &&
                                  capsule_gap(make_float4(p[u].x, p[u].y, p[u].z, 0.f), s_cA[j], s_cD[j]) <= s_thr[j];
                        b[u] = __ballot_sync(0xffffffffu, take[u]);
                        cnt += __popc(b[u]);
                    }
                    if (!cnt) continue;
                    int base = 0;
                    if (lane == 0) base = atomicAdd(&s_qn, cnt);
                    base = __shfl_sync(0xffffffffu, base, 0);
#pragma unroll
                    for (int u = 0; u < kSurTake; ++u) {
                        if (take[u]) {
                            const int slot = base + __popc(b[u] & ((1u << lane) - 1u));
                            s_q[slot] = make_query(A, l, s_M[jj[u]], p[u]);
                            s_tag[slot] = ((unsigned)jj[u] << 24) | (unsigned)__float_as_int(p[u].w);
                        }
                        base += __popc(b[u]);
                    }
                }
                __syncthreads();
                stamp(&ns_prod);
                const int nq = s_qn;
                const bool done = s_lnext >= n_list;
                if (nq == 0) break;   // then done as well: production stops only at kSurFill or at the end
                const int take_q = done ? nq : (nq & ~127);
                if (A.stats && t == 0) n_cull_q += (unsigned)take_q;
                if (take_q <= 128)
                    evaluate_block(l, take_q);   // one tile: the whole block on it
                else
                    evaluate_ring(l, take_q);
                __syncthreads();
                stamp(&ns_eval);
                // the rest (under one tile) to the front of the ring; thresholds tighten
                const int left = nq - take_q;
                float4 mq;
                uint32_t mt = kNoTag;
                if (t < left) {
                    mq = s_q[take_q + t];
                    mt = s_tag[take_q + t];
                }
                if (t < nw) {
                    const unsigned long long k = s_key[t];
                    const float best = k == ~0ull ? INFINITY : from_ordered((unsigned)(k >> 32));
                    s_thr[t] = best < A.decided_below ? -INFINITY : fminf(s_thr[t], best + A.slack + s_cA[t].w);
                }
                __syncthreads();
                if (t < left) {
                    s_q[t] = mq;
                    s_tag[t] = mt;
                }
                if (t == 0) s_qn = left;
                __syncthreads();
                stamp(&ns_prod);
                if (done && left == 0) break;
            }
        }
        // publish the group's minima (and the waypoints whose list overflowed)
        if (t < nw) {
            if (s_key[t] != ~0ull) atomicMin(&A.keys[w0 + t * w_step], s_key[t]);
            if (s_over & (1u << t)) A.recheck[w0 + t * w_step] = 1;
        }
    }
    if (A.stats) {
        if (lane == 0) {
            unsigned long long v = n_seed_q;
            if (v) atomicAdd(&A.stats[26], v);
        }
        if (t == 0 && n_cull_q) atomicAdd(&A.stats[27], n_cull_q);
        if (timed) {
            const unsigned long long cta = sur_ns() - t_cta0;
            atomicAdd(&A.stats[19], cta);
            atomicAdd(&A.stats[28], ns_prod);
            atomicAdd(&A.stats[29], ns_eval);
            atomicAdd(&A.stats[30], ns_list);
            atomicMax(&A.stats[31], cta);
        }
    }
    if (!ok) {
        // a wait gave up: report it, then let the MMA still in flight end before the
        // tensor memory is released
        if (r == 0) atomicOr(A.status, kStatusTimeout);
        tc::mbar_wait(&mbar[pipe], phase ^ 1u, kWaitPolls);
        tc::mbar_wait(&mbar[kEvalPipes], phase_b ^ 1u, kWaitPolls);
    }
    tc::fence_before_sync();
    __threadfence();   // this CTA's key updates and flags, before it counts itself done
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_free(tm, 512);
    // the last CTA to finish decodes every waypoint's key into the results and selects
    // the waypoints for the grid re-check (the other CTAs' updates are visible: each
    // fenced them before counting itself done)
    __shared__ int s_last;
    if (t == 0) s_last = atomicAdd(A.work + 1, 1) == (int)gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    for (int w = t; w < A.W; w += kEvalThreads) {
        const unsigned long long key = __ldcg(&A.keys[w]);
        float d;
        if (key == ~0ull) {
            d = INFINITY;
            A.arg_link[w] = -1;
            A.arg_point[w] = -1;
        } else {
            d = from_ordered((unsigned)(key >> 32));
            A.arg_link[w] = (int)(key & 15u);
            A.arg_point[w] = (int)((key & 0xffffffffu) >> 4);
        }
        A.dist[w] = d;
        if (A.sur_dist) A.sur_dist[w] = d;
        const uint8_t r = (__ldcg(&A.recheck[w]) || d < A.limit) ? 1 : 0;
        A.recheck[w] = r;
        if (A.recheck_out) A.recheck_out[w] = r;
    }
}

}  // namespace

// ------------------------------------------------------------------ launchers

cudaError_t configure_surrogate_kernels() {
    cudaError_t e = cudaFuncSetAttribute(mlp_train_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kTrainSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(mlp_eval_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kEvalSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(sur_check_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSurSmem);
    return e;
}

}  // namespace sdf

// ====================================================================== C ABI

struct sdf_surrogate {
    int device = 0;
    int L = 0;
    uint64_t id = 0;                        // unique over the process (never reused)
    std::atomic<uint64_t> version{0};       // incremented by every training call
    const sdf_grids* grids = nullptr;
    float* master = nullptr;   // [L][PARAMS], W2/W3 blocks [in][out]
    float* adam_m = nullptr;
    float* adam_v = nullptr;
    int* step = nullptr;
    float* loss = nullptr;     // [L]
    float box_m[SDF_MAX_LINKS][3];
    float box_a[SDF_MAX_LINKS];
};

namespace sdf {
const sdf_grids* surrogate_grids(const sdf_surrogate* s) { return s ? s->grids : nullptr; }
}  // namespace sdf

namespace {

using sdf::kH;
using sdf::kPar;
using sdf::kParStride;

std::atomic<uint64_t> g_surrogate_ids{0};

int sfail(sdf_ctx* ctx, int code, const std::string& msg) {
    if (ctx) ctx->err = msg;
    return code;
}
int scuda(sdf_ctx* ctx, cudaError_t e, const char* what) {
    return sfail(ctx, e == cudaErrorMemoryAllocation ? SDF_ERR_OOM : SDF_ERR_CUDA,
                 std::string(what) + ": " + cudaGetErrorString(e));
}

struct Dev {
    int prev = -1;
    explicit Dev(int d) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != d) cudaSetDevice(d);
    }
    ~Dev() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// public layout (W2, W3 [out][in]) <-> device layout ([in][out])
void to_device_layout(const float* in, float* out) {
    std::memcpy(out, in, sizeof(float) * kPar);
    for (int blk = 0; blk < 2; ++blk) {
        const int base = blk == 0 ? sdf::kOW2 : sdf::kOW3;
        for (int o = 0; o < kH; ++o)
            for (int i = 0; i < kH; ++i) out[base + i * kH + o] = in[base + o * kH + i];
    }
}
void to_public_layout(const float* in, float* out) {
    std::memcpy(out, in, sizeof(float) * kPar);
    for (int blk = 0; blk < 2; ++blk) {
        const int base = blk == 0 ? sdf::kOW2 : sdf::kOW3;
        for (int o = 0; o < kH; ++o)
            for (int i = 0; i < kH; ++i) out[base + o * kH + i] = in[base + i * kH + o];
    }
}

bool surrogate_configured(int device) {
    static bool done[64] = {};
    if (device < 0 || device >= 64) return false;
    if (!done[device]) done[device] = sdf::configure_surrogate_kernels() == cudaSuccess;
    return done[device];
}

sdf::SampleArgs sample_args(const sdf_grids* G, int link) {
    sdf::SampleArgs A{};
    const sdf_grid_meta& m = G->meta[link];
    const int n = G->n;
    A.grid = G->values + (size_t)link * n * n * n;
    A.n = n;
    A.o_ih = make_float4(m.origin[0], m.origin[1], m.origin[2], 1.0f / m.h);
    A.h = m.h;
    const double a = 0.5 * (n - 1) * (double)m.h;
    for (int k = 0; k < 3; ++k) {
        A.lo[k] = m.origin[k];
        A.span[k] = (float)(2.0 * a);
        A.m[k] = (float)(m.origin[k] + a);
    }
    A.inv_a = (float)(1.0 / a);
    return A;
}

}  // namespace

extern "C" {

int sdf_surrogate_create(sdf_ctx* ctx, const sdf_grids* grids, const float* params_host, sdf_surrogate** out) {
    if (!ctx || !grids || !params_host || !out) return sfail(ctx, SDF_ERR_INVALID_ARG, "sdf_surrogate_create: null");
    *out = nullptr;
    if (grids->device != ctx->device) return sfail(ctx, SDF_ERR_INVALID_ARG, "sdf_surrogate_create: other device");
    Dev guard(ctx->device);
    if (!surrogate_configured(ctx->device)) return sfail(ctx, SDF_ERR_CUDA, "surrogate kernels: attributes");
    sdf_surrogate* S = new (std::nothrow) sdf_surrogate();
    if (!S) return sfail(ctx, SDF_ERR_OOM, "sdf_surrogate_create");
    S->id = ++g_surrogate_ids;
    S->device = ctx->device;
    S->L = grids->n_links;
    S->grids = grids;
    const size_t bytes = sizeof(float) * (size_t)kParStride * S->L;
    cudaError_t e = sdf::dmalloc(&S->master, bytes);
    if (e == cudaSuccess) e = sdf::dmalloc(&S->adam_m, bytes);
    if (e == cudaSuccess) e = sdf::dmalloc(&S->adam_v, bytes);
    if (e == cudaSuccess) e = sdf::dmalloc(&S->step, sizeof(int) * S->L);
    if (e == cudaSuccess) e = sdf::dmalloc(&S->loss, sizeof(float) * S->L);
    std::vector<float> dev((size_t)kParStride * S->L, 0.f);
    for (int l = 0; l < S->L; ++l) to_device_layout(params_host + (size_t)l * kPar, dev.data() + (size_t)l * kParStride);
    if (e == cudaSuccess) e = cudaMemcpy(S->master, dev.data(), bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(S->adam_m, 0, bytes);
    if (e == cudaSuccess) e = cudaMemset(S->adam_v, 0, bytes);
    if (e == cudaSuccess) e = cudaMemset(S->step, 0, sizeof(int) * S->L);
    if (e == cudaSuccess) e = cudaMemset(S->loss, 0, sizeof(float) * S->L);
    if (e != cudaSuccess) {
        sdf_surrogate_destroy(S);
        return scuda(ctx, e, "sdf_surrogate_create");
    }
    for (int l = 0; l < S->L; ++l) {
        const sdf_grid_meta& m = grids->meta[l];
        const double a = 0.5 * (grids->n - 1) * (double)m.h;
        for (int k = 0; k < 3; ++k) S->box_m[l][k] = (float)(m.origin[k] + a);
        S->box_a[l] = (float)a;
    }
    *out = S;
    return SDF_OK;
}

void sdf_surrogate_destroy(sdf_surrogate* S) {
    if (!S) return;
    Dev guard(S->device);
    sdf::dfree(S->master);
    sdf::dfree(S->adam_m);
    sdf::dfree(S->adam_v);
    sdf::dfree(S->step);
    sdf::dfree(S->loss);
    delete S;
}

int sdf_surrogate_params(sdf_ctx* ctx, const sdf_surrogate* S, float* params_host) {
    if (!ctx || !S || !params_host) return sfail(ctx, SDF_ERR_INVALID_ARG, "sdf_surrogate_params: null");
    Dev guard(S->device);
    std::vector<float> dev((size_t)kParStride * S->L);
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpy(dev.data(), S->master, dev.size() * sizeof(float), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return scuda(ctx, e, "sdf_surrogate_params");
    for (int l = 0; l < S->L; ++l) to_public_layout(dev.data() + (size_t)l * kParStride, params_host + (size_t)l * kPar);
    return SDF_OK;
}

int sdf_surrogate_sample(sdf_ctx* ctx, const sdf_grids* G, int32_t link, int64_t n, int32_t near_per_10, float band,
                         uint64_t seed, float* x_dev, float* y_dev, int64_t* source_dev) {
    if (!ctx || !G || !x_dev || !y_dev || link < 0 || link >= G->n_links || n < 0 || near_per_10 < 0 ||
        near_per_10 > 10 || !(band > 0.f))
        return sfail(ctx, SDF_ERR_INVALID_ARG, "sdf_surrogate_sample: invalid argument");
    if (n == 0) return SDF_OK;
    Dev guard(ctx->device);
    sdf::SampleArgs A = sample_args(G, link);
    A.key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    A.band = band;
    A.near10 = near_per_10;
    A.n_samples = n;
    A.n_near = (n / 10) * near_per_10 + std::min<int64_t>(n % 10, near_per_10);
    A.x = x_dev;
    A.y = y_dev;
    A.source = reinterpret_cast<long long*>(source_dev);
    cudaStream_t st = ctx->stream;
    sdf::sample_uniform_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(A);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return scuda(ctx, e, "sample_uniform_kernel");
    if (A.n_near == 0) return SDF_OK;
    // near samples: chunks of candidates until enough are accepted
    const int chunk = (int)std::min<int64_t>(std::max<int64_t>(4 * A.n_near, 1 << 20), 1 << 26);
    const int nb = (chunk + 1023) / 1024;
    int* counts = nullptr;
    long long* found = nullptr;   // [0] found, [1] found before this chunk
    e = sdf::dmalloc(&counts, sizeof(int) * nb);
    if (e == cudaSuccess) e = sdf::dmalloc(&found, 2 * sizeof(long long));
    if (e == cudaSuccess) e = cudaMemsetAsync(found, 0, 2 * sizeof(long long), st);
    long long have = 0;
    long long start = 0;
    const long long max_candidates = 1ll << 32;   // the counter is 32 bits wide
    while (e == cudaSuccess && have < A.n_near) {
        if (start >= max_candidates) {
            sdf::dfree(counts);
            sdf::dfree(found);
            return sfail(ctx, SDF_ERR_INVALID_ARG, "sdf_surrogate_sample: too few candidates within the band");
        }
        A.start = start;
        A.count = chunk;
        A.block_count = counts;
        A.found = found;
        sdf::sample_count_kernel<<<nb, 1024, 0, st>>>(A);
        e = cudaGetLastError();
        if (e == cudaSuccess) sdf::sample_scan_kernel<<<1, 1024, 0, st>>>(counts, nb, found, found + 1);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) sdf::sample_scatter_kernel<<<nb, 1024, 0, st>>>(A, found + 1);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(&have, found, sizeof(long long), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        start += chunk;
    }
    sdf::dfree(counts);
    sdf::dfree(found);
    if (e != cudaSuccess) return scuda(ctx, e, "sdf_surrogate_sample");
    return SDF_OK;
}

namespace {
int launch_train(sdf_ctx* ctx, sdf_surrogate* S, int link0, int links, const float* x, const float* y, long long n,
                 long long batch0, int steps, float lr, float* grad_out, float* loss_out) {
    if (!surrogate_configured(ctx->device)) return sfail(ctx, SDF_ERR_CUDA, "surrogate kernels: attributes");
    sdf::TrainArgs A{};
    A.master = S->master;
    A.adam_m = S->adam_m;
    A.adam_v = S->adam_v;
    A.step = S->step;
    A.x = x;
    A.y = y;
    A.n = n;
    A.batch0 = batch0;
    A.steps = steps;
    A.link0 = link0;
    A.lr = lr;
    A.beta1 = 0.9f;
    A.beta2 = 0.999f;
    A.eps = 1e-8f;
    A.grad_out = grad_out;
    A.loss_out = loss_out;
    A.status = ctx->status;
    A.wait_polls = ctx->wait_polls;
    sdf::mlp_train_kernel<<<links, sdf::kTrainThreads, sdf::kTrainSmem, ctx->stream>>>(A);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SDF_OK : scuda(ctx, e, "mlp_train_kernel");
}
}  // namespace

int sdf_surrogate_grad(sdf_ctx* ctx, const sdf_surrogate* S, int32_t link, const float* x_dev, const float* y_dev,
                       float* grad_dev, float* loss_dev) {
    if (!ctx || !S || !x_dev || !y_dev || !grad_dev || link < 0 || link >= S->L)
        return sfail(ctx, SDF_ERR_INVALID_ARG, "sdf_surrogate_grad: invalid argument");
    Dev guard(ctx->device);
    // one batch of SDF_MLP_BATCH samples, read as link `link`'s samples: the kernel
    // indexes x[link][n][3] with n = SDF_MLP_BATCH, so shift the base pointers back
    const float* xb = x_dev - (size_t)link * SDF_MLP_BATCH * 3;
    const float* yb = y_dev - (size_t)link * SDF_MLP_BATCH;
    float* lb = loss_dev ? loss_dev - link : nullptr;
    return launch_train(ctx, const_cast<sdf_surrogate*>(S), link, 1, xb, yb, SDF_MLP_BATCH, 0, 1, 0.f, grad_dev,
                        lb);
}

int sdf_surrogate_train(sdf_ctx* ctx, sdf_surrogate* S, const float* x_dev, const float* y_dev, int64_t n,
                        int64_t first_batch, int32_t steps, float lr, float* loss_dev) {
    if (!ctx || !S || !x_dev || !y_dev || n < 1 || first_batch < 0 || steps < 0 || !(lr >= 0.f))
        return sfail(ctx, SDF_ERR_INVALID_ARG, "sdf_surrogate_train: invalid argument");
    if (steps == 0) return SDF_OK;
    Dev guard(ctx->device);
    float* loss = loss_dev ? loss_dev : S->loss;
    cudaError_t e = cudaMemsetAsync(loss, 0, sizeof(float) * S->L, ctx->stream);
    if (e != cudaSuccess) return scuda(ctx, e, "sdf_surrogate_train");
    ++S->version;   // the checks' cached weight images are stale from here on
    return launch_train(ctx, S, 0, S->L, x_dev, y_dev, n, first_batch, steps, lr, nullptr, loss);
}

int sdf_surrogate_eval(sdf_ctx* ctx, const sdf_surrogate* S, int32_t link, const float* x_dev, int32_t n,
                       float* f_dev) {
    if (!ctx || !S || link < 0 || link >= S->L || n < 0 || (n > 0 && (!x_dev || !f_dev)))
        return sfail(ctx, SDF_ERR_INVALID_ARG, "sdf_surrogate_eval: invalid argument");
    if (n == 0) return SDF_OK;
    Dev guard(ctx->device);
    if (!surrogate_configured(ctx->device)) return sfail(ctx, SDF_ERR_CUDA, "surrogate kernels: attributes");
    sdf::EvalArgs A{};
    A.master = S->master;
    A.x3 = x_dev;
    A.L = S->L;
    A.n = n;
    A.link0 = link;
    A.f_out = f_dev;
    A.status = ctx->status;
    A.wait_polls = ctx->wait_polls;
    const int tiles = (n + 127) / 128;
    const int grid = std::min(tiles, ctx->num_sms);
    sdf::mlp_eval_kernel<<<grid, sdf::kEvalThreads, sdf::kEvalSmem, ctx->stream>>>(A);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SDF_OK : scuda(ctx, e, "mlp_eval_kernel");
}


int check_trajectory_surrogate(sdf_ctx* ctx, const sdf_robot* R, const sdf_surrogate* Sc, const float* q_dev,
                               int32_t W, const float* points_dev, int32_t N, float margin, float eps,
                               float* dist_dev, int32_t* argmin_link_dev, int32_t* argmin_point_dev,
                               uint8_t* rechecked_dev, float* surrogate_dist_dev) {
    sdf_surrogate* S = const_cast<sdf_surrogate*>(Sc);
    if (!ctx || !R || !S) return sfail(ctx, SDF_ERR_INVALID_ARG, "check_trajectory_surrogate: null");
    if (R->grids != S->grids || R->device != ctx->device)
        return sfail(ctx, SDF_ERR_INVALID_ARG, "check_trajectory_surrogate: robot and surrogate use different grids");
    if (W < 0 || N < 0 || N > SDF_MAX_POINTS || !(margin >= 0.f) || !(eps >= 0.f))
        return sfail(ctx, SDF_ERR_INVALID_ARG, "check_trajectory_surrogate: invalid sizes or bounds");
    if (W == 0) return SDF_OK;
    if (!dist_dev || !argmin_link_dev || !argmin_point_dev || (R->dof > 0 && !q_dev) || (N > 0 && !points_dev))
        return sfail(ctx, SDF_ERR_INVALID_ARG, "check_trajectory_surrogate: null buffer");
    Dev guard(ctx->device);
    if (!surrogate_configured(ctx->device)) return sfail(ctx, SDF_ERR_CUDA, "surrogate kernels: attributes");
    const int L = S->L;
    cudaStream_t st = ctx->stream;
    cudaError_t e = cudaSuccess;
    // workspace (the context's): poses, keys and re-check mask per waypoint, the item counter
    if ((size_t)W > ctx->sur_w_cap || !ctx->sur_count) {
        const size_t cap = std::max<size_t>((size_t)W, 2 * ctx->sur_w_cap);
        cudaStreamSynchronize(st);
        sdf::dfree(ctx->sur_poses);
        sdf::dfree(ctx->sur_keys);
        sdf::dfree(ctx->sur_mask);
        ctx->sur_poses = nullptr;
        ctx->sur_keys = nullptr;
        ctx->sur_mask = nullptr;
        ctx->sur_w_cap = 0;
        e = sdf::dmalloc(&ctx->sur_poses, sizeof(float) * 16 * SDF_MAX_LINKS * cap);
        if (e == cudaSuccess) e = sdf::dmalloc(&ctx->sur_keys, sizeof(unsigned long long) * cap);
        if (e == cudaSuccess) e = sdf::dmalloc(&ctx->sur_mask, cap);
        if (e == cudaSuccess && !ctx->sur_count) e = sdf::dmalloc(&ctx->sur_count, sizeof(int) * SDF_MAX_LINKS);
        if (e != cudaSuccess) return scuda(ctx, e, "check_trajectory_surrogate: workspace");
        ctx->sur_w_cap = cap;
    }
    if ((size_t)L * sdf::kImgBytes > ctx->sur_wimg_cap) {
        cudaStreamSynchronize(st);
        sdf::dfree(ctx->sur_wimg);
        ctx->sur_wimg = nullptr;
        ctx->sur_wimg_cap = 0;
        e = sdf::dmalloc(&ctx->sur_wimg, (size_t)SDF_MAX_LINKS * sdf::kImgBytes);
        if (e != cudaSuccess) return scuda(ctx, e, "check_trajectory_surrogate: weight image");
        ctx->sur_wimg_cap = (size_t)SDF_MAX_LINKS * sdf::kImgBytes;
        ctx->sur_wimg_id = 0;
    }
    // the weights in the fused kernel's shared-memory layout, made again only when the
    // context last made them for another surrogate or before its latest training
    const uint64_t version = S->version.load();
    e = cudaSuccess;
    if (ctx->sur_wimg_id != S->id || ctx->sur_wimg_version != version) {
        sdf::weight_image_kernel<<<(unsigned)L, 512, 0, st>>>(S->master, ctx->sur_wimg);
        e = cudaGetLastError();
        if (e == cudaSuccess) {
            ctx->sur_wimg_id = S->id;
            ctx->sur_wimg_version = version;
        }
    }
    if (e != cudaSuccess) return scuda(ctx, e, "check_trajectory_surrogate");
    sdf::BatchParams* bp = new (std::nothrow) sdf::BatchParams();
    if (!bp) return sfail(ctx, SDF_ERR_OOM, "host allocation");
    int rc = sdf::sort_cloud(ctx, points_dev, N, bp);
    sdf::SurFusedArgs A{};
    if (rc == SDF_OK) {
        // kinematics and the resets of the keys, flags and work counter, overlapping the sort
        e = sdf::launch_fk_reset(R->table, q_dev, W, ctx->sur_poses, ctx->status, ctx->sur_keys, ctx->sur_mask,
                                 ctx->sur_count, st);
        A.poses = ctx->sur_poses;
        A.W = W;
        A.L = L;
        // waypoints per work item: the most (16, 8 or 4) that still gives every SM about
        // three cull items, so that the items even out across the SMs
        A.group = 4;
        for (int gsz = sdf::kSurGroup; gsz > 4; gsz /= 2)
            if ((long long)L * ((W + gsz - 1) / gsz) >= 3LL * ctx->num_sms) {
                A.group = gsz;
                break;
            }
        A.n_groups = (W + A.group - 1) / A.group;
        A.sorted = bp->sorted;
        A.tiles = bp->tiles;
        A.supers = bp->supers;
        A.n_valid = bp->n_valid;
        const sdf_grids* G = S->grids;
        for (int l = 0; l < L; ++l) {
            const double a = 0.5 * (G->n - 1) * (double)G->meta[l].h;
            for (int k = 0; k < 3; ++k) {
                A.lo[l][k] = G->meta[l].origin[k];
                A.hi[l][k] = (float)(G->meta[l].origin[k] + 2.0 * a);
                A.m[l][k] = S->box_m[l][k];
            }
            A.inv_a[l] = (float)(1.0 / a);
            A.scale[l] = S->box_a[l];
            A.cap_a[l] = R->table.cap_a[l];
            A.cap_b[l] = R->table.cap_b[l];
        }
        A.image = ctx->sur_wimg;
        A.seed_group = sdf::kSurGroup;
        A.keys = ctx->sur_keys;
        A.recheck = ctx->sur_mask;
        A.slack = eps + sdf::kCullSlack;
        A.decided_below = surrogate_dist_dev ? -INFINITY : margin + eps;
        A.work = ctx->sur_count;
        A.limit = margin + eps;
        A.dist = dist_dev;
        A.arg_link = argmin_link_dev;
        A.arg_point = argmin_point_dev;
        A.sur_dist = surrogate_dist_dev;
        A.recheck_out = rechecked_dev;
        A.status = ctx->status;
        A.wait_polls = ctx->wait_polls;
        A.stats = ctx->stats ? ctx->d_stats : nullptr;
    }
    delete bp;
    const int items = L * ((W + sdf::kSurGroup - 1) / sdf::kSurGroup) + L * A.n_groups;
    if (rc == SDF_OK && e == cudaSuccess) {
        sdf::sur_check_kernel<<<(unsigned)std::min(items, ctx->num_sms), sdf::kEvalThreads, sdf::kSurSmem, st>>>(A);
        e = cudaGetLastError();
    }
    if (rc == SDF_OK && e != cudaSuccess) rc = scuda(ctx, e, "check_trajectory_surrogate");
    if (rc == SDF_OK) {
        // the grid path re-checks the selected waypoints on the cloud sorted above
        sdf_check_request r{};
        r.robot = R;
        r.q_dev = q_dev;
        r.W = W;
        r.points_dev = points_dev;
        r.N = N;
        r.dist_dev = dist_dev;
        r.argmin_link_dev = argmin_link_dev;
        r.argmin_point_dev = argmin_point_dev;
        r.mask_dev = ctx->sur_mask;
        ctx->reuse_sort = 1;
        rc = check_batch(ctx, &r, 1);
        ctx->reuse_sort = 0;
    }
    return rc;
}

int sdf_surrogate_error(sdf_ctx* ctx, const sdf_surrogate* S, int32_t link, int64_t n, int32_t near_per_10,
                        float band, uint64_t seed, float* max_abs, float* mean_abs) {
    if (!ctx || !S || link < 0 || link >= S->L || n < 1 || n > (1 << 30))
        return sfail(ctx, SDF_ERR_INVALID_ARG, "sdf_surrogate_error: invalid argument");
    Dev guard(ctx->device);
    float *x = nullptr, *y = nullptr, *f = nullptr;
    unsigned* mx = nullptr;
    double* sum = nullptr;
    cudaError_t e = sdf::dmalloc(&x, sizeof(float) * 3 * n);
    if (e == cudaSuccess) e = sdf::dmalloc(&y, sizeof(float) * n);
    if (e == cudaSuccess) e = sdf::dmalloc(&f, sizeof(float) * n);
    if (e == cudaSuccess) e = sdf::dmalloc(&mx, sizeof(unsigned));
    if (e == cudaSuccess) e = sdf::dmalloc(&sum, sizeof(double));
    int rc = e == cudaSuccess ? SDF_OK : scuda(ctx, e, "sdf_surrogate_error");
    if (rc == SDF_OK) rc = sdf_surrogate_sample(ctx, S->grids, link, n, near_per_10, band, seed, x, y, nullptr);
    if (rc == SDF_OK) rc = sdf_surrogate_eval(ctx, S, link, x, (int32_t)n, f);
    unsigned hm = 0;
    double hs = 0.0;
    if (rc == SDF_OK) {
        e = cudaMemsetAsync(mx, 0, sizeof(unsigned), ctx->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(sum, 0, sizeof(double), ctx->stream);
        if (e == cudaSuccess)
            sdf::error_reduce_kernel<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(f, y, (int)n,
                                                                                       S->box_a[link], mx, sum);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(&hm, mx, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, sum, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) rc = scuda(ctx, e, "sdf_surrogate_error");
    }
    sdf::dfree(x);
    sdf::dfree(y);
    sdf::dfree(f);
    sdf::dfree(mx);
    sdf::dfree(sum);
    if (rc == SDF_OK) {
        float m;
        std::memcpy(&m, &hm, sizeof(float));
        if (max_abs) *max_abs = m;
        if (mean_abs) *mean_abs = (float)(hs / (double)n);
    }
    return rc;
}

}  // extern "C"
