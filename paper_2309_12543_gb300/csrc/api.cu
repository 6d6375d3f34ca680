// C ABI of the sdfcheck library: argument checks, object lifetimes, scratch
// management and launch configuration.  All device work is in check.cu and
// grid_build.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "internal.h"

namespace {

int fail(sdf_ctx* ctx, int code, const char* fmt, ...) {
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        ctx->err = buf;
    }
    return code;
}

int cuda_fail(sdf_ctx* ctx, cudaError_t e, const char* what) {
    return fail(ctx, e == cudaErrorMemoryAllocation ? SDF_ERR_OOM : SDF_ERR_CUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

#define SDF_CUDA(ctx, call)                                   \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
    } while (0)

// Make ctx->device current for the duration of a call and restore the caller's.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// Cached host-call graphs capture device addresses of the scratch: drop them
// before any of it moves.
void drop_host_graphs(sdf_ctx* ctx) {
    for (auto& g : ctx->host_graphs) cudaGraphExecDestroy(g.exec);
    ctx->host_graphs.clear();
}

template <typename T>
int grow(sdf_ctx* ctx, T** buf, size_t* cap, size_t need, bool fill_ff) {
    if (need <= *cap) return SDF_OK;
    drop_host_graphs(ctx);
    size_t n = std::max(need, *cap * 2);
    if (*buf) sdf::dfree(*buf);
    *buf = nullptr;
    *cap = 0;
    cudaError_t e = sdf::dmalloc(buf, n * sizeof(T));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "device allocation (scratch)");
    e = cudaMemsetAsync(*buf, fill_ff ? 0xff : 0, n * sizeof(T), ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMemsetAsync(scratch)");
    *cap = n;
    return SDF_OK;
}

}  // namespace

extern "C" {

// ------------------------------------------------------------------ context

int sdf_ctx_create(sdf_ctx** out, int device, void* cuda_stream) {
    if (!out) return SDF_ERR_INVALID_ARG;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count)
        return SDF_ERR_INVALID_ARG;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return SDF_ERR_CUDA;
    if (prop.major != 10 || prop.minor != 3) return SDF_ERR_UNSUPPORTED;
    sdf_ctx* ctx = new (std::nothrow) sdf_ctx();
    if (!ctx) return SDF_ERR_OOM;
    ctx->device = device;
    ctx->num_sms = prop.multiProcessorCount;
    ctx->stream = (cudaStream_t)cuda_stream;
    DeviceGuard g(device);
    if (sdf::dmalloc(&ctx->status, sizeof(int)) != cudaSuccess ||
        cudaMemset(ctx->status, 0, sizeof(int)) != cudaSuccess ||
        sdf::hmalloc(&ctx->h_status, sizeof(int)) != cudaSuccess ||
        sdf::dmalloc(&ctx->d_seq, sizeof(unsigned)) != cudaSuccess ||
        cudaMemset(ctx->d_seq, 0, sizeof(unsigned)) != cudaSuccess ||
        sdf::hmalloc(&ctx->h_done, sizeof(unsigned)) != cudaSuccess ||
        cudaEventCreate(&ctx->ev0) != cudaSuccess || cudaEventCreate(&ctx->ev1) != cudaSuccess ||
        cudaEventCreate(&ctx->ev2) != cudaSuccess) {
        sdf_ctx_destroy(ctx);
        return SDF_ERR_OOM;
    }
    if (sdf::configure_kernels() != cudaSuccess) {
        sdf_ctx_destroy(ctx);
        return SDF_ERR_CUDA;
    }
    *out = ctx;
    return SDF_OK;
}

void sdf_ctx_destroy(sdf_ctx* ctx) {
    if (!ctx) return;
    DeviceGuard g(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    drop_host_graphs(ctx);
    if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
    sdf::dfree(ctx->sorted);
    sdf::dfree(ctx->tiles);
    sdf::dfree(ctx->supers);
    sdf::dfree(ctx->n_valid);
    sdf::dfree(ctx->d_stats);
    sdf::dfree(ctx->status);
    if (ctx->h_status) sdf::hfree(ctx->h_status);
    sdf::dfree(ctx->d_seq);
    if (ctx->h_done) sdf::hfree(ctx->h_done);
    sdf::dfree(ctx->st_q);
    sdf::dfree(ctx->st_pts);
    sdf::dfree(ctx->st_dist);
    sdf::dfree(ctx->st_link);
    sdf::dfree(ctx->st_point);
    sdf::dfree(ctx->rs_sdf);
    sdf::dfree(ctx->rs_bits);
    sdf::dfree(ctx->rs_list);
    sdf::dfree(ctx->rs_poses);
    sdf::dfree(ctx->sur_poses);
    sdf::dfree(ctx->sur_keys);
    sdf::dfree(ctx->sur_mask);
    sdf::dfree(ctx->sur_count);
    sdf::dfree(ctx->sur_wimg);
    if (ctx->ev0) cudaEventDestroy(ctx->ev0);
    if (ctx->ev1) cudaEventDestroy(ctx->ev1);
    if (ctx->ev2) cudaEventDestroy(ctx->ev2);
    delete ctx;
}

int sdf_ctx_set_stream(sdf_ctx* ctx, void* cuda_stream) {
    if (!ctx) return SDF_ERR_INVALID_ARG;
    ctx->stream = (cudaStream_t)cuda_stream;
    return SDF_OK;
}

const char* sdf_last_error(const sdf_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int sdf_ctx_set_option(sdf_ctx* ctx, int32_t key, int64_t v) {
    if (!ctx) return SDF_ERR_INVALID_ARG;
    {
        DeviceGuard g(ctx->device);
        drop_host_graphs(ctx);   // captured launches follow the options
    }
    switch (key) {
        case SDF_OPT_CULL: ctx->cull = v ? 1 : 0; return SDF_OK;
        case SDF_OPT_POINT_STRIDE:
            if (v != 3 && v != 4) return fail(ctx, SDF_ERR_INVALID_ARG, "point stride must be 3 or 4");
            ctx->point_stride = (int)v;
            return SDF_OK;
        case SDF_OPT_WAYPOINTS_PER_BLOCK:
            if (v < 0 || v > sdf::kCheckWarps)
                return fail(ctx, SDF_ERR_INVALID_ARG, "waypoints per block must be 0..%d", sdf::kCheckWarps);
            ctx->tw = (int)v;
            return SDF_OK;
        case SDF_OPT_TILE_BATCH:
            if (v != 0 && v != 1 && v != 2 && v != 4)
                return fail(ctx, SDF_ERR_INVALID_ARG, "tile batch must be 0, 1, 2 or 4");
            ctx->tile_batch = (int)v;
            return SDF_OK;
        case SDF_OPT_TIME_KERNELS: ctx->time_kernels = v ? 1 : 0; return SDF_OK;
        case SDF_OPT_BLOCK_WARPS:
            if (v != 0 && v != 8 && v != 16) return fail(ctx, SDF_ERR_INVALID_ARG, "block warps must be 0, 8 or 16");
            ctx->block_warps = (int)v;
            return SDF_OK;
        case SDF_OPT_WAIT_POLLS:
            if (v < 0 || v > (int64_t)UINT32_MAX) return fail(ctx, SDF_ERR_INVALID_ARG, "wait polls must be 0..2^32-1");
            ctx->wait_polls = (unsigned)v;
            return SDF_OK;
        case SDF_OPT_TEX3D: ctx->tex3d = v ? 1 : 0; return SDF_OK;
        case SDF_OPT_SORT_CTAS: {
            if (v != 0 && v != 8 && v != 16) return fail(ctx, SDF_ERR_INVALID_ARG, "sort CTAs must be 0, 8 or 16");
            if (v == 16 && sdf::max_sort_ctas(ctx->device) < 16)
                return fail(ctx, SDF_ERR_UNSUPPORTED, "this device cannot place a 16-CTA cluster for the sort");
            ctx->sort_ctas = (int)v;
            return SDF_OK;
        }
        case SDF_OPT_STATS:
            if (v && !ctx->d_stats) {
                DeviceGuard g(ctx->device);
                cudaError_t e = sdf::dmalloc(&ctx->d_stats, sdf::kStatCount * sizeof(unsigned long long));
                if (e == cudaSuccess) e = cudaMemset(ctx->d_stats, 0, sdf::kStatCount * sizeof(unsigned long long));
                if (e == cudaSuccess) e = cudaMemset(ctx->d_stats + 17, 0xff, sizeof(unsigned long long));
                if (e != cudaSuccess) return cuda_fail(ctx, e, "statistics buffer");
            }
            ctx->stats = v ? 1 : 0;
            return SDF_OK;
        default: return fail(ctx, SDF_ERR_INVALID_ARG, "unknown option %d", (int)key);
    }
}

int sdf_ctx_get_option(const sdf_ctx* ctx, int32_t key, int64_t* v) {
    if (!ctx || !v) return SDF_ERR_INVALID_ARG;
    switch (key) {
        case SDF_OPT_CULL: *v = ctx->cull; return SDF_OK;
        case SDF_OPT_POINT_STRIDE: *v = ctx->point_stride; return SDF_OK;
        case SDF_OPT_WAYPOINTS_PER_BLOCK: *v = ctx->tw; return SDF_OK;
        case SDF_OPT_TILE_BATCH: *v = ctx->tile_batch; return SDF_OK;
        case SDF_OPT_TIME_KERNELS: *v = ctx->time_kernels; return SDF_OK;
        case SDF_OPT_STATS: *v = ctx->stats; return SDF_OK;
        case SDF_OPT_BLOCK_WARPS: *v = ctx->block_warps; return SDF_OK;
        case SDF_OPT_WAIT_POLLS: *v = (int64_t)ctx->wait_polls; return SDF_OK;
        case SDF_OPT_TEX3D: *v = ctx->tex3d; return SDF_OK;
        case SDF_OPT_SORT_CTAS: {
            if (ctx->sort_ctas) {
                *v = ctx->sort_ctas;
                return SDF_OK;
            }
            *v = sdf::max_sort_ctas(ctx->device);
            return SDF_OK;
        }
        default: return SDF_ERR_INVALID_ARG;
    }
}

}  // extern "C"

namespace {
// Enqueue: the status word to page-locked host memory, then cleared on the device.
cudaError_t enqueue_status_readback(sdf_ctx* ctx, cudaStream_t st) {
    cudaError_t e = cudaMemcpyAsync(ctx->h_status, ctx->status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->status, 0, sizeof(int), st);
    return e;
}
// Polls the host-buffer path's completion word for the value `want` (written by
// finish_kernel after the status); gives up after 2 s, after which the caller
// synchronises the stream.  The acquire load orders the later reads of the results.
bool wait_done(sdf_ctx* ctx, unsigned want) {
    const auto t0 = std::chrono::steady_clock::now();
    for (unsigned i = 0;; ++i) {
        if (__atomic_load_n(ctx->h_done, __ATOMIC_ACQUIRE) == want) return true;
        if ((i & 1023u) == 1023u && std::chrono::steady_clock::now() - t0 > std::chrono::seconds(2)) return false;
    }
}

// The status word read back by enqueue_status_readback, as a return code.
int status_code(sdf_ctx* ctx) {
    const int st = *ctx->h_status;
    if (st & sdf::kStatusTimeout)
        return fail(ctx, SDF_ERR_TIMEOUT, "a bounded device wait gave up; results of that call are invalid");
    if (st & sdf::kStatusNonFinite) return fail(ctx, SDF_ERR_NONFINITE, "non-finite joint value or point in a check");
    return SDF_OK;
}
}  // namespace

extern "C" {

int sdf_ctx_synchronize(sdf_ctx* ctx) {
    if (!ctx) return SDF_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    SDF_CUDA(ctx, enqueue_status_readback(ctx, ctx->stream));
    SDF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return status_code(ctx);
}

int sdf_ctx_stats(sdf_ctx* ctx, int64_t* out, int32_t n, int32_t reset) {
    if (!ctx || (n > 0 && !out) || n < 0) return SDF_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    unsigned long long h[sdf::kStatCount] = {0};
    if (ctx->d_stats) {
        SDF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        SDF_CUDA(ctx, cudaMemcpy(h, ctx->d_stats, sizeof h, cudaMemcpyDeviceToHost));
        if (reset) {
            SDF_CUDA(ctx, cudaMemset(ctx->d_stats, 0, sizeof h));
            SDF_CUDA(ctx, cudaMemset(ctx->d_stats + 17, 0xff, sizeof(unsigned long long)));
        }
        h[16] = h[18] > h[17] ? h[18] - h[17] : 0;   // first block start to last block end
        h[17] = h[18] = 0;
    }
    for (int i = 0; i < n && i < sdf::kStatCount; ++i) out[i] = (int64_t)h[i];
    return SDF_OK;
}

int sdf_ctx_last_kernel_ms(sdf_ctx* ctx, int32_t kernel, float* ms) {
    if (!ctx || !ms || (kernel != SDF_KERNEL_PREP && kernel != SDF_KERNEL_CHECK)) return SDF_ERR_INVALID_ARG;
    if (!ctx->timed_valid) return fail(ctx, SDF_ERR_INVALID_ARG, "no timed check recorded");
    DeviceGuard g(ctx->device);
    SDF_CUDA(ctx, cudaEventSynchronize(ctx->ev2));
    if (kernel == SDF_KERNEL_PREP)
        SDF_CUDA(ctx, cudaEventElapsedTime(ms, ctx->ev0, ctx->ev1));
    else
        SDF_CUDA(ctx, cudaEventElapsedTime(ms, ctx->ev1, ctx->ev2));
    return SDF_OK;
}

// -------------------------------------------------------------------- grids

static bool finite3(const float* v) { return std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]); }

int sdf_build_grids(sdf_ctx* ctx, const sdf_mesh* links, int32_t n_links, int32_t resolution,
                    float margin, sdf_grids** out) {
    if (!ctx || !out) return SDF_ERR_INVALID_ARG;
    *out = nullptr;
    if (!links || n_links < 1 || n_links > SDF_MAX_LINKS)
        return fail(ctx, SDF_ERR_INVALID_ARG, "n_links must be 1..%d", SDF_MAX_LINKS);
    if (resolution < 2 || resolution > SDF_MAX_RESOLUTION)
        return fail(ctx, SDF_ERR_INVALID_ARG, "resolution must be 2..%d", SDF_MAX_RESOLUTION);
    if (!(margin >= 0.f) || !std::isfinite(margin)) return fail(ctx, SDF_ERR_INVALID_ARG, "bad margin");
    for (int l = 0; l < n_links; ++l) {
        const sdf_mesh& m = links[l];
        if (!m.verts || !m.tris || m.n_verts < 3 || m.n_tris < 1 || m.n_components < 1)
            return fail(ctx, SDF_ERR_INVALID_ARG, "link %d: empty mesh", l);
        if (m.n_components > 1 && !m.comp_tri_offsets)
            return fail(ctx, SDF_ERR_INVALID_ARG, "link %d: component offsets missing", l);
        for (int v = 0; v < m.n_verts; ++v)
            if (!finite3(m.verts + 3 * v)) return fail(ctx, SDF_ERR_INVALID_ARG, "link %d: non-finite vertex", l);
        for (int t = 0; t < 3 * m.n_tris; ++t)
            if (m.tris[t] < 0 || m.tris[t] >= m.n_verts)
                return fail(ctx, SDF_ERR_INVALID_ARG, "link %d: triangle index out of range", l);
        if (m.comp_tri_offsets) {
            if (m.comp_tri_offsets[0] != 0 || m.comp_tri_offsets[m.n_components] != m.n_tris)
                return fail(ctx, SDF_ERR_INVALID_ARG, "link %d: component offsets must span 0..n_tris", l);
            for (int c = 0; c < m.n_components; ++c)
                if (m.comp_tri_offsets[c + 1] <= m.comp_tri_offsets[c])
                    return fail(ctx, SDF_ERR_INVALID_ARG, "link %d: empty or unordered component", l);
        }
    }
    DeviceGuard g(ctx->device);
    const int n = resolution;
    const size_t per = (size_t)n * n * n;
    sdf_grids* G = new (std::nothrow) sdf_grids();
    if (!G) return fail(ctx, SDF_ERR_OOM, "host allocation");
    G->device = ctx->device;
    G->n_links = n_links;
    G->n = n;
    cudaError_t e = sdf::dmalloc(&G->values, per * n_links * sizeof(float));
    if (e != cudaSuccess) {
        delete G;
        return cuda_fail(ctx, e, "device allocation (grids)");
    }
    float* d_tris = nullptr;
    int* d_off = nullptr;
    int rc = SDF_OK;
    for (int l = 0; l < n_links && rc == SDF_OK; ++l) {
        const sdf_mesh& m = links[l];
        // box and bounding sphere in double from the FP32 vertices
        double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int v = 0; v < m.n_verts; ++v)
            for (int k = 0; k < 3; ++k) {
                lo[k] = std::min(lo[k], (double)m.verts[3 * v + k]);
                hi[k] = std::max(hi[k], (double)m.verts[3 * v + k]);
            }
        double mid[3], span = 0.0;
        for (int k = 0; k < 3; ++k) {
            mid[k] = 0.5 * (lo[k] + hi[k]);
            span = std::max(span, hi[k] - lo[k]);
        }
        span += 2.0 * (double)margin;
        const double h = span / (double)(n - 1);
        double r2 = 0.0;
        for (int v = 0; v < m.n_verts; ++v) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += ((double)m.verts[3 * v + k] - mid[k]) * ((double)m.verts[3 * v + k] - mid[k]);
            r2 = std::max(r2, s);
        }
        sdf_grid_meta& md = G->meta[l];
        for (int k = 0; k < 3; ++k) {
            md.origin[k] = (float)(mid[k] - 0.5 * span);
            md.center[k] = (float)mid[k];
        }
        md.h = (float)h;
        md.n = n;
        // round the radius up so the FP32 sphere still holds every vertex
        md.radius = nextafterf((float)std::sqrt(r2), INFINITY) * (1.f + 1e-6f);
        md.margin = margin;
        // triangles as 9 floats each, components as offsets
        std::vector<float> tri9((size_t)m.n_tris * 9);
        for (int t = 0; t < m.n_tris; ++t)
            for (int c = 0; c < 3; ++c)
                for (int k = 0; k < 3; ++k) tri9[(size_t)t * 9 + 3 * c + k] = m.verts[3 * m.tris[3 * t + c] + k];
        std::vector<int> off(m.n_components + 1);
        if (m.comp_tri_offsets) {
            for (int c = 0; c <= m.n_components; ++c) off[c] = m.comp_tri_offsets[c];
        } else {
            off[0] = 0;
            off[1] = m.n_tris;
        }
        e = sdf::dmalloc(&d_tris, tri9.size() * sizeof(float));
        if (e == cudaSuccess) e = sdf::dmalloc(&d_off, off.size() * sizeof(int));
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(d_tris, tri9.data(), tri9.size() * sizeof(float), cudaMemcpyHostToDevice, ctx->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(d_off, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice, ctx->stream);
        if (e == cudaSuccess)
            e = sdf::launch_grid_build(d_tris, d_off, m.n_components, m.n_tris, md.origin[0], md.origin[1],
                                       md.origin[2], md.h, n, G->values + per * l, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) rc = cuda_fail(ctx, e, "grid build");
        sdf::dfree(d_tris);
        sdf::dfree(d_off);
        d_tris = nullptr;
        d_off = nullptr;
    }
    if (rc != SDF_OK) {
        sdf_grids_destroy(G);
        return rc;
    }
    *out = G;
    return SDF_OK;
}

int sdf_grids_upload(sdf_ctx* ctx, const float* host_values, const sdf_grid_meta* meta, int32_t n_links,
                     sdf_grids** out) {
    if (!ctx || !out) return SDF_ERR_INVALID_ARG;
    *out = nullptr;
    if (!host_values || !meta || n_links < 1 || n_links > SDF_MAX_LINKS)
        return fail(ctx, SDF_ERR_INVALID_ARG, "bad grids");
    const int n = meta[0].n;
    if (n < 2 || n > SDF_MAX_RESOLUTION) return fail(ctx, SDF_ERR_INVALID_ARG, "bad resolution");
    for (int l = 0; l < n_links; ++l) {
        if (meta[l].n != n) return fail(ctx, SDF_ERR_INVALID_ARG, "all grids need the same resolution");
        if (!(meta[l].h > 0.f) || !std::isfinite(meta[l].h) || !(meta[l].radius >= 0.f) ||
            !finite3(meta[l].origin) || !finite3(meta[l].center))
            return fail(ctx, SDF_ERR_INVALID_ARG, "link %d: bad grid metadata", l);
    }
    DeviceGuard g(ctx->device);
    sdf_grids* G = new (std::nothrow) sdf_grids();
    if (!G) return fail(ctx, SDF_ERR_OOM, "host allocation");
    G->device = ctx->device;
    G->n_links = n_links;
    G->n = n;
    for (int l = 0; l < n_links; ++l) {
        G->meta[l] = meta[l];
        // one ulp up: a nearest-FP32 radius may lie just below the exact bound
        G->meta[l].radius = nextafterf(meta[l].radius, INFINITY);
    }
    const size_t bytes = (size_t)n * n * n * n_links * sizeof(float);
    cudaError_t e = sdf::dmalloc(&G->values, bytes);
    if (e == cudaSuccess) e = cudaMemcpyAsync(G->values, host_values, bytes, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
        sdf_grids_destroy(G);
        return cuda_fail(ctx, e, "grid upload");
    }
    *out = G;
    return SDF_OK;
}

int sdf_grids_download(sdf_ctx* ctx, const sdf_grids* G, float* host_values, sdf_grid_meta* meta) {
    if (!ctx || !G) return SDF_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    if (meta)
        for (int l = 0; l < G->n_links; ++l) meta[l] = G->meta[l];
    if (host_values) {
        const size_t bytes = (size_t)G->n * G->n * G->n * G->n_links * sizeof(float);
        SDF_CUDA(ctx, cudaMemcpyAsync(host_values, G->values, bytes, cudaMemcpyDeviceToHost, ctx->stream));
        SDF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    }
    return SDF_OK;
}

int sdf_grids_info(const sdf_grids* G, int32_t* n_links, int32_t* resolution) {
    if (!G) return SDF_ERR_INVALID_ARG;
    if (n_links) *n_links = G->n_links;
    if (resolution) *resolution = G->n;
    return SDF_OK;
}

void sdf_grids_destroy(sdf_grids* G) {
    if (!G) return;
    DeviceGuard g(G->device);
    for (int l = 0; l < SDF_MAX_LINKS; ++l) {
        if (G->tex[l]) cudaDestroyTextureObject(G->tex[l]);
        sdf::afree(G->tex_arr[l]);
    }
    sdf::dfree(G->values);
    delete G;
}

// -------------------------------------------------------------------- robot

}  // extern "C"

namespace {

// A capsule (segment a-b, radius r) containing the link's surface, found from its
// grid: every surface point lies within p = h sqrt(3)/2 of a node whose value has
// magnitude <= p, so the capsule around those nodes, grown by p, contains the
// surface and hence the (bounded) solid.  The signed distance to a convex superset
// bounds the link SDF from below at every node, and so (convexity, 1-Lipschitz)
// the interpolated value everywhere: the same exact cull as the bounding sphere,
// tighter for elongated links.  The axis is the principal axis of those nodes; the
// segment ends are pulled in as far as the radius allows.  When the sphere is the
// smaller volume, the capsule degenerates to it (a = b = centre).
void link_capsule(const float* v, int n, const sdf_grid_meta& m, float4* ca, float4* cb) {
    const double h = m.h, pad = h * std::sqrt(3.0) * 0.5 * 1.0001 + 1e-7;
    std::vector<double> P;
    for (int k = 0; k < n; ++k)
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
                const float x = v[((size_t)k * n + j) * n + i];
                if (std::fabs((double)x) <= pad) {
                    P.push_back(m.origin[0] + i * h);
                    P.push_back(m.origin[1] + j * h);
                    P.push_back(m.origin[2] + k * h);
                }
            }
    const double R = m.radius;
    *ca = make_float4(m.center[0], m.center[1], m.center[2], m.radius);
    *cb = make_float4(m.center[0], m.center[1], m.center[2], 0.f);
    const size_t np = P.size() / 3;
    if (np < 2) return;
    double mu[3] = {0, 0, 0}, C[9] = {0};
    for (size_t q = 0; q < np; ++q)
        for (int a = 0; a < 3; ++a) mu[a] += P[3 * q + a] / (double)np;
    for (size_t q = 0; q < np; ++q)
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) C[3 * a + b] += (P[3 * q + a] - mu[a]) * (P[3 * q + b] - mu[b]);
    double u[3] = {0.577, 0.578, 0.576};
    for (int it = 0; it < 100; ++it) {   // power iteration: principal axis
        double w[3];
        for (int a = 0; a < 3; ++a) w[a] = C[3 * a] * u[0] + C[3 * a + 1] * u[1] + C[3 * a + 2] * u[2];
        const double nw = std::sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
        if (!(nw > 0)) break;
        for (int a = 0; a < 3; ++a) u[a] = w[a] / nw;
    }
    double rp2 = 0;
    std::vector<double> s(np), rho2(np);
    for (size_t q = 0; q < np; ++q) {
        double d[3], t = 0;
        for (int a = 0; a < 3; ++a) {
            d[a] = P[3 * q + a] - mu[a];
            t += d[a] * u[a];
        }
        double r2 = 0;
        for (int a = 0; a < 3; ++a) r2 += (d[a] - t * u[a]) * (d[a] - t * u[a]);
        s[q] = t;
        rho2[q] = r2;
        rp2 = std::max(rp2, r2);
    }
    double s_lo = INFINITY, s_hi = -INFINITY;
    for (size_t q = 0; q < np; ++q) {
        const double e = std::sqrt(std::max(rp2 - rho2[q], 0.0));
        s_hi = std::max(s_hi, s[q] - e);
        s_lo = std::min(s_lo, s[q] + e);
    }
    if (s_lo > s_hi) s_lo = s_hi = 0.5 * (s_lo + s_hi);
    double A[3], B[3], D[3], dd = 0;
    for (int a = 0; a < 3; ++a) {
        A[a] = mu[a] + s_lo * u[a];
        B[a] = mu[a] + s_hi * u[a];
        D[a] = B[a] - A[a];
        dd += D[a] * D[a];
    }
    double r = 0;
    for (size_t q = 0; q < np; ++q) {
        double x[3], t = 0;
        for (int a = 0; a < 3; ++a) {
            x[a] = P[3 * q + a] - A[a];
            t += x[a] * D[a];
        }
        t = dd > 0 ? std::min(std::max(t / dd, 0.0), 1.0) : 0.0;
        double r2 = 0;
        for (int a = 0; a < 3; ++a) r2 += (x[a] - t * D[a]) * (x[a] - t * D[a]);
        r = std::max(r, std::sqrt(r2));
    }
    r += pad;
    const double pi = 3.14159265358979323846;
    const double vol_c = pi * r * r * std::sqrt(dd) + 4.0 / 3.0 * pi * r * r * r;
    const double vol_s = 4.0 / 3.0 * pi * R * R * R;
    if (!(vol_c < vol_s)) return;
    const float rf = std::nextafter((float)r, INFINITY);
    *ca = make_float4((float)A[0], (float)A[1], (float)A[2], rf);
    *cb = make_float4((float)B[0], (float)B[1], (float)B[2], 0.f);
}

// The hardware-filtered copy of the grids (SDF_OPT_TEX3D): per link a 3-D array of
// the FP32 values and a texture object with linear filtering, clamped addressing
// and unnormalised coordinates (texel (i,j,k) is sampled at (i,j,k) + 1/2).  Made
// once per grids object; allocates and synchronises.
int grid_textures(sdf_ctx* ctx, sdf_grids* G) {
    if (G->tex_ready) return SDF_OK;
    const int n = G->n;
    const size_t n3 = (size_t)n * n * n;
    cudaError_t e = cudaSuccess;
    for (int l = 0; l < G->n_links && e == cudaSuccess; ++l) {
        if (!G->tex_arr[l]) e = sdf::amalloc3d(&G->tex_arr[l], n);
        if (e != cudaSuccess) break;
        cudaMemcpy3DParms cp = {};
        cp.srcPtr = make_cudaPitchedPtr(G->values + l * n3, (size_t)n * sizeof(float), (size_t)n, (size_t)n);
        cp.dstArray = G->tex_arr[l];
        cp.extent = make_cudaExtent((size_t)n, (size_t)n, (size_t)n);
        cp.kind = cudaMemcpyDeviceToDevice;
        e = cudaMemcpy3DAsync(&cp, ctx->stream);
        if (e != cudaSuccess) break;
        if (!G->tex[l]) {
            cudaResourceDesc rd = {};
            rd.resType = cudaResourceTypeArray;
            rd.res.array.array = G->tex_arr[l];
            cudaTextureDesc td = {};
            td.addressMode[0] = td.addressMode[1] = td.addressMode[2] = cudaAddressModeClamp;
            td.filterMode = cudaFilterModeLinear;
            td.readMode = cudaReadModeElementType;
            td.normalizedCoords = 0;
            e = cudaCreateTextureObject(&G->tex[l], &rd, &td, nullptr);
        }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    // on failure the arrays and objects made so far stay with G (sdf_grids_destroy frees them)
    if (e != cudaSuccess) return cuda_fail(ctx, e, "texture copy of the grids");
    G->tex_ready = true;
    return SDF_OK;
}

int grid_capsules(sdf_ctx* ctx, sdf_grids* G) {
    if (G->capsules) return SDF_OK;
    const size_t n3 = (size_t)G->n * G->n * G->n;
    std::vector<float> v(n3);
    for (int l = 0; l < G->n_links; ++l) {
        const cudaError_t e = cudaMemcpy(v.data(), G->values + l * n3, n3 * sizeof(float), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "grid download (capsules)");
        link_capsule(v.data(), G->n, G->meta[l], &G->cap_a[l], &G->cap_b[l]);
    }
    G->capsules = true;
    return SDF_OK;
}

}  // namespace

extern "C" {

int sdf_robot_create(sdf_ctx* ctx, const sdf_dh* dh, int32_t dof, const float* base_3x4,
                     const sdf_grids* grids, sdf_robot** out) {
    if (!ctx || !out) return SDF_ERR_INVALID_ARG;
    *out = nullptr;
    if (!grids || dof < 0 || dof + 1 > SDF_MAX_LINKS || (dof > 0 && !dh))
        return fail(ctx, SDF_ERR_INVALID_ARG, "dof must be 0..%d with a DH table", SDF_MAX_LINKS - 1);
    if (grids->n_links != dof + 1)
        return fail(ctx, SDF_ERR_INVALID_ARG, "robot with %d joints needs %d grids, got %d", dof, dof + 1,
                    grids->n_links);
    for (int j = 0; j < dof; ++j)
        if (!std::isfinite(dh[j].a) || !std::isfinite(dh[j].alpha) || !std::isfinite(dh[j].d) ||
            !std::isfinite(dh[j].theta_offset))
            return fail(ctx, SDF_ERR_INVALID_ARG, "joint %d: non-finite DH row", j);
    if (base_3x4)
        for (int k = 0; k < 12; ++k)
            if (!std::isfinite(base_3x4[k])) return fail(ctx, SDF_ERR_INVALID_ARG, "non-finite base transform");
    sdf_robot* R = new (std::nothrow) sdf_robot();
    if (!R) return fail(ctx, SDF_ERR_OOM, "host allocation");
    static std::atomic<uint64_t> next_robot_id{1};
    R->device = ctx->device;
    R->dof = dof;
    R->grids = grids;
    R->id = next_robot_id.fetch_add(1);
    sdf::LinkTable& T = R->table;
    memset(&T, 0, sizeof T);
    T.L = dof + 1;
    T.dof = dof;
    T.n = grids->n;
    static const float kId[12] = {1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0};
    memcpy(T.base, base_3x4 ? base_3x4 : kId, sizeof T.base);
    for (int j = 0; j < dof; ++j) {
        T.dh_a[j] = dh[j].a;
        T.dh_d[j] = dh[j].d;
        T.dh_ca[j] = (float)std::cos((double)dh[j].alpha);
        T.dh_sa[j] = (float)std::sin((double)dh[j].alpha);
        T.dh_th[j] = dh[j].theta_offset;
    }
    {
        DeviceGuard g0(ctx->device);
        const int rc = grid_capsules(ctx, const_cast<sdf_grids*>(grids));
        if (rc != SDF_OK) {
            delete R;
            return rc;
        }
    }
    for (int l = 0; l < T.L; ++l) {
        const sdf_grid_meta& m = grids->meta[l];
        T.sph_local[l] = make_float4(m.center[0], m.center[1], m.center[2], m.radius);
        T.cap_a[l] = grids->cap_a[l];
        T.cap_b[l] = grids->cap_b[l];
        T.grid_o[l] = make_float4(m.origin[0], m.origin[1], m.origin[2], (float)(1.0 / (double)m.h));
        T.grid_h[l] = m.h;
    }
    T.values = grids->values;
    DeviceGuard g(ctx->device);
    cudaError_t e = sdf::dmalloc(&R->d_table, sizeof(sdf::LinkTable));
    if (e == cudaSuccess) e = cudaMemcpy(R->d_table, &T, sizeof(sdf::LinkTable), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        sdf_robot_destroy(R);
        return cuda_fail(ctx, e, "robot table upload");
    }
    *out = R;
    return SDF_OK;
}

void sdf_robot_destroy(sdf_robot* R) {
    if (!R) return;
    if (R->d_table) {
        DeviceGuard g(R->device);
        sdf::dfree(R->d_table);
    }
    delete R;
}

int sdf_forward_kinematics(sdf_ctx* ctx, const sdf_robot* R, const float* q_dev, int32_t W, float* out_dev) {
    if (!ctx || !R || W < 0) return SDF_ERR_INVALID_ARG;
    if (W == 0) return SDF_OK;
    if ((R->dof > 0 && !q_dev) || !out_dev) return fail(ctx, SDF_ERR_INVALID_ARG, "null buffer");
    if ((reinterpret_cast<uintptr_t>(out_dev) & 15u) != 0)
        return fail(ctx, SDF_ERR_INVALID_ARG, "output must be 16-byte aligned");
    DeviceGuard g(ctx->device);
    SDF_CUDA(ctx, sdf::launch_fk(R->table, q_dev, W, out_dev, ctx->status, ctx->stream));
    return SDF_OK;
}

// -------------------------------------------------------------------- check

// ------------------------------------------------------------------ batches

static int validate_request(sdf_ctx* ctx, const sdf_check_request& r, int idx) {
    if (!r.robot) return fail(ctx, SDF_ERR_INVALID_ARG, "request %d: null robot", idx);
    if (r.robot->device != ctx->device) return fail(ctx, SDF_ERR_INVALID_ARG, "request %d: robot on another device", idx);
    if (r.W < 0 || r.N < 0) return fail(ctx, SDF_ERR_INVALID_ARG, "request %d: negative size", idx);
    if (r.N > SDF_MAX_POINTS) return fail(ctx, SDF_ERR_INVALID_ARG, "request %d: N > %d", idx, SDF_MAX_POINTS);
    if (r.W == 0) return SDF_OK;
    if (!r.dist_dev || !r.argmin_link_dev || !r.argmin_point_dev || (r.robot->dof > 0 && !r.q_dev) ||
        (r.N > 0 && !r.points_dev))
        return fail(ctx, SDF_ERR_INVALID_ARG, "request %d: null buffer", idx);
    const uintptr_t pa = reinterpret_cast<uintptr_t>(r.points_dev);
    if ((ctx->point_stride == 4 && (pa & 15u) != 0) || (pa & 3u) != 0)
        return fail(ctx, SDF_ERR_INVALID_ARG, "request %d: points misaligned", idx);
    return SDF_OK;
}

// Scratch for up to the given totals; growth synchronises the device, so a launch
// that fits needs no allocation (and can be captured in a CUDA graph).
static int reserve_scratch(sdf_ctx* ctx, size_t points, size_t tiles, size_t supers, size_t instances) {
    int rc = grow(ctx, &ctx->sorted, &ctx->sorted_cap, std::max<size_t>(points, 1), false);
    if (rc == SDF_OK) rc = grow(ctx, &ctx->tiles, &ctx->tiles_cap, std::max<size_t>(tiles, 1), false);
    if (rc == SDF_OK) rc = grow(ctx, &ctx->supers, &ctx->supers_cap, std::max<size_t>(supers, 1), false);
    if (rc == SDF_OK) rc = grow(ctx, &ctx->n_valid, &ctx->n_valid_cap, std::max<size_t>(instances, 1), false);
    return rc;
}

}  // extern "C"

namespace sdf {

// Sort one cloud into the context's scratch (the layout check_batch uses for a
// single request) and fill p for kernels that read it.  Asynchronous.
int sort_cloud(sdf_ctx* ctx, const float* points_dev, int N, BatchParams* p) {
    const uintptr_t pa = reinterpret_cast<uintptr_t>(points_dev);
    if (N < 0 || N > SDF_MAX_POINTS || (N > 0 && !points_dev) || (pa & 3u) != 0 ||
        (ctx->point_stride == 4 && (pa & 15u) != 0))
        return fail(ctx, SDF_ERR_INVALID_ARG, "cloud: invalid points");
    const size_t tiles = ((size_t)N + 31) / 32;
    int rc = reserve_scratch(ctx, (size_t)N, tiles, (tiles + 31) / 32, 1);
    if (rc != SDF_OK) return rc;
    CloudDesc& C = p->cloud[0];
    C.points = points_dev;
    C.N = N;
    C.point_base = C.tile_base = C.super_base = 0;
    p->n_cloud = 1;
    p->stride = ctx->point_stride;
    p->cull = ctx->cull;
    p->sorted = ctx->sorted;
    p->tiles = ctx->tiles;
    p->supers = ctx->supers;
    p->n_valid = ctx->n_valid;
    p->status = ctx->status;
    p->wait_polls = ctx->wait_polls;
    p->sort_ctas = ctx->sort_ctas;
    p->stats = nullptr;
    const cudaError_t e = launch_prep(*p, ctx->stream);
    return e == cudaSuccess ? SDF_OK : cuda_fail(ctx, e, "cloud sort");
}

}  // namespace sdf

extern "C" {

int sdf_ctx_reserve(sdf_ctx* ctx, int64_t max_points, int64_t max_waypoints, int64_t max_pairs, int32_t max_requests) {
    if (!ctx || max_points < 0 || max_waypoints < 0 || max_pairs < 0 || max_requests < 0 || max_requests > SDF_MAX_BATCH)
        return SDF_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    const size_t P = (size_t)max_points, R = (size_t)std::max(max_requests, 1);
    const size_t tiles = (P + 31) / 32 + R, supers = tiles / 32 + R;
    return reserve_scratch(ctx, P, tiles, supers, R);
}

// Launch-shape key of a batch for the tuning cache: request count, the largest
// link count, and power-of-two buckets of the total waypoints and points.
static uint64_t shape_key(const sdf_check_request* reqs, int n) {
    uint64_t W = 0, N = 0, L = 0, k = 0;
    for (int i = 0; i < n; ++i) {
        if (reqs[i].W == 0) continue;
        ++k;
        W += (uint64_t)reqs[i].W;
        N += (uint64_t)reqs[i].N;
        L = std::max<uint64_t>(L, (uint64_t)reqs[i].robot->table.L);
    }
    auto lg = [](uint64_t v) { uint64_t b = 0; while (v > 1) { v >>= 1; ++b; } return b; };
    return (k << 40) | (L << 32) | (lg(W) << 16) | lg(N);
}

// Warps per check block for a launch whose largest robot has Lmax links and that
// checks W_total waypoints: the option, else the tuned value for this shape, else
// 8 when one-waypoint blocks would leave SMs idle (W_total <= SMs), 16 otherwise
// (two interleaved waypoints a block even out uneven waypoints); 8 only when a
// waypoint's links fit (one warp per waypoint and link).
static int launch_warps(const sdf_ctx* ctx, uint64_t key, int Lmax, size_t W_total) {
    int nw = ctx->block_warps;
    if (nw == 0) {
        auto it = ctx->tuned.find(key);
        nw = it != ctx->tuned.end() ? it->second.nw : (W_total <= (size_t)ctx->num_sms ? 8 : 16);
    }
    return (nw == 8 && Lmax <= 8) ? 8 : 16;
}

// Waypoints per check block for a robot with L links in blocks of nw warps, and
// list entries per warp step: explicit options first, then a tuned configuration
// for this launch shape, then the defaults.
static void launch_shape(const sdf_ctx* ctx, uint64_t key, int L, int nw, int* tw, int* tb) {
    const int fit = std::max(1, nw / L);
    int t = ctx->tw, b = ctx->tile_batch;
    auto it = ctx->tuned.find(key);
    if (it != ctx->tuned.end()) {
        if (t == 0) t = it->second.tw;
        if (b == 0) b = it->second.tb;
    }
    *tw = t > 0 ? std::min(t, fit) : fit;
    *tb = b > 0 ? b : sdf::kDefaultTileBatch;
}

int check_batch(sdf_ctx* ctx, const sdf_check_request* reqs, int32_t n) {
    if (!ctx) return SDF_ERR_INVALID_ARG;
    if (n < 0 || n > SDF_MAX_BATCH) return fail(ctx, SDF_ERR_INVALID_ARG, "batch size must be 0..%d", SDF_MAX_BATCH);
    if (n > 0 && !reqs) return fail(ctx, SDF_ERR_INVALID_ARG, "null request array");
    for (int i = 0; i < n; ++i) {
        const int rc = validate_request(ctx, reqs[i], i);
        if (rc != SDF_OK) return rc;
    }
    const sdf_grids* tex_grids = nullptr;
    if (ctx->tex3d) {   // the texture copy of the grids (made once; may synchronise)
        for (int i = 0; i < n; ++i)
            if (reqs[i].W > 0) {
                if (tex_grids && reqs[i].robot->grids != tex_grids)
                    return fail(ctx, SDF_ERR_UNSUPPORTED, "SDF_OPT_TEX3D: every request of a launch must use one grids object");
                tex_grids = reqs[i].robot->grids;
            }
        if (tex_grids) {
            DeviceGuard g(ctx->device);
            const int rc = grid_textures(ctx, const_cast<sdf_grids*>(tex_grids));
            if (rc != SDF_OK) return rc;
        }
    }
    sdf::BatchParams* p = new (std::nothrow) sdf::BatchParams();
    if (!p) return fail(ctx, SDF_ERR_OOM, "host allocation");
    const uint64_t key = shape_key(reqs, n);
    int tile_batch = sdf::kDefaultTileBatch;
    size_t points = 0, tiles = 0, supers = 0, blocks = 0, max_tiles = 0;
    int Lmax = 1;
    size_t W_total = 0;
    for (int i = 0; i < n; ++i)
        if (reqs[i].W > 0) {
            Lmax = std::max(Lmax, reqs[i].robot->table.L);
            W_total += (size_t)reqs[i].W;
        }
    const int nw = launch_warps(ctx, key, Lmax, W_total);
    int k = 0, nc = 0;
    for (int i = 0; i < n; ++i) {
        const sdf_check_request& r = reqs[i];
        if (r.W == 0) continue;
        // requests passing the same cloud share its sort
        int c = 0;
        while (c < nc && !(p->cloud[c].points == r.points_dev && p->cloud[c].N == r.N)) ++c;
        if (c == nc) {
            sdf::CloudDesc& C = p->cloud[nc++];
            C.points = r.points_dev;
            C.N = r.N;
            C.point_base = (int)points;
            C.tile_base = (int)tiles;
            C.super_base = (int)supers;
            const size_t nt = ((size_t)r.N + 31) / 32;
            points += (size_t)r.N;
            tiles += nt;
            supers += (nt + 31) / 32;
            max_tiles = std::max(max_tiles, nt);
        }
        sdf::InstDesc& I = p->inst[k++];
        I.robot = r.robot->d_table;
        I.q = r.q_dev;
        I.dist = r.dist_dev;
        I.arg_link = r.argmin_link_dev;
        I.arg_point = r.argmin_point_dev;
        I.W = r.W;
        I.L = r.robot->table.L;
        I.dof = r.robot->dof;
        I.cloud = c;
        I.mask = r.mask_dev;
        // the linear grids are prefetched into L2 only when the lookups read them
        I.warm = ctx->tex3d ? nullptr : r.robot->table.values;
        I.warm_bytes = (unsigned long long)I.L * r.robot->table.n * r.robot->table.n * r.robot->table.n * sizeof(float);
        for (int j = 0; j < k - 1 && I.warm; ++j)
            if (p->inst[j].warm == I.warm) I.warm = nullptr;   // warmed by an earlier trajectory
        launch_shape(ctx, key, I.L, nw, &I.tw, &tile_batch);
        I.block_base = (int)blocks;
        blocks += ((size_t)r.W + I.tw - 1) / I.tw;
    }
    if (k == 0 || points > (size_t)INT32_MAX || blocks > (size_t)INT32_MAX) {
        delete p;
        return k == 0 ? SDF_OK : fail(ctx, SDF_ERR_INVALID_ARG, "batch too large");
    }
    DeviceGuard g(ctx->device);
    int rc = reserve_scratch(ctx, points, tiles, supers, (size_t)nc);
    if (rc != SDF_OK) {
        delete p;
        return rc;
    }
    p->n_inst = k;
    p->n_cloud = nc;
    p->n_blocks = (int)blocks;
    for (int i = 0; i < k; ++i)
        p->inst[i].interleave = sdf::interleave_waypoints((long long)blocks, p->inst[i].tw, nw, ctx->num_sms);
    p->stride = ctx->point_stride;
    p->cull = ctx->cull;
    p->stage_tiles = (int)std::min<size_t>(max_tiles, (size_t)sdf::kMaxStagedTiles);
    p->skip_prep = ctx->reuse_sort;
    p->warm_l2 = !ctx->reuse_sort && !ctx->time_kernels;   // the launches that overlap check and sort
    p->warps = nw;
    p->tex = tex_grids ? 1 : 0;
    if (tex_grids)
        for (int l = 0; l < tex_grids->n_links; ++l) p->tex_h[l] = (unsigned long long)tex_grids->tex[l];
    p->sorted = ctx->sorted;
    p->tiles = ctx->tiles;
    p->supers = ctx->supers;
    p->n_valid = ctx->n_valid;
    p->status = ctx->status;
    p->wait_polls = ctx->wait_polls;
    p->sort_ctas = ctx->sort_ctas;
    if (p->sort_ctas == 0) {   // the tuned width for this launch shape, else the widest
        auto it = ctx->tuned.find(key);
        if (it != ctx->tuned.end()) p->sort_ctas = it->second.sort;
    }
    p->stats = ctx->stats ? ctx->d_stats : nullptr;
    cudaError_t e = cudaSuccess;
    if (ctx->time_kernels) e = cudaEventRecord(ctx->ev0, ctx->stream);
    if (e == cudaSuccess) e = sdf::launch_batch(*p, tile_batch, ctx->stream, ctx->time_kernels ? ctx->ev1 : nullptr);
    if (e == cudaSuccess && ctx->time_kernels) {
        e = cudaEventRecord(ctx->ev2, ctx->stream);
        ctx->timed_valid = true;
    }
    delete p;
    if (e != cudaSuccess) return cuda_fail(ctx, e, "check launch");
    return SDF_OK;
}

int sdf_autotune(sdf_ctx* ctx, const sdf_check_request* reqs, int32_t n, int32_t repeats, int32_t* best_tw,
                 int32_t* best_tile_batch, float* best_us) {
    if (!ctx || repeats < 1) return SDF_ERR_INVALID_ARG;
    if (n < 1 || n > SDF_MAX_BATCH || !reqs) return fail(ctx, SDF_ERR_INVALID_ARG, "autotune needs 1..%d requests", SDF_MAX_BATCH);
    int Lmin = sdf::kMaxLinks;
    for (int i = 0; i < n; ++i) {
        const int rc = validate_request(ctx, reqs[i], i);
        if (rc != SDF_OK) return rc;
        if (reqs[i].W > 0) Lmin = std::min(Lmin, reqs[i].robot->table.L);
    }
    DeviceGuard g(ctx->device);
    const uint64_t key = shape_key(reqs, n);
    const int save_tw = ctx->tw, save_tb = ctx->tile_batch, save_time = ctx->time_kernels,
              save_nw = ctx->block_warps, save_sort = ctx->sort_ctas;
    ctx->time_kernels = 0;
    ctx->tuned.erase(key);
    cudaEvent_t a = nullptr, b = nullptr;
    SDF_CUDA(ctx, cudaEventCreate(&a));
    SDF_CUDA(ctx, cudaEventCreate(&b));
    float best = INFINITY;
    int btw = 0, btb = 0, bnw = 16, rc = SDF_OK;
    const int tbs[3] = {1, 2, 4};
    int Lmax = 1;
    for (int i = 0; i < n; ++i)
        if (reqs[i].W > 0) Lmax = std::max(Lmax, reqs[i].robot->table.L);
    for (int nw = 16; nw >= 8 && rc == SDF_OK; nw -= 8) {
      if (nw == 8 && Lmax > 8) break;
      const int fit = std::max(1, nw / Lmin);
      for (int tw = 1; tw <= fit && rc == SDF_OK; ++tw) {
        for (int tb : tbs) {
            ctx->tw = tw;
            ctx->tile_batch = tb;
            ctx->block_warps = nw;
            rc = check_batch(ctx, reqs, n);   // warm-up, grows scratch if needed
            std::vector<float> ms;
            for (int r = 0; r < repeats && rc == SDF_OK; ++r) {
                cudaEventRecord(a, ctx->stream);
                rc = check_batch(ctx, reqs, n);
                cudaEventRecord(b, ctx->stream);
                float t = 0.f;
                if (cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&t, a, b) != cudaSuccess) rc = SDF_ERR_CUDA;
                ms.push_back(t);
            }
            if (rc != SDF_OK) break;
            std::nth_element(ms.begin(), ms.begin() + ms.size() / 2, ms.end());
            const float med = ms[ms.size() / 2];
            if (med < best) {
                best = med;
                btw = tw;
                btb = tb;
                bnw = nw;
            }
        }
      }
    }
    // the sort's cluster width at the best shape: 8, and 16 where the device allows it
    int bsort = 0;
    if (rc == SDF_OK && sdf::max_sort_ctas(ctx->device) == 16) {
        ctx->tw = btw;
        ctx->tile_batch = btb;
        ctx->block_warps = bnw;
        float best_sort = INFINITY;
        for (int width : {16, 8}) {
            ctx->sort_ctas = width;
            rc = check_batch(ctx, reqs, n);
            std::vector<float> ms;
            for (int r = 0; r < repeats && rc == SDF_OK; ++r) {
                cudaEventRecord(a, ctx->stream);
                rc = check_batch(ctx, reqs, n);
                cudaEventRecord(b, ctx->stream);
                float t = 0.f;
                if (cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&t, a, b) != cudaSuccess) rc = SDF_ERR_CUDA;
                ms.push_back(t);
            }
            if (rc != SDF_OK) break;
            std::nth_element(ms.begin(), ms.begin() + ms.size() / 2, ms.end());
            const float med = ms[ms.size() / 2];
            if (med < best_sort) {
                best_sort = med;
                bsort = width;
            }
        }
        if (rc == SDF_OK) best = std::min(best, best_sort);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    ctx->tw = save_tw;
    ctx->tile_batch = save_tb;
    ctx->time_kernels = save_time;
    ctx->block_warps = save_nw;
    ctx->sort_ctas = save_sort;
    if (rc != SDF_OK) return rc;
    ctx->tuned[key] = sdf_ctx::Shape{btw, btb, bnw, bsort};
    drop_host_graphs(ctx);
    if (best_tw) *best_tw = btw;
    if (best_tile_batch) *best_tile_batch = btb;
    if (best_us) *best_us = best * 1e3f;
    return SDF_OK;
}

int check_trajectory(sdf_ctx* ctx, const sdf_robot* R, const float* q_dev, int32_t W, const float* points_dev,
                     int32_t N, float* dist_dev, int32_t* argmin_link_dev, int32_t* argmin_point_dev) {
    if (!ctx || !R) return SDF_ERR_INVALID_ARG;
    sdf_check_request r{};
    r.robot = R;
    r.q_dev = q_dev;
    r.W = W;
    r.points_dev = points_dev;
    r.N = N;
    r.dist_dev = dist_dev;
    r.argmin_link_dev = argmin_link_dev;
    r.argmin_point_dev = argmin_point_dev;
    return check_batch(ctx, &r, 1);
}

int check_trajectory_host(sdf_ctx* ctx, const sdf_robot* R, const float* q_host, int32_t W,
                          const float* points_host, int32_t N, float* dist_host, int32_t* argmin_link_host,
                          int32_t* argmin_point_host) {
    if (!ctx || !R) return SDF_ERR_INVALID_ARG;
    if (W < 0 || N < 0) return fail(ctx, SDF_ERR_INVALID_ARG, "negative size");
    if (W == 0) return SDF_OK;
    if (!dist_host || !argmin_link_host || !argmin_point_host || (R->dof > 0 && !q_host) ||
        (N > 0 && !points_host))
        return fail(ctx, SDF_ERR_INVALID_ARG, "null buffer");
    DeviceGuard g(ctx->device);
    const size_t nq = (size_t)W * std::max(R->dof, 1);
    const size_t np = (size_t)std::max(N, 1) * ctx->point_stride;
    int rc = grow(ctx, &ctx->st_q, &ctx->st_q_cap, nq, false);
    if (rc == SDF_OK) rc = grow(ctx, &ctx->st_pts, &ctx->st_pts_cap, np, false);
    if (rc == SDF_OK && (size_t)W > ctx->st_out_cap) {
        drop_host_graphs(ctx);
        sdf::dfree(ctx->st_dist);
        sdf::dfree(ctx->st_link);
        sdf::dfree(ctx->st_point);
        ctx->st_dist = nullptr;
        ctx->st_link = ctx->st_point = nullptr;
        ctx->st_out_cap = 0;
        const size_t cap = std::max((size_t)W, (size_t)1024);
        if (sdf::dmalloc(&ctx->st_dist, cap * sizeof(float)) != cudaSuccess ||
            sdf::dmalloc(&ctx->st_link, cap * sizeof(int32_t)) != cudaSuccess ||
            sdf::dmalloc(&ctx->st_point, cap * sizeof(int32_t)) != cudaSuccess)
            rc = fail(ctx, SDF_ERR_OOM, "staging allocation");
        else
            ctx->st_out_cap = cap;
    }
    if (rc != SDF_OK) return rc;
    // scratch for this cloud before any capture (growing it synchronises)
    {
        const size_t tiles = ((size_t)N + 31) / 32;
        rc = reserve_scratch(ctx, (size_t)N, tiles, (tiles + 31) / 32, 1);
        if (rc != SDF_OK) return rc;
    }
    // Page-locked host buffers are read and written by the kernels themselves over
    // the CPU-GPU link (no copies); other host memory goes through device staging.
    bool zero_copy = true;
    const void* hp[5] = {q_host, points_host, dist_host, argmin_link_host, argmin_point_host};
    void* dp[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    for (int k = 0; k < 5 && zero_copy; ++k) {
        if ((k == 0 && R->dof == 0) || (k == 1 && N == 0)) continue;
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, hp[k]) != cudaSuccess || a.type != cudaMemoryTypeHost || !a.devicePointer)
            zero_copy = false;
        else
            dp[k] = a.devicePointer;
    }
    cudaGetLastError();   // a pointer unknown to CUDA is not an error here
    // copies in, the check, copies out
    auto enqueue = [&](cudaStream_t st) -> int {
        if (zero_copy) {
            cudaStream_t saved = ctx->stream;
            ctx->stream = st;
            int r = check_trajectory(ctx, R, static_cast<const float*>(dp[0]), W, static_cast<const float*>(dp[1]),
                                     N, static_cast<float*>(dp[2]), static_cast<int32_t*>(dp[3]),
                                     static_cast<int32_t*>(dp[4]));
            if (r == SDF_OK && sdf::launch_finish(ctx->status, ctx->h_status, ctx->d_seq, ctx->h_done, st) !=
                                   cudaSuccess)
                r = SDF_ERR_CUDA;
            ctx->stream = saved;
            return r;
        }
        cudaStream_t saved = ctx->stream;
        ctx->stream = st;
        int r = SDF_OK;
        if (R->dof > 0 && cudaMemcpyAsync(ctx->st_q, q_host, (size_t)W * R->dof * sizeof(float),
                                          cudaMemcpyHostToDevice, st) != cudaSuccess)
            r = SDF_ERR_CUDA;
        if (r == SDF_OK && N > 0 &&
            cudaMemcpyAsync(ctx->st_pts, points_host, (size_t)N * ctx->point_stride * sizeof(float),
                            cudaMemcpyHostToDevice, st) != cudaSuccess)
            r = SDF_ERR_CUDA;
        if (r == SDF_OK) r = check_trajectory(ctx, R, ctx->st_q, W, ctx->st_pts, N, ctx->st_dist, ctx->st_link,
                                              ctx->st_point);
        if (r == SDF_OK && (cudaMemcpyAsync(dist_host, ctx->st_dist, (size_t)W * sizeof(float),
                                            cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                            cudaMemcpyAsync(argmin_link_host, ctx->st_link, (size_t)W * sizeof(int32_t),
                                            cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                            cudaMemcpyAsync(argmin_point_host, ctx->st_point, (size_t)W * sizeof(int32_t),
                                            cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                            enqueue_status_readback(ctx, st) != cudaSuccess))
            r = SDF_ERR_CUDA;
        ctx->stream = saved;
        return r;
    };
    if (ctx->time_kernels || ctx->stats) {   // per-kernel events and counters: no graph
        rc = enqueue(ctx->stream);
        if (rc != SDF_OK) return rc == SDF_ERR_CUDA ? cuda_fail(ctx, cudaGetLastError(), "host check") : rc;
        SDF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        ctx->seq = *ctx->h_done;
        return status_code(ctx);
    }
    const void* ptr[5] = {q_host, points_host, dist_host, argmin_link_host, argmin_point_host};
    cudaGraphExec_t exec = nullptr;
    for (auto& hg : ctx->host_graphs)
        if (hg.robot == R->id && hg.W == W && hg.N == N && hg.zero_copy == zero_copy &&
            std::equal(ptr, ptr + 5, hg.ptr))
            exec = hg.exec;
    if (!exec) {
        // capture the call once on the context's own stream, then replay it; when the
        // capture is refused (some host memory cannot be captured), run it directly
        if (!ctx->capture_stream)
            SDF_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking));
        cudaGraph_t graph = nullptr;
        int r = SDF_ERR_CUDA;
        if (cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            r = enqueue(ctx->capture_stream);
            if (cudaStreamEndCapture(ctx->capture_stream, &graph) != cudaSuccess) r = SDF_ERR_CUDA;
        }
        if (r == SDF_OK && graph && cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) exec = nullptr;
        if (graph) cudaGraphDestroy(graph);
        if (!exec) {
            cudaGetLastError();   // clear the refused capture's error
            rc = enqueue(ctx->stream);
            if (rc != SDF_OK) return rc == SDF_ERR_CUDA ? cuda_fail(ctx, cudaGetLastError(), "host check") : rc;
            SDF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
            ctx->seq = *ctx->h_done;
            return status_code(ctx);
        }
        if (ctx->host_graphs.size() >= 8) drop_host_graphs(ctx);
        sdf_ctx::HostGraph hg{R->id, {}, W, N, zero_copy, exec};
        std::copy(ptr, ptr + 5, hg.ptr);
        ctx->host_graphs.push_back(hg);
    }
    SDF_CUDA(ctx, cudaGraphLaunch(exec, ctx->stream));
    if (zero_copy && wait_done(ctx, ++ctx->seq)) return status_code(ctx);
    SDF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    ctx->seq = *ctx->h_done;   // back in step after a synchronisation
    return status_code(ctx);
}

}  // extern "C"
