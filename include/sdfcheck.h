/*
 * sdfcheck -- batched runtime robot/obstacle distance check on one GPU (C ABI).
 *
 * Method: Fujii & Pham, "Real-time Batched Distance Computation for Time-Optimal
 * Safe Path Tracking" (arXiv 2309.12543).  For every configuration (waypoint) of a
 * trajectory the library returns the minimum signed distance between the robot's
 * links and a set of obstacle points, with the arg-min link and point (Sec. III-A:
 * "extracting the distances at the voxels occupied by the obstacles and taking the
 * minimum").  Distances come from Link SDFs -- signed distance grids of each link
 * in its own frame (Sec. III-A, "Link SDFs").  Obstacle points are mapped into
 * every link frame (the per-point form contrasted in Sec. II-B and Fig. 2) and the
 * link grid is interpolated trilinearly (the grid-sample interpolation of Sec.
 * III-A).
 *
 * Conventions (all entry points):
 *   - Units are metres and radians; the world frame is the robot base frame unless
 *     a base transform is given.
 *   - Transforms are 3x4 row-major [R | t] (world-from-frame), FP32.
 *   - Link 0 is the static base link (frame 0); link j (1..dof) is DH frame j.
 *     A robot with `dof` joints has L = dof + 1 links and needs L grids.
 *   - Pointers named *_dev are CUDA device pointers, *_host host pointers.  The
 *     caller owns every buffer it passes; the library copies host meshes and
 *     tables during the call and owns the objects it creates (ctx, grids,
 *     robot), freed by the matching *_destroy.
 *   - Work is enqueued on the context's CUDA stream and the call returns without
 *     waiting, except where a function says it synchronises.  Results are valid
 *     after the stream has been synchronised.  Calls on one context must not be
 *     made from several host threads at once.
 *   - Every int-returning function returns SDF_OK (0) or a negative SDF_ERR_*
 *     code; no C++ exception crosses this boundary.  sdf_last_error() gives a
 *     message for the last failure on a context.  Faults that happen on the
 *     device after a call returned surface in sdf_ctx_synchronize().
 */
#ifndef SDFCHECK_H
#define SDFCHECK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status codes */
#define SDF_OK 0
#define SDF_ERR_INVALID_ARG (-1)  /* bad pointer, size, layout or mismatched objects */
#define SDF_ERR_OOM (-2)          /* device or host allocation failed                 */
#define SDF_ERR_CUDA (-3)         /* a CUDA runtime call failed (message has details)  */
#define SDF_ERR_TIMEOUT (-4)      /* a bounded device wait gave up                     */
#define SDF_ERR_UNSUPPORTED (-5)  /* device or option not supported by this build      */
#define SDF_ERR_NONFINITE (-6)    /* a NaN/Inf joint value or point was seen           */
#define SDF_PENDING 1             /* sdf_server_poll: the request is not finished yet  */

#define SDF_MAX_LINKS 16          /* L = dof + 1 <= 16                                  */
#define SDF_MAX_POINTS 16777215   /* N < 2^24 (point index packed with waypoint/link)  */
#define SDF_MAX_RESOLUTION 512    /* grid nodes per axis                               */
#define SDF_MAX_BATCH 128         /* trajectories per check_batch call                 */

typedef struct sdf_ctx sdf_ctx;       /* device, stream, scratch, options          */
typedef struct sdf_grids sdf_grids;   /* device Link SDF grids + per-link metadata */
typedef struct sdf_robot sdf_robot;   /* DH table + base transform + grids          */

/* A link mesh in its own frame: closed, outward (counter-clockwise seen from
 * outside) triangles.  Several closed components may form one link (a union);
 * component c is triangles [comp_tri_offsets[c], comp_tri_offsets[c+1]).  With
 * n_components == 1, comp_tri_offsets may be NULL. */
typedef struct {
    const float* verts;               /* host, n_verts x 3                          */
    int32_t n_verts;
    const int32_t* tris;              /* host, n_tris x 3 vertex indices            */
    int32_t n_tris;
    int32_t n_components;
    const int32_t* comp_tri_offsets;  /* host, n_components + 1 entries, or NULL    */
} sdf_mesh;

/* Standard Denavit-Hartenberg row of one revolute joint: the joint transform is
 * Rz(theta_offset + q) Tz(d) Tx(a) Rx(alpha).  q_min/q_max are informational. */
typedef struct {
    float a, alpha, d, theta_offset, q_min, q_max;
} sdf_dh;

/* Grid of one link: node (i,j,k) sits at origin + (i,j,k) h, value index
 * i + n (j + n k) (x fastest).  center/radius bound the link mesh (every vertex
 * lies within radius of center).  margin is informational. */
typedef struct {
    float origin[3];
    float h;
    int32_t n;
    float center[3];
    float radius;
    float margin;
} sdf_grid_meta;

/* ------------------------------------------------------------------- context */

/* Create a context on `device` that enqueues on `cuda_stream` (a cudaStream_t;
 * NULL = the legacy default stream).  Errors: INVALID_ARG (out NULL, bad device),
 * UNSUPPORTED (device is not compute capability 10.3), CUDA, OOM. */
int sdf_ctx_create(sdf_ctx** out, int device, void* cuda_stream);
void sdf_ctx_destroy(sdf_ctx* ctx);
/* Change the stream later calls enqueue on. */
int sdf_ctx_set_stream(sdf_ctx* ctx, void* cuda_stream);
/* Message of the last failure on ctx ("" if none).  Valid until the next call. */
const char* sdf_last_error(const sdf_ctx* ctx);

/* Options (sdf_ctx_set_option / sdf_ctx_get_option). */
#define SDF_OPT_CULL 1            /* 1 (default): bounding-sphere culling; 0: evaluate every pair */
#define SDF_OPT_POINT_STRIDE 2    /* floats per point: 3 (default, x y z) or 4 (x y z pad)       */
#define SDF_OPT_WAYPOINTS_PER_BLOCK 3 /* waypoints per check block, 1..16; 0 (default) = tuned or 16 / links */
#define SDF_OPT_TILE_BATCH 4      /* list entries per warp step: 1, 2 or 4; 0 (default) = tuned or 1  */
#define SDF_OPT_TIME_KERNELS 6    /* 1: record CUDA events around the two kernels of a check      */
#define SDF_OPT_STATS 7           /* 1: count culls/lookups and time kernel phases (adds atomics)  */
#define SDF_OPT_BLOCK_WARPS 8     /* warps per check block, 8 or 16 (0 = tuned, else 8 when the
                                     launch has no more waypoints than SMs, else 16; always
                                     16 when a robot has more than 8 links).  Blocks of
                                     several waypoints take interleaved ones (b, b + blocks,
                                     ...) when the whole launch is resident at once. */
#define SDF_OPT_WAIT_POLLS 9      /* polls a bounded device wait makes before it gives up (the
                                     staging copy of the check kernel, the tensor-core MMA
                                     completions of the surrogate kernels), 0..2^32-1; default
                                     2^22.  A wait that gives up sets SDF_ERR_TIMEOUT (reported
                                     by sdf_ctx_synchronize and the synchronising calls) and
                                     every output of that launch is invalid; the block first
                                     drains its own copies or MMAs with a wait of the default
                                     length, then leaves.  Small values exist for tests of the
                                     timeout path. */
#define SDF_OPT_TEX3D 10          /* 1: grid lookups by the texture unit's trilinear filter
                                     (Sec. III-A's grid-sample interpolation in hardware)
                                     instead of the FP32 software interpolation; 0 (default).
                                     The filter keeps each axis weight with 8 fractional bits,
                                     so a value may differ from the FP32 interpolation by up
                                     to about 3 h / 256 (h the grid spacing): at h = 5 mm it
                                     does not meet a 1e-5 m tolerance, hence off by default.
                                     The culls stay exact for the filtered values (each link's
                                     bounding volume grows by sqrt(3) h / 256).  The first
                                     check of a grids object with the option on makes its
                                     texture copy (n^3 FP32 per link; allocates and
                                     synchronises); sdf_grids_destroy frees it.  The texture
                                     form is its own kernel and always takes 1 list entry
                                     per warp step (SDF_OPT_TILE_BATCH does not apply); every
                                     request of one launch must use the same grids object
                                     (else SDF_ERR_UNSUPPORTED). */
#define SDF_OPT_SORT_CTAS 11     /* CTAs of the thread-block cluster that sorts each cloud: 8
                                     (the portable cluster size), 16 (a non-portable size;
                                     SDF_ERR_UNSUPPORTED where the device cannot place it), or
                                     0 (default) = the width sdf_autotune picked for the
                                     launch shape, else 16 where the device can place it,
                                     else 8.
                                     The sorted order and every result are the same either
                                     way; a wider cluster gives each CTA fewer points.  Get
                                     returns the size in use. */
int sdf_ctx_set_option(sdf_ctx* ctx, int32_t key, int64_t value);
int sdf_ctx_get_option(const sdf_ctx* ctx, int32_t key, int64_t* value);

/* Wait for the context's stream, then return and clear the device-side status:
 * NONFINITE if a non-finite joint value or point was met since the last call,
 * CUDA if the stream reported an error, else OK. */
int sdf_ctx_synchronize(sdf_ctx* ctx);

/* With SDF_OPT_TIME_KERNELS set: device time in milliseconds of one kernel of the
 * last check_trajectory call -- SDF_KERNEL_PREP (spatial sort of the points) or
 * SDF_KERNEL_CHECK (FK + cull + lookup + reduction).  Synchronises on that call. */
#define SDF_KERNEL_PREP 0
#define SDF_KERNEL_CHECK 1
int sdf_ctx_last_kernel_ms(sdf_ctx* ctx, int32_t kernel, float* ms);

/* Statistics accumulated by checks while SDF_OPT_STATS is 1 (cleared by
 * sdf_ctx_stats with reset != 0).  Counts are over all checks since the reset;
 * times are sums (or maxima) over check blocks of %globaltimer nanoseconds.
 * Fills min(n, SDF_STAT_COUNT) entries; synchronises. */
#define SDF_STAT_PAIRS 0          /* (waypoint, link) pairs                        */
#define SDF_STAT_SEED_LOOKUPS 1   /* lookups of the seed tiles                      */
#define SDF_STAT_SUPER_TESTS 2    /* super-tile sphere tests                        */
#define SDF_STAT_SUPER_PASS 3     /* super-tiles that survived                      */
#define SDF_STAT_TILE_TESTS 4     /* tile sphere tests                              */
#define SDF_STAT_TILE_PASS 5      /* (pair, tile) entries that survived             */
#define SDF_STAT_POINT_TESTS 6    /* point sphere tests                             */
#define SDF_STAT_LOOKUPS 7        /* grid lookups of surviving points (seed excluded) */
#define SDF_STAT_LIST_OVERFLOW 8  /* entries tested in place (block list full)      */
#define SDF_STAT_BLOCKS 9         /* check blocks                                   */
#define SDF_STAT_NS_FK 10         /* sum over blocks: kinematics and staging        */
#define SDF_STAT_NS_SEED 11       /* sum over blocks: seeding                       */
#define SDF_STAT_NS_CULL 12       /* sum over blocks: super-tile and tile culls     */
#define SDF_STAT_NS_POINTS 13     /* sum over blocks: point tests and lookups       */
#define SDF_STAT_NS_BLOCK 14      /* sum over blocks: whole block                   */
#define SDF_STAT_NS_BLOCK_MAX 15  /* longest block                                  */
#define SDF_STAT_NS_SPAN 16       /* first block start to last block end, over the calls */
#define SDF_STAT_SUR_NS_CTA 19    /* surrogate check, sum over CTAs: whole CTA       */
#define SDF_STAT_NS_SORT_BOX 20   /* sort phases, first cluster only: bounding box    */
#define SDF_STAT_NS_SORT_HIST 21  /* histogram                                      */
#define SDF_STAT_NS_SORT_SCAN 22  /* scan                                           */
#define SDF_STAT_NS_SORT_SCATTER 23 /* scatter                                      */
#define SDF_STAT_NS_SORT_TILES 24 /* tile and super-tile spheres                   */
#define SDF_STAT_NS_SORT_SUPERS 25 /* 0: counted with the tile spheres             */
#define SDF_STAT_SUR_SEED_QUERIES 26 /* surrogate check: seed queries evaluated      */
#define SDF_STAT_SUR_QUERIES 27   /* surrogate check: queries after the cull        */
#define SDF_STAT_SUR_NS_PRODUCE 28 /* surrogate check, sum over CTAs: weight copies, seed picks,
                                      culls and point tests (query production)   */
#define SDF_STAT_SUR_NS_EVAL 29   /* surrogate check, sum over CTAs: network evaluation rounds */
#define SDF_STAT_SUR_NS_LIST 30   /* surrogate check, sum over CTAs: the cull lists (part of 28) */
#define SDF_STAT_SUR_NS_CTA_MAX 31 /* surrogate check: longest CTA                    */
#define SDF_STAT_COUNT 32
int sdf_ctx_stats(sdf_ctx* ctx, int64_t* out, int32_t n, int32_t reset);

/* Gather roofline (measurement only).  A grid lookup (Sec. III-B, trilinear
 * interpolation) reads the 8 corner values of one cell of one link grid at a
 * data-dependent place, so the ceiling of the lookup rate is the rate of such reads.
 * Times, with CUDA events on the context stream, kernels that read `grids`' values
 * at pseudo-random places over 2, 4 and 8 blocks of 256 threads per SM and keeps the
 * best:  gathers_per_s = independent random 4-byte loads per second;
 * cells_per_s = random 8-corner cell reads per second.  Either output may be NULL.
 * Allocates 4 bytes; synchronises.  Errors: INVALID_ARG, CUDA. */
int sdf_measure_gather(sdf_ctx* ctx, const sdf_grids* grids, double* gathers_per_s, double* cells_per_s);

/* --------------------------------------------------------------------- grids */

/* Pre-processing (Sec. III-A, "Link SDFs"): build one signed distance grid per link
 * mesh on the GPU.  For link i: box = mesh bounding box grown by `margin` on every
 * side and made cubic (span s = max extent + 2 margin), n = `resolution` nodes per
 * axis, h = s / (n - 1).  Node value = signed distance to the mesh: distance to
 * the closest triangle, negative where the generalised winding number (sum of
 * triangle solid angles / 4 pi) is >= 1/2; a multi-component mesh takes the
 * minimum over components.  Synchronises.  Errors: INVALID_ARG (n_links outside
 * 1..SDF_MAX_LINKS, resolution outside 2..SDF_MAX_RESOLUTION, margin < 0, empty or
 * out-of-range mesh), OOM, CUDA. */
int sdf_build_grids(sdf_ctx* ctx, const sdf_mesh* links, int32_t n_links, int32_t resolution,
                    float margin, sdf_grids** out);

/* Link SDFs built elsewhere (Sec. III-A, "Link SDFs": one signed distance grid per
 * link in the link's own frame), e.g. by an offline tool: host_values holds n_links
 * grids of n^3 FP32 values each, x fastest (value index i + n (j + n k) at
 * origin + (i,j,k) h), the same n for every link; meta[l] gives link l's origin,
 * h, n, bounding-sphere centre and radius.  The radius is rounded up by one FP32
 * ulp on the way in, so a radius that is the nearest-FP32 rounding of an exact
 * bound (which may lie below it) still bounds every vertex; the culls rely on it.
 * Values and metadata are copied (the caller keeps its arrays).  Synchronises.
 * Errors: INVALID_ARG (NULL arrays, n_links outside 1..SDF_MAX_LINKS, n outside
 * 2..SDF_MAX_RESOLUTION or different between links, h <= 0, non-finite origin or
 * centre, negative radius), OOM, CUDA. */
int sdf_grids_upload(sdf_ctx* ctx, const float* host_values, const sdf_grid_meta* meta,
                     int32_t n_links, sdf_grids** out);

/* Copy grids back: host_values (n_links x n^3 floats) and/or meta (n_links
 * entries) may be NULL.  Synchronises. */
int sdf_grids_download(sdf_ctx* ctx, const sdf_grids* grids, float* host_values,
                       sdf_grid_meta* meta);
int sdf_grids_info(const sdf_grids* grids, int32_t* n_links, int32_t* resolution);
void sdf_grids_destroy(sdf_grids* grids);

/* --------------------------------------------------------------------- robot */

/* The robot whose links the check poses by forward kinematics (Sec. III-A, the
 * kinematic chain behind "parallel forward kinematics"; the paper's arm, a DENSO
 * VS-060 in Sec. IV-C, is not given, so joints are standard DH rows): a serial
 * arm of `dof` revolute joints dh[0..dof-1] (host, copied) with world-from-base
 * transform base_3x4 (host, 3x4 row-major, copied; NULL = identity) whose
 * L = dof + 1 links use `grids` (which must hold exactly L grids and outlive the
 * robot; link 0 is the static base).  Derives each link's bounding capsule for the
 * culls from its grid (downloads the grids once per sdf_grids object, which
 * synchronises).  Errors: INVALID_ARG (dof outside 0..SDF_MAX_LINKS-1, DH table
 * missing, non-finite DH row or base, grid count != dof + 1), OOM, CUDA. */
int sdf_robot_create(sdf_ctx* ctx, const sdf_dh* dh, int32_t dof, const float* base_3x4,
                     const sdf_grids* grids, sdf_robot** out);
void sdf_robot_destroy(sdf_robot* robot);

/* Parallel forward kinematics (Sec. III-A): for each waypoint w and link l write
 * 16 floats to out_dev[(w L + l) 16 ...]: the link-from-world transform
 * [R^T | -R^T t] (12 floats, row-major) followed by the world position of the
 * link's bounding-sphere centre (3 floats) and its radius.  q_dev: W x dof FP32
 * row-major.  Asynchronous. */
int sdf_forward_kinematics(sdf_ctx* ctx, const sdf_robot* robot, const float* q_dev, int32_t W,
                           float* out_dev);

/* ------------------------------------------------------------------- check */

/* The runtime distance check (Sec. III-A, runtime): for each waypoint w,
 *   dist[w] = min over links l and points p of g_l(T_{w,l}^{-1} p)
 * where T_{w,l} is link l's pose from forward kinematics of q[w] and g_l is link
 * l's grid interpolated trilinearly; a point outside the grid box gets the
 * distance to the box plus the interpolated value at the nearest box point.
 * argmin_link[w], argmin_point[w] attain the minimum (ties: smallest point, then
 * smallest link; results equal to within FP32 rounding may pick either).
 *
 * q_dev: W x dof FP32 row-major.  points_dev: N x 3 FP32 (or N x 4 with
 * SDF_OPT_POINT_STRIDE = 4, then 16-byte aligned).  Outputs: W entries each.
 * N = 0 gives dist = +inf and argmins = -1; W = 0 is a no-op.  Pairs whose value
 * is NaN are ignored; non-finite inputs also raise SDF_ERR_NONFINITE in
 * sdf_ctx_synchronize.  Asynchronous: enqueues two kernels (a spatial sort of the
 * points, then forward kinematics, culls, lookups and the reduction) and uses
 * context-owned scratch (about 17 bytes per point), grown when a call needs more
 * (which synchronises).
 * Errors: INVALID_ARG (NULL pointer with W, N > 0, N > SDF_MAX_POINTS, W < 0,
 * misaligned points), OOM (growing scratch), CUDA. */
int check_trajectory(sdf_ctx* ctx, const sdf_robot* robot, const float* q_dev, int32_t W,
                     const float* points_dev, int32_t N, float* dist_dev,
                     int32_t* argmin_link_dev, int32_t* argmin_point_dev);

/* One trajectory of a batch: the arguments of check_trajectory, and an optional
 * per-waypoint mask (device, W bytes): when set, only waypoints whose byte is
 * non-zero are checked and written; the other outputs are left as they are. */
typedef struct {
    const sdf_robot* robot;
    const float* q_dev;
    int32_t W;
    const float* points_dev;
    int32_t N;
    float* dist_dev;
    int32_t* argmin_link_dev;
    int32_t* argmin_point_dev;
    const uint8_t* mask_dev;
} sdf_check_request;

/* Batching (the paper batches all configurations of a trajectory, Sec. III-A;
 * this batches trajectories too): n <= SDF_MAX_BATCH independent checks of
 * uneven sizes -- each with its own robot (same device), trajectory and cloud --
 * in one launch of the same two kernels: one cluster per request sorts its cloud,
 * and the check blocks of all requests share one grid.
 * Each request's results are exactly those check_trajectory gives it alone.
 * Asynchronous; errors as check_trajectory (the message names the request). */
int check_batch(sdf_ctx* ctx, const sdf_check_request* requests, int32_t n);

/* Autotuner: times every launch shape (waypoints per block 1..16/links x list
 * entries per warp step 1, 2, 4) on these requests, `repeats` runs each (median,
 * caches warm), then the width of the sort's cluster (8 or 16, where the device
 * allows 16) at the fastest shape, and remembers the best for launches of the same shape -- the
 * request count, the largest link count and the power-of-two buckets of the total
 * waypoints and points.  Later check_trajectory / check_batch calls of that shape
 * use it unless SDF_OPT_WAYPOINTS_PER_BLOCK / SDF_OPT_TILE_BATCH / SDF_OPT_SORT_CTAS are set.  Runs the
 * checks (their outputs are overwritten) and synchronises.  Outputs may be NULL. */
int sdf_autotune(sdf_ctx* ctx, const sdf_check_request* requests, int32_t n, int32_t repeats,
                 int32_t* best_waypoints_per_block, int32_t* best_tile_batch, float* best_us);

/* Grow the context's scratch for launches of up to these totals (sums over a
 * batch) so that later checks allocate nothing: a prerequisite for capturing
 * check_trajectory / check_batch in a CUDA graph.  Synchronises. */
int sdf_ctx_reserve(sdf_ctx* ctx, int64_t max_points, int64_t max_waypoints, int64_t max_pairs,
                    int32_t max_requests);

/* The same check on HOST buffers, synchronising.  When all five buffers are
 * page-locked (cudaHostAlloc / cudaHostRegister) the kernels read q and the points
 * and write the outputs over the CPU-GPU link directly; otherwise q and the
 * points are copied to context-owned device staging and the outputs copied back.
 * The first call with a given set of buffers and sizes captures the whole call
 * (copies, kernels, copies back) in a CUDA graph that later identical calls replay
 * (where the capture is refused the call runs directly); the graphs are dropped
 * when the context's scratch grows or an option changes.  In the page-locked case
 * the call returns as soon as the graph's last kernel has published the status
 * and a completion count to page-locked memory (polled, at most 2 s before it
 * falls back to synchronising the stream), so the results are in the caller's
 * buffers but the stream may not yet be idle; later work on the context's stream
 * is ordered after it as usual.
 * Returns the check's status (including NONFINITE). */
int check_trajectory_host(sdf_ctx* ctx, const sdf_robot* robot, const float* q_host, int32_t W,
                          const float* points_host, int32_t N, float* dist_host,
                          int32_t* argmin_link_host, int32_t* argmin_point_host);

/* ------------------------------------------------------------------- serving */

/* A serving engine for the paper's use: the controller needs the distances along
 * the executing trajectory every control cycle (about 10 ms, 8 ms for the b-CAP
 * protocol; Sec. I).  Clients publish the latest obstacle cloud and submit
 * trajectories from any thread; an engine thread batches the requests as they
 * arrive (continuous batching): whenever one of `slots` in-flight slots is free it
 * takes waiting requests in arrival order while the batch fits the slot
 * (max_batch requests, max_waypoints in total) and the device-memory budget
 * (the request buffers and sort scratch of every in-flight batch count against
 * it), and launches it with check_batch on the slot's own stream, so batches
 * overlap on the device.  The kernels read the joint values from and write the
 * results to the slot's page-locked buffers; the engine learns of completion by
 * polling a count published in page-locked memory (it spins while batches are in
 * flight).  Every request of a batch is checked against the cloud current when
 * the batch forms.  Robots (grids) stay resident; the server owns its streams,
 * buffers and contexts. */
typedef struct sdf_server sdf_server;
typedef struct {
    int32_t device;
    int64_t memory_budget_bytes;  /* 0 = a quarter of the device's free memory          */
    int32_t slots;                /* batches in flight at once, 1..16                    */
    int32_t max_batch;            /* requests per batch, 1..SDF_MAX_BATCH                */
    int32_t max_waypoints;        /* waypoints per batch (and per request)               */
    int32_t max_points;           /* points per published cloud                          */
    int32_t max_dof;              /* largest robot dof submitted                         */
    int32_t batch_window_us;      /* 0: launch as soon as a slot is free; > 0: a batch
                                     short of max_batch waits until its oldest request
                                     has waited this long (more requests per batch)      */
} sdf_server_config;

/* Allocates every buffer up front (errors: INVALID_ARG, OOM, CUDA). */
int sdf_server_create(const sdf_server_config* config, sdf_server** out);
/* Stops the engine after the batches in flight; pending requests are dropped. */
void sdf_server_destroy(sdf_server* server);
/* Publish a cloud (host N x 3, copied).  Requests batched after this call use it.
 * SDF_ERR_TIMEOUT if every cloud buffer is still held by in-flight batches. */
int sdf_server_set_cloud(sdf_server* server, const float* points_host, int32_t N);
/* Queue one trajectory (host W x dof, copied); returns at once with a ticket.
 * SDF_ERR_OOM if the request alone exceeds the memory budget (it is not queued),
 * SDF_ERR_INVALID_ARG if W > max_waypoints or dof > max_dof. */
int sdf_server_submit(sdf_server* server, const sdf_robot* robot, const float* q_host, int32_t W,
                      uint64_t* ticket);
/* Results of a ticket (W entries each, any output may be NULL) and its latency
 * from submission to results in host memory.  wait_us: 0 = do not wait (returns
 * SDF_PENDING if unfinished), > 0 = wait up to that long (SDF_ERR_TIMEOUT),
 * < 0 = wait up to 60 s.  A finished ticket is released by this call. */
int sdf_server_poll(sdf_server* server, uint64_t ticket, int64_t wait_us, float* dist_host,
                    int32_t* argmin_link_host, int32_t* argmin_point_host, double* latency_us);
/* Statistics since creation or the last reset. */
#define SDF_SERVER_STAT_P50_US 0
#define SDF_SERVER_STAT_P99_US 1
#define SDF_SERVER_STAT_MEAN_US 2
#define SDF_SERVER_STAT_COMPLETED 3
#define SDF_SERVER_STAT_REJECTED 4
#define SDF_SERVER_STAT_BATCHES 5
#define SDF_SERVER_STAT_MEAN_BATCH 6
#define SDF_SERVER_STAT_PEAK_IN_FLIGHT 7
#define SDF_SERVER_STAT_PENDING 8
#define SDF_SERVER_STAT_MAX_US 9
#define SDF_SERVER_STAT_COUNT 10
int sdf_server_stats(sdf_server* server, double* out, int32_t n, int32_t reset);

/* ------------------------------------------------------------ learned surrogate
 *
 * No counterpart in the paper (its only network, Eq. (5), approximates its grid
 * transform).  One network per link stands in for the link's grid lookup
 * (Sec. III-A): f(x) = w4 . s(W3 s(W2 s(W1 x + b1) + b2) + b3) + b4 with
 * s(z) = z / (1 + exp(-z)), hidden width SDF_MLP_HIDDEN, on the point normalised to
 * the link's grid box, x = (p_loc - m) / a (m the box centre, a its half-span);
 * the distance is a f(x), and outside the box the grid path's rule applies
 * (distance to the box + the value at the nearest box point).  The two 128 x 128
 * layers run on the tensor cores with bfloat16 operands and FP32 accumulation;
 * training and its gradients do too.
 *
 * Parameter vector of one link (SDF_MLP_PARAMS FP32, row-major, output index
 * first): W1[128][3], b1[128], W2[128][128], b2[128], W3[128][128], b3[128],
 * w4[128], b4.  Host arrays of several links are [links][SDF_MLP_PARAMS]. */
#define SDF_MLP_HIDDEN 128
#define SDF_MLP_PARAMS 33665
#define SDF_MLP_BATCH 128
typedef struct sdf_surrogate sdf_surrogate;

/* One network per link of `grids` (which must outlive it), initial parameters
 * copied from params_host [n_links][SDF_MLP_PARAMS]; Adam state zeroed.
 * Errors: INVALID_ARG, OOM, CUDA.  Synchronous. */
int sdf_surrogate_create(sdf_ctx* ctx, const sdf_grids* grids, const float* params_host, sdf_surrogate** out);
void sdf_surrogate_destroy(sdf_surrogate* surrogate);
/* Current parameters of every link to params_host [n_links][SDF_MLP_PARAMS].
 * Synchronises the context stream. */
int sdf_surrogate_params(sdf_ctx* ctx, const sdf_surrogate* surrogate, float* params_host);

/* Training samples of one link, labelled by its grid.  Sample j (0 <= j < n) is a
 * "near" sample if j % 10 < near_per_10, else a uniform one.  Uniform sample u is
 * candidate u of stream 1; near sample k is the k-th candidate of stream 0 (in
 * counter order) whose grid value g satisfies |g| <= band (metres).  Candidate i of
 * stream s is lo + U (hi - lo) componentwise over the grid box [lo, hi], with U
 * the first three words of Philox4x32-10(counter (i, s, 0, 0), key (seed low,
 * seed high)) as (word >> 8) 2^-24.  Outputs (device, caller-owned): x_dev n x 3
 * normalised points, y_dev n normalised labels g / a, source_dev (optional) n
 * int64 = stream << 40 | counter.  Synchronises (the number of candidates to draw
 * is found on the way).  Errors: INVALID_ARG (also when 2^32 candidates give too
 * few within the band), OOM, CUDA. */
int sdf_surrogate_sample(sdf_ctx* ctx, const sdf_grids* grids, int32_t link, int64_t n, int32_t near_per_10,
                         float band, uint64_t seed, float* x_dev, float* y_dev, int64_t* source_dev);

/* Gradient of the mean absolute error over one batch of SDF_MLP_BATCH samples of
 * link `link` (x_dev 128 x 3 normalised, y_dev 128 normalised labels) with respect
 * to that link's parameters: grad_dev SDF_MLP_PARAMS FP32 in the parameter layout;
 * loss_dev (optional) one FP32, the batch's mean absolute error.  The parameters
 * are not changed.  Asynchronous. */
int sdf_surrogate_grad(sdf_ctx* ctx, const sdf_surrogate* surrogate, int32_t link, const float* x_dev,
                       const float* y_dev, float* grad_dev, float* loss_dev);

/* `steps` Adam steps (beta1 0.9, beta2 0.999, eps 1e-8, rate lr) on every link at
 * once, one CTA per link.  Step s uses the batch of samples
 * ((first_batch + s) * SDF_MLP_BATCH + j) mod n, j < SDF_MLP_BATCH, of x_dev
 * [n_links][n][3] / y_dev [n_links][n] (as sdf_surrogate_sample writes them).
 * loss_dev (optional, n_links FP32): the sum over the steps of each batch's mean
 * absolute error.  Asynchronous. */
int sdf_surrogate_train(sdf_ctx* ctx, sdf_surrogate* surrogate, const float* x_dev, const float* y_dev, int64_t n,
                        int64_t first_batch, int32_t steps, float lr, float* loss_dev);

/* f(x) of link `link` at n normalised points x_dev (n x 3) into f_dev (n FP32, in
 * units of the half-span a).  Asynchronous. */
int sdf_surrogate_eval(sdf_ctx* ctx, const sdf_surrogate* surrogate, int32_t link, const float* x_dev, int32_t n,
                       float* f_dev);

/* Error of link `link`'s network against its grid, in metres: n fresh samples
 * drawn as by sdf_surrogate_sample (near_per_10, band, seed), *max_abs and
 * *mean_abs of |a f(x) - g|.  Synchronises. */
int sdf_surrogate_error(sdf_ctx* ctx, const sdf_surrogate* surrogate, int32_t link, int64_t n, int32_t near_per_10,
                        float band, uint64_t seed, float* max_abs, float* mean_abs);

/* The check with the surrogate in place of the grid lookup, and the grid path as
 * fallback.  For each waypoint: forward kinematics, then every (link, point) pair
 * whose capsule bound (the distance from p to the link's bounding capsule) is within
 * the surrogate minimum found so far plus `eps` (seeded, per link, by the 8 points of
 * the tile nearest to the capsule that lie nearest to it) is evaluated by the link's
 * network, with the out-of-box rule; the minimum and its
 * arg-min are the surrogate result.  Waypoints whose surrogate minimum is below
 * margin + eps -- eps being the caller's bound on the surrogate's error, e.g. from
 * sdf_surrogate_error -- are checked again by the grid path, whose result replaces
 * the surrogate's (exactly what check_trajectory returns for them).  Outputs as
 * check_trajectory; rechecked_dev (optional, W bytes) is 1 where the grid path
 * decided, surrogate_dist_dev (optional, W FP32) the surrogate minimum before the
 * re-check (for a waypoint whose work item's (waypoint, tile) list overflowed, an upper
 * bound of it; such a waypoint is always re-checked).  Without surrogate_dist_dev, a
 * waypoint whose surrogate minimum so far
 * is already below margin + eps stops being culled and evaluated (the grid path
 * decides it whatever the rest would give), which changes no output; with it, every
 * waypoint's surrogate minimum is completed.  Uses workspace owned by the context (grown on demand, which
 * synchronises); contexts on different streams may share one surrogate.  The context keeps
 * the networks' weights in the check's layout and makes them again after any
 * sdf_surrogate_train of that surrogate (a check must be ordered after the training it
 * is to see, as for any use of the parameters).
 * Asynchronous.
 * Errors: INVALID_ARG (robot and surrogate built on different grids, bad sizes),
 * OOM, CUDA. */
int check_trajectory_surrogate(sdf_ctx* ctx, const sdf_robot* robot, const sdf_surrogate* surrogate,
                               const float* q_dev, int32_t W, const float* points_dev, int32_t N, float margin,
                               float eps, float* dist_dev, int32_t* argmin_link_dev, int32_t* argmin_point_dev,
                               uint8_t* rechecked_dev, float* surrogate_dist_dev);

/* Serving in the surrogate form: requests whose robot uses `surrogate`'s grids are
 * checked by check_trajectory_surrogate (margin, eps as there) on their slot's
 * stream, one after the other; other requests keep the batched grid path.  NULL
 * returns to the grid form.  Applies to batches formed after the call. */
int sdf_server_set_surrogate(sdf_server* server, const sdf_surrogate* surrogate, float margin, float eps);

/* --------------------------------------------------- the paper's Robot-SDF form
 *
 * The paper's own formulation of the check (Sec. III-A), for comparison with the
 * per-point form above: for every configuration, each Link SDF is transformed into
 * an environment voxel grid (Eq. (1)-(4): the samples land on voxel centres) over
 * the voxels of its block -- the "grids in sphere" of Sec. III-B, radius
 * R_link + reach + sqrt(3) voxel / 2 around the link's bounding-sphere centre --
 * and the Robot SDF of the configuration is the minimum over links per voxel.  The
 * cloud is voxelised (a point occupies voxel floor((p - origin) * fl32(1/voxel))
 * per axis, in single precision; points outside the grid occupy none) and the
 * distance of a configuration is the minimum of its Robot SDF over the occupied
 * voxels (+inf when none lies in a block).
 *
 * Memory: W x dims[0] x dims[1] x dims[2] x 4 bytes of context workspace (grown on
 * demand, which synchronises), the cost that formulation carries. */
typedef struct {
    float origin[3];   /* lower corner of the grid (world frame, metres)          */
    float voxel;       /* voxel edge (metres)                                     */
    int32_t dims[3];   /* voxels per axis; their product at most 2^31 - 1          */
    float reach;       /* distance range covered beyond a link's bounding sphere  */
} sdf_env_grid;

/* dist_dev: W FP32 distances; argmin_voxel_dev: W int32 linear voxel indices
 * (i + dims[0] (j + dims[1] k); smallest index on ties; -1 with +inf).
 * Asynchronous.  Errors: INVALID_ARG (null, sizes, grid), OOM, CUDA. */
int check_trajectory_robot_sdf(sdf_ctx* ctx, const sdf_robot* robot, const sdf_env_grid* env,
                               const float* q_dev, int32_t W, const float* points_dev, int32_t N,
                               float* dist_dev, int32_t* argmin_voxel_dev);

/* ------------------------------------------------------------ fault injection
 *
 * The paper has no counterpart: these serve tests of the library's error paths.
 * Every device or page-locked host allocation the library makes is counted.
 * sdf_debug_fail_alloc(k), k >= 1: the k-th allocation from now (in any thread,
 * on any device) fails as if the memory were exhausted, so the call making it
 * returns SDF_ERR_OOM (and must free what it had allocated); 0 disarms.  Nothing
 * happens on the GPU.  sdf_debug_alloc_live: the library's live allocations, their
 * total bytes and the remaining countdown (0 = disarmed); any output may be NULL.
 * Errors: INVALID_ARG (k < 0). */
int sdf_debug_fail_alloc(int64_t k);
int sdf_debug_alloc_live(int64_t* count, int64_t* bytes, int64_t* countdown);

/* ----------------------------------------------------------- allocation-free check */

/* The paper has no counterpart to this entry point; it serves deployment.
 *
 * check_trajectory_noalloc: the same check as check_trajectory, for callers that
 * must not allocate GPU memory while checking -- typically a fixed-period
 * control loop, where an allocation's unpredictable latency (and the device
 * synchronisation cudaMalloc/cudaFree can imply) would miss the cycle deadline,
 * or a process whose memory budget is fixed at start-up.  It needs no context:
 * it calls no cudaMalloc, cudaFree or other allocating routine.  Its scratch is
 * one file-scope device array of about 0.5 MiB that every GPU loading this
 * library holds until the process exits.
 *
 * Limits: N <= SDF_NOALLOC_MAX_POINTS, else SDF_ERR_INVALID_ARG (nothing is
 * enqueued); W up to 2^31 - 1 (any int32).  Points are N x 3 FP32; culling is on.
 *
 * robot: as for check_trajectory (its device is made current for the call).
 * cuda_stream: the cudaStream_t to enqueue on (NULL = legacy default stream).
 * status_dev: optional device int that the call clears and the kernels OR their
 *   status bits into (bit 0: a non-finite input was seen); NULL = not reported.
 * Returns SDF_OK after enqueueing (asynchronous), SDF_ERR_INVALID_ARG or
 * SDF_ERR_CUDA (launch or set-up failure).
 *
 * The first call on each device looks up the array's device address; make that
 * first call before any stream capture.  A set-up that failed (SDF_ERR_CUDA) is
 * tried again by the next call.  Every call shares the one array and it
 * keeps the previous call's contents (the call resets what must start cleared),
 * so calls whose work overlaps on the GPU -- on different streams, or from
 * different host threads -- race and must be serialised by the caller. */
#define SDF_NOALLOC_MAX_POINTS 32768
int check_trajectory_noalloc(const sdf_robot* robot, void* cuda_stream, const float* q_dev, int32_t W,
                             const float* points_dev, int32_t N, float* dist_dev,
                             int32_t* argmin_link_dev, int32_t* argmin_point_dev, int32_t* status_dev);

#ifdef __cplusplus
}
#endif

#endif /* SDFCHECK_H */
