/*
 * lfp.h -- C ABI of the GB300 light-field-probe ray tracer.
 *
 * Method: Liu, Nowrouzezahrai & McGuire, "Real-Time Scene Reconstruction
 * using Light Field Probes" (arXiv 2507.14624). A camera ray (X, w1) is traced
 * through a uniform 3D grid of probes (Sec. 3, multiple probes; Sec. 4.3 grid
 * iterator). Each probe stores octahedral maps (Sec. 3, octahedral mapping) of
 * radial distance, surface normal and radiance, plus a low-resolution distance
 * map (Sec. 5.1; here a conservative per-block min/max). Per probe the ray is
 * split at the probe's axis planes into at most 4 segments, marched on the
 * low-resolution map and then on the full-resolution map, and classified HIT /
 * MISS / UNKNOWN (Sec. 4.2; Appendix A, traceOneRaySegment,
 * lowResolutionTracing, highResolutionTracing). UNKNOWN falls through to the
 * next probe of the 8-probe cage. A HIT is shaded by a bilinear radiance fetch
 * (Sec. 3: L_o(X, w1) = L_p(w2)).
 *
 * Conventions shared by every entry point
 *   - Octahedral maps are N x N, row-major, row j, column i; texel (i, j)
 *     holds direction decode(((i + .5) / N * 2 - 1, (j + .5) / N * 2 - 1)),
 *     pole +z, lower octants unfolded onto the square's corners.
 *   - Probe index p = ix + nx * (iy + ny * iz); probe p sits at
 *     origin + spacing * (ix, iy, iz) (float32 arithmetic).
 *   - Pixel (x, y) of a view (x to the right, y down) is written at flat index
 *     out_offset + y * W + x of every per-pixel output.
 *   - Every call that takes a stream is asynchronous on that stream (a
 *     cudaStream_t passed as void*, NULL = the legacy default stream) unless
 *     stated otherwise; device pointers must stay valid until the stream has
 *     executed the call. No call allocates on behalf of the caller's outputs.
 *   - Every call returns a status; no C++ exception crosses the ABI. A launch
 *     failure is reported as LFP_ERR_CUDA (checked with cudaGetLastError).
 *   - The library is not thread-safe per grid: calls on one grid must come
 *     from one host thread at a time. Distinct grids are independent.
 *   - Renders of one grid share its work-queue head (a device counter that
 *     every launch resets and then consumes): lfp_render, lfp_render_ex,
 *     lfp_render_to_host, lfp_autotune and lfp_render_levels. Such calls
 *     must run one after another on the GPU: issue them on one stream, and
 *     do not replay a CUDA graph that recorded one of them while another
 *     render of the same grid may run. Two that overlap corrupt each other's
 *     queue (rays skipped or rendered twice). lfp_render_to_host_async uses
 *     two queue heads of its own and lfp_render_static one per process (see
 *     there); the adjoint and the probe builder use none.
 */
#ifndef LFP_H
#define LFP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LFP_OK = 0,
    LFP_ERR_INVALID_ARG = 1, /* a pointer, size or descriptor field is invalid */
    LFP_ERR_OOM = 2,         /* a device allocation failed */
    LFP_ERR_CUDA = 3,        /* a CUDA runtime call or launch failed */
    LFP_ERR_STATE = 4,       /* call order violated (e.g. render before upload) */
    LFP_ERR_CAPACITY = 5,    /* request larger than a fixed-size buffer allows */
    LFP_ERR_BOUNDS = 6,      /* an index out of range was caught (lfp_check_flags) */
    LFP_WARN_STEPLIMIT = 100 /* some ray hit the per-ray step cap (class 3) */
} lfp_status;

typedef enum { LFP_TEXEL_F32 = 0, LFP_TEXEL_F16 = 1 } lfp_texel_fmt;

/* per-pixel classes written to `cls` */
enum {
    LFP_CLASS_MISS = 0,      /* the ray left the grid in front of every surface */
    LFP_CLASS_HIT = 1,       /* a probe saw the intersection (rgb valid) */
    LFP_CLASS_UNKNOWN = 2,   /* no probe could decide (all UNKNOWN somewhere) */
    LFP_CLASS_STEPLIMIT = 3  /* max_steps texel visits reached */
};

/* Grid of probes (Sec. 3: probes sit at the vertices of a uniform 3D grid).
 *   nx, ny, nz >= 2          probes per axis (cells: (nx-1)(ny-1)(nz-1));
 *                            >= 1 with traversal LFP_TRAVERSAL_NEAREST
 *   origin, spacing > 0      probe (0,0,0) position and grid pitch
 *   N                        full-resolution map side, even, 2..8192
 *   M                        low-resolution map side, even, N % M == 0, M <= N
 *                            (blocks of k = N / M texels; the grid keeps the
 *                            min/max maps of a few more block sides for the
 *                            walk to skip with: lfp_skip_blocks)
 *   radiance_fmt, normal_fmt device storage of radiance (RGB) and normals
 *                            (octahedral-encoded RG); distance is always float32
 *   thickness_rel            th: a texel crossing counts while the ray's
 *                            nearest radial distance is <= d (1 + 4 th / N);
 *                            th < 0 selects the two-way rule of Appendix A
 *                            highResolutionTracing (every crossing -> normal test)
 *   eye_eps                  |X - O| < eye_eps counts as the eye aligned with a probe
 *                            (Sec. 4.2, O(1) lookup); 0 -> 1e-6 * spacing
 *   max_steps                cap on texel visits per ray, 0 = none
 *   eye_lookup               LFP_EYE_BILINEAR (default): the eye-aligned
 *                            lookup filters like every other hit;
 *                            LFP_EYE_NEAREST: the value of the texel holding
 *                            oct(w) (Appendix A traceOneProbe's texel fetch)
 *   traversal                LFP_TRAVERSAL_GRID (default): grid iterator over
 *                            the cells, 8-probe cage per cell (Sec. 4.3);
 *                            LFP_TRAVERSAL_NEAREST: the mode Sec. 4.3 gives
 *                            for fewer than 8 probes: all probes (at most 8)
 *                            nearest to the eye first, each traced over the
 *                            whole ray; MISS or UNKNOWN goes to the next probe. */
enum { LFP_EYE_BILINEAR = 0, LFP_EYE_NEAREST = 1 };
enum { LFP_TRAVERSAL_GRID = 0, LFP_TRAVERSAL_NEAREST = 1 };
#define LFP_NEAREST_MAX_PROBES 8
typedef struct {
    int nx, ny, nz;
    float origin[3];
    float spacing;
    int N, M;
    lfp_texel_fmt radiance_fmt, normal_fmt;
    float thickness_rel;
    float eye_eps;
    int max_steps;
    int eye_lookup;
    int traversal;
} lfp_grid_desc;

/* Pinhole camera (the ray (X, w1) of Sec. 3). The ray through pixel (x, y)
 * starts at pos and runs along normalize(fwd + a right + b up) with
 * a = ((x + .5) / W * 2 - 1) tan(fov_y / 2) W / H and
 * b = (1 - (y + .5) / H * 2) tan(fov_y / 2); fov_y is vertical, in radians.
 * right/up/fwd need not be orthonormal. out_offset: first flat output index. */
typedef struct {
    float pos[3], right[3], up[3], fwd[3];
    float fov_y;
    int W, H;
    long long out_offset;
} lfp_view;

/* Probe maps for `count` consecutive probes, float32, tightly packed:
 *   dist      [count][N][N]     radial distance from the probe to the nearest surface
 *   normal    [count][N][N][3]  unit surface normal at that surface point
 *   radiance  [count][N][N][3]  linear RGB leaving that point towards the probe
 * is_device: 0 = host pointers (copied), 1 = device pointers (read in place). */
typedef struct {
    const float* dist;
    const float* normal;
    const float* radiance;
    int is_device;
} lfp_probe_planes;

typedef struct lfp_grid lfp_grid;

/* Optional per-pixel outputs and statistics of lfp_render_ex. Any pointer
 * may be NULL. All device pointers, flat per-pixel arrays (see conventions).
 *   rgb [P][3] f32, cls [P] u8, aux_probe [P] i32 (-1 unless HIT),
 *   aux_uv [P][2] f32 (shading coordinate in [0,1]^2, HIT only),
 *   hit_texel [P] i32: i + N * j of the full-resolution texel that decided
 *   the HIT (-1 otherwise), counters [8] u64, accumulated (not cleared):
 *   low-res texel visits, full-res texel visits, normal fetches, radiance
 *   texel fetches, cells entered, probes traced, HIT pixels, rays. */
typedef struct {
    float* rgb;
    uint8_t* cls;
    int32_t* aux_probe;
    float* aux_uv;
    int32_t* hit_texel;
    unsigned long long* counters;
} lfp_outputs;

/* Launch options for lfp_render_ex (zero-initialised = defaults). */
enum { LFP_MARCH_HIER = 0, LFP_MARCH_FLAT = 1 };
enum { LFP_SCHED_AUTO = 0, LFP_SCHED_TILES = 1, LFP_SCHED_PERSISTENT = 2 };
enum { LFP_ENGINE_AUTO = 0, LFP_ENGINE_STREAM = 1, LFP_ENGINE_NESTED = 2 };
typedef struct {
    int march;      /* LFP_MARCH_HIER (low-res then full-res) or LFP_MARCH_FLAT
                       (Appendix A RayMarching over the full-res map only) */
    int tile_w;     /* ray tile width x height per CTA; 0 = autotuned/default.
                       Valid shapes: 8x4, 8x8, 16x8, 16x16, 32x8 */
    int tile_h;
    int schedule;   /* LFP_SCHED_*: one CTA per tile, or a persistent grid
                       pulling tiles from a queue (nested engine only) */
    int engine;     /* LFP_ENGINE_STREAM (default): a persistent per-lane
                       state machine, one texel visit per lane per step, lanes
                       refilled from 8x4 ray tiles; LFP_ENGINE_NESTED: the
                       loop nest of Appendix A, one ray per thread (tile_w,
                       tile_h, schedule and LFP_MARCH_FLAT apply to it only).
                       Both give identical results. */
    int occupancy;  /* streaming engine: LFP_OCC_AUTO (the grid's default,
                       set by lfp_autotune), LFP_OCC_8 (8 blocks of 128
                       threads per SM, up to 64 registers per thread) or
                       LFP_OCC_9 (9 blocks, up to 56 registers); identical
                       results, different speed per workload */
    int skip_block; /* side, in full-resolution texels, of the min/max
                       blocks the walk skips over: one of lfp_skip_blocks,
                       or 0 for the grid's default. Both engines; the same
                       decisions up to near-ties, different speed per
                       workload */
} lfp_render_opts;
enum { LFP_OCC_AUTO = 0, LFP_OCC_8 = 1, LFP_OCC_9 = 2 };

/* Create a grid; allocates the device planes for all nx*ny*nz probes on the
 * current device. *out receives the handle (owned by the caller, release with
 * lfp_destroy_grid). Errors: INVALID_ARG (desc), OOM, CUDA. */
lfp_status lfp_create_grid(const lfp_grid_desc* desc, lfp_grid** out);

/* Upload maps for probes [first_probe, first_probe + count) and rebuild their
 * low-resolution min/max maps (Sec. 5.1) at every skip level and the least
 * distance of each quadrant of their maps (where a segment's walk starts).
 * Host planes are copied before the call returns only if the stream is
 * synchronous; otherwise they must stay valid until the stream has run the
 * copy. Errors: INVALID_ARG, OOM, CUDA. */
lfp_status lfp_upload_probes(lfp_grid* grid, int first_probe, int count,
                             const lfp_probe_planes* planes, void* cuda_stream);

/* Render n_views views (Sec. 3 problem statement; Sec. 4.2-4.3; Appendix A).
 * `views` is host memory, read before the call returns. rgb [P][3] f32 and
 * cls [P] u8 are required; aux_probe [P] i32 and aux_uv [P][2] f32 are the
 * saved state for lfp_render_backward and may be NULL. Pixels that are not
 * HIT get rgb 0. Returns LFP_ERR_STATE if any probe was never uploaded, and
 * LFP_ERR_INVALID_ARG if a view has more than 2^31 pixels or a group of 128
 * consecutive views more than 2^30 ray tiles of 8 x 4 pixels. */
lfp_status lfp_render(lfp_grid* grid, const lfp_view* views, int n_views,
                      float* rgb, uint8_t* cls, int32_t* aux_probe, float* aux_uv,
                      void* cuda_stream);

/* lfp_render with optional outputs and launch options (opts may be NULL). */
lfp_status lfp_render_ex(lfp_grid* grid, const lfp_view* views, int n_views,
                         const lfp_outputs* out, const lfp_render_opts* opts,
                         void* cuda_stream);

/* Autotuner: first the skip level (lfp_skip_blocks), timed on the
 * streaming engine with the 8-block register budget; then, at that level,
 * every launch configuration (streaming engine with each register budget,
 * the loop-nest engine with each ray-tile shape, one CTA per tile or
 * persistent) on these views. Keeps the fastest as the grid's default for
 * calls that leave the options zero, and returns it in *best (may be
 * NULL). A configuration whose first launch takes more than twice the best
 * per-launch time so far is dropped after that launch; the others get a
 * second warm-up and three timed launches. Synchronises the stream; the
 * outputs (rgb and cls required) are overwritten with the last run. Do not
 * call it during stream capture. */
lfp_status lfp_autotune(lfp_grid* grid, const lfp_view* views, int n_views,
                        const lfp_outputs* out, lfp_render_opts* best, void* cuda_stream);

/* Make `opts` the grid's default launch configuration, as lfp_autotune does
 * with the one it picks (e.g. a pick it returned earlier for the same views
 * and GPU, kept by the caller). Fields left zero keep the current default;
 * march must be LFP_MARCH_HIER. Host-only, no stream. Errors: INVALID_ARG
 * (a field out of range, an invalid tile shape, or a skip_block that is not
 * one of the grid's skip levels). */
lfp_status lfp_set_defaults(lfp_grid* grid, const lfp_render_opts* opts);

/* Render into HOST memory: one call that runs lfp_render on device buffers
 * owned by the grid and copies rgb [P][3] f32 and cls [P] u8 back, then
 * synchronises the stream. rgb_host / cls_host: host memory (pinned memory
 * gives asynchronous copies), either may be NULL. */
lfp_status lfp_render_to_host(lfp_grid* grid, const lfp_view* views, int n_views,
                              float* rgb_host, uint8_t* cls_host, void* cuda_stream);

/* Frame-loop form of lfp_render_to_host: renders into one of two grid-owned
 * device buffers (used in turn), each on its own grid-owned stream that
 * first waits for the work queued so far on `cuda_stream`, and queues the
 * copy of rgb / cls to the host buffers on a grid-owned copy stream; returns
 * without waiting. The copy of one call and the end of its render overlap
 * the render of the next. Later work on `cuda_stream` does not wait for
 * these renders; lfp_sync_host does.
 * Copies run in call order. The host buffers of a call hold its result
 * once lfp_sync_host(grid) has returned (read them only then). Pinned host
 * memory is needed for the overlap. */
lfp_status lfp_render_to_host_async(lfp_grid* grid, const lfp_view* views, int n_views,
                                    float* rgb_host, uint8_t* cls_host, void* cuda_stream);
/* Wait for every copy queued by lfp_render_to_host_async on this grid. */
lfp_status lfp_sync_host(lfp_grid* grid);

/* Adjoint of lfp_render with respect to radiance (the paper has no adjoint;
 * it follows from L_o(X, w1) = L_p(w2): for fixed distance and normal maps
 * the HIT texel and bilinear weights do not depend on radiance, so
 * d rgb_c / d radiance[p, texel_k, c] = w_k). For each HIT pixel, adds
 * w_k * grad_rgb[c] into grad_radiance [P_total][N][N][3] f32 (device,
 * ACCUMULATED: the caller zeroes it). cls, aux_probe, aux_uv: the forward's
 * outputs for the same views; the grid must not have changed in between
 * except through lfp_set_radiance. */
lfp_status lfp_render_backward(lfp_grid* grid, const lfp_view* views, int n_views,
                               const float* grad_rgb, const uint8_t* cls,
                               const int32_t* aux_probe, const float* aux_uv,
                               float* grad_radiance, void* cuda_stream);

/* lfp_render_backward with a choice of how the scatter-add is reduced:
 *   LFP_REDUCE_AUTO      the library default (warp-aggregated)
 *   LFP_REDUCE_ATOMIC    12 f32 atomics per HIT pixel
 *   LFP_REDUCE_WARP      pixels of a warp that hit the same texel are summed
 *                        with shuffles first, one atomic per distinct texel
 *   LFP_REDUCE_SORT      each block sorts its taps by texel in shared memory
 *                        and issues one atomic per run of equal texels
 * All give the same sums up to the order of f32 additions. */
enum { LFP_REDUCE_AUTO = 0, LFP_REDUCE_ATOMIC = 1, LFP_REDUCE_WARP = 2, LFP_REDUCE_SORT = 3 };
lfp_status lfp_render_backward_ex(lfp_grid* grid, const lfp_view* views, int n_views,
                                  const float* grad_rgb, const uint8_t* cls,
                                  const int32_t* aux_probe, const float* aux_uv,
                                  float* grad_radiance, int reduction, void* cuda_stream);

/* Replace every probe's radiance from a device array [P_total][N][N][3] f32
 * (the fitted parameters); converted to the grid's radiance format. */
lfp_status lfp_set_radiance(lfp_grid* grid, const float* dev_radiance_f32, void* cuda_stream);

/* Synchronise the stream and report (then clear) the device flag word:
 * LFP_ERR_BOUNDS if an index out of range was caught since the last call (an
 * adjoint given saved state whose probe index is outside the grid, or, in
 * the checked library liblfp_checked.so, any texel index of a render or
 * adjoint; the access was redirected to texel 0), else LFP_WARN_STEPLIMIT if
 * some ray reached max_steps, else LFP_OK. */
lfp_status lfp_check_flags(lfp_grid* grid, void* cuda_stream);

/* Device bytes the grid's probe storage takes for a descriptor (maps, the
 * min/max maps of every skip level, and per probe the least distance of
 * each quadrant of its map, 16 B), the byte accounting of Sec. 6 (memory
 * efficient representation). */
lfp_status lfp_grid_bytes(const lfp_grid_desc* desc, unsigned long long* bytes);

/* Skip levels (Sec. 5.1 hierarchical tracing; the paper uses one
 * low-resolution map and studies its size in Sec. 6). Besides the
 * descriptor's map of blocks of k = N / M full-resolution texels, a grid
 * keeps per-block min/max maps at the block sides k / 4, k / 2 and 2 k,
 * those of them that are whole numbers >= 2 and cut the map into an even
 * number of blocks per side; all are rebuilt by every upload. The walk
 * skips over the blocks of one level (lfp_render_opts.skip_block; the
 * grid's default is k until lfp_autotune or lfp_set_defaults picks
 * another). A block is skipped only while the ray stays in front of its
 * minimum, so every level finds the same crossings: the level changes the
 * speed, while classes and colours agree to rounding of the walk's start
 * inside a block. Writes the block sides, ascending, to blocks[0 .. *count)
 * (room for LFP_MAX_SKIP_LEVELS ints). Host-only. Errors: INVALID_ARG. */
#define LFP_MAX_SKIP_LEVELS 4
lfp_status lfp_skip_blocks(const lfp_grid_desc* desc, int* blocks, int* count);

/* Most views one lfp_render_static call accepts. */
#define LFP_STATIC_MAX_VIEWS 4096

/* Forward render that allocates nothing (the paper has no counterpart). It
 * is for callers that cannot allocate device memory at render time: a
 * real-time frame loop that must not touch the allocator after start-up
 * (cudaMalloc and cudaFree can synchronise the whole device and stall the
 * loop), or a host application or plug-in whose device memory comes from its
 * own fixed-budget allocator, which a library allocating behind its back
 * would break. Same results and outputs as lfp_render_ex with
 * LFP_ENGINE_NESTED, LFP_SCHED_PERSISTENT and 16x8 ray tiles, in one
 * persistent launch for all n_views <= LFP_STATIC_MAX_VIEWS views (more ->
 * LFP_ERR_CAPACITY, nothing is launched). The work-queue head and the view
 * table live in one file-scope device array of 256 B + LFP_STATIC_MAX_VIEWS
 * * 80 B (about 320 KiB) that every GPU loading the library keeps until the
 * process exits. The call issues small fill kernels that carry the view
 * entries in their parameters, a 4-byte memset of the queue head, and the
 * render; it calls no cudaMalloc, cudaFree or other allocating routine.
 *   - The first call on a device sets that device up (looks up the array's
 *     device address with cudaGetSymbolAddress, sizes the persistent grid);
 *     make that first call before any stream capture.
 *   - All calls share the array: every call rewrites the view table and
 *     clears the queue head, so calls that overlap on the GPU (other streams,
 *     other host threads' streams) race; serialise them on one stream.
 *   - `views` is host memory, read before the call returns (the call does
 *     not wait for the stream).
 *   - grid: created and uploaded beforehand (those calls do allocate). */
lfp_status lfp_render_static(lfp_grid* grid, const lfp_view* views, int n_views,
                             const lfp_outputs* out, void* cuda_stream);

/* A point cloud, e.g. merged laser scans in one world frame (Sec. 4.1, Sec. 5.1).
 *   xyz     [n][3] float32 world positions
 *   rgb     [n][3] float32 colour (stored as the probe radiance)
 *   normal  [n][3] float32 unit surface normals, or NULL: the builder then
 *           stores the incoming direction (point -> probe), the content
 *           Sec. 5.1 gives its normal map
 *   n       1 .. 2^32 - 1 points
 *   is_device 1: device pointers, read in place; 0: host pointers, copied
 *           on the stream into a grid-owned device buffer (kept for later
 *           calls); pinned host memory copies asynchronously and must stay
 *           valid until the stream has passed the call */
typedef struct {
    const float* xyz;
    const float* rgb;
    const float* normal;
    long long n;
    int is_device;
} lfp_point_cloud;

/* Probe maps of probes [first_probe, first_probe + count) from a point cloud
 * (Sec. 4.1 simulated probe data: any grid position can become a probe;
 * Sec. 5.1 probe data generation): every point is moved into the probe's
 * frame (v = p - O), projected onto the octahedral map, and per texel the
 * point nearest to the probe is kept: distance |v|, its colour, its normal
 * (or -v/|v|). Texels no point reaches get distance empty_dist, radiance 0
 * and normal minus the texel-centre direction (empty_dist 0: any ray through
 * them passes behind and is UNKNOWN; a large value: they never stop a ray).
 * The min/max map is rebuilt and the probes count as uploaded.
 * The texel and the ranking are decided in float32 with this sequence of
 * correctly rounded operations (no fused multiply-add), so other
 * implementations following it bin identically:
 *   v = p - O per component; q = (v.x v.x + v.y v.y) + v.z v.z;
 *   s = (|v.x| + |v.y|) + |v.z| (s = 0 or non-finite q or s: point skipped);
 *   r = 1 / s; px = v.x r, py = v.y r; if v.z < 0:
 *   (px, py) = ((1 - |py|) sgn px, (1 - |px|) sgn py), sgn 0 = +1;
 *   i = floor((px + 1) (N / 2)) clamped to [0, N - 1], j likewise from py;
 *   the smallest q wins, ties to the lower point index; distance = sqrt(q).
 * Work: probes in chunks whose (distance, index) table fits 64 MiB; per chunk
 * one pass over the points (64-bit atomicMin per point and probe) and one
 * over the texels. Errors: LFP_ERR_INVALID_ARG (NULL xyz/rgb, range,
 * n out of range, non-finite empty_dist), LFP_ERR_OOM. */
lfp_status lfp_build_probes_from_points(lfp_grid* grid, int first_probe, int count, const lfp_point_cloud* cloud,
                                        float empty_dist, void* cuda_stream);

/* Read probe maps back as float32 device arrays: dist [count][N][N], normal
 * [count][N][N][3] (unit xyz decoded from the stored octahedral pair),
 * radiance [count][N][N][3] (from the stored texels: FP16 storage returns
 * the rounded values). LFP_ERR_STATE if a probe was never filled. */
lfp_status lfp_read_probes(lfp_grid* grid, int first_probe, int count, float* dist, float* normal, float* radiance,
                           void* cuda_stream);

/* Multi-scale hierarchy (the multi-scale representation named in the
 * abstract; the hierarchical scene representation of the teaser figure):
 * several grids of one scene at different spacings, typically nested (coarse
 * grids over the whole scene, fine grids where the eye goes).
 *   levels      n_levels (1..16) grid handles on one device, any order
 * Every ray of a view starts at the camera, so a view is traced in one level:
 * the finest (smallest spacing, ties to the lower index) whose probe box
 * [origin, origin + spacing (n - 1)] per axis (closed, float32) holds the
 * camera position; a camera outside every box uses the coarsest level
 * (largest spacing, ties to the lower index).
 *
 * lfp_pick_levels writes that level for each view (host int32[n_views]).
 * lfp_render_levels renders every view with its level into the shared flat
 * outputs (each view at its own out_offset): one lfp_render_ex call per
 * level that has views, on `cuda_stream`, same options (a nonzero skip_block
 * must be a skip level of every level that has views; 0 takes each grid's
 * default); aux_probe indexes the probes of the view's level. lfp_render_backward_levels is the adjoint:
 * grad_radiance is a host array of n_levels device pointers, entry k the
 * [P_k][N_k][N_k][3] f32 accumulator of level k (may be NULL for a level no
 * view uses); each level's views go to lfp_render_backward_ex.
 * Errors: NULL or mismatched arguments, grids on different devices, invalid
 * views -> LFP_ERR_INVALID_ARG before anything is launched; a failing level
 * returns its status (levels before it have been launched). */
lfp_status lfp_pick_levels(lfp_grid* const* levels, int n_levels, const lfp_view* views, int n_views,
                           int32_t* level_of_view);
lfp_status lfp_render_levels(lfp_grid* const* levels, int n_levels, const lfp_view* views, int n_views,
                             const lfp_outputs* out, const lfp_render_opts* opts, void* cuda_stream);
lfp_status lfp_render_backward_levels(lfp_grid* const* levels, int n_levels, const lfp_view* views,
                                      int n_views, const float* grad_rgb, const uint8_t* cls,
                                      const int32_t* aux_probe, const float* aux_uv,
                                      float* const* grad_radiance, int reduction, void* cuda_stream);

/* Release a grid (NULL-safe; synchronises the device first). */
void lfp_destroy_grid(lfp_grid* grid);

/* Static string for a status code. */
const char* lfp_status_string(lfp_status status);

#ifdef __cplusplus
}
#endif

#endif /* LFP_H */
