/*
 * curast.h -- C ABI of the GB300 visibility-buffer rasterizer.
 *
 * The calls follow the paper's statement of the problem (Schuetz, Lipp,
 * Kristmann, Wimmer: "CuRast: Cuda-Based Software Rasterization for Billions
 * of Triangles"): indexed meshes and their instances (Section 4, "Method";
 * Section 4.5 "Instancing") are rasterized by brute force into a 64-bit
 * visibility buffer holding 28 depth bits and a 36-bit global triangle id
 * (Section 4.1 "Rasterization"), which a screen pass then resolves into
 * colours (Section 4.4).
 *
 * Conventions for every call
 *   - Pointers marked "device" are CUDA device pointers on the context's
 *     device; "host" pointers are ordinary memory read during the call.
 *   - Matrices are 16 host floats, row-major (m[4*row + col]).  view and
 *     model must be affine (last row 0 0 0 1).  proj must be a symmetric
 *     perspective matrix: proj[1]=proj[2]=proj[3]=proj[4]=proj[6]=proj[7]=
 *     proj[8]=proj[9]=0, last row (0, 0, -1, 0); the projection vector of
 *     Eq. 2 is read off it as fx = proj[0] (f/aspect), fy = proj[5] (f), and
 *     the near plane as proj[11] / (proj[10] - 1) (double, rounded to float).
 *   - Images (visibility buffers, colours, gradients) are W x H pixels,
 *     row-major, row 0 = the BOTTOM row (y up), pixel (x, y) at y * W + x.
 *     1 <= W, H <= 16384.
 *   - A visibility word is (depth28 << 36) | id, where depth28 is the FP32
 *     bit pattern of the pixel's positive linear view depth shifted right by
 *     3 (sign and 3 low mantissa bits dropped) and id is the global triangle
 *     id; an empty pixel holds 0xFFFFFFFFFFFFFFFF.
 *   - Global id of triangle t of instance i = base[i] + t, where base is the
 *     exclusive prefix sum of the triangle counts of all instances in the
 *     order they were added (Section 4, host frame setup; Section 4.4).
 *   - Work is enqueued on the given CUDA stream (NULL = legacy default
 *     stream) and the call returns without waiting for the GPU.  Inputs
 *     must stay valid and unmodified until the stream reaches the work.
 *   - Every call returns a status; no C++ exception crosses this boundary.
 *     Conditions found on the device (an index out of range when checking
 *     is on, a queue overflow) are latched in the context and reported by
 *     curast_sync.
 *   - A context is not thread-safe: one host thread at a time.
 */
#ifndef CURAST_H
#define CURAST_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t curast_status;
#define CURAST_OK                        0
#define CURAST_ERR_INVALID_ARG          -1  /* null pointer, bad size, bad id  */
#define CURAST_ERR_OUT_OF_MEMORY        -2  /* a context allocation failed      */
#define CURAST_ERR_ID_SPACE_OVERFLOW    -3  /* total triangles > 2^36 - 1       */
#define CURAST_ERR_INDEX_OUT_OF_RANGE   -4  /* device check found index >= V    */
#define CURAST_ERR_DEVICE_TIMEOUT       -5  /* a bounded device wait gave up    */
#define CURAST_ERR_CUDA                 -6  /* a CUDA runtime call failed       */
#define CURAST_ERR_NOT_AFFINE           -7  /* view/model last row not 0 0 0 1  */
#define CURAST_ERR_BAD_CAMERA           -8  /* proj is not symmetric perspective*/
#define CURAST_ERR_NOT_BUILT            -9  /* no kernel image for this device  */
#define CURAST_ERR_TOO_LARGE           -10  /* over a fixed capacity of curast_render_static */

typedef struct curast_ctx curast_ctx;

/* A CUDA stream handle (cudaStream_t) passed as an opaque pointer. */
typedef void *curast_stream;

/* One view of a batched render: camera, size and its visibility buffer
 * (device, W*H words, caller-owned). */
typedef struct {
    float view[16];
    float proj[16];
    int32_t W, H;
    uint64_t *vis;
} curast_view;

/* Tunables.  None of them but stage3_raycast changes a visibility buffer:
 * every triangle is covered by the same exact rule whichever stage
 * rasterizes it.  With stage3_raycast on, stage1_max_pixels and
 * stage2_max_pixels also decide which triangles are ray cast. */
typedef struct {
    uint32_t stage1_max_pixels;  /* stage 1 rasterizes bbox <= this (paper: 128), 1..1024   */
    uint32_t stage2_max_pixels;  /* stage 2 rasterizes bbox <= this (paper: 4096), >= 32     */
    uint32_t tile_log2;          /* stage-3 tile side 2^k px (paper: 64 -> 6), 4..7          */
    uint32_t stage1_tri_per_thread; /* triangles per thread per stage-1 work grab, 1..4      */
    uint32_t pairs_per_segment;  /* instance-view pairs one stage-1 work item loops over     */
    uint64_t queue1_capacity;    /* stage 1 -> 2 queue entries; overflow is rasterized in place */
    uint64_t queue2_capacity;    /* stage 2 -> 3 tile parts;   overflow is rasterized in place */
    uint32_t check_indices;      /* 1: bounds-check every index on the device               */
    uint32_t collect_stats;      /* 1: count culled / forwarded triangles (slower)           */
    uint64_t stage1_bitmap_bytes; /* survivor bitmap of the stage-1 cull (1 bit per triangle x
                                    pair); a frame needing more runs stage 1 in several
                                    rounds, 2^12..2^36                                       */
    uint32_t stage1_group_min_pairs; /* work items with at least this many (instance, view)
                                    pairs test each step's 64 triangles as one box per pair
                                    before the per-triangle cull (default 2); 0 turns the
                                    group test off, 0..64                                    */
    uint32_t stage3_raycast;     /* 1: the paper's stage 3 (Section 4.3): a triangle whose
                                    visible bbox, on reaching stage 2, holds more than
                                    stage2_max_pixels pixel centres is covered by view-space
                                    pixel-centre rays instead of the fixed-point rule (the
                                    result then follows the ray-cast reading, not the
                                    default one); 0 (default): one fixed-point rule for all */
    uint32_t stage1_exact_all;   /* 1: no conservative cull in stage 1 -- every (triangle,
                                    pair) takes the exact path, which culls tiny and
                                    off-screen triangles itself (the result is the same;
                                    for measuring what the conservative cull saves);
                                    0 (default)                                              */
    uint32_t stage1_vertex_reuse; /* 1: single-pair items of uncompressed meshes stage the
                                    vertex ranges their indices reference in shared memory
                                    and transform each vertex once (Section 6, vertex
                                    reuse); 0 (default): every triangle gathers and
                                    transforms its three vertices, which runs faster on
                                    GB300 (the result is the same)                           */
    uint32_t stage3_tile_buffer; /* 1: stage 3 sorts its tile parts by tile and gives each
                                    tile a shared-memory framebuffer (Section 4.3): up to 8
                                    parts of a tile meet there, and each covered pixel takes
                                    one global atomic minimum; 0 (default, faster on most of
                                    the workloads measured): every covered pixel of every
                                    part goes to the global buffer after a plain read (the
                                    result is the same)                                      */
    uint32_t reserved;           /* 0                                                        */
} curast_config;

/* Counters read back by curast_sync.  Stats fields are filled only when
 * collect_stats is on. */
typedef struct {
    uint64_t triangles_in;       /* triangle x (instance, view) pairs entering stage 1 */
    uint64_t culled_clip;        /* whole triangle beyond one clip plane               */
    uint64_t culled_backface;    /* area <= 0 after snapping (stage 1)                 */
    uint64_t culled_tiny;        /* bbox holds no pixel centre (stage 1)               */
    uint64_t stage1_rasterized;
    uint64_t queued_stage2;
    uint64_t stage2_rasterized;  /* sub-triangles rasterized by stage 2                */
    uint64_t queued_stage3;      /* tile parts                                          */
    uint64_t queue1_overflow;    /* rasterized in place because queue 1 was full        */
    uint64_t queue2_overflow;
    uint64_t exact_path;         /* (triangle, pair)s the conservative tiny cull passed on */
    uint32_t device_error;       /* nonzero: an index >= V was found (check_indices)    */
    uint32_t reserved;
} curast_stats;

/* ------------------------------------------------------------ context --- */

/* Creates a context on CUDA device `device`: queues, frame tables and the
 * tuning state.  Fails with CURAST_ERR_NOT_BUILT when the library holds no
 * kernels for that device (it is built for sm_103a only). */
curast_status curast_create(curast_ctx **out, int device);

/* Waits for the context's work and frees what the context allocated (never
 * the caller's buffers).  NULL is ignored. */
void curast_destroy(curast_ctx *ctx);

const char *curast_status_string(curast_status s);

curast_status curast_get_config(const curast_ctx *ctx, curast_config *out);
/* Validates and installs a configuration; queue capacities are reallocated
 * when they change. */
curast_status curast_set_config(curast_ctx *ctx, const curast_config *cfg);

/* ------------------------------------------------------- scene objects --- */

/* Registers an indexed triangle mesh (Section 4: indexed meshes; Section
 * 4.1: only indices and positions are read while rasterizing).
 *   pos    device, V x 3 FP32 (x, y, z), 4-byte aligned
 *   idx    device, T x 3 uint32 vertex indices, triangles wound CCW = front
 *   rgba8  device, V x 4 bytes of vertex colour for curast_resolve, or NULL
 *   flags  0, or CURAST_MESH_COMPRESSED
 * The buffers are BORROWED: they must stay allocated until curast_destroy;
 * their contents may change between renders.  T may be 0.
 *
 * CURAST_MESH_COMPRESSED (Section 4.6) encodes the mesh on the device into
 * buffers the context owns, and pos and idx are read only during this call
 * (rgba8 stays borrowed):
 *   indices  bit-packed as (index - min) in ceil(log2(max - min + 1)) bits
 *            each, index k at bit k * bits of little-endian 32-bit words;
 *   positions  16 bits an axis over the mesh bounds lo..hi, per axis
 *            q = rint(65535 (p - lo) / (hi - lo)) computed in double.
 * Every stage then renders the decoded positions fma(q, step, lo) in FP32,
 * step = (float)((hi - lo) / 65535), and the decoded indices.  Meshes whose
 * indices reach V are rejected with CURAST_ERR_INDEX_OUT_OF_RANGE.  A
 * compressed mesh cannot be updated and has no differentiable path. */
#define CURAST_MESH_COMPRESSED 1u
curast_status curast_upload_mesh(curast_ctx *ctx, const float *pos, uint64_t V, const uint32_t *idx,
                                 uint64_t T, const uint8_t *rgba8, uint32_t flags, uint32_t *mesh_id);

/* Points a registered mesh at other buffers of the same V and T (e.g. new
 * positions for the differentiable path).  NULL keeps the current one. */
curast_status curast_update_mesh(curast_ctx *ctx, uint32_t mesh_id, const float *pos, const uint32_t *idx,
                                 const uint8_t *rgba8);

/* How a registered mesh is held.  For a compressed mesh the encoding's
 * parameters and read-only device pointers to the context's buffers. */
typedef struct {
    uint64_t V, T;
    uint32_t compressed;          /* 1: Section 4.6 encoding held by the context              */
    uint32_t index_bits;          /* bits per index (compressed)                              */
    uint32_t index_min;
    uint32_t pad;
    float pos_lo[3];              /* decoded position = fma(q, pos_step, pos_lo) per axis     */
    float pos_step[3];
    uint64_t geometry_bytes;      /* device bytes of the index and position data a frame reads */
    const void *packed_indices;   /* device: ceil(3 T bits / 32) words, then zero padding     */
    const void *quantized_positions; /* device: V x 3 uint16                                  */
    const void *grid_flags;       /* device: ceil(ceil(T / 128) / 32) uint32 words; bit G (word
                                     G / 32, bit G % 32) set when the 128 triangles 128 G ..
                                     128 G + 127 all exist and each run of four, 128 G + 4 l ..
                                     + 3, lists (s0 s1 s2) (s2 s1 s3) (s2 s3 s4) (s4 s3 s5) with
                                     s2 = s0 + 1, s4 = s0 + 2, s3 = s1 + 1, s5 = s1 + 2, all
                                     below V (a row of a row-major grid): the compressed cull
                                     then decodes s0 and s1 alone (compressed meshes)         */
} curast_mesh_info;

curast_status curast_get_mesh_info(const curast_ctx *ctx, uint32_t mesh_id, curast_mesh_info *out);

/* Adds an instance of a mesh with an affine model matrix (Section 4.5).
 * Its ids start at the running total of triangles of the instances added
 * before it.  Fails with CURAST_ERR_ID_SPACE_OVERFLOW when the total would
 * exceed 2^36 - 1 triangles. */
curast_status curast_add_instance(curast_ctx *ctx, uint32_t mesh_id, const float model[16],
                                  uint32_t *instance_id);

/* Removes all instances (meshes stay registered). */
curast_status curast_clear_instances(curast_ctx *ctx);

/* ------------------------------------------------------------ render --- */

/* Fills a visibility buffer with 0xFF..FF (device, n words). */
curast_status curast_clear(uint64_t *vis, uint64_t n, curast_stream stream);

/* One frame of every instance into one view (Section 4: host setup, then
 * stages 1, 2 and 3): clears vis, then for every triangle of every instance
 * whose bounds intersect the view frustum keeps, per pixel, the minimum
 * visibility word of the covered fragments.  vis: device, W*H words,
 * caller-owned, 8-byte aligned. */
curast_status curast_render(curast_ctx *ctx, const float view[16], const float proj[16], int W, int H,
                            uint64_t *vis, curast_stream stream);

/* Renders only the instances of one mesh into vis WITHOUT clearing it (the
 * one-launch-per-mesh-per-view path the batched form is compared with). */
curast_status curast_render_mesh(curast_ctx *ctx, uint32_t mesh_id, const float view[16],
                                 const float proj[16], int W, int H, uint64_t *vis, curast_stream stream);

/* Batched frame: every instance into every view in ONE persistent launch
 * sequence (Section 4.1 "Looping Through Batches", Section 4.5 extended to
 * several views: each triangle is loaded once and rasterized into every
 * (instance, view) pair whose bounds meet that view).  Clears every view's
 * buffer first.  With use_graph = 1 the launch sequence is captured once in
 * a CUDA graph (re-captured when the views' sizes or buffers change) and
 * replayed; the frame's matrices are uploaded before the replay.  The
 * result is identical to curast_render per view. */
curast_status curast_render_batch(curast_ctx *ctx, const curast_view *views, int n_views, int use_graph,
                                  curast_stream stream);

/* ------------------------------------------------------------ resolve --- */

/* Screen pass (Section 4.4): per pixel, decode the id, find its instance by
 * binary search of the prefix sum, fetch the triangle, intersect the pixel
 * centre ray with it in view space and interpolate the RGBA8 vertex colours
 * (c = byte / 255).  rgba_f32: device W*H*4 floats or NULL; rgba8: device
 * W*H*4 bytes (rint(clamp(c, 0, 1) * 255)) or NULL.  Empty pixels, and
 * pixels of meshes without colours, get all zeros.  The camera must be the
 * one vis was rendered with, and the instance list unchanged since. */
curast_status curast_resolve(curast_ctx *ctx, const float view[16], const float proj[16], int W, int H,
                             const uint64_t *vis, float *rgba_f32, uint8_t *rgba8, curast_stream stream);

/* Super-sampled resolve (anti-aliasing by super sampling, Section 5): vis
 * holds the view rendered by curast_render at (ss W) x (ss H), i.e. an
 * ss x ss grid of samples at the sub-pixel centres of every output pixel.
 * Each sample is resolved as by curast_resolve; output pixel (x, y) is the
 * box filter of its samples -- FP32 colours summed row by row (sample rows
 * outer, columns inner) and divided by ss^2 -- then converted to RGBA8 as
 * by curast_resolve.  W, H: the output size; ss: 1..8 with ss W, ss H <=
 * 16384; ss = 1 is curast_resolve.  Buffers as for curast_resolve. */
curast_status curast_resolve_ss(curast_ctx *ctx, const float view[16], const float proj[16], int W, int H, int ss,
                                const uint64_t *vis, float *rgba_f32, uint8_t *rgba8, curast_stream stream);

/* Textured resolve (Section 4.4 "Shading and Mip Mapping").  Registers a
 * texture for a mesh:
 *   uv      device, V x 2 FP32 texture coordinates (8-byte aligned)
 *   texels  device, a square RGBA8 texture of side 2^log2_size with its whole
 *           mip chain: level l (0 .. log2_size) holds (2^(log2_size - l))^2
 *           texels, row-major with row 0 at v = 0, each level right after
 *           the one before (4-byte aligned); NULL removes the texture
 *   log2_size  0..15
 * Both buffers are BORROWED like the mesh's: they must stay allocated and
 * unchanged while resolves that use them run.  Fails with
 * CURAST_ERR_INVALID_ARG for a bad mesh id, size or alignment. */
curast_status curast_set_mesh_texture(curast_ctx *ctx, uint32_t mesh_id, const float *uv, const uint8_t *texels,
                                      int log2_size);

/* Screen pass with textures: as curast_resolve, but pixels of a textured
 * mesh take their colour from the texture.  Rays through the centres of the
 * pixel and of its right (x + 1), top (y + 1) and top-right neighbours meet
 * the plane of the pixel's triangle; their barycentrics (unclamped, so
 * points off the triangle extrapolate) interpolate the vertex uv; the
 * footprint F is the larger side of the four samples' uv bounding box times
 * 2^log2_size, and the mip level is floor(log2 F) clamped to 0..log2_size
 * (0 when F < 1).  The colour is the nearest texel of that level at the
 * pixel's own uv -- column floor(u s), row floor(v s), s the level's side,
 * clamped to the level -- as byte / 255.  rgba_f32 (16-byte aligned),
 * rgba8 (4-byte aligned) and level (W*H bytes: the level per pixel, 255 for
 * background and untextured pixels) are device buffers or NULL. */
curast_status curast_resolve_textured(curast_ctx *ctx, const float view[16], const float proj[16], int W, int H,
                                      const uint64_t *vis, float *rgba_f32, uint8_t *rgba8, uint8_t *level,
                                      curast_stream stream);

/* --------------------------------------------------- differentiable step --- */

/* Forward of the differentiable interpolation (perspective-correct
 * barycentrics of Section 4.4 applied to a float attribute): for pixels
 * whose triangle belongs to an instance of mesh_id,
 * out[p] = sum_k b_k(p) attr[v_k]; other pixels get 0.
 *   pos   device V x 3 positions to use instead of the registered ones, or NULL
 *   attr  device V x C floats (1 <= C <= 16); out device W*H*C floats. */
curast_status curast_interpolate(curast_ctx *ctx, uint32_t mesh_id, const float *pos, const float view[16],
                                 const float proj[16], int W, int H, const uint64_t *vis, const float *attr,
                                 int C, float *out, curast_stream stream);

/* Backward of curast_interpolate with the visibility held fixed: given
 * grad_out = dL/dout (device W*H*C), ACCUMULATES dL/dattr into grad_attr
 * (device V*C, may be NULL) and dL/dpos into grad_pos (device V*3, world
 * space through the instance's model-view, may be NULL) with FP32 atomics
 * aggregated per warp.  The caller zeroes the gradients first.  The order of
 * the atomic additions is not fixed, so results vary in the last bits. */
curast_status curast_interpolate_backward(curast_ctx *ctx, uint32_t mesh_id, const float *pos,
                                          const float view[16], const float proj[16], int W, int H,
                                          const uint64_t *vis, const float *attr, int C, const float *grad_out,
                                          float *grad_attr, float *grad_pos, curast_stream stream);

/* Size of the last frame built by a render call (host-side numbers, valid
 * as soon as the call returns). */
typedef struct {
    uint64_t pairs;              /* (instance, view) pairs left after frustum culling     */
    uint64_t segments;           /* stage-1 work segments (mesh x run of pairs)           */
    uint64_t work_items;         /* stage-1 work grabs                                    */
    uint64_t triangles;          /* sum over pairs of the mesh's triangle count           */
    uint64_t unique_triangles;   /* sum of T over meshes with at least one pair           */
    uint64_t unique_vertices;    /* sum of V over the same meshes                         */
    uint64_t rounds;             /* stage-1 rounds (cull + exact kernel pairs)            */
} curast_frame_info;

curast_status curast_last_frame(const curast_ctx *ctx, curast_frame_info *out);

/* ------------------------------------------------------- sync & tuning --- */

/* Waits for the stream, then reads the device counters of the last render
 * into *stats (may be NULL) and returns CURAST_ERR_INDEX_OUT_OF_RANGE if a
 * device check failed since the previous curast_sync, else CURAST_OK. */
curast_status curast_sync(curast_ctx *ctx, curast_stream stream, curast_stats *stats);

/* Per-stage device times (ms) of the last render issued on this context:
 * out[0] clear, [1] stage-1 cull, [2] stage-1 exact path, [3] stage 2,
 * [4] stage 3; waits for them. */
curast_status curast_stage_times(curast_ctx *ctx, float out[5]);

/* Picks stage thresholds, tile size, batch shape, pairs per work item and the
 * group-test threshold for the given views by timing candidate
 * configurations with curast_render_batch (coordinate descent).  A candidate is
 * kept only if its visibility buffers equal the default configuration's bit
 * for bit.  The winner is installed and returned in *chosen (may be NULL).
 * The views' buffers are overwritten. */
curast_status curast_autotune(curast_ctx *ctx, const curast_view *views, int n_views, curast_stream stream,
                              curast_config *chosen);

/* ------------------------------------------------- no-allocation render --- */

/* The paper has no counterpart of this call; it exists for callers that
 * cannot allocate device memory -- real-time loops that must not allocate
 * (an allocation may synchronize the device and take milliseconds), and
 * plug-ins whose host hands out device memory only from its own pools or
 * reserves all of it up front.
 *
 * Renders n_instances (1..CURAST_STATIC_MAX_INSTANCES) instances of one mesh
 * into one view, like curast_render with the same mesh and instances, and
 * with bit-identical results, but without a context and without allocating:
 *   pos, V, idx, T   as in curast_upload_mesh (device buffers)
 *   models           host, n_instances row-major affine 4x4 matrices, or
 *                    NULL for one identity instance (n_instances must be 1);
 *                    instance i owns ids i*T .. i*T + T - 1
 *   view, proj, W, H, vis, stream   as in curast_render (vis is cleared first)
 * The pipeline's scratch (frame tables, counters, stage queues) is one fixed
 * array of about 2 MB in the library's device memory, which every GPU that
 * loads the library holds until the process exits.  Consequences:
 *   - the first call on a device (with that device current) looks the
 *     array's address up and sets the kernels' shared-memory limits; make
 *     that first call before any stream capture; if it fails, the next call
 *     tries again;
 *   - every call uses the same array and leaves its contents behind (the
 *     counters are cleared at the start of each call): calls that overlap on
 *     the GPU -- on two streams, or from two host threads -- race and corrupt
 *     each other's frames; serialize them;
 *   - indices >= V are skipped but not reported (no context to latch them),
 *     and neither is a bounded wait of the stage-1 kernel that gave up (its
 *     triangles are then missing from the frame) -- the call still returns
 *     CURAST_OK;
 *   - the call works on the current CUDA device, which must hold pos, idx,
 *     vis and the stream;
 *   - the stage-1 cull runs its exact path for every triangle (no mesh
 *     bounds are computed), so it is slower than curast_render.
 * Fails with CURAST_ERR_TOO_LARGE for n_instances outside 1..32 or V, T at
 * or above 2^32. */
#define CURAST_STATIC_MAX_INSTANCES 32
curast_status curast_render_static(const float *pos, uint64_t V, const uint32_t *idx, uint64_t T,
                                   const float *models, int n_instances, const float view[16],
                                   const float proj[16], int W, int H, uint64_t *vis, curast_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* CURAST_H */
