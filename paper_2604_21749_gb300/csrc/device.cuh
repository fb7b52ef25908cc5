// device.cuh -- frame tables and the exact per-vertex / per-pixel arithmetic
// shared by every rasterization stage.
//
// All stages cover pixels with one rule (exact integer edge functions on
// vertices snapped to 1/256 px, sampled at pixel centres, top-left fill
// rule, y up, CCW front), so which stage handles a triangle never changes the
// visibility buffer.  Every floating-point operation uses an explicitly
// rounded intrinsic (__fmul_rn, __fadd_rn, ...) so the compiler cannot fuse
// or reorder it; the order of operations is the one stated in each comment.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace curast {

constexpr float kGuard = 128.0f;             // clip guard band |x|,|y| <= 128 w
constexpr float kSnapLimit = 536870912.0f;   // 2^29: bound of snapped coordinates
constexpr uint64_t kIdMask = (1ull << 36) - 1;
constexpr uint64_t kEmpty = ~0ull;
constexpr int kMaxPoly = 9;                  // clipped polygon <= 3 + 5 vertices

// ---------------------------------------------------------------- tables --
struct ViewDev {             // one view of a frame
    float fx, fy, nearv;     // projection vector (Eq. 2) and near plane
    float hw, hh;            // W/2, H/2
    int32_t W, H;
    uint32_t tile0;          // stage-3 tiles: index of this view's first tile in the frame
    uint32_t ntx;            // tiles per row (ceil(W / tile side))
    uint64_t *vis;           // W*H visibility words
};

struct PairDev {             // one (instance, view) pair that survived host culling
    float mv[12];            // rows 0..2 of view * model, FP32 (the exact transform)
    // conservative tiny-triangle cull: rows giving X'*w, Y'*w and w with FMA,
    // where X' = X - 1/2 and Y' = Y - 1/2 put the pixel centres on integers;
    // the estimate and the exact snapped position lie at most
    // margin = max(1/w) * (fk0 + fk1 a) + fk2 a + fk3 pixels apart, a the
    // largest |X'|, |Y'| of the triangle, while every w exceeds wsafe and
    // every |X'|, |Y'| < win; wsafe = +inf disables the test
    float fn[12];
    float fk[4];
    float wsafe, win;
    // bound on the rounding of a row evaluated anywhere in the mesh bounds,
    // for the X'*w, Y'*w and w rows (2^-19 times the row's magnitude bound)
    float fs[3];
    // near-plane cull: a vertex whose estimated w (the w row) lies below nlo
    // has an exact w below the near plane; -inf disables the test
    float nlo;
    uint64_t base;           // global id of the instance's triangle 0
    uint32_t view;
    uint32_t mesh;
};

// Constants of the division of 32-bit numbers by a fixed d >= 2 with a
// multiply-high (Granlund and Montgomery, unsigned division by invariant
// integers): l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1, s = l - 1;
// then n / d = (t + ((n - t) >> 1)) >> s with t = mulhi(n, m).
__host__ __device__ inline void fastdiv_consts(uint32_t d, uint32_t &m, uint32_t &s) {
    uint32_t l = 0;
    while ((1ull << l) < d) ++l;
    m = (uint32_t)((((1ull << 32) * ((1ull << l) - d)) / d) + 1ull);
    s = l - 1u;
}

struct SegDev {              // a stage-1 work item: one mesh x a run of its pairs
    uint32_t mesh;
    uint32_t pair0;
    uint32_t npairs;
    uint32_t pad;
    uint64_t T;              // triangles of the mesh
    uint64_t batch0;         // first work-grab index of this segment
    uint64_t word0;          // first survivor-bitmap word of this segment (frame-wide)
};

// The frame's work items in rounds, each small enough for the survivor
// bitmap: round r culls items [b0, b1) into bitmap words [w0, w1).
struct RoundDev {
    uint64_t b0, b1, w0, w1;
};
constexpr int kMaxRounds = 64;

struct MeshDev {
    const float *pos;        // V x 3 FP32, or nullptr when compressed
    const uint32_t *idx;     // T x 3 uint32, or nullptr when compressed
    const uint8_t *rgba;
    uint64_t V, T;
    // Section 4.6 compression (cidx != nullptr): index k of the 3T index
    // words is imin + the `bits` bits at bit k * bits of cidx (little-endian
    // 32-bit words); vertex i is fma(qpos[3i + a], step[a], lo[a]) in FP32
    const uint32_t *cidx;
    const uint16_t *qpos;
    // bit G: 128-triangle group G is a row of a grid, whose index fields
    // follow from its runs' first two (k_grid_flags); nullptr: none known
    const uint32_t *gflag;
    uint32_t bits, mask, imin, pad;
    float lo[3], step[3];
    // texture of the textured resolve (Section 4.4): per-vertex uv (V x 2)
    // and a square RGBA8 mip chain of side 2^tex_log2; uv == nullptr: none
    const float *uv;
    const uint8_t *tex;
    int32_t tex_log2, pad2;
};

__device__ __forceinline__ bool compressed(const MeshDev &m) { return m.cidx != nullptr; }

// Index word k (= 3 t + corner) of a mesh, decoded when compressed.
__device__ __forceinline__ uint32_t mesh_index(const MeshDev &m, uint64_t k) {
    if (!m.cidx) return __ldg(m.idx + k);
    const uint64_t bit = k * m.bits;
    const uint32_t *w = m.cidx + (bit >> 5);
    return m.imin + (__funnelshift_r(__ldg(w), __ldg(w + 1), (uint32_t)bit & 31u) & m.mask);
}

// A 16-bit value as a float, exactly: its bits OR-ed into the mantissa of
// 2^23 give the float 2^23 + q, and subtracting 2^23 is exact (an OR and an
// add instead of a conversion instruction).
__device__ __forceinline__ float u16_to_float(uint32_t q) {
    return __fsub_rn(__int_as_float(0x4B000000 | q), 8388608.0f);
}

// The three coordinates of vertex i as every stage renders them.
__device__ __forceinline__ void mesh_vertex(const MeshDev &m, uint32_t i, float &x, float &y, float &z) {
    if (!m.qpos) {
        const float *q = m.pos + 3 * (uint64_t)i;
        x = __ldg(q); y = __ldg(q + 1); z = __ldg(q + 2);
    } else {
        const uint16_t *q = m.qpos + 3 * (uint64_t)i;
        x = __fmaf_rn(u16_to_float(__ldg(q)), m.step[0], m.lo[0]);
        y = __fmaf_rn(u16_to_float(__ldg(q + 1)), m.step[1], m.lo[1]);
        z = __fmaf_rn(u16_to_float(__ldg(q + 2)), m.step[2], m.lo[2]);
    }
}

struct Q1Entry {             // stage 1 -> stage 2: a whole triangle of one pair
    uint64_t id;
    uint32_t pair;
    uint32_t pad;
};

struct Q2Entry {             // stage 2 -> stage 3: one tile of one sub-triangle
    int32_t X[3], Y[3];      // ray entries: X = (x0, x1, 0), Y = (y0, y1, 0), the pixel range
    float iz[3];
    uint32_t view;
    uint64_t id;
    uint32_t tx, ty;         // tile coordinates
    uint32_t pair;           // ray entries: the (instance, view) pair
    uint32_t ray;            // 1: the paper's ray-cast stage 3 over the whole triangle
};

struct Counters {
    unsigned long long work[kMaxRounds];   // stage-1 work grabs of each round
    unsigned long long q1_count, q1_next;
    unsigned long long q2_count, q2_next;
    unsigned long long overflow1, overflow2;
    unsigned int error, pad;
    unsigned long long stats[8];      // see Stat
    unsigned long long s3_next;       // binned stage 3: tiles taken
    unsigned long long s3_tiles;      // binned stage 3: units of work (parts of one tile)
};

enum Stat { kStatIn = 0, kStatClip, kStatBack, kStatTiny, kStatS1, kStatS2, kStatParts, kStatFast, kStatCount };

// Frame sizes that vary from frame to frame live in device memory, so a
// launch sequence captured in a CUDA graph stays valid.
struct FrameHdr {
    uint64_t n_batches;      // stage-1 work items
    uint32_t n_segs;
    uint32_t n_views;
    uint32_t n_rounds;
    uint32_t pad;
};

struct FrameDev {
    const FrameHdr *hdr;
    const ViewDev *views;
    const PairDev *pairs;
    const SegDev *segs;
    const RoundDev *rounds;
    const MeshDev *meshes;
    Q1Entry *q1;
    Q2Entry *q2;
    uint32_t *bits;          // survivor bitmap of the current round (nullptr: fused stage 1)
    Counters *ctr;
    unsigned *err;           // sticky error bits, cleared by curast_sync
    uint64_t q1_cap, q2_cap;
    uint32_t s1_max;         // stage-1 bbox pixel limit
    uint32_t s2_max;         // stage-2 bbox pixel limit
    uint32_t tile_log2;
    uint32_t tpt;            // stage-1 triangles per thread per grab
    uint32_t g_m, g_s;       // multiply-high division by G = 8 tpt words (fastdiv_consts)
    uint32_t check;          // bounds-check indices
    uint32_t stats;          // count statistics
    uint32_t group_min;      // instanced items with >= this many pairs (> 0) run the group test
    uint32_t s3_ray;         // 1: triangles past s2_max take the paper's ray-cast stage 3
    // binned stage 3 (s3_bin = 1): queue-2 parts sorted by tile, one block per tile
    uint32_t s3_bin;
    uint32_t n_tiles;        // tiles of all views
    uint32_t *tile_cnt;      // n_tiles: parts per tile (counted by stage 2)
    uint32_t *tile_start;    // n_tiles + 1: exclusive prefix sum of tile_cnt
    uint32_t *tile_fill;     // n_tiles: scatter cursors
    uint2 *units;            // (tile, first part in part_sorted): up to 8 parts of one tile
    uint32_t *part_sorted;   // q2_cap: queue-2 indices in tile order
};

constexpr unsigned kErrIndex = 1u;     // a vertex index >= V was skipped
constexpr unsigned kErrTimeout = 2u;   // a bounded wait on a bulk copy gave up

// ------------------------------------------------------------ transform --
struct CV { float x, y, w; };   // clip-space vertex: fx*vx, fy*vy, -vz

// Section 4.1: view-space transform, each row as ((m0 x + m1 y) + m2 z) + m3,
// then the projection vector of Eq. 2 (x, y scaled by fx, fy; depth = -z).
__device__ __forceinline__ CV to_clip(const float *mv, float x, float y, float z, float fx, float fy) {
    float vx = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(mv[0], x), __fmul_rn(mv[1], y)), __fmul_rn(mv[2], z)), mv[3]);
    float vy = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(mv[4], x), __fmul_rn(mv[5], y)), __fmul_rn(mv[6], z)), mv[7]);
    float vz = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(mv[8], x), __fmul_rn(mv[9], y)), __fmul_rn(mv[10], z)), mv[11]);
    CV c;
    c.x = __fmul_rn(fx, vx);
    c.y = __fmul_rn(fy, vy);
    c.w = -vz;
    return c;
}

// Signed distance-like value of plane p (0 near, 1 left, 2 right, 3 bottom,
// 4 top of the guard band); the vertex is inside when the value is >= 0.
__device__ __forceinline__ float plane_value(int p, CV v, float nearv) {
    const float gw = __fmul_rn(kGuard, v.w);
    switch (p) {
    case 0: return __fsub_rn(v.w, nearv);
    case 1: return __fadd_rn(v.x, gw);
    case 2: return __fsub_rn(gw, v.x);
    case 3: return __fadd_rn(v.y, gw);
    default: return __fsub_rn(gw, v.y);
    }
}

// Bit p set when the vertex is outside plane p (NaN counts as outside).
__device__ __forceinline__ unsigned outcode(CV v, float nearv) {
    unsigned o = 0;
#pragma unroll
    for (int p = 0; p < 5; ++p) o |= (plane_value(p, v, nearv) >= 0.0f) ? 0u : (1u << p);
    return o;
}

// Edge from an inside vertex to an outside vertex cut by plane p:
// t = f_in / (f_in - f_out), r = in + t (out - in); depth of the near-plane
// point set to near exactly, other points kept at depth >= near.
__device__ __forceinline__ CV intersect(CV in, CV out, float fin, float fout, int p, float nearv) {
    float t = __fdiv_rn(fin, __fsub_rn(fin, fout));
    CV r;
    r.x = __fadd_rn(in.x, __fmul_rn(t, __fsub_rn(out.x, in.x)));
    r.y = __fadd_rn(in.y, __fmul_rn(t, __fsub_rn(out.y, in.y)));
    r.w = __fadd_rn(in.w, __fmul_rn(t, __fsub_rn(out.w, in.w)));
    if (p == 0) r.w = nearv;
    else if (r.w < nearv) r.w = nearv;
    return r;
}

// Sutherland-Hodgman (Section 4.2) against near, left, right, bottom, top.
// Returns 0 or the vertex count (3..8); a triangle inside every plane comes
// back unchanged.
static __device__ __noinline__ int clip_polygon(const CV tri[3], float nearv, CV out[kMaxPoly]) {
    CV a[kMaxPoly], b[kMaxPoly];
    int n = 3;
    a[0] = tri[0]; a[1] = tri[1]; a[2] = tri[2];
    for (int p = 0; p < 5 && n > 0; ++p) {
        int m = 0;
        CV prev = a[n - 1];
        float fprev = plane_value(p, prev, nearv);
        for (int i = 0; i < n; ++i) {
            CV cur = a[i];
            float fcur = plane_value(p, cur, nearv);
            if (fcur >= 0.0f) {
                if (fprev < 0.0f) b[m++] = intersect(cur, prev, fcur, fprev, p, nearv);
                b[m++] = cur;
            } else if (fprev >= 0.0f) {
                b[m++] = intersect(prev, cur, fprev, fcur, p, nearv);
            }
            prev = cur;
            fprev = fcur;
        }
        for (int i = 0; i < m; ++i) a[i] = b[i];
        n = m;
    }
    if (n < 3) return 0;
    for (int i = 0; i < n; ++i) out[i] = a[i];
    return n;
}

// Eq. 2 division by depth, viewport map and snap to 1/256 px:
// iz = 1/w, s = c * iz, X = (s + 1) * (W/2), Xq = rint(clamp(256 X, +-2^29)).
__device__ __forceinline__ void snap(CV v, float hw, float hh, int &X, int &Y, float &iz) {
    float r = __frcp_rn(v.w);
    float xs = __fmul_rn(__fmul_rn(__fadd_rn(__fmul_rn(v.x, r), 1.0f), hw), 256.0f);
    float ys = __fmul_rn(__fmul_rn(__fadd_rn(__fmul_rn(v.y, r), 1.0f), hh), 256.0f);
    xs = fminf(fmaxf(xs, -kSnapLimit), kSnapLimit);
    ys = fminf(fmaxf(ys, -kSnapLimit), kSnapLimit);
    X = __float2int_rn(xs);
    Y = __float2int_rn(ys);
    iz = r;
}

// ---------------------------------------------------------------- raster --
__device__ __forceinline__ int64_t floor_div256(int64_t a) { return a >> 8; }        // arithmetic shift = floor
__device__ __forceinline__ int64_t ceil_div256(int64_t a) { return -((-a) >> 8); }

// top-left rule, y up, CCW: the edge a->b owns samples on it iff it runs
// downwards, or horizontally to the left.
__device__ __forceinline__ bool top_left(int ax, int ay, int bx, int by) {
    int dx = bx - ax, dy = by - ay;
    return dy < 0 || (dy == 0 && dx < 0);
}

// A snapped (sub-)triangle ready for pixel loops.
struct SubTri {
    int X[3], Y[3];
    float iz[3];
    int64_t A;              // twice the signed area, > 0
    int x0, x1, y0, y1;     // pixel-centre range clamped to the screen (may be empty)
    unsigned bias;          // bit k set: edge k is NOT top-left (needs E_k > 0)
    uint64_t id;
};

// Sets up a sub-triangle; returns false when it is back-facing, degenerate
// or covers no pixel centre of the W x H screen.
__device__ __forceinline__ bool setup_subtri(SubTri &s, int W, int H) {
    const int64_t A = (int64_t)(s.X[1] - s.X[0]) * (int64_t)(s.Y[2] - s.Y[0]) -
                      (int64_t)(s.X[2] - s.X[0]) * (int64_t)(s.Y[1] - s.Y[0]);
    if (A <= 0) return false;
    s.A = A;
    int minX = min(s.X[0], min(s.X[1], s.X[2])), maxX = max(s.X[0], max(s.X[1], s.X[2]));
    int minY = min(s.Y[0], min(s.Y[1], s.Y[2])), maxY = max(s.Y[0], max(s.Y[1], s.Y[2]));
    int64_t x0 = ceil_div256((int64_t)minX - 128), x1 = floor_div256((int64_t)maxX - 128);
    int64_t y0 = ceil_div256((int64_t)minY - 128), y1 = floor_div256((int64_t)maxY - 128);
    x0 = max(x0, (int64_t)0); y0 = max(y0, (int64_t)0);
    x1 = min(x1, (int64_t)W - 1); y1 = min(y1, (int64_t)H - 1);
    if (x0 > x1 || y0 > y1) return false;
    s.x0 = (int)x0; s.x1 = (int)x1; s.y0 = (int)y0; s.y1 = (int)y1;
    unsigned b = 0;
    if (!top_left(s.X[1], s.Y[1], s.X[2], s.Y[2])) b |= 1u;
    if (!top_left(s.X[2], s.Y[2], s.X[0], s.Y[0])) b |= 2u;
    if (!top_left(s.X[0], s.Y[0], s.X[1], s.Y[1])) b |= 4u;
    s.bias = b;
    return true;
}

// Depth (Section 4.1, perspective-correct): A / sum_k float(E_k) * iz_k, the
// sum taken as (t0 + t1) + t2; then the 64-bit word depth28 << 36 | id.
__device__ __forceinline__ uint64_t frag_key(int64_t E0, int64_t E1, int64_t E2, int64_t A, const float iz[3],
                                             uint64_t id) {
    float s = __fadd_rn(__fadd_rn(__fmul_rn(__ll2float_rn(E0), iz[0]), __fmul_rn(__ll2float_rn(E1), iz[1])),
                        __fmul_rn(__ll2float_rn(E2), iz[2]));
    float depth = __fdiv_rn(__ll2float_rn(A), s);
    return ((uint64_t)(__float_as_uint(depth) >> 3) << 36) | (id & kIdMask);
}

// Section 3.1: the closest fragment wins by a 64-bit atomic minimum.
// Stage 1's tiny triangles cover a pixel or two each: a reduction that needs
// no answer, issued directly.
__device__ __forceinline__ void depth_min(uint64_t *vis, size_t pix, uint64_t key) {
    atomicMin(reinterpret_cast<unsigned long long *>(vis + pix), (unsigned long long)key);
}

// Stages 2 and 3 write many pixels of one triangle, often behind nearer
// ones: a plain read first skips the atomic when the stored word is already
// smaller (words only ever decrease, so a stale read is still safe).
__device__ __forceinline__ void depth_test_write(uint64_t *vis, size_t pix, uint64_t key) {
    unsigned long long *p = reinterpret_cast<unsigned long long *>(vis + pix);
    if (key < __ldcg(p)) atomicMin(p, (unsigned long long)key);
}

// Exact coverage test and write of one pixel (int64 edge functions).
__device__ __forceinline__ void shade_pixel(const SubTri &s, int x, int y, uint64_t *vis, int W) {
    const int64_t px = 256 * (int64_t)x + 128, py = 256 * (int64_t)y + 128;
    const int64_t E0 = (int64_t)(s.X[2] - s.X[1]) * (py - s.Y[1]) - (int64_t)(s.Y[2] - s.Y[1]) * (px - s.X[1]);
    const int64_t E1 = (int64_t)(s.X[0] - s.X[2]) * (py - s.Y[2]) - (int64_t)(s.Y[0] - s.Y[2]) * (px - s.X[2]);
    const int64_t E2 = (int64_t)(s.X[1] - s.X[0]) * (py - s.Y[0]) - (int64_t)(s.Y[1] - s.Y[0]) * (px - s.X[0]);
    const int64_t b0 = s.bias & 1u, b1 = (s.bias >> 1) & 1u, b2 = (s.bias >> 2) & 1u;
    if (((E0 - b0) | (E1 - b1) | (E2 - b2)) < 0) return;
    depth_test_write(vis, (size_t)y * (size_t)W + (size_t)x, frag_key(E0, E1, E2, s.A, s.iz, s.id));
}

// The coverage test and word of shade_pixel without the write: false when the
// pixel centre is not covered.
__device__ __forceinline__ bool pixel_key(const SubTri &s, int x, int y, uint64_t &key) {
    const int64_t px = 256 * (int64_t)x + 128, py = 256 * (int64_t)y + 128;
    const int64_t E0 = (int64_t)(s.X[2] - s.X[1]) * (py - s.Y[1]) - (int64_t)(s.Y[2] - s.Y[1]) * (px - s.X[1]);
    const int64_t E1 = (int64_t)(s.X[0] - s.X[2]) * (py - s.Y[2]) - (int64_t)(s.Y[0] - s.Y[2]) * (px - s.X[2]);
    const int64_t E2 = (int64_t)(s.X[1] - s.X[0]) * (py - s.Y[0]) - (int64_t)(s.Y[1] - s.Y[0]) * (px - s.X[0]);
    const int64_t b0 = s.bias & 1u, b1 = (s.bias >> 1) & 1u, b2 = (s.bias >> 2) & 1u;
    if (((E0 - b0) | (E1 - b1) | (E2 - b2)) < 0) return false;
    key = frag_key(E0, E1, E2, s.A, s.iz, s.id);
    return true;
}

// Pixels i = start, start + stride, ... of the sub-triangle's pixel range
// (x = x0 + i mod w, y = y0 + i / w: the 1D loop of Section 4.2), optionally
// restricted to a sub-rectangle.  The int64 edge functions of shade_pixel are
// evaluated at the thread's first pixel and then stepped exactly: a step of
// `stride` pixels is q rows and r columns (stride = q w + r), one column
// changes E_k by -256 dy_k and one row by +256 dx_k, and a column past x1
// wraps to the next row.  U > 1: U pixels at a time -- their words first,
// then the reads of the stored words all in flight together, then the
// atomic minimums (their order does not change the result); stage 2, a warp
// per triangle, waits on those reads (U = 4 there), while stage 3's blocks
// and the overflow paths run faster one pixel at a time (U = 1).
template <int U = 1>
__device__ __forceinline__ void raster_range(const SubTri &s, int x0, int x1, int y0, int y1, int start, int stride,
                                             uint64_t *vis, int W) {
    const int w = x1 - x0 + 1;
    const int64_t n = (int64_t)w * (int64_t)(y1 - y0 + 1);
    if ((int64_t)start >= n) return;
    int y = y0 + start / w, x = x0 + start % w;
    const int q = stride / w, r = stride % w;
    const int64_t px = 256 * (int64_t)x + 128, py = 256 * (int64_t)y + 128;
    const int64_t dx0 = (int64_t)s.X[2] - s.X[1], dy0 = (int64_t)s.Y[2] - s.Y[1];
    const int64_t dx1 = (int64_t)s.X[0] - s.X[2], dy1 = (int64_t)s.Y[0] - s.Y[2];
    const int64_t dx2 = (int64_t)s.X[1] - s.X[0], dy2 = (int64_t)s.Y[1] - s.Y[0];
    int64_t E0 = dx0 * (py - s.Y[1]) - dy0 * (px - s.X[1]);
    int64_t E1 = dx1 * (py - s.Y[2]) - dy1 * (px - s.X[2]);
    int64_t E2 = dx2 * (py - s.Y[0]) - dy2 * (px - s.X[0]);
    const int64_t S0 = 256 * ((int64_t)q * dx0 - (int64_t)r * dy0), S1 = 256 * ((int64_t)q * dx1 - (int64_t)r * dy1),
                  S2 = 256 * ((int64_t)q * dx2 - (int64_t)r * dy2);
    const int64_t R0 = 256 * (dx0 + (int64_t)w * dy0), R1 = 256 * (dx1 + (int64_t)w * dy1),
                  R2 = 256 * (dx2 + (int64_t)w * dy2);
    const int64_t b0 = s.bias & 1u, b1 = (s.bias >> 1) & 1u, b2 = (s.bias >> 2) & 1u;
    if (U == 1) {
        for (int64_t i = start; i < n; i += stride) {
            if (((E0 - b0) | (E1 - b1) | (E2 - b2)) >= 0)
                depth_test_write(vis, (size_t)y * (size_t)W + (size_t)x, frag_key(E0, E1, E2, s.A, s.iz, s.id));
            x += r;
            y += q;
            E0 += S0; E1 += S1; E2 += S2;
            if (x > x1) {
                x -= w;
                ++y;
                E0 += R0; E1 += R1; E2 += R2;
            }
        }
        return;
    }
    for (int64_t i = start; i < n; i += U * (int64_t)stride) {
        uint64_t key[U];
        unsigned long long *px[U];
        bool cov[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            cov[u] = i + u * (int64_t)stride < n && ((E0 - b0) | (E1 - b1) | (E2 - b2)) >= 0;
            px[u] = reinterpret_cast<unsigned long long *>(vis + (size_t)y * (size_t)W + (size_t)x);
            key[u] = cov[u] ? frag_key(E0, E1, E2, s.A, s.iz, s.id) : 0ull;
            x += r;
            y += q;
            E0 += S0; E1 += S1; E2 += S2;
            if (x > x1) {
                x -= w;
                ++y;
                E0 += R0; E1 += R1; E2 += R2;
            }
        }
        unsigned long long old[U];
#pragma unroll
        for (int u = 0; u < U; ++u) old[u] = cov[u] ? __ldcg(px[u]) : 0ull;
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (cov[u] && key[u] < old[u]) atomicMin(px[u], (unsigned long long)key[u]);
    }
}

// ---------------------------------------------------- view-space rays --
// view-space vertex: row r of MV as ((m0 x + m1 y) + m2 z) + m3 (Section 4.1)
__device__ __forceinline__ float3 view_space(const float *m, const float *p) {
    float3 v;
    v.x = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(m[0], p[0]), __fmul_rn(m[1], p[1])), __fmul_rn(m[2], p[2])), m[3]);
    v.y = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(m[4], p[0]), __fmul_rn(m[5], p[1])), __fmul_rn(m[6], p[2])), m[7]);
    v.z = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(m[8], p[0]), __fmul_rn(m[9], p[1])), __fmul_rn(m[10], p[2])), m[11]);
    return v;
}

__device__ __forceinline__ float3 sub3(float3 a, float3 b) {
    return make_float3(__fsub_rn(a.x, b.x), __fsub_rn(a.y, b.y), __fsub_rn(a.z, b.z));
}

__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
    return make_float3(__fsub_rn(__fmul_rn(a.y, b.z), __fmul_rn(a.z, b.y)),
                       __fsub_rn(__fmul_rn(a.z, b.x), __fmul_rn(a.x, b.z)),
                       __fsub_rn(__fmul_rn(a.x, b.y), __fmul_rn(a.y, b.x)));
}

__device__ __forceinline__ float dot3(float3 a, float3 b) {
    return __fadd_rn(__fadd_rn(__fmul_rn(a.x, b.x), __fmul_rn(a.y, b.y)), __fmul_rn(a.z, b.z));
}

// Pixel-centre ray through (x, y): (ndx / fx, ndy / fy, -1) with
// ndx = (2x + 1) / W - 1 (camera at the origin of view space).
__device__ __forceinline__ float3 pixel_ray(int x, int y, int W, int H, float fx, float fy) {
    const float ndx = __fsub_rn(__fdiv_rn(__int2float_rn(2 * x + 1), __int2float_rn(W)), 1.0f);
    const float ndy = __fsub_rn(__fdiv_rn(__int2float_rn(2 * y + 1), __int2float_rn(H)), 1.0f);
    return make_float3(__fdiv_rn(ndx, fx), __fdiv_rn(ndy, fy), -1.0f);
}

// Pixel centres 256 i + 128 inside the snapped range [mn, mx] (1/256 px) of
// an n-pixel axis (arithmetic shifts are floor divisions), clamped to the
// screen; lo > hi when there are none.
__device__ __forceinline__ void centre_range(int mn, int mx, int n, int &lo, int &hi) {
    lo = max(-((128 - mn) >> 8), 0);
    hi = min((mx - 128) >> 8, n - 1);
}

// The paper's stage 3 (Section 4.3): a ray from the camera through each
// pixel centre, intersected with the triangle in view space.  With
// e1 = v1 - v0, e2 = v2 - v0, p = r x e2, det = e1.p, u = (-v0).p / det,
// q = (-v0) x e1, w = r.q / det, b0 = (1 - u) - w and t = e2.q / det, the
// pixel is covered when det > 0 (the front side faces the camera), u, w and
// b0 are >= 0 and t >= near, at depth t (the view-space distance along -z).
struct RayTri { float3 e1, e2, tv, qv; };

__device__ __forceinline__ RayTri ray_setup(float3 v0, float3 v1, float3 v2) {
    RayTri R;
    R.e1 = sub3(v1, v0);
    R.e2 = sub3(v2, v0);
    R.tv = make_float3(-v0.x, -v0.y, -v0.z);
    R.qv = cross3(R.tv, R.e1);
    return R;
}

__device__ __forceinline__ bool ray_key(const RayTri &R, int x, int y, const ViewDev &vw, uint64_t id, uint64_t &key) {
    const float3 r = pixel_ray(x, y, vw.W, vw.H, vw.fx, vw.fy);
    const float3 pv = cross3(r, R.e2);
    const float det = dot3(R.e1, pv);
    if (!(det > 0.0f)) return false;
    const float u = __fdiv_rn(dot3(R.tv, pv), det);
    const float w = __fdiv_rn(dot3(r, R.qv), det);
    const float b0 = __fsub_rn(__fsub_rn(1.0f, u), w);
    const float t = __fdiv_rn(dot3(R.e2, R.qv), det);
    if (!(u >= 0.0f && w >= 0.0f && b0 >= 0.0f && t >= vw.nearv)) return false;
    key = ((uint64_t)(__float_as_uint(t) >> 3) << 36) | (id & kIdMask);
    return true;
}

__device__ __forceinline__ void ray_pixel(const RayTri &R, int x, int y, const ViewDev &vw, uint64_t id) {
    uint64_t key;
    if (ray_key(R, x, y, vw, id, key)) depth_test_write(vw.vis, (size_t)y * (size_t)vw.W + (size_t)x, key);
}

// Pixels i = start, start + stride, ... of [x0, x1] x [y0, y1] by ray cast.
__device__ __forceinline__ void ray_range(const RayTri &R, int x0, int x1, int y0, int y1, int start, int stride,
                                          const ViewDev &vw, uint64_t id) {
    const int w = x1 - x0 + 1;
    const int64_t n = (int64_t)w * (int64_t)(y1 - y0 + 1);
    for (int64_t i = start; i < n; i += stride) {
        const int y = y0 + (int)(i / w);
        const int x = x0 + (int)(i - (int64_t)(y - y0) * w);
        ray_pixel(R, x, y, vw, id);
    }
}

}  // namespace curast
