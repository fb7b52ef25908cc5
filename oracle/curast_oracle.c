/*
 * curast_oracle.c -- the ORACLE: a plain, slow, single-threaded CPU
 * rasterizer that defines the result the GPU path must reproduce bit for bit.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header or constant table with the CUDA path.
 *
 * Build: gcc -O2 -ffp-contract=off -fno-fast-math -shared -fPIC
 * (contraction off: every float expression below is evaluated one IEEE
 * operation at a time, in the order written).
 *
 * What it computes (paper = Schuetz et al., "CuRast", 2026):
 *   - the visibility buffer: for every pixel the minimum over all covered
 *     fragments of the 64-bit word  depth28 << 36 | global triangle id
 *     (Section 4.1 "Rasterization": 28 depth bits taken from the FP32 depth
 *     by dropping the sign bit and 3 mantissa bits, 36 ID bits; Section 3.1:
 *     the closest fragment wins through a 64-bit minimum);
 *   - global triangle ids from the exclusive prefix sum of triangle counts
 *     over the instance list (Section 4, host frame setup; Section 4.4);
 *   - view-space transform, projection by the element-wise vector
 *     P = [f/aspect, f, -1] and division of x, y by depth (Section 4.1,
 *     Eq. 1 and Eq. 2);
 *   - near-plane handling by Sutherland-Hodgman clipping (Section 4.2);
 *   - bounding-box scan over pixel centres (Section 4.1 "Rasterization");
 *   - backface culling (Section 4.1);
 *   - the resolve pass: binary search of the prefix sum, per-pixel
 *     barycentrics of the pixel ray and the triangle in view space, and
 *     vertex-colour interpolation (Section 4.4);
 *   - the textured resolve: the mip level from the texture-space footprint
 *     of four pixel rays, and the nearest texel of that level (Section 4.4
 *     "Shading and Mip Mapping"; reading R17 below).
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   R1 coverage is exact integer arithmetic on vertices snapped to 1/256 px,
 *      sampled at pixel centres, with the top-left fill rule (y-up, CCW);
 *   R2 depth = A / sum_k(float(E_k) * iz_k) with IEEE division (the paper's
 *      approximate __fdividef is replaced so that the result is defined);
 *   R3 clipping also runs against guard-band planes |x|,|y| <= 128 w so
 *      snapped coordinates stay below 2^29; intersections always
 *      interpolate from the inside vertex towards the outside vertex, which
 *      makes shared edges clip identically in both triangles (watertight);
 *   R4 one coverage rule for every triangle size (the paper's stage-3 world
 *      space ray cast is replaced by the same fixed-point rule); the ray
 *      cast itself is orc_render_paper at the end of this file (R16);
 *   R5 ids are numbered over all instances, culled or not;
 *   R6 ties in depth28 go to the smaller id (64-bit minimum);
 *   R17 the footprint is the larger side of the uv bounding box of the four
 *      samples in level-0 texels, the level floor(log2) of it clamped to the
 *      chain, and the texel the nearest one at the pixel's own uv.
 *
 * Every step is pinned by tests/test_oracle_pins.py; among them, a point cut
 * by the near plane takes w = near exactly, the w of every point of that
 * plane (the interpolated w would carry rounding).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_ID_MASK   ((1ull << 36) - 1ull)
#define ORC_EMPTY     0xFFFFFFFFFFFFFFFFull
#define ORC_GUARD     128.0f
#define ORC_SNAP_LIM  536870912.0f /* 2^29 */
#define ORC_MAX_WH    16384

enum { ORC_OK = 0, ORC_BAD_CAMERA = -1, ORC_BAD_INDEX = -2, ORC_ID_OVERFLOW = -3,
       ORC_BAD_ARG = -4, ORC_NOT_AFFINE = -5 };

typedef struct {
    const float *pos;      /* V x 3 */
    uint64_t V;
    const uint32_t *idx;   /* T x 3 */
    uint64_t T;
    const uint8_t *rgba8;  /* V x 4 or NULL */
} orc_mesh;

typedef struct {
    uint32_t mesh;
    uint32_t pad;
    float model[16];       /* row-major affine */
} orc_instance;

typedef struct {
    float view[16];        /* row-major affine world -> view */
    float proj[16];        /* row-major symmetric perspective */
    int32_t W, H;
} orc_camera;

/* clip-space vertex: x = fx * vx, y = fy * vy, w = -vz (positive depth) */
typedef struct { float x, y, w; } orc_cv;

/* ------------------------------------------------------------------ camera */

/* Projection vector of Eq. 2 read off a symmetric perspective matrix:
 * fx = f/aspect = proj[0][0], fy = f = proj[1][1]; near plane from the depth
 * row, near = proj[2][3] / (proj[2][2] - 1), computed in double and rounded. */
int orc_camera_params(const float proj[16], float out[3])
{
    if (proj[1] != 0.0f || proj[2] != 0.0f || proj[3] != 0.0f) return ORC_BAD_CAMERA;
    if (proj[4] != 0.0f || proj[6] != 0.0f || proj[7] != 0.0f) return ORC_BAD_CAMERA;
    if (proj[8] != 0.0f || proj[9] != 0.0f) return ORC_BAD_CAMERA;
    if (proj[12] != 0.0f || proj[13] != 0.0f || proj[14] != -1.0f || proj[15] != 0.0f)
        return ORC_BAD_CAMERA;
    double nearv = (double)proj[11] / ((double)proj[10] - 1.0);
    float fx = proj[0], fy = proj[5], nr = (float)nearv;
    if (!(fx > 0.0f) || !(fy > 0.0f) || !(nr > 0.0f) || !isfinite(nr)) return ORC_BAD_CAMERA;
    out[0] = fx; out[1] = fy; out[2] = nr;
    return ORC_OK;
}

static int is_affine(const float m[16])
{
    return m[12] == 0.0f && m[13] == 0.0f && m[14] == 0.0f && m[15] == 1.0f;
}

/* Model-view: MV = view * model, each entry summed over k = 0..3 left to
 * right in double (the products of two floats are exact), rounded once. */
void orc_model_view(const float view[16], const float model[16], float mv[12])
{
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 4; ++c) {
            double acc = 0.0;
            for (int k = 0; k < 4; ++k)
                acc = acc + (double)view[4 * r + k] * (double)model[4 * k + c];
            mv[4 * r + c] = (float)acc;
        }
}

/* Section 4.1: transform a vertex to view space (row r of MV applied as
 * ((m0*x + m1*y) + m2*z) + m3), then form the clip-space triple. */
static void view_space(const float mv[12], const float *p, float v[3])
{
    for (int r = 0; r < 3; ++r) {
        float a = mv[4 * r + 0] * p[0];
        float b = mv[4 * r + 1] * p[1];
        float s = a + b;
        float c = mv[4 * r + 2] * p[2];
        s = s + c;
        s = s + mv[4 * r + 3];
        v[r] = s;
    }
}

static orc_cv to_clip(const float v[3], float fx, float fy)
{
    orc_cv o;
    o.x = fx * v[0];
    o.y = fy * v[1];
    o.w = -v[2];
    return o;
}

/* ---------------------------------------------------------------- clipping */

static float plane_value(int p, orc_cv v, float nearv)
{
    switch (p) {
    case 0: return v.w - nearv;                  /* near: w >= near   */
    case 1: return v.x + ORC_GUARD * v.w;        /* left guard        */
    case 2: return ORC_GUARD * v.w - v.x;        /* right guard       */
    case 3: return v.y + ORC_GUARD * v.w;        /* bottom guard      */
    default: return ORC_GUARD * v.w - v.y;       /* top guard         */
    }
}

/* Point where the edge from an inside vertex to an outside vertex meets
 * plane p: t = f_in / (f_in - f_out), r = in + t * (out - in). */
static orc_cv intersect(orc_cv in, orc_cv out, float fin, float fout, int p, float nearv)
{
    float den = fin - fout;
    float t = fin / den;
    orc_cv r;
    float d, m;
    d = out.x - in.x; m = t * d; r.x = in.x + m;
    d = out.y - in.y; m = t * d; r.y = in.y + m;
    d = out.w - in.w; m = t * d; r.w = in.w + m;
    if (p == 0) r.w = nearv;
    else if (r.w < nearv) r.w = nearv;
    return r;
}

/* Sutherland-Hodgman against near, left, right, bottom, top, in that order.
 * Returns the vertex count (0 or 3..8); a triangle inside every plane comes
 * back unchanged and in its own vertex order -- every pass would keep its
 * three vertices and cut nothing, so such a triangle is returned at once. */
int orc_clip(const float tri[9], float nearv, float out[24])
{
    orc_cv a[9], b[9];
    int n = 3;
    for (int k = 0; k < 3; ++k) { a[k].x = tri[3 * k]; a[k].y = tri[3 * k + 1]; a[k].w = tri[3 * k + 2]; }
    int inside = 1;
    for (int k = 0; k < 3; ++k)
        for (int p = 0; p < 5; ++p) inside = inside && plane_value(p, a[k], nearv) >= 0.0f;
    if (inside) {
        memcpy(out, tri, sizeof(float) * 9);
        return 3;
    }
    for (int p = 0; p < 5 && n > 0; ++p) {
        int m = 0;
        orc_cv prev = a[n - 1];
        float fprev = plane_value(p, prev, nearv);
        for (int i = 0; i < n; ++i) {
            orc_cv cur = a[i];
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
        memcpy(a, b, sizeof(orc_cv) * (size_t)m);
        n = m;
    }
    if (n < 3) n = 0;
    for (int k = 0; k < n; ++k) { out[3 * k] = a[k].x; out[3 * k + 1] = a[k].y; out[3 * k + 2] = a[k].w; }
    return n;
}

/* -------------------------------------------------------------- projection */

/* Eq. 2 and the division by depth, then the viewport map and the snap to
 * 1/256 pixel: iz = 1/w, s = c * iz, X = (s + 1) * (W/2), Xq = rint(256 X)
 * (round half to even), with 256 X clamped to [-2^29, 2^29]. */
static void snap_vertex(orc_cv v, float hw, float hh, int32_t *X, int32_t *Y, float *iz)
{
    float r = 1.0f / v.w;
    float sx = v.x * r;
    float sy = v.y * r;
    float px = sx + 1.0f;
    float py = sy + 1.0f;
    float X0 = px * hw;
    float Y0 = py * hh;
    float xs = X0 * 256.0f;
    float ys = Y0 * 256.0f;
    if (!(xs >= -ORC_SNAP_LIM)) xs = -ORC_SNAP_LIM;
    if (xs > ORC_SNAP_LIM) xs = ORC_SNAP_LIM;
    if (!(ys >= -ORC_SNAP_LIM)) ys = -ORC_SNAP_LIM;
    if (ys > ORC_SNAP_LIM) ys = ORC_SNAP_LIM;
    *X = (int32_t)rintf(xs);
    *Y = (int32_t)rintf(ys);
    *iz = r;
}

/* --------------------------------------------------------------- raster */

static int64_t floor_div256(int64_t a)
{
    int64_t q = a / 256;
    if ((a % 256) != 0 && a < 0) q -= 1;
    return q;
}

static int64_t ceil_div256(int64_t a)
{
    int64_t q = a / 256;
    if ((a % 256) != 0 && a > 0) q += 1;
    return q;
}

/* edge function of the directed edge a -> b at sample (px, py): the cross
 * product (b - a) x (p - a); positive when p lies to the left of a -> b. */
static int64_t edge(int64_t ax, int64_t ay, int64_t bx, int64_t by, int64_t px, int64_t py)
{
    return (bx - ax) * (py - ay) - (by - ay) * (px - ax);
}

/* top-left rule for a CCW triangle in y-up screen space: an edge owns the
 * samples exactly on it when it runs downwards, or horizontally leftwards. */
static int top_left(int64_t ax, int64_t ay, int64_t bx, int64_t by)
{
    int64_t dx = bx - ax, dy = by - ay;
    return dy < 0 || (dy == 0 && dx < 0);
}

static void raster_tri(const int32_t Xi[3], const int32_t Yi[3], const float izi[3], uint64_t id,
                       int W, int H, int mode, int cull_back, uint64_t *vis)
{
    int64_t X[3] = {Xi[0], Xi[1], Xi[2]};
    int64_t Y[3] = {Yi[0], Yi[1], Yi[2]};
    float iz[3] = {izi[0], izi[1], izi[2]};
    int64_t A = (X[1] - X[0]) * (Y[2] - Y[0]) - (X[2] - X[0]) * (Y[1] - Y[0]);
    if (A == 0) return;
    if (A < 0) {
        if (cull_back) return;
        /* count mode without culling: mirror the winding to CCW */
        int64_t t;
        float f;
        t = X[1]; X[1] = X[2]; X[2] = t;
        t = Y[1]; Y[1] = Y[2]; Y[2] = t;
        f = iz[1]; iz[1] = iz[2]; iz[2] = f;
        A = -A;
    }
    int64_t minX = X[0], maxX = X[0], minY = Y[0], maxY = Y[0];
    for (int k = 1; k < 3; ++k) {
        if (X[k] < minX) minX = X[k];
        if (X[k] > maxX) maxX = X[k];
        if (Y[k] < minY) minY = Y[k];
        if (Y[k] > maxY) maxY = Y[k];
    }
    int64_t x0 = ceil_div256(minX - 128), x1 = floor_div256(maxX - 128);
    int64_t y0 = ceil_div256(minY - 128), y1 = floor_div256(maxY - 128);
    if (x0 < 0) x0 = 0;
    if (y0 < 0) y0 = 0;
    if (x1 > W - 1) x1 = W - 1;
    if (y1 > H - 1) y1 = H - 1;
    int tl0 = top_left(X[1], Y[1], X[2], Y[2]);
    int tl1 = top_left(X[2], Y[2], X[0], Y[0]);
    int tl2 = top_left(X[0], Y[0], X[1], Y[1]);
    for (int64_t y = y0; y <= y1; ++y) {
        for (int64_t x = x0; x <= x1; ++x) {
            int64_t px = 256 * x + 128, py = 256 * y + 128;
            int64_t E0 = edge(X[1], Y[1], X[2], Y[2], px, py);
            int64_t E1 = edge(X[2], Y[2], X[0], Y[0], px, py);
            int64_t E2 = edge(X[0], Y[0], X[1], Y[1], px, py);
            int in0 = E0 > 0 || (E0 == 0 && tl0);
            int in1 = E1 > 0 || (E1 == 0 && tl1);
            int in2 = E2 > 0 || (E2 == 0 && tl2);
            if (!(in0 && in1 && in2)) continue;
            size_t pix = (size_t)y * (size_t)W + (size_t)x;
            if (mode == 1) { vis[pix] += 1; continue; }
            float s0 = (float)E0 * iz[0];
            float s1 = (float)E1 * iz[1];
            float s = s0 + s1;
            float s2 = (float)E2 * iz[2];
            s = s + s2;
            float depth = (float)A / s;
            uint32_t bits;
            memcpy(&bits, &depth, 4);
            uint64_t key = ((uint64_t)(bits >> 3) << 36) | (id & ORC_ID_MASK);
            if (key < vis[pix]) vis[pix] = key;
        }
    }
}

/* ----------------------------------------------------------------- ids */

/* exclusive prefix sum of triangle counts over the instance list (base has
 * n_inst + 1 entries); fails if the total does not fit the 36-bit id field. */
int orc_bases(const orc_mesh *meshes, int n_meshes, const orc_instance *inst, int n_inst, uint64_t *base)
{
    uint64_t acc = 0;
    for (int i = 0; i < n_inst; ++i) {
        if (inst[i].mesh >= (uint32_t)n_meshes) return ORC_BAD_ARG;
        base[i] = acc;
        acc += meshes[inst[i].mesh].T;
        if (acc > ORC_ID_MASK) return ORC_ID_OVERFLOW;
    }
    base[n_inst] = acc;
    return ORC_OK;
}

/* ----------------------------------------------------------- render */

/* Renders instances [first, first + count) of the scene into vis (W x H,
 * row 0 = bottom).  mode 0: visibility words (vis must start all ones);
 * mode 1: coverage counts (vis must start at zero; cull_back selects whether
 * clockwise triangles are dropped).  Ids use bases over ALL instances. */
int orc_render(const orc_mesh *meshes, int n_meshes, const orc_instance *inst, int n_inst,
               const orc_camera *cam, int first, int count, int mode, int cull_back, uint64_t *vis)
{
    float cp[3];
    if (orc_camera_params(cam->proj, cp) != ORC_OK) return ORC_BAD_CAMERA;
    if (cam->W <= 0 || cam->H <= 0 || cam->W > ORC_MAX_WH || cam->H > ORC_MAX_WH) return ORC_BAD_ARG;
    if (!is_affine(cam->view)) return ORC_NOT_AFFINE;
    if (first < 0 || count < 0 || first + count > n_inst) return ORC_BAD_ARG;
    uint64_t *base = (uint64_t *)malloc(sizeof(uint64_t) * ((size_t)n_inst + 1));
    int st = orc_bases(meshes, n_meshes, inst, n_inst, base);
    if (st != ORC_OK) { free(base); return st; }
    float fx = cp[0], fy = cp[1], nearv = cp[2];
    float hw = 0.5f * (float)cam->W, hh = 0.5f * (float)cam->H;
    if (mode == 0) cull_back = 1;
    for (int i = first; i < first + count; ++i) {
        const orc_mesh *m = &meshes[inst[i].mesh];
        if (!is_affine(inst[i].model)) { free(base); return ORC_NOT_AFFINE; }
        float mv[12];
        orc_model_view(cam->view, inst[i].model, mv);
        for (uint64_t t = 0; t < m->T; ++t) {
            float tri[9], poly[24];
            for (int k = 0; k < 3; ++k) {
                uint32_t vi = m->idx[3 * t + (uint64_t)k];
                if ((uint64_t)vi >= m->V) { free(base); return ORC_BAD_INDEX; }
                float v[3];
                view_space(mv, m->pos + 3 * (uint64_t)vi, v);
                orc_cv c = to_clip(v, fx, fy);
                tri[3 * k] = c.x; tri[3 * k + 1] = c.y; tri[3 * k + 2] = c.w;
            }
            int n = orc_clip(tri, nearv, poly);
            if (n < 3) continue;
            int32_t X[8], Y[8];
            float iz[8];
            for (int k = 0; k < n; ++k) {
                orc_cv c = {poly[3 * k], poly[3 * k + 1], poly[3 * k + 2]};
                snap_vertex(c, hw, hh, &X[k], &Y[k], &iz[k]);
            }
            for (int j = 1; j + 1 < n; ++j) {
                int32_t sx[3] = {X[0], X[j], X[j + 1]}, sy[3] = {Y[0], Y[j], Y[j + 1]};
                float sz[3] = {iz[0], iz[j], iz[j + 1]};
                raster_tri(sx, sy, sz, base[i] + t, cam->W, cam->H, mode, cull_back, vis);
            }
        }
    }
    free(base);
    return ORC_OK;
}

/* Rasterizes triangles given directly in snapped fixed point (X, Y per
 * vertex, 6 ints per triangle) with per-vertex iz; triangle t gets id0 + t. */
int orc_raster_fixed(const int32_t *XY, const float *iz, uint64_t n_tri, uint64_t id0,
                     int W, int H, int mode, int cull_back, uint64_t *vis)
{
    for (uint64_t t = 0; t < n_tri; ++t) {
        int32_t X[3] = {XY[6 * t], XY[6 * t + 2], XY[6 * t + 4]};
        int32_t Y[3] = {XY[6 * t + 1], XY[6 * t + 3], XY[6 * t + 5]};
        raster_tri(X, Y, iz + 3 * t, id0 + t, W, H, mode, mode == 0 ? 1 : cull_back, vis);
    }
    return ORC_OK;
}

/* Per-vertex clip-space triple and, for vertices inside every clip plane,
 * the snapped screen position: out = (cx, cy, cw) per vertex, XY = 2 ints,
 * inside = 1 if the vertex lies inside all five planes. */
int orc_project(const float mv[12], const float cp[3], int W, int H, const float *pos, uint64_t n,
                float *clip, int32_t *XY, float *iz, int32_t *inside)
{
    float hw = 0.5f * (float)W, hh = 0.5f * (float)H;
    for (uint64_t i = 0; i < n; ++i) {
        float v[3];
        view_space(mv, pos + 3 * i, v);
        orc_cv c = to_clip(v, cp[0], cp[1]);
        clip[3 * i] = c.x; clip[3 * i + 1] = c.y; clip[3 * i + 2] = c.w;
        int ok = 1;
        for (int p = 0; p < 5; ++p) ok = ok && (plane_value(p, c, cp[2]) >= 0.0f);
        inside[i] = ok;
        if (ok) snap_vertex(c, hw, hh, &XY[2 * i], &XY[2 * i + 1], &iz[i]);
        else { XY[2 * i] = 0; XY[2 * i + 1] = 0; iz[i] = 0.0f; }
    }
    return ORC_OK;
}

/* ---------------------------------------------------------------- resolve */

static void cross3(const float a[3], const float b[3], float o[3])
{
    float p, q;
    p = a[1] * b[2]; q = a[2] * b[1]; o[0] = p - q;
    p = a[2] * b[0]; q = a[0] * b[2]; o[1] = p - q;
    p = a[0] * b[1]; q = a[1] * b[0]; o[2] = p - q;
}

static float dot3(const float a[3], const float b[3])
{
    float p = a[0] * b[0];
    float q = a[1] * b[1];
    float s = p + q;
    float r = a[2] * b[2];
    return s + r;
}

static uint64_t upper_bound_u64(const uint64_t *a, int n, uint64_t key)
{
    int lo = 0, hi = n;           /* first index with a[i] > key */
    while (lo < hi) {
        int mid = lo + (hi - lo) / 2;
        if (a[mid] <= key) lo = mid + 1; else hi = mid;
    }
    return (uint64_t)lo;
}

/* Barycentrics of the ray through the centre of pixel (x, y) -- which may
 * lie just outside the screen -- with the triangle whose view-space
 * vertices are v (camera at the origin; Moeller-Trumbore form, unclamped). */
static void ray_bary(const float v[3][3], const orc_camera *cam, const float cp[3], int x, int y, float b[3])
{
    float ndx = ((float)(2 * x + 1) / (float)cam->W) - 1.0f;
    float ndy = ((float)(2 * y + 1) / (float)cam->H) - 1.0f;
    float r[3] = {ndx / cp[0], ndy / cp[1], -1.0f};
    float e1[3], e2[3], tv[3], pv[3], qv[3];
    for (int k = 0; k < 3; ++k) { e1[k] = v[1][k] - v[0][k]; e2[k] = v[2][k] - v[0][k]; tv[k] = -v[0][k]; }
    cross3(r, e2, pv);
    float det = dot3(e1, pv);
    float u = dot3(tv, pv) / det;
    cross3(tv, e1, qv);
    float w = dot3(r, qv) / det;
    float b0 = 1.0f - u;
    b0 = b0 - w;
    b[0] = b0; b[1] = u; b[2] = w;
}

/* Section 4.4: pixel -> (instance, triangle) by binary search of the prefix
 * sum, then the barycentrics of the pixel-centre ray with the triangle in
 * view space (camera at the origin; Moeller-Trumbore form, unclamped).
 * Returns 0 for background, 1 otherwise. */
static int pixel_bary(const orc_mesh *meshes, const orc_instance *inst, int n_inst, const uint64_t *base,
                      const orc_camera *cam, const float cp[3], int x, int y, uint64_t key,
                      float b[3], const orc_mesh **mesh_out, uint32_t vidx[3])
{
    if (key == ORC_EMPTY) return 0;
    uint64_t id = key & ORC_ID_MASK;
    int i = (int)upper_bound_u64(base, n_inst, id) - 1;
    uint64_t t = id - base[i];
    const orc_mesh *m = &meshes[inst[i].mesh];
    float mv[12];
    orc_model_view(cam->view, inst[i].model, mv);
    float v[3][3];
    for (int k = 0; k < 3; ++k) {
        vidx[k] = m->idx[3 * t + (uint64_t)k];
        view_space(mv, m->pos + 3 * (uint64_t)vidx[k], v[k]);
    }
    ray_bary(v, cam, cp, x, y, b);
    *mesh_out = m;
    return 1;
}

static float interp3(const float b[3], float c0, float c1, float c2)
{
    float p = b[0] * c0;
    float q = b[1] * c1;
    float s = p + q;
    float r = b[2] * c2;
    return s + r;
}

/* One resolved pixel: FP32 RGBA, and RGBA8 = rint(clamp(c, 0, 1) * 255). */
static void put_pixel(const float out[4], size_t pix, float *rgba, uint8_t *rgba8)
{
    for (int ch = 0; ch < 4; ++ch) {
        if (rgba) rgba[4 * pix + ch] = out[ch];
        if (rgba8) {
            float c = out[ch];
            if (!(c >= 0.0f)) c = 0.0f;
            if (c > 1.0f) c = 1.0f;
            rgba8[4 * pix + ch] = (uint8_t)rintf(c * 255.0f);
        }
    }
}

/* Resolve with the meshes' RGBA8 vertex colours (c = byte / 255): FP32 RGBA
 * and RGBA8 = rint(clamp(rgba, 0, 1) * 255); background is all zero. */
int orc_resolve(const orc_mesh *meshes, int n_meshes, const orc_instance *inst, int n_inst,
                const orc_camera *cam, const uint64_t *vis, float *rgba, uint8_t *rgba8)
{
    float cp[3];
    if (orc_camera_params(cam->proj, cp) != ORC_OK) return ORC_BAD_CAMERA;
    uint64_t *base = (uint64_t *)malloc(sizeof(uint64_t) * ((size_t)n_inst + 1));
    int st = orc_bases(meshes, n_meshes, inst, n_inst, base);
    if (st != ORC_OK) { free(base); return st; }
    for (int y = 0; y < cam->H; ++y)
        for (int x = 0; x < cam->W; ++x) {
            size_t pix = (size_t)y * (size_t)cam->W + (size_t)x;
            float b[3], out[4] = {0.0f, 0.0f, 0.0f, 0.0f};
            const orc_mesh *m;
            uint32_t vi[3];
            if (pixel_bary(meshes, inst, n_inst, base, cam, cp, x, y, vis[pix], b, &m, vi) && m->rgba8) {
                for (int ch = 0; ch < 4; ++ch) {
                    float c0 = (float)m->rgba8[4 * (uint64_t)vi[0] + ch] / 255.0f;
                    float c1 = (float)m->rgba8[4 * (uint64_t)vi[1] + ch] / 255.0f;
                    float c2 = (float)m->rgba8[4 * (uint64_t)vi[2] + ch] / 255.0f;
                    out[ch] = interp3(b, c0, c1, c2);
                }
            }
            put_pixel(out, pix, rgba, rgba8);
        }
    free(base);
    return ORC_OK;
}

/* ------------------------------------------------- textured resolve (R17) */

/* A mesh's texture: per-vertex texture coordinates and a square RGBA8 mip
 * chain of side 2^log2_size: level l (0 .. log2_size) holds (2^(log2_size-l))^2
 * texels, row-major with row 0 at v = 0, and the levels follow one another. */
typedef struct {
    const float *uv;        /* V x 2, or NULL: the mesh has no texture */
    const uint8_t *texels;
    int32_t log2_size;
    int32_t pad;
} orc_texture;

/* floor(log2(F)) for a finite F >= 1, read off the exponent of the float. */
static int floor_log2f(float F)
{
    int e;
    frexpf(F, &e);         /* F = m 2^e with m in [0.5, 1) */
    return e - 1;
}

/* Section 4.4 "Shading and Mip Mapping": the mip level of a pixel comes from
 * the pixel footprint in texture space.  Rays through the centres of the
 * pixel and of its right (x + 1), top (y + 1) and top-right neighbours meet
 * the plane of the pixel's triangle; their barycentrics (unclamped, so
 * points off the triangle extrapolate) interpolate the vertex texture
 * coordinates; the footprint is the larger side of the four samples' uv
 * bounding box in level-0 texels, F = max(du, dv) 2^log2_size, and the level
 * is floor(log2(F)), clamped to 0 .. log2_size (0 when F < 1).  The colour is
 * the nearest texel of that level at the pixel's own uv -- column
 * floor(u s), row floor(v s) with s the level's side, clamped to the level --
 * as c = byte / 255; RGBA8 as in orc_resolve.  Pixels of meshes without a
 * texture take orc_resolve's vertex colours.  level: W*H bytes or NULL, the
 * chosen level, 255 for background and untextured pixels. */
int orc_resolve_textured(const orc_mesh *meshes, int n_meshes, const orc_texture *tex,
                         const orc_instance *inst, int n_inst, const orc_camera *cam, const uint64_t *vis,
                         float *rgba, uint8_t *rgba8, uint8_t *level)
{
    float cp[3];
    if (orc_camera_params(cam->proj, cp) != ORC_OK) return ORC_BAD_CAMERA;
    uint64_t *base = (uint64_t *)malloc(sizeof(uint64_t) * ((size_t)n_inst + 1));
    int st = orc_bases(meshes, n_meshes, inst, n_inst, base);
    if (st != ORC_OK) { free(base); return st; }
    for (int y = 0; y < cam->H; ++y)
        for (int x = 0; x < cam->W; ++x) {
            size_t pix = (size_t)y * (size_t)cam->W + (size_t)x;
            float out[4] = {0.0f, 0.0f, 0.0f, 0.0f};
            int lev = 255;
            uint64_t key = vis[pix];
            if (key != ORC_EMPTY) {
                uint64_t id = key & ORC_ID_MASK;
                int i = (int)upper_bound_u64(base, n_inst, id) - 1;
                uint64_t t = id - base[i];
                const orc_mesh *m = &meshes[inst[i].mesh];
                const orc_texture *tx = &tex[inst[i].mesh];
                float mv[12], v[3][3];
                uint32_t vi[3];
                orc_model_view(cam->view, inst[i].model, mv);
                for (int k = 0; k < 3; ++k) {
                    vi[k] = m->idx[3 * t + (uint64_t)k];
                    view_space(mv, m->pos + 3 * (uint64_t)vi[k], v[k]);
                }
                if (tx->uv) {
                    /* the four samples: (x, y), (x + 1, y), (x, y + 1), (x + 1, y + 1) */
                    float us[4], vs[4];
                    for (int q = 0; q < 4; ++q) {
                        float b[3];
                        ray_bary(v, cam, cp, x + (q & 1), y + (q >> 1), b);
                        us[q] = interp3(b, tx->uv[2 * (uint64_t)vi[0]], tx->uv[2 * (uint64_t)vi[1]],
                                        tx->uv[2 * (uint64_t)vi[2]]);
                        vs[q] = interp3(b, tx->uv[2 * (uint64_t)vi[0] + 1], tx->uv[2 * (uint64_t)vi[1] + 1],
                                        tx->uv[2 * (uint64_t)vi[2] + 1]);
                    }
                    float umin = fminf(fminf(us[0], us[1]), fminf(us[2], us[3]));
                    float umax = fmaxf(fmaxf(us[0], us[1]), fmaxf(us[2], us[3]));
                    float vmin = fminf(fminf(vs[0], vs[1]), fminf(vs[2], vs[3]));
                    float vmax = fmaxf(fmaxf(vs[0], vs[1]), fmaxf(vs[2], vs[3]));
                    float du = umax - umin;
                    float dv = vmax - vmin;
                    float F = fmaxf(du, dv) * (float)(1 << tx->log2_size);
                    lev = 0;
                    if (F >= 1.0f) lev = isfinite(F) ? floor_log2f(F) : tx->log2_size;
                    if (lev > tx->log2_size) lev = tx->log2_size;
                    /* level lev starts after the (4^L - 4^(L - lev)) / 3 texels of the finer levels */
                    int side = 1 << (tx->log2_size - lev);
                    uint64_t off = 0;
                    for (int l = 0; l < lev; ++l) {
                        uint64_t sl = (uint64_t)1 << (tx->log2_size - l);
                        off += sl * sl;
                    }
                    float fs = (float)side;
                    float cu = floorf(us[0] * fs);
                    float cv = floorf(vs[0] * fs);
                    if (!(cu >= 0.0f)) cu = 0.0f;
                    if (cu > fs - 1.0f) cu = fs - 1.0f;
                    if (!(cv >= 0.0f)) cv = 0.0f;
                    if (cv > fs - 1.0f) cv = fs - 1.0f;
                    uint64_t texel = off + (uint64_t)cv * (uint64_t)side + (uint64_t)cu;
                    for (int ch = 0; ch < 4; ++ch) out[ch] = (float)tx->texels[4 * texel + (uint64_t)ch] / 255.0f;
                } else if (m->rgba8) {
                    float b[3];
                    ray_bary(v, cam, cp, x, y, b);
                    for (int ch = 0; ch < 4; ++ch) {
                        float c0 = (float)m->rgba8[4 * (uint64_t)vi[0] + ch] / 255.0f;
                        float c1 = (float)m->rgba8[4 * (uint64_t)vi[1] + ch] / 255.0f;
                        float c2 = (float)m->rgba8[4 * (uint64_t)vi[2] + ch] / 255.0f;
                        out[ch] = interp3(b, c0, c1, c2);
                    }
                }
            }
            if (level) level[pix] = (uint8_t)lev;
            put_pixel(out, pix, rgba, rgba8);
        }
    free(base);
    return ORC_OK;
}

/* ------------------------------------------------------------ compression */

/* Section 4.6, indices: the number of bits for indices in [min, max] is
 * ceil(log2(span + 1)), span = max - min (span + 1 distinct values; the
 * paper's ceil(log2(span)) undercounts when span is a power of two). */
int orc_index_bits(uint32_t span)
{
    int b = 0;
    while (b < 32 && ((uint64_t)1 << b) < (uint64_t)span + 1) ++b;
    return b;
}

/* Packs n indices as (index - min) in `bits` bits each, index k at bit
 * k * bits of a little-endian stream of 32-bit words (words must hold
 * ceil(n * bits / 32) + 1 zeroed words). */
void orc_pack_indices(const uint32_t *idx, uint64_t n, uint32_t imin, int bits, uint32_t *words)
{
    for (uint64_t k = 0; k < n; ++k) {
        uint64_t v = (uint64_t)(idx[k] - imin);
        for (int b = 0; b < bits; ++b) {
            uint64_t bit = k * (uint64_t)bits + (uint64_t)b;
            if ((v >> b) & 1u) words[bit >> 5] |= 1u << (bit & 31);
        }
    }
}

/* Index k of a packed stream: min + the `bits` bits at bit k * bits. */
void orc_unpack_indices(const uint32_t *words, uint64_t n, uint32_t imin, int bits, uint32_t *idx)
{
    for (uint64_t k = 0; k < n; ++k) {
        uint64_t v = 0;
        for (int b = 0; b < bits; ++b) {
            uint64_t bit = k * (uint64_t)bits + (uint64_t)b;
            v |= (uint64_t)((words[bit >> 5] >> (bit & 31)) & 1u) << b;
        }
        idx[k] = imin + (uint32_t)v;
    }
}

/* Section 4.6, positions: 16-bit fixed point over the mesh bounds.  Per
 * axis, with lo the minimum and size = max - min (in double),
 * q = rint(65535 (p - lo) / size) clamped to [0, 65535] (q = 0 when
 * size = 0), in double; the paper's 65536 would overflow 16 bits at
 * p = max.  The decoded position is fma(q, step, lo) in FP32 with
 * step = (float)(size / 65535); it is what every stage renders. */
void orc_quantize_positions(const float *pos, uint64_t V, const float lo[3], const double size[3], uint16_t *q)
{
    for (uint64_t i = 0; i < V; ++i)
        for (int a = 0; a < 3; ++a) {
            double v = 0.0;
            if (size[a] > 0.0) v = rint(65535.0 * (((double)pos[3 * i + a] - (double)lo[a]) / size[a]));
            if (!(v >= 0.0)) v = 0.0;
            if (v > 65535.0) v = 65535.0;
            q[3 * i + a] = (uint16_t)v;
        }
}

void orc_dequantize_positions(const uint16_t *q, uint64_t V, const float lo[3], const float step[3], float *pos)
{
    for (uint64_t i = 0; i < V; ++i)
        for (int a = 0; a < 3; ++a) pos[3 * i + a] = fmaf((float)q[3 * i + a], step[a], lo[a]);
}

/* Anti-aliasing by super sampling (Section 5): the view is rendered and
 * resolved at ss times the output size per axis (fine, FP32 RGBA,
 * (ss W) x (ss H) pixels); output pixel (x, y) is the box filter of its
 * ss x ss samples -- summed one IEEE float addition at a time, sample rows
 * outer and columns inner, then divided by ss^2 -- and RGBA8 =
 * rint(clamp(c, 0, 1) * 255) as for the plain resolve. */
int orc_box_filter(const float *fine, int W, int H, int ss, float *rgba, uint8_t *rgba8)
{
    if (ss < 1 || W < 1 || H < 1) return ORC_BAD_ARG;
    const int Wf = ss * W;
    const float n = (float)(ss * ss);
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            size_t pix = (size_t)y * (size_t)W + (size_t)x;
            for (int ch = 0; ch < 4; ++ch) {
                float sum = 0.0f;
                for (int sy = 0; sy < ss; ++sy)
                    for (int sx = 0; sx < ss; ++sx) {
                        size_t f = (size_t)(ss * y + sy) * (size_t)Wf + (size_t)(ss * x + sx);
                        sum = sum + fine[4 * f + ch];
                    }
                float c = sum / n;
                if (rgba) rgba[4 * pix + ch] = c;
                if (rgba8) {
                    if (!(c >= 0.0f)) c = 0.0f;
                    if (c > 1.0f) c = 1.0f;
                    rgba8[4 * pix + ch] = (uint8_t)rintf(c * 255.0f);
                }
            }
        }
    return ORC_OK;
}

/* Interpolation of a C-channel float attribute of one mesh (the
 * differentiable forward): pixels whose triangle belongs to an instance of
 * mesh `mesh` get sum_k b_k attr_k; all others get zero.  The barycentrics
 * are written too (3 floats per pixel, zero for other pixels). */
int orc_interpolate(const orc_mesh *meshes, int n_meshes, const orc_instance *inst, int n_inst,
                    const orc_camera *cam, const uint64_t *vis, uint32_t mesh, const float *attr, int C,
                    float *out, float *bary)
{
    float cp[3];
    if (orc_camera_params(cam->proj, cp) != ORC_OK) return ORC_BAD_CAMERA;
    uint64_t *base = (uint64_t *)malloc(sizeof(uint64_t) * ((size_t)n_inst + 1));
    int st = orc_bases(meshes, n_meshes, inst, n_inst, base);
    if (st != ORC_OK) { free(base); return st; }
    for (int y = 0; y < cam->H; ++y)
        for (int x = 0; x < cam->W; ++x) {
            size_t pix = (size_t)y * (size_t)cam->W + (size_t)x;
            float b[3] = {0.0f, 0.0f, 0.0f};
            const orc_mesh *m;
            uint32_t vi[3];
            int hit = pixel_bary(meshes, inst, n_inst, base, cam, cp, x, y, vis[pix], b, &m, vi);
            if (hit && m != &meshes[mesh]) { hit = 0; b[0] = b[1] = b[2] = 0.0f; }
            for (int ch = 0; ch < C; ++ch)
                out[(size_t)C * pix + ch] = hit ? interp3(b, attr[(uint64_t)C * vi[0] + ch],
                                                          attr[(uint64_t)C * vi[1] + ch],
                                                          attr[(uint64_t)C * vi[2] + ch]) : 0.0f;
            if (bary) { bary[3 * pix] = b[0]; bary[3 * pix + 1] = b[1]; bary[3 * pix + 2] = b[2]; }
        }
    free(base);
    return ORC_OK;
}

/* ------------------------------------------- paper-faithful stage 3 */

/* Bit p set when clip-space vertex v lies outside plane p (0 near, 1..4 the
 * guard band), NaN counting as outside. */
static unsigned outcode5(orc_cv v, float nearv)
{
    unsigned o = 0;
    for (int p = 0; p < 5; ++p)
        if (!(plane_value(p, v, nearv) >= 0.0f)) o |= 1u << p;
    return o;
}

/* Pixel centres covered by the snapped range [mn, mx] (1/256 px), clamped
 * to [0, n - 1]; lo > hi when there are none. */
static void centre_range(int64_t mn, int64_t mx, int n, int64_t *lo, int64_t *hi)
{
    *lo = ceil_div256(mn - 128);
    *hi = floor_div256(mx - 128);
    if (*lo < 0) *lo = 0;
    if (*hi > n - 1) *hi = n - 1;
}

/* Section 4.3 as the paper describes it: the large-triangle stage casts, for
 * every pixel centre of the triangle's visible bbox, a ray from the camera
 * in view space (camera at the origin) and intersects it with the triangle.
 * r = (ndx / fx, ndy / fy, -1) with ndx = (2x + 1) / W - 1; with
 * e1 = v1 - v0, e2 = v2 - v0, p = r x e2, det = e1.p, u = (-v0).p / det,
 * q = (-v0) x e1, w = r.q / det, b0 = (1 - u) - w and t = e2.q / det, the
 * pixel is covered when det > 0 (the front side faces the camera), u, w and
 * b0 are >= 0 and t >= near; its depth is t, the view-space distance along
 * -z that the edge-function depth of Eq. 2 also gives. */
static void raycast_range(const float v[3][3], float fx, float fy, float nearv, int W, int H, int64_t x0,
                          int64_t x1, int64_t y0, int64_t y1, uint64_t id, uint64_t *vis)
{
    float e1[3], e2[3], tv[3], qv[3];
    for (int k = 0; k < 3; ++k) { e1[k] = v[1][k] - v[0][k]; e2[k] = v[2][k] - v[0][k]; tv[k] = -v[0][k]; }
    cross3(tv, e1, qv);
    for (int64_t y = y0; y <= y1; ++y)
        for (int64_t x = x0; x <= x1; ++x) {
            float ndx = ((float)(2 * x + 1) / (float)W) - 1.0f;
            float ndy = ((float)(2 * y + 1) / (float)H) - 1.0f;
            float r[3] = {ndx / fx, ndy / fy, -1.0f};
            float pv[3];
            cross3(r, e2, pv);
            float det = dot3(e1, pv);
            if (!(det > 0.0f)) continue;
            float u = dot3(tv, pv) / det;
            float w = dot3(r, qv) / det;
            float b0 = 1.0f - u;
            b0 = b0 - w;
            float t = dot3(e2, qv) / det;
            if (!(u >= 0.0f && w >= 0.0f && b0 >= 0.0f && t >= nearv)) continue;
            uint32_t bits;
            memcpy(&bits, &t, 4);
            uint64_t key = ((uint64_t)(bits >> 3) << 36) | (id & ORC_ID_MASK);
            size_t pix = (size_t)y * (size_t)W + (size_t)x;
            if (key < vis[pix]) vis[pix] = key;
        }
    (void)H;
}

/* The visibility buffer with the paper's ray-cast stage 3 (reading R16).
 * Which triangles reach it follows the stage thresholds of Sections 4.1 and
 * 4.2, s1_max and s2_max pixel centres:
 *   - a vertex outside the near plane or the guard band sends the triangle
 *     on to stage 2, unless all three lie outside one plane (dropped);
 *   - otherwise the snapped triangle decides: area <= 0 is dropped (back
 *     face), a bbox without a pixel centre on screen is dropped, an extent of
 *     2^14 subpixels or more, or more than s1_max pixel centres, goes on to
 *     stage 2, and every other triangle is rasterized with edge functions;
 *   - in stage 2 the clipped polygon's snapped bbox, clamped to the screen,
 *     decides: more than s2_max pixel centres take the ray cast over exactly
 *     those pixels, fewer take edge functions like everything else.
 * vis (W x H, row 0 = bottom) must start all ones. */
int orc_render_paper(const orc_mesh *meshes, int n_meshes, const orc_instance *inst, int n_inst,
                     const orc_camera *cam, uint32_t s1_max, uint32_t s2_max, uint64_t *vis)
{
    float cp[3];
    if (orc_camera_params(cam->proj, cp) != ORC_OK) return ORC_BAD_CAMERA;
    if (cam->W <= 0 || cam->H <= 0 || cam->W > ORC_MAX_WH || cam->H > ORC_MAX_WH) return ORC_BAD_ARG;
    if (!is_affine(cam->view)) return ORC_NOT_AFFINE;
    uint64_t *base = (uint64_t *)malloc(sizeof(uint64_t) * ((size_t)n_inst + 1));
    int st = orc_bases(meshes, n_meshes, inst, n_inst, base);
    if (st != ORC_OK) { free(base); return st; }
    float fx = cp[0], fy = cp[1], nearv = cp[2];
    int W = cam->W, H = cam->H;
    float hw = 0.5f * (float)W, hh = 0.5f * (float)H;
    for (int i = 0; i < n_inst; ++i) {
        const orc_mesh *m = &meshes[inst[i].mesh];
        if (!is_affine(inst[i].model)) { free(base); return ORC_NOT_AFFINE; }
        float mv[12];
        orc_model_view(cam->view, inst[i].model, mv);
        for (uint64_t t = 0; t < m->T; ++t) {
            uint64_t id = base[i] + t;
            float v[3][3], tri[9];
            orc_cv c[3];
            unsigned o[3];
            for (int k = 0; k < 3; ++k) {
                uint32_t vi = m->idx[3 * t + (uint64_t)k];
                if ((uint64_t)vi >= m->V) { free(base); return ORC_BAD_INDEX; }
                view_space(mv, m->pos + 3 * (uint64_t)vi, v[k]);
                c[k] = to_clip(v[k], fx, fy);
                tri[3 * k] = c[k].x; tri[3 * k + 1] = c[k].y; tri[3 * k + 2] = c[k].w;
                o[k] = outcode5(c[k], nearv);
            }
            if (o[0] & o[1] & o[2]) continue;
            if (!(o[0] | o[1] | o[2])) {
                int32_t X[3], Y[3];
                float iz[3];
                for (int k = 0; k < 3; ++k) snap_vertex(c[k], hw, hh, &X[k], &Y[k], &iz[k]);
                int64_t A = ((int64_t)X[1] - X[0]) * ((int64_t)Y[2] - Y[0]) -
                            ((int64_t)X[2] - X[0]) * ((int64_t)Y[1] - Y[0]);
                if (A <= 0) continue;
                int64_t mnx = X[0], mxx = X[0], mny = Y[0], mxy = Y[0];
                for (int k = 1; k < 3; ++k) {
                    if (X[k] < mnx) mnx = X[k];
                    if (X[k] > mxx) mxx = X[k];
                    if (Y[k] < mny) mny = Y[k];
                    if (Y[k] > mxy) mxy = Y[k];
                }
                int64_t x0, x1, y0, y1;
                centre_range(mnx, mxx, W, &x0, &x1);
                centre_range(mny, mxy, H, &y0, &y1);
                if (x0 > x1 || y0 > y1) continue;
                int large = mxx - mnx >= 16384 || mxy - mny >= 16384 ||
                            (x1 - x0 + 1) * (y1 - y0 + 1) > (int64_t)s1_max;
                if (!large) {
                    raster_tri(X, Y, iz, id, W, H, 0, 1, vis);
                    continue;
                }
            }
            /* stage 2: the clipped polygon */
            float poly[24];
            int n = orc_clip(tri, nearv, poly);
            if (n < 3) continue;
            int32_t PX[8], PY[8];
            float piz[8];
            for (int k = 0; k < n; ++k) {
                orc_cv q = {poly[3 * k], poly[3 * k + 1], poly[3 * k + 2]};
                snap_vertex(q, hw, hh, &PX[k], &PY[k], &piz[k]);
            }
            int64_t mnx = PX[0], mxx = PX[0], mny = PY[0], mxy = PY[0];
            for (int k = 1; k < n; ++k) {
                if (PX[k] < mnx) mnx = PX[k];
                if (PX[k] > mxx) mxx = PX[k];
                if (PY[k] < mny) mny = PY[k];
                if (PY[k] > mxy) mxy = PY[k];
            }
            int64_t x0, x1, y0, y1;
            centre_range(mnx, mxx, W, &x0, &x1);
            centre_range(mny, mxy, H, &y0, &y1);
            if (x0 > x1 || y0 > y1) continue;
            if ((x1 - x0 + 1) * (y1 - y0 + 1) > (int64_t)s2_max) {
                raycast_range(v, fx, fy, nearv, W, H, x0, x1, y0, y1, id, vis);
                continue;
            }
            for (int j = 1; j + 1 < n; ++j) {
                int32_t sx[3] = {PX[0], PX[j], PX[j + 1]}, sy[3] = {PY[0], PY[j], PY[j + 1]};
                float sz[3] = {piz[0], piz[j], piz[j + 1]};
                raster_tri(sx, sy, sz, id, W, H, 0, 1, vis);
            }
        }
    }
    free(base);
    return ORC_OK;
}
