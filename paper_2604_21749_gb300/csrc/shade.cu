// shade.cu -- resolve pass (Section 4.4) and the differentiable interpolation
// step (forward and backward) on a fixed visibility buffer.
#include "internal.h"

namespace curast {

__device__ __forceinline__ float interp3(float b0, float b1, float b2, float c0, float c1, float c2) {
    return __fadd_rn(__fadd_rn(__fmul_rn(b0, c0), __fmul_rn(b1, c1)), __fmul_rn(b2, c2));
}

// Section 4.4: the mesh instance owning a global id is found by binary
// search of the exclusive prefix sum (last instance with base <= id).
__device__ __forceinline__ int find_instance(const uint64_t *base, int n, uint64_t id) {
    int lo = 0, hi = n;   // first index with base[i] > id
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (base[mid] <= id) lo = mid + 1; else hi = mid;
    }
    return lo - 1;
}

// Barycentrics of the ray hit with the triangle's plane (Moeller-Trumbore
// form, unclamped): e1 = v1 - v0, e2 = v2 - v0, p = r x e2, det = e1.p,
// u = (-v0).p / det, q = (-v0) x e1, w = r.q / det, b = (1 - u - w, u, w).
__device__ __forceinline__ void ray_bary(float3 r, float3 v0, float3 v1, float3 v2, float &b0, float &b1, float &b2) {
    const float3 e1 = sub3(v1, v0), e2 = sub3(v2, v0);
    const float3 tv = make_float3(-v0.x, -v0.y, -v0.z);
    const float3 pv = cross3(r, e2);
    const float det = dot3(e1, pv);
    const float u = __fdiv_rn(dot3(tv, pv), det);
    const float3 qv = cross3(tv, e1);
    const float w = __fdiv_rn(dot3(r, qv), det);
    b0 = __fsub_rn(__fsub_rn(1.0f, u), w);
    b1 = u;
    b2 = w;
}

struct PixelTri {
    int inst;
    uint64_t t;
    uint32_t vi[3];
    float3 v[3];
};

__device__ __forceinline__ bool lookup(const ShadeArgs &a, uint64_t key, PixelTri &o, MeshDev &m) {
    if (key == kEmpty) return false;
    const uint64_t id = key & kIdMask;
    const int i = find_instance(a.base, a.n_inst, id);
    if (i < 0) return false;
    o.inst = i;
    o.t = id - a.base[i];
    m = a.meshes[a.inst_mesh[i]];
    if (o.t >= m.T) return false;
    const float *mv = a.inst_mv + 12 * (size_t)i;
    const bool over = a.pos && a.inst_mesh[i] == a.mesh;    // positions given by the caller
    for (int k = 0; k < 3; ++k) {
        o.vi[k] = mesh_index(m, 3 * o.t + k);
        if (o.vi[k] >= m.V) return false;
    }
    for (int k = 0; k < 3; ++k) {
        float p[3];
        if (over) {
            p[0] = a.pos[3 * (size_t)o.vi[k]]; p[1] = a.pos[3 * (size_t)o.vi[k] + 1]; p[2] = a.pos[3 * (size_t)o.vi[k] + 2];
        } else {
            mesh_vertex(m, o.vi[k], p[0], p[1], p[2]);
        }
        o.v[k] = view_space(mv, p);
    }
    return true;
}

// ---------------------------------------------------------------- resolve --
// Colour of the sample at pixel (x, y) of a W x H visibility buffer:
// barycentrics of the pixel-centre ray, vertex colours byte / 255; 0 where
// the pixel is empty or the mesh has no colours.
__device__ __forceinline__ void resolve_sample(const ShadeArgs &a, int x, int y, int W, int H, float c[4]) {
    c[0] = c[1] = c[2] = c[3] = 0.0f;
    PixelTri pt;
    MeshDev m;
    if (lookup(a, a.vis[(size_t)y * W + x], pt, m) && m.rgba) {
        float b0, b1, b2;
        ray_bary(pixel_ray(x, y, W, H, a.fx, a.fy), pt.v[0], pt.v[1], pt.v[2], b0, b1, b2);
        const uchar4 q0 = reinterpret_cast<const uchar4 *>(m.rgba)[pt.vi[0]];
        const uchar4 q1 = reinterpret_cast<const uchar4 *>(m.rgba)[pt.vi[1]];
        const uchar4 q2 = reinterpret_cast<const uchar4 *>(m.rgba)[pt.vi[2]];
        const unsigned char s0[4] = {q0.x, q0.y, q0.z, q0.w}, s1[4] = {q1.x, q1.y, q1.z, q1.w},
                            s2[4] = {q2.x, q2.y, q2.z, q2.w};
#pragma unroll
        for (int ch = 0; ch < 4; ++ch)
            c[ch] = interp3(b0, b1, b2, __fdiv_rn(__uint2float_rn(s0[ch]), 255.0f),
                            __fdiv_rn(__uint2float_rn(s1[ch]), 255.0f), __fdiv_rn(__uint2float_rn(s2[ch]), 255.0f));
    }
}

__device__ __forceinline__ void store_rgba(const ShadeArgs &a, size_t pix, const float c[4]) {
    if (a.rgba_f32) reinterpret_cast<float4 *>(a.rgba_f32)[pix] = make_float4(c[0], c[1], c[2], c[3]);
    if (a.rgba8) {
        unsigned char q[4];
#pragma unroll
        for (int ch = 0; ch < 4; ++ch)
            q[ch] = (unsigned char)__float2uint_rn(__fmul_rn(fminf(fmaxf(c[ch], 0.0f), 1.0f), 255.0f));
        reinterpret_cast<uchar4 *>(a.rgba8)[pix] = make_uchar4(q[0], q[1], q[2], q[3]);
    }
}

__global__ void __launch_bounds__(256) k_resolve(ShadeArgs a) {
    const int x = blockIdx.x * 32 + (threadIdx.x & 31), y = blockIdx.y * 8 + (threadIdx.x >> 5);
    if (x >= a.W || y >= a.H) return;
    float c[4];
    resolve_sample(a, x, y, a.W, a.H, c);
    store_rgba(a, (size_t)y * a.W + x, c);
}

// Super-sampled resolve: the visibility buffer holds (ss W) x (ss H)
// samples (the same view rendered at ss times the resolution per axis);
// output pixel (x, y) is the box filter of its ss x ss samples -- their
// colours summed row by row, y outer and x inner, then divided by ss^2.
__global__ void __launch_bounds__(256) k_resolve_ss(ShadeArgs a, int W, int H) {
    const int x = blockIdx.x * 32 + (threadIdx.x & 31), y = blockIdx.y * 8 + (threadIdx.x >> 5);
    if (x >= W || y >= H) return;
    const int ss = a.ss;
    float sum[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    for (int sy = 0; sy < ss; ++sy)
        for (int sx = 0; sx < ss; ++sx) {
            float c[4];
            resolve_sample(a, ss * x + sx, ss * y + sy, a.W, a.H, c);
#pragma unroll
            for (int ch = 0; ch < 4; ++ch) sum[ch] = __fadd_rn(sum[ch], c[ch]);
        }
    const float n = __int2float_rn(ss * ss);
#pragma unroll
    for (int ch = 0; ch < 4; ++ch) sum[ch] = __fdiv_rn(sum[ch], n);
    store_rgba(a, (size_t)y * W + x, sum);
}

// ------------------------------------------------------- textured resolve --
// Section 4.4 "Shading and Mip Mapping": rays through the centres of the
// pixel and of its right (x + 1), top (y + 1) and top-right neighbours meet
// the plane of the pixel's triangle; their barycentrics (unclamped: points
// off the triangle extrapolate) interpolate the vertex uv; the footprint is
// the larger side of the four samples' uv bounding box in level-0 texels,
// F = max(du, dv) 2^L, and the level is floor(log2 F) -- read off the
// float's exponent -- clamped to 0..L (0 when F < 1).  The colour is the
// nearest texel of that level at the pixel's own uv (column floor(u s), row
// floor(v s), s the level's side, clamped to it), c = byte / 255.  Pixels of
// meshes without a texture take the vertex colours of k_resolve.
__global__ void __launch_bounds__(256) k_resolve_tex(ShadeArgs a) {
    const int x = blockIdx.x * 32 + (threadIdx.x & 31), y = blockIdx.y * 8 + (threadIdx.x >> 5);
    if (x >= a.W || y >= a.H) return;
    float c[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    int lev = 255;
    PixelTri pt;
    MeshDev m;
    if (lookup(a, a.vis[(size_t)y * a.W + x], pt, m)) {
        if (m.uv) {
            const float2 t0 = reinterpret_cast<const float2 *>(m.uv)[pt.vi[0]];
            const float2 t1 = reinterpret_cast<const float2 *>(m.uv)[pt.vi[1]];
            const float2 t2 = reinterpret_cast<const float2 *>(m.uv)[pt.vi[2]];
            float us[4], vs[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float b0, b1, b2;
                ray_bary(pixel_ray(x + (q & 1), y + (q >> 1), a.W, a.H, a.fx, a.fy), pt.v[0], pt.v[1], pt.v[2], b0,
                         b1, b2);
                us[q] = interp3(b0, b1, b2, t0.x, t1.x, t2.x);
                vs[q] = interp3(b0, b1, b2, t0.y, t1.y, t2.y);
            }
            const float du = __fsub_rn(fmaxf(fmaxf(us[0], us[1]), fmaxf(us[2], us[3])),
                                       fminf(fminf(us[0], us[1]), fminf(us[2], us[3])));
            const float dv = __fsub_rn(fmaxf(fmaxf(vs[0], vs[1]), fmaxf(vs[2], vs[3])),
                                       fminf(fminf(vs[0], vs[1]), fminf(vs[2], vs[3])));
            const int L = m.tex_log2;
            const float F = __fmul_rn(fmaxf(du, dv), __int2float_rn(1 << L));
            lev = 0;
            if (F >= 1.0f) lev = isfinite(F) ? (int)((__float_as_uint(F) >> 23) & 0xFFu) - 127 : L;
            lev = min(lev, L);
            // level lev follows the finer levels' sum of (2^(L - l))^2 texels
            uint64_t off = 0;
            for (int l = 0; l < lev; ++l) off += 1ull << (2 * (L - l));
            const int side = 1 << (L - lev);
            const float fs = __int2float_rn(side);
            float cu = floorf(__fmul_rn(us[0], fs)), cv = floorf(__fmul_rn(vs[0], fs));
            if (!(cu >= 0.0f)) cu = 0.0f;
            if (cu > __fsub_rn(fs, 1.0f)) cu = __fsub_rn(fs, 1.0f);
            if (!(cv >= 0.0f)) cv = 0.0f;
            if (cv > __fsub_rn(fs, 1.0f)) cv = __fsub_rn(fs, 1.0f);
            const uint64_t texel = off + (uint64_t)(uint32_t)cv * (uint64_t)side + (uint64_t)(uint32_t)cu;
            const uchar4 q = reinterpret_cast<const uchar4 *>(m.tex)[texel];
            c[0] = __fdiv_rn(__uint2float_rn(q.x), 255.0f);
            c[1] = __fdiv_rn(__uint2float_rn(q.y), 255.0f);
            c[2] = __fdiv_rn(__uint2float_rn(q.z), 255.0f);
            c[3] = __fdiv_rn(__uint2float_rn(q.w), 255.0f);
        } else if (m.rgba) {
            float b0, b1, b2;
            ray_bary(pixel_ray(x, y, a.W, a.H, a.fx, a.fy), pt.v[0], pt.v[1], pt.v[2], b0, b1, b2);
            const uchar4 q0 = reinterpret_cast<const uchar4 *>(m.rgba)[pt.vi[0]];
            const uchar4 q1 = reinterpret_cast<const uchar4 *>(m.rgba)[pt.vi[1]];
            const uchar4 q2 = reinterpret_cast<const uchar4 *>(m.rgba)[pt.vi[2]];
            const unsigned char s0[4] = {q0.x, q0.y, q0.z, q0.w}, s1[4] = {q1.x, q1.y, q1.z, q1.w},
                                s2[4] = {q2.x, q2.y, q2.z, q2.w};
#pragma unroll
            for (int ch = 0; ch < 4; ++ch)
                c[ch] = interp3(b0, b1, b2, __fdiv_rn(__uint2float_rn(s0[ch]), 255.0f),
                                __fdiv_rn(__uint2float_rn(s1[ch]), 255.0f), __fdiv_rn(__uint2float_rn(s2[ch]), 255.0f));
        }
    }
    const size_t pix = (size_t)y * a.W + x;
    if (a.level) a.level[pix] = (uint8_t)lev;
    store_rgba(a, pix, c);
}

// ------------------------------------------------------- interpolate fwd --
__global__ void __launch_bounds__(256) k_interp_fwd(ShadeArgs a) {
    const int x = blockIdx.x * 32 + (threadIdx.x & 31), y = blockIdx.y * 8 + (threadIdx.x >> 5);
    if (x >= a.W || y >= a.H) return;
    const size_t pix = (size_t)y * a.W + x;
    PixelTri pt;
    MeshDev m;
    float *o = a.out + (size_t)a.C * pix;
    if (lookup(a, a.vis[pix], pt, m) && a.inst_mesh[pt.inst] == a.mesh) {
        float b0, b1, b2;
        ray_bary(pixel_ray(x, y, a.W, a.H, a.fx, a.fy), pt.v[0], pt.v[1], pt.v[2], b0, b1, b2);
        for (int ch = 0; ch < a.C; ++ch)
            o[ch] = interp3(b0, b1, b2, a.attr[(size_t)a.C * pt.vi[0] + ch], a.attr[(size_t)a.C * pt.vi[1] + ch],
                            a.attr[(size_t)a.C * pt.vi[2] + ch]);
    } else {
        for (int ch = 0; ch < a.C; ++ch) o[ch] = 0.0f;
    }
}

// ------------------------------------------------------- interpolate bwd --
// Sums `val` over the lanes of the warp holding the same key and adds the
// sum once per group as an FP32 atomicAdd (warp-aggregated atomics).  All
// 32 lanes must call it; key 0xFFFFFFFF marks lanes with nothing to add.
__device__ __forceinline__ void aggregated_add(unsigned key, float *addr, float val) {
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(peers) - 1;
    float sum = val;
    if (__popc(peers) > 1) {
        sum = 0.0f;
        unsigned m = peers;
        while (m) {
            const int j = __ffs(m) - 1;
            m &= m - 1;
            sum = __fadd_rn(sum, __shfl_sync(peers, val, j));
        }
    }
    if (lane == leader && key != 0xffffffffu) atomicAdd(addr, sum);
}

constexpr int kMaxC = 16;

// Double-float numbers (hi + lo, |lo| <= ulp(hi) / 2) for the two
// quantities whose cancellation the backward cannot afford: the view-space
// vertex v0 and the pixel ray r.  Error-free product by FMA, error-free sum
// (Knuth's two-sum), and a sum of two double-floats.
struct DF { float hi, lo; };
__device__ __forceinline__ DF two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ DF two_sum(float a, float b) {
    const float s = __fadd_rn(a, b), bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ DF df_add(DF x, DF y) {
    const DF s = two_sum(x.hi, y.hi);
    const float lo = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
    const float hi = __fadd_rn(s.hi, lo);
    return {hi, __fsub_rn(lo, __fsub_rn(hi, s.hi))};
}
// x / d for a double-float x and a float d, as a double-float: the first
// quotient rounded, its remainder exact by FMA, the remainder's quotient.
__device__ __forceinline__ DF df_div(DF x, float d) {
    const float q = __fdiv_rn(x.hi, d);
    const float rem = __fadd_rn(__fmaf_rn(-q, d, x.hi), x.lo);
    return two_sum(q, __fdiv_rn(rem, d));
}

// One coordinate of the pixel-centre ray, ((2 i + 1) / n - 1) / f, as a
// double-float (2 i + 1 and n are exact floats below 2^24).
__device__ __forceinline__ DF ray_coord(int i, int n, float f) {
    DF t = df_div({__int2float_rn(2 * i + 1), 0.0f}, __int2float_rn(n));
    t = df_add(t, {-1.0f, 0.0f});
    return df_div(t, f);
}

// a b - c d for double-floats: the hi products error-free, their difference
// as a double-float, the cross terms in FP32 (they are ulp-sized).
__device__ __forceinline__ float df_cross1(DF a, DF b, DF c, DF d) {
    const DF p = two_prod(a.hi, b.hi), q = two_prod(c.hi, d.hi);
    const DF t = df_add(p, {-q.hi, -q.lo});
    const float x = __fsub_rn(__fadd_rn(__fmul_rn(a.hi, b.lo), __fmul_rn(a.lo, b.hi)),
                              __fadd_rn(__fmul_rn(c.hi, d.lo), __fmul_rn(c.lo, d.hi)));
    return __fadd_rn(t.hi, __fadd_rn(t.lo, x));
}

// Gradient of I = sum_k b_k c_k with the visibility held fixed.  With
// D_k = r . (v_{k+1} x v_{k+2}) and S = sum_k D_k the barycentrics are
// b_k = D_k / S, so for g = dL/dI, gamma_k = g . c_k and gbar = sum b_k gamma_k:
//   dL/dc_k = g b_k,
//   dL/dv_j = [ (gamma_{j-1} - gbar) (v_{j+1} x r) + (gamma_{j+1} - gbar) (r x v_{j-1}) ] / S,
//   dL/dp_j = M^T dL/dv_j   (M = the 3x3 part of the instance's model-view).
// A pixel's ray passes ~100x closer to its triangle than the triangle lies
// to the camera, so written naively these cancel in FP32.  Everything is
// expressed instead through the ray's moment about v0, m = v0 x r, and the
// edges E_1 = e1 = v1 - v0, E_2 = e2 = v2 - v0 (E_0 = 0):
//   D_1 = e2 . m,  D_2 = -(e1 . m),  S = r . (e1 x e2),  D_0 = S - D_1 - D_2,
//   v_{j+1} x r = m + E_{j+1} x r,  r x v_{j-1} = -(m + E_{j-1} x r),
// which are all well conditioned once m is: m alone carries the
// cancellation, and is computed from v0 and r held as double-floats (v0 from
// the FP32 model-view and position with error-free products, r by
// double-float division) with a compensated cross product.  The edges come from the model-space
// differences rotated by M.  Everything else is plain FP32.
__global__ void __launch_bounds__(256) k_interp_bwd(ShadeArgs a) {
    const int x = blockIdx.x * 32 + (threadIdx.x & 31), y = blockIdx.y * 8 + (threadIdx.x >> 5);
    const bool inside = x < a.W && y < a.H;
    PixelTri pt;
    MeshDev m;
    bool hit = false;
    size_t pix = 0;
    if (inside) {
        pix = (size_t)y * a.W + x;
        hit = lookup(a, a.vis[pix], pt, m) && a.inst_mesh[pt.inst] == a.mesh;
    }
    float b[3] = {0.0f, 0.0f, 0.0f};
    float dv[3][3] = {{0.0f, 0.0f, 0.0f}, {0.0f, 0.0f, 0.0f}, {0.0f, 0.0f, 0.0f}};
    float g[kMaxC];
    for (int ch = 0; ch < a.C; ++ch) g[ch] = 0.0f;
    if (hit) {
        const float *mv = a.inst_mv + 12 * (size_t)pt.inst;
        const float *pos = (a.pos && a.inst_mesh[pt.inst] == a.mesh) ? a.pos : m.pos;
        const float *p0 = pos + 3 * (size_t)pt.vi[0];
        const float *p1 = pos + 3 * (size_t)pt.vi[1];
        const float *p2 = pos + 3 * (size_t)pt.vi[2];
        // v0 as double-floats, row by row
        DF v0[3];
        for (int r = 0; r < 3; ++r) {
            DF acc = two_prod(mv[4 * r], p0[0]);
            acc = df_add(acc, two_prod(mv[4 * r + 1], p0[1]));
            acc = df_add(acc, two_prod(mv[4 * r + 2], p0[2]));
            v0[r] = df_add(acc, {mv[4 * r + 3], 0.0f});
        }
        // the pixel-centre ray as double-floats
        const DF rx = ray_coord(x, a.W, a.fx), ry = ray_coord(y, a.H, a.fy);
        const DF rz = {-1.0f, 0.0f};
        const float3 r = make_float3(rx.hi, ry.hi, -1.0f);
        // m = v0 x r
        const float3 mm = make_float3(df_cross1(v0[1], rz, v0[2], ry), df_cross1(v0[2], rx, v0[0], rz),
                                      df_cross1(v0[0], ry, v0[1], rx));
        // edges: model-space differences through M
        float3 E[3];
        E[0] = make_float3(0.0f, 0.0f, 0.0f);
        for (int k = 1; k < 3; ++k) {
            const float *pk = k == 1 ? p1 : p2;
            const float d0 = __fsub_rn(pk[0], p0[0]), d1 = __fsub_rn(pk[1], p0[1]), d2 = __fsub_rn(pk[2], p0[2]);
            E[k] = make_float3(__fadd_rn(__fadd_rn(__fmul_rn(mv[0], d0), __fmul_rn(mv[1], d1)), __fmul_rn(mv[2], d2)),
                               __fadd_rn(__fadd_rn(__fmul_rn(mv[4], d0), __fmul_rn(mv[5], d1)), __fmul_rn(mv[6], d2)),
                               __fadd_rn(__fadd_rn(__fmul_rn(mv[8], d0), __fmul_rn(mv[9], d1)), __fmul_rn(mv[10], d2)));
        }
        const float S = dot3(r, cross3(E[1], E[2]));
        float D[3];
        D[1] = dot3(E[2], mm);
        D[2] = -dot3(E[1], mm);
        D[0] = __fsub_rn(__fsub_rn(S, D[1]), D[2]);
        const float invS = __frcp_rn(S);
        for (int k = 0; k < 3; ++k) b[k] = __fmul_rn(D[k], invS);
        for (int ch = 0; ch < a.C; ++ch) g[ch] = a.grad_out[(size_t)a.C * pix + ch];
        float gam[3];
        for (int k = 0; k < 3; ++k) {
            float s = 0.0f;
            for (int ch = 0; ch < a.C; ++ch) s = __fmaf_rn(g[ch], a.attr[(size_t)a.C * pt.vi[k] + ch], s);
            gam[k] = s;
        }
        const float gbar = __fmaf_rn(b[0], gam[0], __fmaf_rn(b[1], gam[1], __fmul_rn(b[2], gam[2])));
        for (int j = 0; j < 3; ++j) {
            const int jm = (j + 2) % 3, jp = (j + 1) % 3;
            const float w1 = __fmul_rn(__fsub_rn(gam[jm], gbar), invS), w2 = __fmul_rn(__fsub_rn(gam[jp], gbar), invS);
            const float3 cp = cross3(E[jp], r), cm = cross3(E[jm], r);
            const float wd = __fsub_rn(w1, w2);
            const float3 d = make_float3(__fmaf_rn(wd, mm.x, __fsub_rn(__fmul_rn(w1, cp.x), __fmul_rn(w2, cm.x))),
                                         __fmaf_rn(wd, mm.y, __fsub_rn(__fmul_rn(w1, cp.y), __fmul_rn(w2, cm.y))),
                                         __fmaf_rn(wd, mm.z, __fsub_rn(__fmul_rn(w1, cp.z), __fmul_rn(w2, cm.z))));
            for (int ax = 0; ax < 3; ++ax)
                dv[j][ax] = __fmaf_rn(mv[ax], d.x, __fmaf_rn(mv[4 + ax], d.y, __fmul_rn(mv[8 + ax], d.z)));
        }
    }
    for (int j = 0; j < 3; ++j) {
        const unsigned key = hit ? pt.vi[j] : 0xffffffffu;
        const size_t vj = hit ? pt.vi[j] : 0;
        if (a.grad_pos)
            for (int ax = 0; ax < 3; ++ax) aggregated_add(key, a.grad_pos + 3 * vj + ax, dv[j][ax]);
        if (a.grad_attr)
            for (int ch = 0; ch < a.C; ++ch)
                aggregated_add(key, a.grad_attr + (size_t)a.C * vj + ch, __fmul_rn(g[ch], b[j]));
    }
}

// -------------------------------------------------------------- launchers --
static dim3 pixel_grid(int W, int H) { return dim3((unsigned)((W + 31) / 32), (unsigned)((H + 7) / 8)); }

cudaError_t launch_resolve_ss(const ShadeArgs &a, int W, int H, cudaStream_t s) {
    k_resolve_ss<<<pixel_grid(W, H), 256, 0, s>>>(a, W, H);
    return cudaGetLastError();
}

cudaError_t launch_resolve(const ShadeArgs &a, cudaStream_t s) {
    k_resolve<<<pixel_grid(a.W, a.H), 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_resolve_textured(const ShadeArgs &a, cudaStream_t s) {
    k_resolve_tex<<<pixel_grid(a.W, a.H), 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_interpolate(const ShadeArgs &a, cudaStream_t s) {
    k_interp_fwd<<<pixel_grid(a.W, a.H), 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_interpolate_backward(const ShadeArgs &a, cudaStream_t s) {
    k_interp_bwd<<<pixel_grid(a.W, a.H), 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace curast
