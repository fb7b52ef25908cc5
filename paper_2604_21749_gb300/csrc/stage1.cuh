// stage1.cuh -- the persistent stage-1 kernel (Section 4.1), included by raster.cu.
//
// Warp-specialized pipeline: one producer warp grabs work items from the
// global counter, stages each item's index triples in shared memory with a
// TMA bulk copy and fills the item's per-(instance, view) constants; eight
// consumer warps cull and rasterize.  Producer and consumers meet only at
// full / empty mbarriers of a three-slot ring, so no block-wide barrier
// stalls the consumers.
#pragma once

// ------------------------------------------------------- TMA / mbarrier --
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// 1D bulk copy global -> shared (TMA engine), completion counted in bytes
// on the mbarrier.  dst, src and bytes must be multiples of 16.
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for a phase of an mbarrier; false after 2^24 polls.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    for (int it = 0; it < (1 << 24); ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// --------------------------------------------- conservative tiny cull --
// Per (instance, view) constants of the fast test, staged in shared memory:
// rows giving X'*w, Y'*w and w by FMA (X' = X - 1/2, so pixel centres sit on
// integers), the error bound margin = max(1/w) (ka + kb a) + kc a + kd with
// a the largest |X'|, |Y'| of the triangle, and the region the bound holds in.
struct __align__(16) FastPair {
    float4 rx, ry, rw;          // (fn[4r], fn[4r+1], fn[4r+2], fn[4r+3])
    float4 k;                   // ka, kb, kc, kd
    float4 lim;                 // wsafe, win, W - 1, H - 1 (every w > wsafe and |X'|, |Y'| < win;
                                // the last pixel centre)
    float4 sl;                  // rounding bound of the rows over the mesh bounds (group test), and
                                // nlo: every w below it is beyond the near plane in the exact path
};

struct Tri9 { float v[9]; };    // the three vertices of a triangle

// The "bbox holds no pixel centre" test of Section 4.1, done before the
// exact arithmetic: the estimated bbox widened by the error bound must hold
// no pixel centre of the screen while every vertex lies safely in front of
// the near plane and inside the window -- then the exact snapped bbox holds
// none either and the exact path would drop the triangle as well.
// Evaluated without branches.
__device__ __forceinline__ bool fast_cull(const FastPair &fp, const Tri9 &p) {
    // vertex by vertex into running bounds (few live registers); the host
    // chose wsafe so that every w > wsafe keeps each exact vertex of a
    // tested triangle inside the guard band (no clipping in the exact path)
    float xmn, xmx, ymn, ymx, wmn, wmx, rmx;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float x = p.v[3 * c], y = p.v[3 * c + 1], z = p.v[3 * c + 2];
        const float4 rx = fp.rx, ry = fp.ry, rw = fp.rw;
        const float xw = __fmaf_rn(rx.x, x, __fmaf_rn(rx.y, y, __fmaf_rn(rx.z, z, rx.w)));
        const float yw = __fmaf_rn(ry.x, x, __fmaf_rn(ry.y, y, __fmaf_rn(ry.z, z, ry.w)));
        const float w = __fmaf_rn(rw.x, x, __fmaf_rn(rw.y, y, __fmaf_rn(rw.z, z, rw.w)));
        const float r = rcp_approx(w);
        const float X = xw * r, Y = yw * r;
        if (c == 0) {
            xmn = xmx = X; ymn = ymx = Y; wmn = wmx = w; rmx = r;
        } else {
            xmn = fminf(xmn, X); xmx = fmaxf(xmx, X);
            ymn = fminf(ymn, Y); ymx = fmaxf(ymx, Y);
            wmn = fminf(wmn, w); wmx = fmaxf(wmx, w); rmx = fmaxf(rmx, r);
        }
    }
    const float4 k = fp.k, lim = fp.lim;
    const float a = fmaxf(fmaxf(fabsf(xmn), fabsf(xmx)), fmaxf(fabsf(ymn), fabsf(ymx)));
    const float m = __fmaf_rn(rmx, __fmaf_rn(k.y, a, k.x), __fmaf_rn(k.z, a, k.w));
    const bool safe = (wmn > lim.x) & (a < lim.y);
    // no integer in [lo, hi] within [0, last] on one axis: floor(min(hi, last)) < max(lo, 0)
    const bool nx = floorf(fminf(xmx + m, lim.z)) < fmaxf(xmn - m, 0.0f);
    const bool ny = floorf(fminf(ymx + m, lim.w)) < fmaxf(ymn - m, 0.0f);
    // or every vertex beyond the near plane
    return (safe & (nx | ny)) | (wmx < fp.sl.w);
}

// Packed FP32 pairs (Blackwell f32x2): two independent operations in one
// instruction, each half rounded exactly like the scalar __fmaf_rn,
// __fmul_rn, __fadd_rn and __fsub_rn.
__device__ __forceinline__ float2 fma_x2(float2 a, float2 b, float2 c) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rc, {%6, %7};\n\t"
        "fma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}
__device__ __forceinline__ float2 mul_x2(float2 a, float2 b) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "mul.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 add_x2(float2 a, float2 b) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "add.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 sub_x2(float2 a, float2 b) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "sub.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 dup(float a) { return make_float2(a, a); }

// Minimum and maximum of three floats in one instruction each (the
// three-input forms of min.f32 / max.f32); a NaN operand is ignored, as by
// fminf / fmaxf.
__device__ __forceinline__ float min3f(float a, float b, float c) {
    float d;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}
__device__ __forceinline__ float max3f(float a, float b, float c) {
    float d;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

// The rows of the conservative cull for two vertices at once (one per half
// of each packed pair): X'w, Y'w and w by FMA, 1/w by rcp.approx, then
// X' = (X'w)(1/w) and Y' = (Y'w)(1/w).
__device__ __forceinline__ void xform2(const FastPair &fp, float2 x, float2 y, float2 z, float2 &X, float2 &Y,
                                       float2 &w, float2 &r) {
    const float4 rx = fp.rx, ry = fp.ry, rw = fp.rw;
    const float2 xw = fma_x2(dup(rx.x), x, fma_x2(dup(rx.y), y, fma_x2(dup(rx.z), z, dup(rx.w))));
    const float2 yw = fma_x2(dup(ry.x), x, fma_x2(dup(ry.y), y, fma_x2(dup(ry.z), z, dup(ry.w))));
    w = fma_x2(dup(rw.x), x, fma_x2(dup(rw.y), y, fma_x2(dup(rw.z), z, dup(rw.w))));
    r = make_float2(rcp_approx(w.x), rcp_approx(w.y));
    X = mul_x2(xw, r);
    Y = mul_x2(yw, r);
}

// The decision of the conservative cull for two triangles (one per half)
// from their vertices' bounds: the margin m, the widened bounds, the
// pixel-centre test on each axis, the region where the bound holds and, with
// NEAR, every vertex beyond the near plane.
template <bool NEAR>
__device__ __forceinline__ void cull_tail2(const FastPair &fp, float2 xmn, float2 xmx, float2 ymn, float2 ymx,
                                           float2 wmn, float2 wmx, float2 rmx, bool &cp, bool &cq) {
    const float4 k = fp.k, lim = fp.lim;
    const float2 a = make_float2(max3f(fabsf(xmn.x), fabsf(xmx.x), fmaxf(fabsf(ymn.x), fabsf(ymx.x))),
                                 max3f(fabsf(xmn.y), fabsf(xmx.y), fmaxf(fabsf(ymn.y), fabsf(ymx.y))));
    const float2 m = fma_x2(rmx, fma_x2(dup(k.y), a, dup(k.x)), fma_x2(dup(k.z), a, dup(k.w)));
    const float2 xh = add_x2(xmx, m), xl = sub_x2(xmn, m), yh = add_x2(ymx, m), yl = sub_x2(ymn, m);
    const bool sp = (wmn.x > lim.x) & (a.x < lim.y), sq = (wmn.y > lim.x) & (a.y < lim.y);
    const bool nxp = floorf(fminf(xh.x, lim.z)) < fmaxf(xl.x, 0.0f), nxq = floorf(fminf(xh.y, lim.z)) < fmaxf(xl.y, 0.0f);
    const bool nyp = floorf(fminf(yh.x, lim.w)) < fmaxf(yl.x, 0.0f), nyq = floorf(fminf(yh.y, lim.w)) < fmaxf(yl.y, 0.0f);
    cp = sp & (nxp | nyp);
    cq = sq & (nxq | nyq);
    if (NEAR) {                                       // or every vertex beyond the near plane
        cp |= wmx.x < fp.sl.w;
        cq |= wmx.y < fp.sl.w;
    }
}

// fast_cull for two triangles of the same pair at once: the same arithmetic,
// with the FMA rows, the products by 1/w, the margin and the widened bounds
// evaluated on packed pairs (one triangle per half).  NEAR = false leaves the
// near-plane test out (frames where no vertex can lie near that plane).
template <bool NEAR = true>
__device__ __forceinline__ void fast_cull2(const FastPair &fp, const Tri9 &p, const Tri9 &q, bool &cp, bool &cq) {
    float2 X[3], Y[3], w[3], r[3];
#pragma unroll
    for (int c = 0; c < 3; ++c)
        xform2(fp, make_float2(p.v[3 * c], q.v[3 * c]), make_float2(p.v[3 * c + 1], q.v[3 * c + 1]),
               make_float2(p.v[3 * c + 2], q.v[3 * c + 2]), X[c], Y[c], w[c], r[c]);
    // bounds over the three vertices, one three-input min or max each
    const float2 xmn = make_float2(min3f(X[0].x, X[1].x, X[2].x), min3f(X[0].y, X[1].y, X[2].y));
    const float2 xmx = make_float2(max3f(X[0].x, X[1].x, X[2].x), max3f(X[0].y, X[1].y, X[2].y));
    const float2 ymn = make_float2(min3f(Y[0].x, Y[1].x, Y[2].x), min3f(Y[0].y, Y[1].y, Y[2].y));
    const float2 ymx = make_float2(max3f(Y[0].x, Y[1].x, Y[2].x), max3f(Y[0].y, Y[1].y, Y[2].y));
    const float2 wmn = make_float2(min3f(w[0].x, w[1].x, w[2].x), min3f(w[0].y, w[1].y, w[2].y));
    const float2 rmx = make_float2(max3f(r[0].x, r[1].x, r[2].x), max3f(r[0].y, r[1].y, r[2].y));
    float2 wmx = wmn;
    if (NEAR) wmx = make_float2(max3f(w[0].x, w[1].x, w[2].x), max3f(w[0].y, w[1].y, w[2].y));
    cull_tail2<NEAR>(fp, xmn, xmx, ymn, ymx, wmn, wmx, rmx, cp, cq);
}

// The bounds of two triangles of a strip (one per half) whose vertices are
// the consecutive vertices (a, b, c) and (b, c, d) of the strip, given as the
// packed pairs ab = (a, b) and cd = (c, d) of one quantity.
__device__ __forceinline__ float2 strip_min(float2 ab, float2 cd) {
    return make_float2(min3f(ab.x, ab.y, cd.x), min3f(ab.y, cd.x, cd.y));
}
__device__ __forceinline__ float2 strip_max(float2 ab, float2 cd) {
    return make_float2(max3f(ab.x, ab.y, cd.x), max3f(ab.y, cd.x, cd.y));
}

// The same test for a whole group of triangles and one pair, from the
// group's object-space bounding box (centre c, half extent e).  With
// X0 = (X' w)(c) / w(c) the projected centre, X' = X0 + d / w where
// d = X' w - X0 w is affine in the position; over the box |d| is at most its
// value at c plus the |coefficient|-weighted extent, and w is at least
// w(c) less its own weighted extent (each widened by the rows' rounding
// bound).  So, with every w above wsafe, X' lies within X0 +- max|d| / min w
// for every vertex of the group, and the margin (doubled: the range and the
// exact snapped vertices each take their error at the group's largest 1/w
// and |X'|) holds every exact snapped vertex.  When the widened ranges hold
// no pixel centre, no triangle's bbox does.
template <bool NEAR = true>
__device__ __forceinline__ bool group_cull(const FastPair &fp, float3 c, float3 e) {
    const float4 rx = fp.rx, ry = fp.ry, rw = fp.rw, sl = fp.sl;
    const float cx = __fmaf_rn(rx.x, c.x, __fmaf_rn(rx.y, c.y, __fmaf_rn(rx.z, c.z, rx.w)));
    const float cy = __fmaf_rn(ry.x, c.x, __fmaf_rn(ry.y, c.y, __fmaf_rn(ry.z, c.z, ry.w)));
    const float cw = __fmaf_rn(rw.x, c.x, __fmaf_rn(rw.y, c.y, __fmaf_rn(rw.z, c.z, rw.w)));
    const float ew = __fmaf_rn(fabsf(rw.x), e.x, __fmaf_rn(fabsf(rw.y), e.y, __fmaf_rn(fabsf(rw.z), e.z, sl.z)));
    const float wl = cw - ew;
    const float r0 = rcp_approx(cw);
    const float X0 = cx * r0, Y0 = cy * r0;
    const float dx = __fmaf_rn(fabsf(__fmaf_rn(-X0, rw.x, rx.x)), e.x,
                     __fmaf_rn(fabsf(__fmaf_rn(-X0, rw.y, rx.y)), e.y,
                     __fmaf_rn(fabsf(__fmaf_rn(-X0, rw.z, rx.z)), e.z,
                     __fmaf_rn(fabsf(X0), sl.z, fabsf(__fmaf_rn(-X0, cw, cx)) + sl.x))));
    const float dy = __fmaf_rn(fabsf(__fmaf_rn(-Y0, rw.x, ry.x)), e.x,
                     __fmaf_rn(fabsf(__fmaf_rn(-Y0, rw.y, ry.y)), e.y,
                     __fmaf_rn(fabsf(__fmaf_rn(-Y0, rw.z, ry.z)), e.z,
                     __fmaf_rn(fabsf(Y0), sl.z, fabsf(__fmaf_rn(-Y0, cw, cy)) + sl.y))));
    const float rh = rcp_approx(wl) * 1.0000039f;           // >= 1/w over the box (2^-18 over rcp's error)
    const float hx = dx * rh, hy = dy * rh;
    const float4 k = fp.k, lim = fp.lim;
    const float a = fmaxf(fabsf(X0) + hx, fabsf(Y0) + hy);
    const float m = 2.0f * __fmaf_rn(rh, __fmaf_rn(k.y, a, k.x), __fmaf_rn(k.z, a, k.w)) + 2.0f * (hx + hy) * 4.0e-6f;
    const bool safe = (wl > lim.x) & (a < lim.y);
    const bool nx = floorf(fminf(X0 + hx + m, lim.z)) < fmaxf(X0 - hx - m, 0.0f);
    const bool ny = floorf(fminf(Y0 + hy + m, lim.w)) < fmaxf(Y0 - hy - m, 0.0f);
    // or the whole box beyond the near plane: w <= w(c) + its weighted extent
    return (safe & (nx | ny)) | (NEAR && __fadd_rn(cw, ew) < sl.w);
}

// The exact path of one (triangle, pair) that the conservative cull kept:
// indices and positions from global memory, FP32 transform in the fixed
// order, clip outcodes, snap, culls, then stage-1 raster or queue 1.
// e = (triangle within its mesh, pair).  f must live in parameter or global
// memory (queue-1 overflow passes its address on).
__device__ __forceinline__ void exact_gather(const FrameDev &f, uint2 e, bool live, Tri9 &p) {
    if (live) {
        const MeshDev &mesh = f.meshes[f.pairs[e.y].mesh];
        if (!compressed(mesh)) {
            const uint32_t *ix = mesh.idx + 3 * (uint64_t)e.x;
            const float *pos = mesh.pos;
            const uint32_t i0 = __ldg(ix), i1 = __ldg(ix + 1), i2 = __ldg(ix + 2);
            const float *q0 = pos + 3 * (uint64_t)i0, *q1 = pos + 3 * (uint64_t)i1, *q2 = pos + 3 * (uint64_t)i2;
            p.v[0] = __ldg(q0); p.v[1] = __ldg(q0 + 1); p.v[2] = __ldg(q0 + 2);
            p.v[3] = __ldg(q1); p.v[4] = __ldg(q1 + 1); p.v[5] = __ldg(q1 + 2);
            p.v[6] = __ldg(q2); p.v[7] = __ldg(q2 + 1); p.v[8] = __ldg(q2 + 2);
        } else {
            const MeshDev m = mesh;
#pragma unroll
            for (int c = 0; c < 3; ++c)
                mesh_vertex(m, mesh_index(m, 3 * (uint64_t)e.x + c), p.v[3 * c], p.v[3 * c + 1], p.v[3 * c + 2]);
        }
    } else {
#pragma unroll
        for (int c = 0; c < 9; ++c) p.v[c] = 0.0f;
    }
}

// The exact path given the triangle's positions (from exact_gather).
template <bool RAY>
__device__ __forceinline__ void exact_compute(const FrameDev &f, uint2 e, bool live, const Tri9 &p) {
    const uint32_t pidx = live ? e.y : 0u;
    const uint64_t t = live ? e.x : 0u;
    const PairDev &pr = f.pairs[pidx];
    const MeshDev *mesh = f.meshes + pr.mesh;
    const ViewDev vw = f.views[pr.view];
    Rec r[3];
    int x0 = 0, x1 = 0, y0 = 0, y1 = 0;
    int64_t A = 0;
    unsigned st = kStatCount;
    int cls = kDrop;
    if (live) {
        float mv[12];
#pragma unroll
        for (int q = 0; q < 12; ++q) mv[q] = pr.mv[q];
#pragma unroll
        for (int k = 0; k < 3; ++k)
            r[k] = make_rec(to_clip(mv, p.v[3 * k], p.v[3 * k + 1], p.v[3 * k + 2], vw.fx, vw.fy), vw);
        cls = classify(f, r, vw, x0, x1, y0, y1, A, st);
    }
    const uint64_t id = pr.base + t;
    q1_append<RAY>(f, cls == kQueue, id, pidx, mesh, t);
    if (cls == kSmall) {
        const int X[3] = {r[0].X, r[1].X, r[2].X}, Y[3] = {r[0].Y, r[1].Y, r[2].Y};
        const float iz[3] = {r[0].iz, r[1].iz, r[2].iz};
        raster_small(X, Y, iz, A, x0, x1, y0, y1, id, vw.vis, vw.W);
    }
    if (f.stats && live) {
        stat_add(f, kStatIn, 1);
        if (st != kStatCount) stat_add(f, st, 1);
        if (cls == kSmall) stat_add(f, kStatS1, 1);
    }
}

// (the fused kernel serves the no-allocation entry point, which has no
// ray-cast mode)
__device__ __forceinline__ void exact_body(const FrameDev &f, uint2 e, bool live) {
    Tri9 p;
    exact_gather(f, e, live, p);
    exact_compute<false>(f, e, live, p);
}

// Out-of-line copy for the fused cull kernel (no survivor bitmap), which
// runs the exact path itself.
__device__ __noinline__ void exact_survivor(const FrameDev *f, uint2 e, bool live) { exact_body(*f, e, live); }

// ----------------------------------------------------------- the kernel --
namespace s1 {
constexpr int kConsumerWarps = 8;
constexpr int kConsumers = 32 * kConsumerWarps;      // 256 consumer threads
constexpr int kThreads = kConsumers + 32;            // + one producer warp
constexpr int kMaxTpt = 4;                           // triangles per consumer per item
constexpr int kItem = kConsumers * kMaxTpt;          // 1024 triangles, 12 KB of index triples
constexpr int kSlots = 4;
constexpr int kQueue = 64;                           // per-warp survivors (fused kernel)
constexpr int kMaxPairs = 64;                        // pairs of one segment (pairs_per_segment <= 64)
constexpr int kNT = 2;                               // triangles a lane loads together
constexpr int kCullBlocks = 3;                       // cull blocks per SM: 72 registers a thread (at 4 blocks
                                                     // and 56 registers the four-triangle cull spills)

struct Desc {
    unsigned long long b;  // work item, >= the round's end: none (consumers stop)
    uint64_t t0;           // first triangle of the item within its mesh
    uint64_t wbase;        // bitmap word of (item, pair 0, group 0), relative to the round
    uint32_t n;            // triangles in the item
    uint32_t mesh, pair0, npairs;
};

template <bool INST, bool FUSED>
struct Smem {
    uint32_t idx[kSlots][3 * kItem + 4];             // index triples, or packed index bits (+1 word read ahead)
    FastPair fp[kSlots][INST ? kMaxPairs : 1];
    MeshDev mesh[kSlots];
    Desc desc[kSlots];
    uint64_t full[kSlots], empty[kSlots];
    uint2 wq[FUSED ? kConsumerWarps : 1][FUSED ? kQueue : 1];   // (triangle, pair) survivors
};
}  // namespace s1

template <bool INST, bool FUSED>
size_t stage1_smem_bytes() { return sizeof(s1::Smem<INST, FUSED>); }

// Producer warp: work grabs (Section 4.1 "Looping Through Batches": a
// global counter hands out items until all triangles are done; the counter
// is read one grab ahead), the forward search for the item's segment, the
// item's pair constants, and the TMA copy of its index triples.  Items
// [rd.b0, rd.b1) form round r of the frame.
template <bool INST, bool FUSED, bool COMP>
__device__ __forceinline__ void stage1_producer(const FrameDev &f, s1::Smem<INST, FUSED> &S, const RoundDev &rd,
                                                uint32_t r, int n_segs, uint64_t per_item, uint32_t G) {
    using namespace s1;
    const int lane = threadIdx.x & 31;
    unsigned long long next = 0;
    int segidx = 0;
    unsigned long long seg_end = 0;
    SegDev seg{};
    bool have = false;
    if (lane == 0) next = rd.b0 + atomicAdd(&f.ctr->work[r], 1ull);
    for (int j = 0;; ++j) {
        const int slot = j % kSlots;
        if (j >= kSlots && !mbar_wait(&S.empty[slot], ((j / kSlots) - 1) & 1u)) {
            if (lane == 0) atomicOr(f.err, kErrTimeout);
            return;
        }
        Desc d{};
        if (lane == 0) {
            const unsigned long long b = next;
            d.b = b;
            if (b < rd.b1) {
                next = rd.b0 + atomicAdd(&f.ctr->work[r], 1ull);
                if (!have || b >= seg_end) {          // galloping forward search: grabs only grow
                    int lo = segidx, step = 1, hi;
                    while (true) {
                        hi = lo + step;
                        if (hi >= n_segs || f.segs[hi].batch0 > b) break;
                        lo = hi;
                        step <<= 1;
                    }
                    if (hi > n_segs) hi = n_segs;
                    while (hi - lo > 1) {
                        const int mid = (lo + hi) >> 1;
                        if (f.segs[mid].batch0 <= b) lo = mid; else hi = mid;
                    }
                    segidx = lo;
                    seg = f.segs[lo];
                    seg_end = lo + 1 < n_segs ? f.segs[lo + 1].batch0 : ~0ull;
                    have = true;
                }
                const uint64_t jb = b - seg.batch0;
                d.t0 = jb * per_item;
                const uint64_t left = seg.T - d.t0;
                d.n = (uint32_t)(left < per_item ? left : per_item);
                d.mesh = seg.mesh;
                d.pair0 = seg.pair0;
                d.npairs = INST ? seg.npairs : 1u;
                d.wbase = seg.word0 + jb * seg.npairs * G - rd.w0;
            }
            S.desc[slot] = d;
        }
        d.b = __shfl_sync(0xffffffffu, d.b, 0);
        if (d.b >= rd.b1) {                           // tell the consumers to stop
            __syncwarp();
            mbar_arrive(&S.full[slot]);
            return;
        }
        d.t0 = __shfl_sync(0xffffffffu, d.t0, 0);
        d.n = __shfl_sync(0xffffffffu, d.n, 0);
        d.mesh = __shfl_sync(0xffffffffu, d.mesh, 0);
        d.pair0 = __shfl_sync(0xffffffffu, d.pair0, 0);
        d.npairs = __shfl_sync(0xffffffffu, d.npairs, 0);
        const MeshDev &mesh = f.meshes[d.mesh];
        if (lane == 0) S.mesh[slot] = mesh;
        for (uint32_t q = lane; q < d.npairs; q += 32) {
            const PairDev &pr = f.pairs[d.pair0 + q];
            const ViewDev &vw = f.views[pr.view];
            FastPair fp;
            fp.rx = make_float4(pr.fn[0], pr.fn[1], pr.fn[2], pr.fn[3]);
            fp.ry = make_float4(pr.fn[4], pr.fn[5], pr.fn[6], pr.fn[7]);
            fp.rw = make_float4(pr.fn[8], pr.fn[9], pr.fn[10], pr.fn[11]);
            fp.k = make_float4(pr.fk[0], pr.fk[1], pr.fk[2], pr.fk[3]);
            fp.lim = make_float4(pr.wsafe, pr.win, (float)(vw.W - 1), (float)(vw.H - 1));
            fp.sl = make_float4(pr.fs[0], pr.fs[1], pr.fs[2], pr.nlo);
            S.fp[slot][q] = fp;
        }
        uint32_t bytes = 12u * d.n;
        const uint32_t *src = mesh.idx + 3 * d.t0;
        if (COMP) {
            // the item's packed bits start on a word: 3 t0 bits is a multiple
            // of 32 (t0 is a multiple of 256); one more word is read ahead and
            // the copy is rounded up to 16 bytes (the packed buffer is padded)
            const uint64_t w0 = (3 * d.t0 * mesh.bits) >> 5;
            const uint32_t nw = (uint32_t)((3ull * d.n * mesh.bits + 31) >> 5) + 1;
            bytes = ((nw + 3u) & ~3u) * 4u;
            src = mesh.cidx + w0;
        }
        const bool tma = (reinterpret_cast<uintptr_t>(src) & 15) == 0 && (bytes & 15) == 0;
        if (!tma)
            for (uint32_t w = lane; w < bytes / 4; w += 32) S.idx[slot][w] = __ldg(src + w);
        __syncwarp();
        if (lane == 0) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive_expect_tx(&S.full[slot], tma ? bytes : 0u);
            if (tma) bulk_copy_g2s(S.idx[slot], src, bytes, &S.full[slot]);
        } else {
            mbar_arrive(&S.full[slot]);
        }
    }
}

// The positions of the two triangles a lane holds, from a compressed mesh
// (Section 4.6): the 16-bit values of both triangles' vertices, converted
// exactly (as u16_to_float) and dequantized as fma(q, step, lo) with one
// packed f32x2 operation per coordinate of the two -- each half rounds like
// the scalar __fmaf_rn of mesh_vertex, so the positions are the same.
__device__ __forceinline__ void decode_pair(const MeshDev &mesh, const uint32_t (&ix)[2][3], const bool (&valid)[2],
                                            Tri9 (&p)[2]) {
    uint32_t q[2][9];
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const uint16_t *src = mesh.qpos + 3 * (uint64_t)ix[u][c];
#pragma unroll
            for (int a = 0; a < 3; ++a) q[u][3 * c + a] = valid[u] ? (uint32_t)__ldg(src + a) : 0u;
        }
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const int a = k % 3;
        const float2 f = sub_x2(make_float2(__int_as_float(0x4B000000 | q[0][k]), __int_as_float(0x4B000000 | q[1][k])),
                                dup(8388608.0f));
        const float2 v = fma_x2(f, dup(mesh.step[a]), dup(mesh.lo[a]));
        p[0].v[k] = valid[0] ? v.x : 0.0f;
        p[1].v[k] = valid[1] ? v.y : 0.0f;
    }
}

// The four triangles of a lane in strip order, (s0 s1 s2) (s2 s1 s3)
// (s2 s3 s4) (s4 s3 s5) with sv = s0 .. s5: the six vertices loaded and
// transformed once, each triangle culled from the bounds of its three.
template <bool NEAR, bool COMP>
__device__ __forceinline__ void strip_cull(const FastPair &fp, const MeshDev &mesh, const float *pos,
                                           const uint32_t (&sv)[6], bool (&cull)[4]) {
    // vertex pairs (s0, s1), (s2, s3), (s4, s5)
    float2 X[3], Y[3], w[3], r[3];
    if constexpr (!COMP) {
        float v[18];
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            const float *q = pos + 3 * (uint64_t)sv[c];
            v[3 * c] = __ldg(q); v[3 * c + 1] = __ldg(q + 1); v[3 * c + 2] = __ldg(q + 2);
        }
#pragma unroll
        for (int c = 0; c < 3; ++c)
            xform2(fp, make_float2(v[6 * c], v[6 * c + 3]), make_float2(v[6 * c + 1], v[6 * c + 4]),
                   make_float2(v[6 * c + 2], v[6 * c + 5]), X[c], Y[c], w[c], r[c]);
    } else {
        // the 16-bit values, converted exactly (as u16_to_float) and
        // dequantized as fma(q, step, lo), two vertices a packed pair
        uint32_t fb[18];   // bits of the floats 2^23 + value
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            const uint16_t *src = mesh.qpos + 3 * (uint64_t)sv[c];
#pragma unroll
            for (int a = 0; a < 3; ++a) fb[3 * c + a] = 0x4B000000u | (uint32_t)__ldg(src + a);
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float2 p[3];
#pragma unroll
            for (int a = 0; a < 3; ++a)
                p[a] = fma_x2(sub_x2(make_float2(__int_as_float(fb[6 * c + a]), __int_as_float(fb[6 * c + 3 + a])),
                                     dup(8388608.0f)),
                              dup(mesh.step[a]), dup(mesh.lo[a]));
            xform2(fp, p[0], p[1], p[2], X[c], Y[c], w[c], r[c]);
        }
    }
    // triangles (t0, t1) from the pairs (s0, s1), (s2, s3); (t2, t3) from (s2, s3), (s4, s5)
#pragma unroll
    for (int h = 0; h < 2; ++h)
        cull_tail2<NEAR>(fp, strip_min(X[h], X[h + 1]), strip_max(X[h], X[h + 1]), strip_min(Y[h], Y[h + 1]),
                         strip_max(Y[h], Y[h + 1]), strip_min(w[h], w[h + 1]),
                         NEAR ? strip_max(w[h], w[h + 1]) : make_float2(0.0f, 0.0f),
                         strip_max(r[h], r[h + 1]), cull[2 * h], cull[2 * h + 1]);
}

// Single-pair items of plain meshes, four consecutive triangles a lane: a
// warp takes the 128-triangle groups g = warp, warp + 8, ... of the item and
// lane l the triangles 128 g + 4 l .. 128 g + 4 l + 3, whose twelve index
// words are three 16-byte loads from shared memory.  Where the four are in
// strip order -- the list a triangle strip s0 s1 s2 s3 s4 s5 unrolls to,
// (s0 s1 s2) (s2 s1 s3) (s2 s3 s4) (s4 s3 s5), which is how a row-major grid
// mesh lists a row of cells -- triangle k has the vertices s_k, s_k+1 and
// s_k+2; when every lane's four are, the warp loads and transforms the six
// vertices once for the four triangles.  The cull's bounds are symmetric in
// a triangle's vertices, so each triangle gets the decision fast_cull2 would
// give it.  Other orders run fast_cull2 on the two pairs of triangles.  The
// 128 decisions are the bitmap words 4 g .. 4 g + 3 of the item (word h:
// triangles 128 g + 32 h + b at bit b), gathered by OR-reductions and stored
// at once.  Compressed meshes (COMP, Section 4.6) decode the twelve index
// fields of a lane from the packed bits, and in strip order only the six
// vertices' 16-bit positions; in a group their grid flag marks as two grid
// rows, only the first two fields (s0, s1) are decoded and the strip check is
// skipped.  The mesh record is read in place in the item's shared-memory
// slot, which stays the warp's until it releases the slot.
template <bool NEAR, bool COMP>
__device__ __forceinline__ void cull_quads(const FrameDev &f, const uint32_t *idx, const FastPair &fp,
                                           const MeshDev &mesh, const s1::Desc &d, uint32_t tpt, int warp, int lane) {
    using namespace s1;
    const bool all_valid = mesh.V > 0xFFFFFFFFull;   // every uint32 index is below V
    const uint32_t v32 = (uint32_t)mesh.V;
    const float *pos = mesh.pos;
    for (uint32_t g = warp; g < 2 * tpt; g += kConsumerWarps) {   // the warp stays converged
        const uint32_t lt = 128 * g + 4 * lane;
        bool cull[4];
        bool valid[4] = {true, true, true, true};
        bool grid = false;
        if constexpr (COMP) {
            // a group flagged as a grid row (k_grid_flags): the lane's first
            // two index fields give the other ten
            const uint64_t G = (d.t0 >> 7) + g;
            grid = mesh.gflag != nullptr && ((__ldg(mesh.gflag + (G >> 5)) >> (G & 31u)) & 1u);
        }
        if (grid) {
            uint32_t bit = 3 * lt * mesh.bits;
            const uint32_t s0 = mesh.imin + (__funnelshift_r(idx[bit >> 5], idx[(bit >> 5) + 1], bit & 31u) & mesh.mask);
            bit += mesh.bits;
            const uint32_t s1 = mesh.imin + (__funnelshift_r(idx[bit >> 5], idx[(bit >> 5) + 1], bit & 31u) & mesh.mask);
            const uint32_t sv[6] = {s0, s1, s0 + 1, s1 + 1, s0 + 2, s1 + 2};
            strip_cull<NEAR, COMP>(fp, mesh, pos, sv, cull);
        } else {
            uint32_t ix[12];
            if constexpr (!COMP) {
                const uint4 *src = reinterpret_cast<const uint4 *>(idx + 3 * lt);
                const uint4 ia = src[0], ib = src[1], ic = src[2];
                ix[0] = ia.x; ix[1] = ia.y; ix[2] = ia.z; ix[3] = ia.w; ix[4] = ib.x; ix[5] = ib.y;
                ix[6] = ib.z; ix[7] = ib.w; ix[8] = ic.x; ix[9] = ic.y; ix[10] = ic.z; ix[11] = ic.w;
            } else {
                // index 3 lt + k of the item sits at bit (3 lt + k) bits of the slot
                uint32_t bit = 3 * lt * mesh.bits;
#pragma unroll
                for (int k = 0; k < 12; ++k, bit += mesh.bits)
                    ix[k] = mesh.imin + (__funnelshift_r(idx[bit >> 5], idx[(bit >> 5) + 1], bit & 31u) & mesh.mask);
            }
            const uint32_t smax = max(max(ix[0], max(ix[1], ix[2])), max(ix[5], max(ix[8], ix[11])));
            const bool strip = (lt + 3 < d.n) & (all_valid | (smax < v32)) & (ix[3] == ix[2]) & (ix[4] == ix[1]) &
                               (ix[6] == ix[2]) & (ix[7] == ix[5]) & (ix[9] == ix[8]) & (ix[10] == ix[5]);
            if (__all_sync(0xffffffffu, strip)) {
                const uint32_t sv[6] = {ix[0], ix[1], ix[2], ix[5], ix[8], ix[11]};
                strip_cull<NEAR, COMP>(fp, mesh, pos, sv, cull);
            } else {
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    valid[u] = lt + u < d.n;
                    if (valid[u] && !all_valid && max(ix[3 * u], max(ix[3 * u + 1], ix[3 * u + 2])) >= v32) {
                        if (f.check) atomicOr(f.err, kErrIndex);
                        valid[u] = false;
                    }
                }
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    Tri9 p[2];
                    if constexpr (COMP) {
                        const uint32_t pix[2][3] = {{ix[6 * h], ix[6 * h + 1], ix[6 * h + 2]},
                                                    {ix[6 * h + 3], ix[6 * h + 4], ix[6 * h + 5]}};
                        const bool pv[2] = {valid[2 * h], valid[2 * h + 1]};
                        decode_pair(mesh, pix, pv, p);
                    } else
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        if (valid[2 * h + u]) {
#pragma unroll
                            for (int c = 0; c < 3; ++c) {
                                const float *q = pos + 3 * (uint64_t)idx[3 * (lt + 2 * h + u) + c];   // (read again)
                                p[u].v[3 * c] = __ldg(q); p[u].v[3 * c + 1] = __ldg(q + 1); p[u].v[3 * c + 2] = __ldg(q + 2);
                            }
                        } else {
#pragma unroll
                            for (int c = 0; c < 9; ++c) p[u].v[c] = 0.0f;
                        }
                    }
                    fast_cull2<NEAR>(fp, p[0], p[1], cull[2 * h], cull[2 * h + 1]);
                }
            }
        }
        uint32_t nib = 0;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const bool live = valid[u] && !cull[u];
            if (f.stats && valid[u] && !live) stat_add(f, kStatIn, 1), stat_add(f, kStatTiny, 1);
            nib |= (uint32_t)live << u;
        }
        const uint32_t sh = nib << (4 * (lane & 7)), h = (uint32_t)lane >> 3;
        uint4 wd;
        wd.x = __reduce_or_sync(0xffffffffu, h == 0 ? sh : 0u);
        wd.y = __reduce_or_sync(0xffffffffu, h == 1 ? sh : 0u);
        wd.z = __reduce_or_sync(0xffffffffu, h == 2 ? sh : 0u);
        wd.w = __reduce_or_sync(0xffffffffu, h == 3 ? sh : 0u);
        // 16-byte aligned: the item's words start at a multiple of 8 tpt
        if (lane == 0) *reinterpret_cast<uint4 *>(f.bits + d.wbase + 4 * g) = wd;
    }
}

// Persistent stage-1 cull kernel, round r of the frame.  Consumers read
// index words from shared memory and position floats from global memory,
// then run the conservative tiny-triangle cull for every pair of the item
// (single-pair items: four consecutive triangles a lane, cull_quads;
// instanced items: two a lane, looped over the pairs).  The warp's
// decisions are stored as words of the survivor bitmap (32 consecutive
// triangles of one pair a word), which k_stage1_exact works through
// afterwards; the cull stays free of the exact path's registers.  The FUSED form (no
// bitmap) queues the survivors per warp and runs the exact path itself,
// 32 at a time.  INST blocks loop over many pairs (Section 4.5, extended to
// several views): a triangle's data is loaded once for all of them.
template <bool INST, bool FUSED, bool COMP, bool NEAR = true>
__global__ void __launch_bounds__(s1::kThreads, (FUSED || INST) ? 3 : s1::kCullBlocks)
    k_stage1(const __grid_constant__ FrameDev f, uint32_t r) {
    static_assert(!(FUSED && COMP), "the fused kernel reads uncompressed meshes only");
    using namespace s1;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Smem<INST, FUSED> &S = *reinterpret_cast<Smem<INST, FUSED> *>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const RoundDev rd = f.rounds[r];
    const int n_segs = (int)f.hdr->n_segs;
    const uint32_t tpt = f.tpt;
    const uint64_t per_item = (uint64_t)kConsumers * tpt;
    const uint32_t G = kConsumerWarps * tpt;          // 32-triangle groups per item

    if (tid == 0) {
        for (int s = 0; s < kSlots; ++s) {
            mbar_init(&S.full[s], 32);                 // the producer warp's lanes
            mbar_init(&S.empty[s], kConsumerWarps);    // one arrival per consumer warp
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (warp == kConsumerWarps) {
        stage1_producer<INST, FUSED, COMP>(f, S, rd, r, n_segs, per_item, G);
        return;
    }

    uint2 *wq = S.wq[FUSED ? warp : 0];
    const unsigned lt_mask = (1u << lane) - 1u;
    int qn = 0;
    for (int j = 0;; ++j) {
        const int slot = j % kSlots;
        if (!mbar_wait(&S.full[slot], (j / kSlots) & 1u)) {
            if (lane == 0) atomicOr(f.err, kErrTimeout);
            return;
        }
        const Desc d = S.desc[slot];
        if (d.b >= rd.b1) break;
        const MeshDev &mesh = S.mesh[slot];   // read in place: the slot is ours until we release it
        const uint32_t *idx = S.idx[slot];
        // index bound as a 32-bit compare: every uint32 index is below V >= 2^32
        const bool all_valid = mesh.V > 0xFFFFFFFFull;
        const uint32_t v32 = (uint32_t)mesh.V;
        const uint32_t np = INST ? d.npairs : 1u;
        if (!FUSED) {
            // NT triangles per lane are loaded together (more loads in flight),
            // then culled for every pair of the item; the pair constants are
            // read from shared memory, which leaves the registers to the loads
            constexpr int NT = kNT;
            constexpr bool comp = COMP;                   // rounds hold one kind of mesh
            if constexpr (!INST) {
                cull_quads<NEAR, COMP>(f, idx, S.fp[slot][0], mesh, d, tpt, warp, lane);
            } else {
                // Instanced items: a lane takes one triangle of each of nv
                // 32-triangle runs a step, the adjacent runs k * 8 + nv * warp
                // + u (the group test wants the step's triangles together);
                // the warp's ballot over run q is bitmap word q of the pair.
                for (uint32_t k = 0; k < tpt; k += NT) {   // uniform trip count: the warp stays converged
                    bool valid[NT];
                    uint32_t ix[NT][3];
#pragma unroll
                    for (int u = 0; u < NT; ++u) {
                        const uint32_t lt = 32 * (k * kConsumerWarps + min((uint32_t)NT, tpt - k) * warp + u) + lane;
                        valid[u] = k + u < tpt && lt < d.n;
                        ix[u][0] = ix[u][1] = ix[u][2] = 0;
                        if (valid[u]) {
                            if (!comp) {
                                ix[u][0] = idx[3 * lt]; ix[u][1] = idx[3 * lt + 1]; ix[u][2] = idx[3 * lt + 2];
                            } else {
#pragma unroll
                                for (int c = 0; c < 3; ++c) {
                                    const uint32_t bit = (3 * lt + c) * mesh.bits;
                                    ix[u][c] = mesh.imin +
                                               (__funnelshift_r(idx[bit >> 5], idx[(bit >> 5) + 1], bit & 31u) & mesh.mask);
                                }
                            }
                            if (max(ix[u][0], max(ix[u][1], ix[u][2])) >= v32 && !all_valid) {
                                if (f.check) atomicOr(f.err, kErrIndex);
                                valid[u] = false;
                            }
                        }
                    }
                    Tri9 p[NT];
                    if (comp) {
                        decode_pair(mesh, ix, valid, p);
                    } else
#pragma unroll
                    for (int u = 0; u < NT; ++u) {
                        if (valid[u]) {
#pragma unroll
                            for (int c = 0; c < 3; ++c) {
                                const float *q = mesh.pos + 3 * (uint64_t)ix[u][c];
                                p[u].v[3 * c] = __ldg(q); p[u].v[3 * c + 1] = __ldg(q + 1); p[u].v[3 * c + 2] = __ldg(q + 2);
                            }
                        } else {
#pragma unroll
                            for (int c = 0; c < 9; ++c) p[u].v[c] = 0.0f;
                        }
                    }
                    static_assert(NT == 2, "the cull evaluates triangles in packed pairs");
                    if (f.group_min != 0 && np >= f.group_min) {
                        const uint32_t nv = min((uint32_t)NT, tpt - k);
                        const uint32_t run0 = k * kConsumerWarps + nv * warp;
                        // Instanced items first test the step's triangles as one
                        // group per pair, one pair a lane; the rejected pairs get
                        // zero words in bulk and only the others run the
                        // per-triangle test.
                        float3 gc, ge;                     // the group's box: centre, half extent
                        {
                            float lo[3], hi[3];
#pragma unroll
                            for (int a = 0; a < 3; ++a) {
                                lo[a] = INFINITY, hi[a] = -INFINITY;
#pragma unroll
                                for (int u = 0; u < NT; ++u)
                                    if (valid[u])
#pragma unroll
                                        for (int c = 0; c < 3; ++c)
                                            lo[a] = fminf(lo[a], p[u].v[3 * c + a]), hi[a] = fmaxf(hi[a], p[u].v[3 * c + a]);
#pragma unroll
                                for (int o = 16; o > 0; o >>= 1) {
                                    lo[a] = fminf(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
                                    hi[a] = fmaxf(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
                                }
                            }
                            gc = make_float3(0.5f * (lo[0] + hi[0]), 0.5f * (lo[1] + hi[1]), 0.5f * (lo[2] + hi[2]));
                            ge = make_float3(fmaxf(hi[0] - gc.x, gc.x - lo[0]), fmaxf(hi[1] - gc.y, gc.y - lo[1]),
                                             fmaxf(hi[2] - gc.z, gc.z - lo[2]));
                        }
                        uint64_t keep = 0;                 // pairs whose group test failed
                        for (uint32_t pb = 0; pb < np; pb += 32) {
                            const uint32_t q = pb + lane;
                            const bool g = q < np && group_cull<NEAR>(S.fp[slot][q < np ? q : 0], gc, ge);
                            keep |= (uint64_t)__ballot_sync(0xffffffffu, q < np && !g) << pb;
                        }
                        for (uint32_t i0 = 0; i0 < 2 * np; i0 += 32) {
                            const uint32_t i = i0 + lane, pi = i >> 1, u = i & 1u;
                            if (i < 2 * np && u < nv && !((keep >> pi) & 1u)) f.bits[d.wbase + pi * G + run0 + u] = 0u;
                        }
                        if (f.stats) {
                            const uint32_t rejected = np - (uint32_t)__popcll(keep);
                            const uint32_t nvalid = (uint32_t)valid[0] + (uint32_t)valid[1];
                            if (rejected && nvalid) stat_add(f, kStatIn, rejected * nvalid), stat_add(f, kStatTiny, rejected * nvalid);
                        }
                        while (keep) {
                            const uint32_t pi = (uint32_t)__ffsll((long long)keep) - 1;
                            keep &= keep - 1;
                            bool cull[NT];
                            fast_cull2<NEAR>(S.fp[slot][pi], p[0], p[1], cull[0], cull[1]);
#pragma unroll
                            for (int u = 0; u < NT; ++u) {
                                const bool live = valid[u] && !cull[u];
                                if (f.stats && valid[u] && !live) stat_add(f, kStatIn, 1), stat_add(f, kStatTiny, 1);
                                const unsigned m = __ballot_sync(0xffffffffu, live);
                                if (u < nv && lane == 0) f.bits[d.wbase + pi * G + run0 + u] = m;
                            }
                        }
                    } else {
                        for (uint32_t pi = 0; pi < np; ++pi) {
                            bool cull[NT];
                            fast_cull2<NEAR>(S.fp[slot][pi], p[0], p[1], cull[0], cull[1]);
#pragma unroll
                            for (int u = 0; u < NT; ++u) {
                                const bool live = valid[u] && !cull[u];
                                if (f.stats && valid[u] && !live) stat_add(f, kStatIn, 1), stat_add(f, kStatTiny, 1);
                                const unsigned m = __ballot_sync(0xffffffffu, live);
                                const uint32_t word = k * kConsumerWarps + min((uint32_t)NT, tpt - k) * warp + u;
                                if (k + u < tpt && lane == 0) f.bits[d.wbase + pi * G + word] = m;
                            }
                        }
                    }
                }
            }
        } else
        for (uint32_t k = 0; k < tpt; ++k) {          // uniform trip count: the warp stays converged
            // three index words from shared memory, nine position floats from
            // global memory; an index >= V skips the triangle (reported when checking)
            const uint32_t lt = k * kConsumers + tid;
            bool valid = lt < d.n;
            uint32_t i0 = 0, i1 = 0, i2 = 0;
            if (valid) {
                i0 = idx[3 * lt]; i1 = idx[3 * lt + 1]; i2 = idx[3 * lt + 2];
                if (i0 >= mesh.V || i1 >= mesh.V || i2 >= mesh.V) {
                    if (f.check) atomicOr(f.err, kErrIndex);
                    valid = false;
                }
            }
            Tri9 p;
            if (valid) {
                const float *q0 = mesh.pos + 3 * (uint64_t)i0, *q1 = mesh.pos + 3 * (uint64_t)i1,
                            *q2 = mesh.pos + 3 * (uint64_t)i2;
                p.v[0] = __ldg(q0); p.v[1] = __ldg(q0 + 1); p.v[2] = __ldg(q0 + 2);
                p.v[3] = __ldg(q1); p.v[4] = __ldg(q1 + 1); p.v[5] = __ldg(q1 + 2);
                p.v[6] = __ldg(q2); p.v[7] = __ldg(q2 + 1); p.v[8] = __ldg(q2 + 2);
            } else {
#pragma unroll
                for (int c = 0; c < 9; ++c) p.v[c] = 0.0f;
            }
            for (uint32_t pi = 0; pi < np; ++pi) {
                const bool live = valid && !fast_cull(S.fp[slot][pi], p);
                if (f.stats && valid && !live) stat_add(f, kStatIn, 1), stat_add(f, kStatTiny, 1);
                const unsigned m = __ballot_sync(0xffffffffu, live);
                if (m) {                               // fused: queue the survivors, run 32 at a time
                    if (f.stats && live) stat_add(f, kStatFast, 1);
                    if (live) wq[qn + __popc(m & lt_mask)] = make_uint2((uint32_t)(d.t0 + lt), d.pair0 + pi);
                    qn += __popc(m);
                    __syncwarp();
                    if (qn >= 32) {
                        qn -= 32;
                        exact_survivor(&f, wq[qn + lane], true);
                        __syncwarp();
                    }
                }
            }
        }
        // the slot is free once every consumer warp is done with it
        __syncwarp();
        if (lane == 0) mbar_arrive(&S.empty[slot]);
    }
    if (FUSED && qn > 0) exact_survivor(&f, wq[lane < qn ? lane : 0], lane < qn);
}

// Stage 1, exact part of round r, from the survivor bitmap of the cull.  A
// warp walks its share of the bitmap 32 words at a time: each lane decodes
// its word to (first triangle, pair) -- the segment is found by a forward
// search from the warp's previous one, since a warp's words only grow --
// and the set bits are compacted into a shared-memory batch of up to
// 32 * kExactK survivors.  A full batch is gathered at once (every lane
// issues the index and position loads of its kExactK survivors before any
// arithmetic), parked in shared memory, and run through the exact path one
// survivor a lane at a time.
__device__ __forceinline__ uint32_t fastdiv(uint32_t n, uint32_t m, uint32_t sh) {   // (fastdiv_consts)
    const uint32_t t = __umulhi(n, m);
    return (t + ((n - t) >> 1)) >> sh;
}

namespace s1 {
constexpr int kExactWarps = 4;
constexpr int kExactBlocks = 5;                      // 96 registers a thread
constexpr int kExactK = 3;                           // survivors a lane gathers together
constexpr int kBatch = 32 * kExactK;
}
template <bool RAY>
__global__ void __launch_bounds__(32 * s1::kExactWarps, s1::kExactBlocks)
    k_stage1_exact(const __grid_constant__ FrameDev f, uint32_t r) {
    using namespace s1;
    __shared__ uint2 buf[kExactWarps][kBatch];
    __shared__ float stage[kExactWarps][kExactK][9][32];   // gathered positions, lane-minor
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const RoundDev rd = f.rounds[r];
    const uint64_t nwords = rd.w1 - rd.w0;
    const int n_segs = (int)f.hdr->n_segs;
    const uint32_t G = kConsumerWarps * f.tpt;
    const uint64_t per_item = (uint64_t)kConsumers * f.tpt;
    const uint64_t nw = (uint64_t)gridDim.x * kExactWarps;
    uint64_t c = (uint64_t)blockIdx.x * kExactWarps + warp;   // the next chunk of 32 words
    uint32_t m_next = 32 * c + lane < nwords ? __ldcs(f.bits + 32 * c + lane) : 0u;
    uint32_t m = 0;                                 // bits of the lane's word not yet batched
    uint64_t t0 = 0;
    uint32_t pair = 0;
    int seg = 0;                                    // segment of the warp's last word so far
    bool more = 32 * c < nwords;
    while (true) {
        int n = 0;                                  // survivors in the batch (warp-uniform)
        while (n < kBatch) {
            if (__ballot_sync(0xffffffffu, m != 0) == 0) {
                if (!more) break;
                m = m_next;                         // advance to chunk c
                const uint64_t gw = rd.w0 + 32 * c + lane;
                const uint64_t cn = c + nw;
                m_next = 32 * cn + lane < nwords ? __ldcs(f.bits + 32 * cn + lane) : 0u;
                if (__ballot_sync(0xffffffffu, m != 0) != 0) {
                    int sl = seg;
                    while (sl + 1 < n_segs && f.segs[sl + 1].word0 <= gw) ++sl;
                    seg = __shfl_sync(0xffffffffu, sl, 31);
                    if (m) {
                        const SegDev &sg = f.segs[sl];
                        const uint64_t local = gw - sg.word0;
                        const uint32_t per = sg.npairs * G;         // words per item (<= 64 * 32)
                        uint64_t jb;
                        uint32_t pi, g;
                        if (sg.npairs == 1 && local < (1ull << 32)) {   // one pair: item and group
                            jb = fastdiv((uint32_t)local, f.g_m, f.g_s);
                            g = (uint32_t)local - (uint32_t)jb * G;
                            pi = 0;
                        } else {
                            jb = local < (1ull << 32) ? (uint64_t)((uint32_t)local / per) : local / per;
                            const uint32_t rem = (uint32_t)(local - jb * per);
                            pi = rem / G;
                            g = rem - pi * G;
                        }
                        t0 = jb * per_item + 32ull * g;
                        pair = sg.pair0 + pi;
                    }
                }
                c = cn;
                more = 32 * c < nwords;
                continue;
            }
            // append the lowest set bits of every lane's word, as many as fit
            const int cnt = __popc(m);
            int incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            const int total = __shfl_sync(0xffffffffu, incl, 31);
            int at = n + incl - cnt;
            while (m && at < kBatch) {
                const int bit = __ffs(m) - 1;
                m &= m - 1u;
                buf[warp][at++] = make_uint2((uint32_t)(t0 + (uint64_t)bit), pair);
            }
            n = min(n + total, kBatch);
        }
        if (n == 0) break;
        __syncwarp();
        if (f.stats && lane == 0) stat_add(f, kStatFast, (unsigned long long)n);
        uint2 e[kExactK];
        bool live[kExactK];
        Tri9 p[kExactK];
#pragma unroll
        for (int u = 0; u < kExactK; ++u) {
            live[u] = lane + 32 * u < n;
            e[u] = buf[warp][live[u] ? lane + 32 * u : 0];
        }
#pragma unroll
        for (int u = 0; u < kExactK; ++u) exact_gather(f, e[u], live[u], p[u]);
        // the positions wait in shared memory, so the exact path of one
        // survivor holds no registers for the others
#pragma unroll
        for (int u = 0; u < kExactK; ++u)
#pragma unroll
            for (int c = 0; c < 9; ++c) stage[warp][u][c][lane] = p[u].v[c];
        __syncwarp();
#pragma unroll 1
        for (int u = 0; u < kExactK; ++u) {
            if (!__any_sync(0xffffffffu, live[u])) continue;
            Tri9 q;
#pragma unroll
            for (int c = 0; c < 9; ++c) q.v[c] = stage[warp][u][c][lane];
            exact_compute<RAY>(f, buf[warp][live[u] ? lane + 32 * u : 0], live[u], q);
        }
    }
}
