// internal.h -- launchers the host runtime calls (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>

#include "device.cuh"

namespace curast {

struct LaunchShape {
    int stage1_blocks_per_sm[2][4];   // [instanced][variant: 0 cull, 1 fused, 2 cull of compressed meshes,
                                      //  3 single-pair cull with vertex windows (not instanced)]
    int stage1x_blocks_per_sm;        // exact kernel of stage 1
    int stage2_blocks_per_sm;
    int stage3_blocks_per_sm;
    int stage3t_blocks_per_sm[4];     // binned stage 3 per tile side 2^4 .. 2^7
    int num_sms;
};

cudaError_t query_launch_shape(LaunchShape *out, int device);

cudaError_t launch_clear(uint64_t *vis, uint64_t n, cudaStream_t s);
// Stage 1 of round r: the cull kernel (fused: it runs the exact path itself
// and needs no bitmap), then the exact kernel over the round's bitmap.
// near = false launches the cull (not the fused form) without its near-plane
// test (valid when no pair's mesh bounds reach the near plane).
cudaError_t launch_stage1(const FrameDev &f, bool instanced, int variant, uint32_t r, int blocks, bool near,
                          cudaStream_t s);
cudaError_t launch_stage1_exact(const FrameDev &f, uint32_t r, int blocks, cudaStream_t s);
cudaError_t launch_stage2(const FrameDev &f, int blocks, cudaStream_t s);
cudaError_t launch_stage3(const FrameDev &f, int blocks, cudaStream_t s);
// Binned stage 3: scan of the per-tile part counts, scatter of the parts into
// tile order, then one block per tile with the tile's words in shared memory.
cudaError_t launch_stage3_binned(const FrameDev &f, int scatter_blocks, int tile_blocks, cudaStream_t s);
// scratch: 256 * 6 floats; out6: xmin ymin zmin xmax ymax zmax
cudaError_t launch_aabb(const float *pos, uint64_t V, float *scratch, float *out6, cudaStream_t s);
// Section 4.6 encoding (compress.cu)
cudaError_t launch_minmax_u32(const uint32_t *v, uint64_t n, unsigned *out2, cudaStream_t s);
cudaError_t launch_pack_indices(const uint32_t *idx, uint64_t n, uint32_t imin, uint32_t bits, uint32_t *words,
                                uint64_t nwords, cudaStream_t s);
// grid flags of the 128-triangle groups of a mesh: ceil(ceil(T / 128) / 32) words
cudaError_t launch_grid_flags(const uint32_t *idx, uint64_t T, uint64_t V, uint32_t *flags, uint64_t nwords,
                              cudaStream_t s);
cudaError_t launch_quantize_positions(const float *pos, uint64_t V, const double lo[3], const double size[3],
                                      uint16_t *q, cudaStream_t s);
cudaError_t launch_count_diff(const uint64_t *a, const uint64_t *b, uint64_t n, unsigned long long *out,
                              cudaStream_t s);

struct ShadeArgs {
    const uint64_t *vis;
    int W, H;
    float fx, fy;
    const float *inst_mv;       // n_inst x 12
    const uint64_t *base;       // n_inst + 1
    const uint32_t *inst_mesh;  // n_inst
    const MeshDev *meshes;
    int n_inst;
    // resolve
    float *rgba_f32;
    uint8_t *rgba8;
    int ss;                     // super-sampled resolve: samples per pixel axis
    uint8_t *level;             // textured resolve: the mip level per pixel (255: none), or null
    // interpolate
    uint32_t mesh;
    const float *pos;           // overrides the mesh's positions when non-null
    const float *attr;
    int C;
    float *out;
    const float *grad_out;
    float *grad_attr;
    float *grad_pos;
};

cudaError_t launch_resolve(const ShadeArgs &a, cudaStream_t s);
// a.W, a.H: the super-sampled buffer (ss W x ss H); W, H: the output
cudaError_t launch_resolve_ss(const ShadeArgs &a, int W, int H, cudaStream_t s);
// resolve with textures and the 4-ray mip-level choice (Section 4.4)
cudaError_t launch_resolve_textured(const ShadeArgs &a, cudaStream_t s);
cudaError_t launch_interpolate(const ShadeArgs &a, cudaStream_t s);
cudaError_t launch_interpolate_backward(const ShadeArgs &a, cudaStream_t s);

}  // namespace curast
