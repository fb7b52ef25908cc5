"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package creates geometry, colours, instance transforms and cameras only;
it holds none of the rasterization arithmetic.  Every function takes a
``device`` so the same code produces bit-identical inputs on the CPU (for the
oracle) and on the GPU (for large workloads generated in place).
"""
from .scenes import (  # noqa: F401
    Mesh, Instance, Camera, Scene,
    value_noise, heightfield_mesh, sphere_mesh, ground_mesh,
    look_at, perspective,
    scene_small, scene_unique, camera_unique_pose, scene_billion, camera_billion,
    scene_batched, scene_differentiable, target_colour_noise, scene_room,
    grid_uv, texture_mip_chain, batched_mesh_specs, batched_mesh,
)
