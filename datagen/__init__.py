"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and bench.py.

This package only generates inputs: oriented points with confidence weights
and the RGB-D views they come from.  It holds none of the reconstruction
arithmetic (no splat, transform, level, marching cubes or texture blend);
the oracle and the CUDA library each implement those on their own.

The paper's captured sequences (Sec. V) are not available; these scenes
stand in for them with the paper's capture geometry: K depth cameras on a
ring (Sec. II-A, V-A: 4 sensors on a ~2.5 m circle), Kinect2-sized depth
maps, raw points back-projected from foreground pixels and normals from an
organised triangulation of the depth map with a depth-step constraint, and
the confidence weights W = W1 * W2 of Sec. III-A.
"""

from .scenes import (  # noqa: F401
    sphere_points,
    ring_cameras,
    human_primitives,
    human_frame,
    frame_config,
    f32_box,
)
