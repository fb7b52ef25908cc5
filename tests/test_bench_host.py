"""Host-side logic of bench.py that runs without a GPU: the choice of the
30-tile frame (1.007 B triangles wholly in view)."""
import numpy as np

import synthetic as S
import bench


def _corners_inside(cam, k, tiles):
    i, j = k % tiles, k // tiles
    V, P = np.asarray(cam.view, np.float64), np.asarray(cam.proj, np.float64)
    pts = [(i + a, y, j + b) for a in (0, 1) for b in (0, 1) for y in (0.0, 0.2)]
    for p in pts:
        h = P @ V @ np.array([*p, 1.0])
        if not (h[3] > 0 and abs(h[0] / h[3]) <= 1 and abs(h[1] / h[3]) <= 1):
            return False
    return True


def test_thirty_tiles_are_wholly_in_view_and_central():
    cam = S.camera_billion(3840, 2160, 8)
    keep = bench.tiles_wholly_in_view(cam, 8)
    assert len(keep) == 30 and len(set(keep)) == 30
    assert all(_corners_inside(cam, k, 8) for k in keep)
    # no tile left out lies wholly in view and nearer the centre than the farthest kept one
    d = lambda k: (k % 8 + 0.5 - 4.0) ** 2 + (k // 8 + 0.5 - 4.0) ** 2
    far = max(d(k) for k in keep)
    for k in range(64):
        if k not in keep and _corners_inside(cam, k, 8):
            assert d(k) >= far
    # 30 tiles of 2 x 4096^2 triangles: the 1.007 B-triangle frame
    assert 30 * 2 * 4096 ** 2 == 1_006_632_960
