"""Pins of the oracle's software rasterizer of the skinned crowd (the picture
the paper draws through a graphics API, Sec. 4 and Fig. 6; here fixed
rules: positions snapped to 1/256 pixel, 64-bit edge functions, a tie rule
for centres on edges, nearest depth then smallest id).

  * a square of side s pixels split into two triangles covers exactly s*s
    pixel centres, each once (the tie rule gives a shared edge to one side);
  * a hexagon split into a fan of 6 triangles covers each centre inside it
    once and nothing outside it (Pick-style lattice count checked by brute
    force over the pixel grid with exact rational arithmetic);
  * a triangle larger than the image covers every pixel;
  * of two overlapping squares the one with the larger Z (nearer) wins the
    overlap, the other keeps the rest;
  * the character grid places character c at column c % cols, row c // cols.
"""
from fractions import Fraction

import numpy as np

import oracle


def _one(tris, zs=None, width=32, height=32, cols=1, spacing=0.0, scale=1.0, ox=0.0, oy=0.0):
    """Rasterize triangles given in screen-space pixel units (Y measured up
    from oy) as the faces of one character."""
    verts, faces = [], []
    for k, tri in enumerate(tris):
        z = zs[k] if zs is not None else 0.0
        for (x, y) in tri:
            verts.append([x, y, z, 0, 0, 1])
        faces.append([3 * k, 3 * k + 1, 3 * k + 2])
    v = np.array(verts, np.float64)
    return oracle.raster([np.array(faces)], v, [0, len(v)], cols, spacing, ox, oy, scale, width, height,
                         with_cover=True)


def test_square_of_two_triangles_covers_each_centre_once():
    for s, (x0, y0) in ((8, (4.0, -20.0)), (5, (3.25, -9.75)), (11, (0.5, -12.5))):
        a, b, c, d = (x0, y0), (x0 + s, y0), (x0 + s, y0 + s), (x0, y0 + s)
        ids, cover = _one([(a, b, c), (a, c, d)])
        # y is measured up, screen rows go down: oy = 0 maps y0..y0+s to rows -y0-s..-y0
        assert cover.max() == 1
        assert int(cover.sum()) == s * s
        assert (ids != oracle.RASTER_EMPTY).sum() == s * s


def test_hexagon_fan_is_watertight():
    cx, cy, r = 15.3, -14.7, 9.1
    pts = [(cx + r * np.cos(t), cy + r * np.sin(t)) for t in np.linspace(0, 2 * np.pi, 7)[:-1]]
    tris = [((cx, cy), pts[i], pts[(i + 1) % 6]) for i in range(6)]
    ids, cover = _one(tris)
    assert cover.max() == 1
    # brute force: centres strictly inside the (snapped) hexagon
    snap = lambda v: Fraction(round(v * 256), 256)
    poly = [(snap(x), snap(-y)) for x, y in pts]  # screen coordinates (rows go down)
    inside = 0
    for py in range(32):
        for px in range(32):
            p = (Fraction(2 * px + 1, 2), Fraction(2 * py + 1, 2))
            sgn = []
            for i in range(6):
                a, b = poly[i], poly[(i + 1) % 6]
                sgn.append((b[0] - a[0]) * (p[1] - a[1]) - (b[1] - a[1]) * (p[0] - a[0]))
            if all(s > 0 for s in sgn) or all(s < 0 for s in sgn):
                inside += 1
    strict = int(cover.sum())
    # centres exactly on the outline may go either way; none here by construction
    assert strict == inside


def test_triangle_larger_than_the_image_covers_everything():
    ids, cover = _one([((-100.0, 100.0), (300.0, 100.0), (-100.0, -300.0))], width=20, height=13)
    assert (cover == 1).all()
    assert (ids == 0).all()


def test_nearer_square_wins_the_overlap():
    sq = lambda x0, y0, s: [((x0, y0), (x0 + s, y0), (x0 + s, y0 + s)), ((x0, y0), (x0 + s, y0 + s), (x0, y0 + s))]
    tris = sq(2.0, -18.0, 12) + sq(8.0, -24.0, 12)
    ids, cover = _one(tris, zs=[0.0, 0.0, 0.5, 0.5])
    overlap = cover == 2
    assert overlap.sum() == 6 * 6
    assert set(np.unique(ids[overlap]) // 1) <= {2, 3}        # the nearer square's faces
    only_first = (cover == 1) & np.isin(ids, [0, 1])
    assert only_first.sum() == 12 * 12 - 36


def test_character_grid_placement():
    tri = [[0.0, 0.0, 0.0, 0, 0, 1], [4.0, 0.0, 0.0, 0, 0, 1], [0.0, -4.0, 0.0, 0, 0, 1]]
    v = np.array(tri * 4, np.float64)
    faces = [np.array([[0, 1, 2]])] * 4
    ids = oracle.raster(faces, v, [0, 3, 6, 9, 12], cols=2, spacing=10.0, ox=1.0, oy=1.0, scale=1.0,
                        width=24, height=24)
    got = {int(i) // 4096 for i in np.unique(ids) if i != oracle.RASTER_EMPTY}
    assert got == {0, 1, 2, 3}
    # character 3 (column 1, row 1) sits 10 px right of and 10 px below character 0
    c0 = np.argwhere(ids // 4096 == 0)
    c3 = np.argwhere(ids // 4096 == 3)
    assert len(c0) == len(c3) and (c3 - c0 == [10, 10]).all()
