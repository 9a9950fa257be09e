"""Exact (float64) pixel coverage of projected triangles by polygon clipping.

Test helper for the oracle pins: the box-filtered pixel integral of a constant
colour triangle is the area of (triangle intersect pixel square); partial
occlusion is handled by clipping one polygon with another convex one.
"""
import numpy as np


def clip(poly, clipper):
    """Sutherland-Hodgman: clip polygon `poly` (list of 2-D points) by the convex
    polygon `clipper` (counter-clockwise or clockwise, consistently)."""
    cl = np.asarray(clipper, np.float64)
    orient = np.sign(area_signed(cl))
    out = [np.asarray(p, np.float64) for p in poly]
    n = len(cl)
    for i in range(n):
        a, b = cl[i], cl[(i + 1) % n]

        def inside(p):
            return orient * ((b[0] - a[0]) * (p[1] - a[1]) - (b[1] - a[1]) * (p[0] - a[0])) >= 0

        def inter(p, q):
            d1 = (b[0] - a[0]) * (p[1] - a[1]) - (b[1] - a[1]) * (p[0] - a[0])
            d2 = (b[0] - a[0]) * (q[1] - a[1]) - (b[1] - a[1]) * (q[0] - a[0])
            t = d1 / (d1 - d2)
            return p + t * (q - p)

        inp = out
        out = []
        if not inp:
            break
        for k in range(len(inp)):
            p, q = inp[k], inp[(k + 1) % len(inp)]
            if inside(q):
                if not inside(p):
                    out.append(inter(p, q))
                out.append(q)
            elif inside(p):
                out.append(inter(p, q))
    return out


def area_signed(poly):
    p = np.asarray(poly, np.float64)
    if len(p) < 3:
        return 0.0
    x, y = p[:, 0], p[:, 1]
    return 0.5 * float(np.dot(x, np.roll(y, -1)) - np.dot(np.roll(x, -1), y))


def area(poly):
    return abs(area_signed(poly))


def project(cam, X):
    """Pinhole projection (float64) of world points with a [20] camera record."""
    R = cam[4:13].astype(np.float64).reshape(3, 3)
    t = cam[13:16].astype(np.float64)
    P = np.asarray(X, np.float64) @ R.T + t
    return np.stack([cam[0] * P[:, 0] / P[:, 2] + cam[2], cam[1] * P[:, 1] / P[:, 2] + cam[3]], 1)


def pixel_square(px, py):
    return [(px, py), (px + 1, py), (px + 1, py + 1), (px, py + 1)]


def coverage(tri2d, H, W):
    out = np.zeros((H, W))
    for py in range(H):
        for px in range(W):
            out[py, px] = area(clip(pixel_square(px, py), tri2d))
    return out


def two_layer_image(front2d, back2d, col_front, col_back, H, W):
    """Exact box-filtered image of a front triangle over a back triangle, black
    elsewhere: I = c_F |F n p| + c_B (|B n p| - |B n F n p|)."""
    img = np.zeros((H, W, 3))
    for py in range(H):
        for px in range(W):
            sq = pixel_square(px, py)
            aF = area(clip(sq, front2d))
            bp = clip(sq, back2d)
            aB = area(bp)
            aBF = area(clip(bp, front2d)) if len(bp) >= 3 else 0.0
            img[py, px] = np.asarray(col_front) * aF + np.asarray(col_back) * (aB - aBF)
    return img
