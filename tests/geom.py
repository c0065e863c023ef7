"""Independent geometric helpers for the oracle pins (tests only).

Nothing here calls the oracle or the CUDA path: exact polygon clipping for
box-filtered pixel values, barycentric gradients by matrix inversion, and a
projection written with homogeneous coordinates.  They give the ground truth
the oracle is pinned to.
"""
from __future__ import annotations

import numpy as np


def project_homogeneous(verts, cam):
    """x_s, y_s, zeta through K [R | t] in homogeneous coordinates."""
    R = np.asarray(cam["R"], dtype=np.float64).reshape(3, 3)
    t = np.asarray(cam["t"], dtype=np.float64).reshape(3)
    K = np.array([[float(cam["fx"]), 0.0, float(cam["cx"])], [0.0, float(cam["fy"]), float(cam["cy"])],
                  [0.0, 0.0, 1.0]])
    Xc = np.asarray(verts, dtype=np.float64) @ R.T + t
    h = Xc @ K.T
    return np.stack([h[:, 0] / h[:, 2], h[:, 1] / h[:, 2], 1.0 / Xc[:, 2]], axis=1)


def clip_polygon(poly, a, b, c):
    """Keep the part of convex polygon ``poly`` (list of (x, y)) with a x + b y + c >= 0."""
    out = []
    n = len(poly)
    for i in range(n):
        p, q = poly[i], poly[(i + 1) % n]
        fp = a * p[0] + b * p[1] + c
        fq = a * q[0] + b * q[1] + c
        if fp >= 0:
            out.append(p)
        if (fp >= 0) != (fq >= 0):
            s = fp / (fp - fq)
            out.append((p[0] + s * (q[0] - p[0]), p[1] + s * (q[1] - p[1])))
    return out


def halfplanes_of_triangle(tri):
    """Inward half-planes (a, b, c) of a triangle given as 3 (x, y) points, any winding."""
    (x0, y0), (x1, y1), (x2, y2) = tri
    area2 = (x1 - x0) * (y2 - y0) - (y1 - y0) * (x2 - x0)
    s = 1.0 if area2 > 0 else -1.0
    hp = []
    pts = [(x0, y0), (x1, y1), (x2, y2)]
    for i in range(3):
        (ax, ay), (bx, by) = pts[i], pts[(i + 1) % 3]
        # left of a->b for positive winding
        a = -(by - ay) * s
        b = (bx - ax) * s
        c = -(a * ax + b * ay)
        hp.append((a, b, c))
    return hp


def polygon_area_centroid(poly):
    if len(poly) < 3:
        return 0.0, (0.0, 0.0)
    A = 0.0
    cx = cy = 0.0
    n = len(poly)
    for i in range(n):
        x0, y0 = poly[i]
        x1, y1 = poly[(i + 1) % n]
        cr = x0 * y1 - x1 * y0
        A += cr
        cx += (x0 + x1) * cr
        cy += (y0 + y1) * cr
    A *= 0.5
    if abs(A) < 1e-300:
        return 0.0, (0.0, 0.0)
    return abs(A), (cx / (6 * A), cy / (6 * A))


def box_filtered_flat(tris2d, colours_fn, layers, H, W, bg):
    """Exact box-filtered image of flat-depth triangles in painter's order.

    ``tris2d``: list of 3x2 arrays.  ``layers``: list of triangle indices from
    front to back (no interpenetration).  ``colours_fn(t, x, y)`` gives the
    colour of triangle t at screen point (x, y) and must be affine in (x, y), so
    the integral over a clipped polygon is area x value at its centroid.
    Returns an [H, W] image (one channel).
    """
    img = np.full((H, W), float(bg))
    for y in range(H):
        for x in range(W):
            pix = [(x, y), (x + 1, y), (x + 1, y + 1), (x, y + 1)]
            remaining = [pix]  # parts of the pixel not yet covered (convex pieces)
            acc = 0.0
            covered = 0.0
            for t in layers:
                hp = halfplanes_of_triangle(tris2d[t])
                new_remaining = []
                for piece in remaining:
                    inside = piece
                    for (a, b, c) in hp:
                        inside = clip_polygon(inside, a, b, c)
                        if len(inside) < 3:
                            break
                    A, cen = polygon_area_centroid(inside) if len(inside) >= 3 else (0.0, (0, 0))
                    if A > 0:
                        acc += A * colours_fn(t, cen[0], cen[1])
                        covered += A
                    # outside pieces: split by each half-plane (convex decomposition)
                    rest = piece
                    for (a, b, c) in hp:
                        out = clip_polygon(rest, -a, -b, -c)
                        if len(out) >= 3 and polygon_area_centroid(out)[0] > 0:
                            new_remaining.append(out)
                        rest = clip_polygon(rest, a, b, c)
                        if len(rest) < 3:
                            break
                remaining = new_remaining
            img[y, x] = acc + (1.0 - covered) * bg
    return img


def lambda_gradients(P2):
    """Screen gradients of the barycentric coordinates of a triangle with 2-D vertices ``P2`` [3,2].

    lambda(P) = M^{-1} [P_x, P_y, 1] with M = [[x0 x1 x2], [y0 y1 y2], [1 1 1]].
    Returns (Minv, grad) with grad[i] = (d lambda_i / dP_x, d lambda_i / dP_y).
    """
    M = np.array([[P2[0, 0], P2[1, 0], P2[2, 0]], [P2[0, 1], P2[1, 1], P2[2, 1]], [1.0, 1.0, 1.0]])
    Minv = np.linalg.inv(M)
    return Minv, Minv[:, :2]


def perspective_weights(P3, px, py):
    """Perspective-correct barycentrics of the camera-space point seen at pixel (px, py), by a direct solve.

    ``P3`` [3,3] holds (x_s, y_s, zeta) of the triangle's vertices.  The point sum_i b_i X_i (camera space,
    sum_i b_i = 1) projects to (px, py) iff sum_i b_i Z_i (x_i - px) = 0 and sum_i b_i Z_i (y_i - py) = 0,
    Z_i = 1 / zeta_i: three linear equations in b.  Returns (b [3], depth = sum_i b_i Z_i).
    """
    Z = 1.0 / P3[:, 2]
    A = np.array([Z * (P3[:, 0] - px), Z * (P3[:, 1] - py), np.ones(3)])
    b = np.linalg.solve(A, np.array([0.0, 0.0, 1.0]))
    return b, float(b @ Z)


def projection_jacobian_fd(verts, cam, h=1e-4):
    """d(x_s, y_s, zeta)/d(world position) [V,3,3] by fourth-order central differences of
    ``project_homogeneous`` (row = output, column = world axis)."""
    v = np.asarray(verts, np.float64)
    J = np.zeros((len(v), 3, 3))
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        f = [project_homogeneous(v + k * e, cam) for k in (-2, -1, 1, 2)]
        J[:, :, a] = (f[0] - 8 * f[1] + 8 * f[2] - f[3]) / (12 * h)
    return J
