"""Seeded synthetic inputs: meshes, cameras, textures, upstream gradients.

This module holds no arithmetic of the rasterizer-gradient method.  It only
draws the scenes that both the CUDA path and the FP64 oracle consume, so the
two can share it without sharing any of the method.  Every array is generated
from an explicit seed with numpy's PCG64 generator, which gives the same
numbers on every machine.

Workload shapes follow the paper's head-reconstruction and multi-view fitting
settings (Sec. 6, Supp. B.1-B.2): closed sphere-like meshes of up to ~130k
triangles, 1024^2 textures, many cameras on a sphere around the object.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# ---------------------------------------------------------------------------
# cameras
# ---------------------------------------------------------------------------

CAMERA_DTYPE = np.dtype([("R", "<f8", (9,)), ("t", "<f8", (3,)), ("fx", "<f8"), ("fy", "<f8"),
                         ("cx", "<f8"), ("cy", "<f8"), ("znear", "<f8")])
"""Packed camera record (136 bytes), identical in layout to ``mer_camera``.

OpenCV convention: camera +X right, +Y down, +Z forward.  A world point X_w maps
to X_c = R X_w + t, then x_s = fx X_c/Z_c + cx, y_s = fy Y_c/Z_c + cy.
"""


def look_at_camera(eye, H: int, W: int, fov_deg: float = 45.0, znear: float = 0.1,
                   target=(0.0, 0.0, 0.0), up=(0.0, 1.0, 0.0)) -> np.ndarray:
    """Pinhole camera at ``eye`` looking at ``target`` with vertical field of view ``fov_deg``."""
    eye = np.asarray(eye, dtype=np.float64)
    f = np.asarray(target, dtype=np.float64) - eye
    f /= np.linalg.norm(f)
    r = np.cross(f, np.asarray(up, dtype=np.float64))
    nr = np.linalg.norm(r)
    if nr < 1e-12:  # looking straight along the up axis: pick another up vector
        r = np.cross(f, np.array([0.0, 0.0, 1.0]))
        nr = np.linalg.norm(r)
    r /= nr
    d = np.cross(f, r)
    R = np.stack([r, d, f])
    cam = np.zeros((), dtype=CAMERA_DTYPE)
    cam["R"] = R.reshape(9)
    cam["t"] = -R @ eye
    foc = (H / 2.0) / math.tan(math.radians(fov_deg) / 2.0)
    cam["fx"] = foc
    cam["fy"] = foc
    cam["cx"] = W / 2.0
    cam["cy"] = H / 2.0
    cam["znear"] = znear
    return cam


def cameras_on_sphere(n: int, radius: float, H: int, W: int, seed: int, fov_deg: float = 45.0,
                      elev_deg: float = 60.0) -> np.ndarray:
    """``n`` cameras at distance ``radius``; azimuth U[0, 2pi), elevation U[-elev, elev]."""
    rng = np.random.default_rng(seed)
    az = rng.uniform(0.0, 2.0 * math.pi, n)
    el = np.radians(rng.uniform(-elev_deg, elev_deg, n))
    cams = np.zeros(n, dtype=CAMERA_DTYPE)
    for i in range(n):
        eye = radius * np.array([math.cos(el[i]) * math.sin(az[i]), math.sin(el[i]),
                                 math.cos(el[i]) * math.cos(az[i])])
        cams[i] = look_at_camera(eye, H, W, fov_deg)
    return cams


def random_direction_camera(radius: float, H: int, W: int, rng: np.random.Generator,
                            fov_deg: float = 45.0) -> np.ndarray:
    v = rng.normal(size=3)
    v /= np.linalg.norm(v)
    return look_at_camera(radius * v, H, W, fov_deg)


# ---------------------------------------------------------------------------
# meshes
# ---------------------------------------------------------------------------

def icosphere(subdiv: int) -> tuple[np.ndarray, np.ndarray]:
    """Unit icosphere; ``subdiv`` midpoint subdivisions (3 -> 642 V / 1280 T, 5 -> 10242 V / 20480 T).

    Faces are wound counter-clockwise seen from outside.
    """
    p = (1.0 + math.sqrt(5.0)) / 2.0
    v = np.array([[-1, p, 0], [1, p, 0], [-1, -p, 0], [1, -p, 0], [0, -1, p], [0, 1, p],
                  [0, -1, -p], [0, 1, -p], [p, 0, -1], [p, 0, 1], [-p, 0, -1], [-p, 0, 1]],
                 dtype=np.float64)
    f = np.array([[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11], [1, 5, 9], [5, 11, 4],
                  [11, 10, 2], [10, 7, 6], [7, 1, 8], [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8],
                  [3, 8, 9], [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]], dtype=np.int64)
    verts = [tuple(x) for x in v / np.linalg.norm(v, axis=1, keepdims=True)]
    faces = f
    for _ in range(subdiv):
        cache: dict[tuple[int, int], int] = {}

        def mid(a: int, b: int) -> int:
            key = (a, b) if a < b else (b, a)
            idx = cache.get(key)
            if idx is None:
                m = (np.asarray(verts[a]) + np.asarray(verts[b])) / 2.0
                m /= np.linalg.norm(m)
                verts.append(tuple(m))
                idx = len(verts) - 1
                cache[key] = idx
            return idx

        nf = []
        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [[a, ab, ca], [b, bc, ab], [c, ca, bc], [ab, bc, ca]]
        faces = np.array(nf, dtype=np.int64)
    V = np.array(verts, dtype=np.float64)
    return _orient_outward(V, faces.astype(np.int32))


def octasphere(n: int) -> tuple[np.ndarray, np.ndarray]:
    """Geodesic sphere from an octahedron of frequency ``n``: 4n^2+2 vertices, 8n^2 triangles.

    Lattice points (i, j, k) with |i|+|j|+|k| = n on the octahedron surface are
    projected to the unit sphere; n = 128 gives 65,538 V / 131,072 T.
    """
    pts = []
    tris = []
    key_to_idx: dict[tuple[int, int, int], int] = {}

    def vid(key):
        idx = key_to_idx.get(key)
        if idx is None:
            idx = len(pts)
            key_to_idx[key] = idx
            pts.append(key)
        return idx

    # per octant, a triangular lattice indexed by (i, j) with k = n - i - j
    ii, jj = np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="ij")
    mask = ii + jj <= n
    ii, jj = ii[mask], jj[mask]
    for sx in (1, -1):
        for sy in (1, -1):
            for sz in (1, -1):
                loc = {}
                for a, b in zip(ii.tolist(), jj.tolist()):
                    c = n - a - b
                    key = (sx * a if a else 0, sy * b if b else 0, sz * c if c else 0)
                    loc[(a, b)] = vid(key)
                for a in range(n):
                    for b in range(n - a):
                        tris.append((loc[(a, b)], loc[(a + 1, b)], loc[(a, b + 1)]))
                        if a + b <= n - 2:
                            tris.append((loc[(a + 1, b)], loc[(a + 1, b + 1)], loc[(a, b + 1)]))
    P = np.array(pts, dtype=np.float64)
    P /= np.linalg.norm(P, axis=1, keepdims=True)
    return _orient_outward(P, np.array(tris, dtype=np.int32))


def _orient_outward(V: np.ndarray, F: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Flip faces so their (v1-v0)x(v2-v0) normal points away from the origin."""
    a, b, c = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    nrm = np.cross(b - a, c - a)
    flip = (nrm * (a + b + c)).sum(axis=1) < 0
    F = F.copy()
    F[flip, 1], F[flip, 2] = F[flip, 2].copy(), F[flip, 1].copy()
    return V, F


def random_radial_field(P: np.ndarray, seed: int, degree: int = 4) -> np.ndarray:
    """Random smooth function on the unit sphere, max |s| = 1 over the given points.

    It is a random polynomial of total degree <= ``degree`` in (x, y, z) restricted
    to the sphere, which spans the same space as the real spherical harmonics of
    degree <= ``degree``.
    """
    rng = np.random.default_rng(seed)
    s = np.zeros(len(P))
    for a in range(degree + 1):
        for b in range(degree + 1 - a):
            for c in range(degree + 1 - a - b):
                s += rng.normal() * P[:, 0] ** a * P[:, 1] ** b * P[:, 2] ** c
    s -= s.mean()
    return s / np.abs(s).max()


def displaced_sphere(n: int, seed: int, amp: float = 0.1, noise: float = 0.005):
    """Octasphere of frequency ``n``, radius 1 + amp*s(theta, phi) + N(0, noise) per vertex."""
    P, F = octasphere(n)
    s = random_radial_field(P, seed)
    rng = np.random.default_rng(seed + 7919)
    r = 1.0 + amp * s + rng.normal(0.0, noise, len(P))
    return P * r[:, None], F, P


def equirect_uv(P: np.ndarray) -> np.ndarray:
    """Per-vertex (u, v) = (phi / 2pi, theta / pi) of unit directions ``P`` (y up)."""
    phi = np.arctan2(P[:, 2], P[:, 0])
    u = (phi / (2.0 * math.pi)) % 1.0
    v = np.arccos(np.clip(P[:, 1], -1.0, 1.0)) / math.pi
    return np.stack([u, v], axis=1)


def vertex_normals(V: np.ndarray, F: np.ndarray) -> np.ndarray:
    """Area-weighted, normalised per-vertex normals (an attribute, not part of the method)."""
    a, b, c = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    fn = np.cross(b - a, c - a)
    vn = np.zeros_like(V)
    for k in range(3):
        np.add.at(vn, F[:, k], fn)
    return vn / np.maximum(np.linalg.norm(vn, axis=1, keepdims=True), 1e-30)


def padded_rgba(tex: np.ndarray) -> np.ndarray:
    """[H, W, 3] -> [H, W, 4] with a zero fourth channel: texels 16 bytes apart, for 128-bit loads."""
    out = np.zeros(tex.shape[:2] + (4,), np.float32)
    out[..., : tex.shape[2]] = tex
    return out


def noise_texture(size: int, channels: int, seed: int, sigma: float = 4.0) -> np.ndarray:
    """Uniform noise blurred by a wrapping Gaussian of ``sigma`` texels, rescaled to [0, 1] per channel."""
    rng = np.random.default_rng(seed)
    t = rng.uniform(0.0, 1.0, (size, size, channels))
    k = np.fft.fftfreq(size)
    g = np.exp(-2.0 * (math.pi * sigma) ** 2 * (k[:, None] ** 2 + k[None, :] ** 2))
    out = np.empty_like(t)
    for c in range(channels):
        out[..., c] = np.real(np.fft.ifft2(np.fft.fft2(t[..., c]) * g))
    lo = out.min(axis=(0, 1), keepdims=True)
    hi = out.max(axis=(0, 1), keepdims=True)
    return ((out - lo) / np.maximum(hi - lo, 1e-12)).astype(np.float32)


# ---------------------------------------------------------------------------
# shading programs: which channels the image holds (see ``mer_shading``)
# ---------------------------------------------------------------------------

@dataclass
class Shading:
    """Layout of the shaded image that is passed through the edge-gradient step.

    Channels [0, n_main) hold interpolated attributes (``uv_offset < 0``) or the
    bilinear texture sampled at the interpolated (u, v) = attribute channels
    ``uv_offset, uv_offset + 1``.  ``mask_ch`` / ``depth_ch`` hold the coverage
    mask and the depth Z, ``backface_ch`` the back-face image (1 where the visible
    triangle faces away from the camera), or are -1.  Background pixels take ``bg``.
    """
    n_main: int
    C: int
    uv_offset: int = -1
    mask_ch: int = -1
    depth_ch: int = -1
    bg: list = field(default_factory=list)
    backface_ch: int = -1

    def bg_array(self) -> np.ndarray:
        b = np.zeros(self.C, dtype=np.float32)
        b[: len(self.bg)] = self.bg
        return b


@dataclass
class Scene:
    name: str
    verts: np.ndarray          # [V,3] float32 world positions
    tris: np.ndarray           # [T,3] int32
    cams: np.ndarray           # [n] CAMERA_DTYPE
    H: int
    W: int
    attr: np.ndarray           # [V,C_a] float32
    shading: Shading
    tex: np.ndarray | None = None   # [TH,TW,tex_c >= n_main] float32
    upstream_seed: int = 0
    target_verts: np.ndarray | None = None

    @property
    def n_views(self) -> int:
        return len(self.cams)

    @property
    def pixels(self) -> int:
        return self.n_views * self.H * self.W

    def upstream(self, kind: str = "normal") -> np.ndarray:
        """Upstream image gradient dL/dI [n,H,W,C] float32, N(0,1) from the scene's seed."""
        rng = np.random.default_rng(self.upstream_seed)
        return rng.standard_normal((self.n_views, self.H, self.W, self.shading.C), dtype=np.float32)


# ---------------------------------------------------------------------------
# the five workloads (tiny, intersection, head-scale, multi-view, uneven batch)
# ---------------------------------------------------------------------------

def tiny_icosphere(H: int = 128, W: int = 128) -> Scene:
    """Icosphere (subdivision 3, 642 V / 1280 T), jitter N(0,0.02) seed 0, camera at distance 3, 45 deg.

    Per-vertex RGB ~ U[0,1] (seed 1), background 0.5.  ``target_verts`` is the base
    icosphere jittered by N(0, 0.05) with seed 2 (an L2 loss target).
    """
    P, F = icosphere(3)
    v = P + np.random.default_rng(0).normal(0.0, 0.02, P.shape)
    tgt = P + np.random.default_rng(2).normal(0.0, 0.05, P.shape)
    rgb = np.random.default_rng(1).uniform(0.0, 1.0, (len(P), 3)).astype(np.float32)
    cams = np.stack([look_at_camera((0.0, 0.0, 3.0), H, W)])
    sh = Shading(n_main=3, C=3, bg=[0.5, 0.5, 0.5])
    return Scene("tiny_icosphere_128", v.astype(np.float32), F, cams, H, W, rgb, sh,
                 upstream_seed=3, target_verts=tgt.astype(np.float32))


def two_spheres(H: int = 512, W: int = 512, subdiv: int = 5) -> Scene:
    """Two interpenetrating icospheres (subdivision 5 each), centres +-0.3(1,1,1)/sqrt3.

    Image channels: interpolated vertex normals (3), mask, depth.  Upstream N(0,1) seed 3.
    """
    P, F = icosphere(subdiv)
    off = 0.3 * np.ones(3) / math.sqrt(3.0)
    V = np.concatenate([P + off, P - off])
    T = np.concatenate([F, F + len(P)]).astype(np.int32)
    nrm = vertex_normals(V, T).astype(np.float32)
    cams = np.stack([look_at_camera((0.0, 0.0, 4.5), H, W)])
    sh = Shading(n_main=3, C=5, mask_ch=3, depth_ch=4, bg=[0, 0, 0, 0, 0])
    return Scene(f"two_spheres_{H}", V.astype(np.float32), T, cams, H, W, nrm, sh, upstream_seed=3)


def open_sphere(H: int = 256, W: int = 256, subdiv: int = 4, cap: float = 0.55) -> Scene:
    """Icosphere (subdivision 4) with the cap of triangles whose centroid has z > ``cap`` removed, seen through
    the hole from (0.9, 0.6, 2.6): the inner surface shows its back faces.

    Image channels: interpolated vertex normals (3), back-face image, mask.  Upstream N(0,1) seed 5.
    """
    P, F = icosphere(subdiv)
    keep = P[F].mean(axis=1)[:, 2] <= cap
    used = np.unique(F[keep])
    remap = -np.ones(len(P), np.int64)
    remap[used] = np.arange(len(used))
    V = P[used]
    T = remap[F[keep]].astype(np.int32)
    nrm = vertex_normals(V, T).astype(np.float32)
    cams = np.stack([look_at_camera((0.9, 0.6, 2.6), H, W)])
    sh = Shading(n_main=3, C=5, backface_ch=3, mask_ch=4, bg=[0, 0, 0, 0, 0])
    return Scene(f"open_sphere_{H}", V.astype(np.float32), T, cams, H, W, nrm, sh, upstream_seed=5)


def head_mesh(n: int = 128, seed: int = 4):
    """Displaced closed sphere standing in for a head: n=128 -> 65,538 V / 131,072 T."""
    V, F, P = displaced_sphere(n, seed)
    uv = equirect_uv(P).astype(np.float32)
    return V.astype(np.float32), F, uv


def head_single_view(H: int = 1024, W: int = 1024, n: int = 128, tex_size: int = 1024) -> Scene:
    """Head-scale single view: textured displaced sphere, RGB + mask, camera at distance 3."""
    V, F, uv = head_mesh(n)
    tex = padded_rgba(noise_texture(tex_size, 3, seed=5))
    cams = np.stack([look_at_camera((0.0, 0.0, 3.0), H, W)])
    sh = Shading(n_main=3, C=4, uv_offset=0, mask_ch=3, bg=[0, 0, 0, 0])
    return Scene(f"head_{H}x{W}", V, F, cams, H, W, uv, sh, tex=tex, upstream_seed=10)


def head_multiview(n_views: int = 32, H: int = 2048, W: int = 1334, n: int = 128,
                   tex_size: int = 1024, seed: int = 6) -> Scene:
    """Multi-view head: the head mesh seen by ``n_views`` cameras at radius 3, RGB + mask + depth."""
    V, F, uv = head_mesh(n)
    tex = padded_rgba(noise_texture(tex_size, 3, seed=5))
    cams = cameras_on_sphere(n_views, 3.0, H, W, seed)
    sh = Shading(n_main=3, C=5, uv_offset=0, mask_ch=3, depth_ch=4, bg=[0, 0, 0, 0, 0])
    return Scene(f"head_{n_views}x{W}x{H}", V, F, cams, H, W, uv, sh, tex=tex, upstream_seed=7)


def uneven_plan(n_items: int = 256, seed: int = 8, res_seed: int = 9, t_min: float = 500.0,
                t_max: float = 200000.0, resolutions=(128, 256, 512, 1024)):
    """Sizes of the uneven batch without building it: per item the octasphere frequency n_i (T = 8 n_i^2) and
    the square resolution."""
    rng = np.random.default_rng(seed)
    T = np.exp(rng.uniform(math.log(t_min), math.log(t_max), n_items))
    rres = np.random.default_rng(res_seed)
    res = rres.choice(list(resolutions), n_items)
    n = [max(8, int(round(math.sqrt(T[i] / 8.0)))) for i in range(n_items)]
    return n, [int(r) for r in res]


def uneven_batch(n_items: int = 256, seed: int = 8, res_seed: int = 9,
                 t_min: float = 500.0, t_max: float = 200000.0, resolutions=(128, 256, 512, 1024), subset=None):
    """Uneven batch: ``n_items`` displaced spheres, T log-uniform in [t_min, t_max], res in {128..1024}^2.

    Returns a list of Scenes (one camera each); item i is displaced with seed 1000+i.  ``subset``: build only
    these item indices (a rank's share), in the order given.
    Channels: normal (3) + mask.
    """
    nis, res = uneven_plan(n_items, seed, res_seed, t_min, t_max, resolutions)
    out = []
    for i in (range(n_items) if subset is None else subset):
        ni = nis[i]
        V, F, P = displaced_sphere(ni, 1000 + i)
        cam = random_direction_camera(3.0, int(res[i]), int(res[i]), np.random.default_rng(2000 + i))
        nrm = vertex_normals(V, F).astype(np.float32)
        sh = Shading(n_main=3, C=4, mask_ch=3, bg=[0, 0, 0, 0])
        out.append(Scene(f"item{i}", V.astype(np.float32), F, np.stack([cam]), int(res[i]), int(res[i]),
                         nrm, sh, upstream_seed=3000 + i))
    return out
