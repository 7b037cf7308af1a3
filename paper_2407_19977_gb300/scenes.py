"""Seeded synthetic scene generators.

These build the inputs that both the CUDA path and the CPU oracle consume:
triangle meshes, per-triangle material ids, OpenPBR parameter tables, quad
lights, a lat-long environment map and a camera.  They stand in for the
paper's proprietary CAD pushbutton models (Appendix A, Table 1 and Table 2)
and hold none of the path tracer's arithmetic: no ray, BSDF or light-transport
code lives here, only geometry, parameter tables and a sky image.

Every generator takes a seed and draws from numpy's Philox bit generator, so
the same seed always gives the same arrays on every machine.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# OpenPBR parameter layout shared by the C-ABI (`pt_openpbr`) and the oracle:
# 34 float32 values per material, in this order.
MATERIAL_FIELDS = (
    "base_weight", "base_color_r", "base_color_g", "base_color_b",
    "base_metalness", "base_diffuse_roughness",
    "specular_weight", "specular_color_r", "specular_color_g", "specular_color_b",
    "specular_roughness", "specular_ior",
    "transmission_weight", "transmission_color_r", "transmission_color_g", "transmission_color_b",
    "coat_weight", "coat_color_r", "coat_color_g", "coat_color_b",
    "coat_roughness", "coat_ior",
    "emission_luminance", "emission_color_r", "emission_color_g", "emission_color_b",
    "geometry_thin_walled", "specular_roughness_anisotropy", "specular_rotation",
    "fuzz_weight", "fuzz_color_r", "fuzz_color_g", "fuzz_color_b", "fuzz_roughness",
)
N_MATERIAL_FLOATS = len(MATERIAL_FIELDS)  # 34
# Quad light layout: p0[3], e1[3], e2[3], radiance[3], two_sided (0/1).
N_LIGHT_FLOATS = 13


def openpbr(base_weight=1.0, base_color=(0.8, 0.8, 0.8), base_metalness=0.0,
            base_diffuse_roughness=0.0, specular_weight=1.0, specular_color=(1.0, 1.0, 1.0),
            specular_roughness=0.3, specular_ior=1.5, transmission_weight=0.0,
            transmission_color=(1.0, 1.0, 1.0), coat_weight=0.0, coat_color=(1.0, 1.0, 1.0),
            coat_roughness=0.0, coat_ior=1.6, emission_luminance=0.0,
            emission_color=(1.0, 1.0, 1.0), geometry_thin_walled=0.0,
            specular_roughness_anisotropy=0.0, specular_rotation=0.0, fuzz_weight=0.0,
            fuzz_color=(1.0, 1.0, 1.0), fuzz_roughness=0.5) -> np.ndarray:
    """One OpenPBR parameter row (defaults follow the OpenPBR surface defaults, Sec. 4)."""
    v = [base_weight, *base_color, base_metalness, base_diffuse_roughness,
         specular_weight, *specular_color, specular_roughness, specular_ior,
         transmission_weight, *transmission_color,
         coat_weight, *coat_color, coat_roughness, coat_ior,
         emission_luminance, *emission_color, geometry_thin_walled,
         specular_roughness_anisotropy, specular_rotation, fuzz_weight, *fuzz_color, fuzz_roughness]
    assert len(v) == N_MATERIAL_FLOATS
    return np.asarray(v, dtype=np.float32)


def diffuse(color) -> np.ndarray:
    """Pure Lambertian base: the specular layer is switched off."""
    return openpbr(base_color=color, specular_weight=0.0)


def quad_light(p0, e1, e2, radiance, two_sided=False) -> np.ndarray:
    return np.asarray([*p0, *e1, *e2, *radiance, 1.0 if two_sided else 0.0], dtype=np.float32)


@dataclass
class Camera:
    origin: tuple
    target: tuple
    up: tuple
    vfov_deg: float
    width: int
    height: int
    lens_radius: float = 0.0      # thin lens; 0 = pinhole
    focus_distance: float = 1.0   # distance of the plane of focus along the view direction


@dataclass
class Scene:
    name: str
    vertices: np.ndarray          # (nv, 3) float32
    indices: np.ndarray           # (nt, 3) uint32
    material_ids: np.ndarray      # (nt,) uint32
    materials: np.ndarray         # (nm, 34) float32
    lights: np.ndarray            # (nq, 13) float32
    env: np.ndarray | None        # (H, W, 3) float32, row 0 = straight up (+y)
    camera: Camera
    spp: int
    max_depth: int
    meta: dict = field(default_factory=dict)

    @property
    def n_triangles(self) -> int:
        return int(self.indices.shape[0])

    def with_camera(self, **kw) -> "Scene":
        cam = Camera(**{**self.camera.__dict__, **kw})
        return Scene(self.name, self.vertices, self.indices, self.material_ids, self.materials,
                     self.lights, self.env, cam, self.spp, self.max_depth, dict(self.meta))


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(int(seed)))


# --------------------------------------------------------------------------------------------
# Mesh helpers
# --------------------------------------------------------------------------------------------

def _box_mesh(center, size, rot_y):
    """Closed box (12 triangles, outward counter-clockwise winding), rotated about +y."""
    sx, sy, sz = size
    c = np.asarray(center, dtype=np.float64)
    corners = np.array([[x, y, z] for x in (-0.5, 0.5) for y in (-0.5, 0.5) for z in (-0.5, 0.5)])
    corners *= np.array([sx, sy, sz])
    ca, sa = math.cos(rot_y), math.sin(rot_y)
    rot = np.array([[ca, 0.0, sa], [0.0, 1.0, 0.0], [-sa, 0.0, ca]])
    v = corners @ rot.T + c
    # vertex index = 4*ix + 2*iy + iz
    faces = [
        (0, 1, 3, 2),  # x = -0.5
        (4, 6, 7, 5),  # x = +0.5
        (0, 4, 5, 1),  # y = -0.5
        (2, 3, 7, 6),  # y = +0.5
        (0, 2, 6, 4),  # z = -0.5
        (1, 5, 7, 3),  # z = +0.5
    ]
    tris = []
    for a, b, cc, d in faces:
        tris.append((a, b, cc))
        tris.append((a, cc, d))
    return v, np.asarray(tris, dtype=np.int64)


def _fix_winding_outward(v, tris, center):
    """Flip triangles whose normal points towards `center` (convex solids only)."""
    p0, p1, p2 = v[tris[:, 0]], v[tris[:, 1]], v[tris[:, 2]]
    n = np.cross(p1 - p0, p2 - p0)
    c = (p0 + p1 + p2) / 3.0 - np.asarray(center)
    flip = np.einsum("ij,ij->i", n, c) < 0
    tris = tris.copy()
    tris[flip] = tris[flip][:, [0, 2, 1]]
    return tris


def _grid_plane(x0, x1, z0, z1, nx, nz, y=0.0):
    """Plane y = const facing +y, split into nx*nz quads (2*nx*nz triangles)."""
    xs = np.linspace(x0, x1, nx + 1)
    zs = np.linspace(z0, z1, nz + 1)
    X, Z = np.meshgrid(xs, zs, indexing="ij")
    v = np.stack([X.ravel(), np.full(X.size, y), Z.ravel()], axis=1)
    idx = np.arange((nx + 1) * (nz + 1)).reshape(nx + 1, nz + 1)
    a = idx[:-1, :-1].ravel()
    b = idx[1:, :-1].ravel()
    c = idx[1:, 1:].ravel()
    d = idx[:-1, 1:].ravel()
    # (a, d, c) has normal +y for x along i, z along j
    t1 = np.stack([a, d, c], axis=1)
    t2 = np.stack([a, c, b], axis=1)
    return v, np.concatenate([t1, t2], axis=0)


class _MeshBuilder:
    def __init__(self):
        self.v, self.t, self.m = [], [], []
        self.nv = 0

    def add(self, v, tris, mat):
        v = np.asarray(v, dtype=np.float64)
        tris = np.asarray(tris, dtype=np.int64)
        self.v.append(v)
        self.t.append(tris + self.nv)
        mat = np.broadcast_to(np.asarray(mat, dtype=np.int64), (tris.shape[0],))
        self.m.append(np.array(mat))
        self.nv += v.shape[0]

    def arrays(self):
        v = np.concatenate(self.v).astype(np.float32)
        t = np.concatenate(self.t).astype(np.uint32)
        m = np.concatenate(self.m).astype(np.uint32)
        return v, t, m


def _frame_camera(lo, hi, direction, vfov_deg, width, height, margin=1.15):
    """3/4 view that fits the bounding sphere of the box [lo, hi] into the vertical FOV."""
    lo, hi = np.asarray(lo, float), np.asarray(hi, float)
    center = 0.5 * (lo + hi)
    radius = 0.5 * float(np.linalg.norm(hi - lo))
    d = np.asarray(direction, float)
    d /= np.linalg.norm(d)
    half = math.radians(vfov_deg) * 0.5
    if width < height:
        half = math.atan(math.tan(half) * width / height)
    dist = margin * radius / math.sin(half)
    origin = center + dist * d
    return Camera(tuple(map(float, origin)), tuple(map(float, center)), (0.0, 1.0, 0.0),
                  float(vfov_deg), int(width), int(height))


# --------------------------------------------------------------------------------------------
# Environment map: procedural analytic sky (own closed form, not a published sky model)
# --------------------------------------------------------------------------------------------

def analytic_sky(width=512, height=256, seed=0) -> np.ndarray:
    """Lat-long RGB float32 sky: zenith/horizon gradient, darker ground, and a sun lobe.

    Row y covers polar angle [y, y+1) * pi / height measured from +y; column x covers
    azimuth phi = ((x + 0.5) / width - 0.5) * 2 pi with direction
    (sin t sin phi, cos t, -sin t cos phi).
    """
    rng = _rng(seed + 7919)
    zenith = np.array([0.22, 0.40, 0.95]) * rng.uniform(0.9, 1.1, 3)
    horizon = np.array([0.95, 0.92, 0.85]) * rng.uniform(0.9, 1.1, 3)
    ground = np.array([0.25, 0.22, 0.20]) * rng.uniform(0.9, 1.1, 3)
    sun_elev = math.radians(rng.uniform(25.0, 50.0))
    sun_az = rng.uniform(-math.pi, math.pi)
    sun = np.array([math.cos(sun_elev) * math.sin(sun_az), math.sin(sun_elev),
                    -math.cos(sun_elev) * math.cos(sun_az)])
    sun_color = np.array([1.0, 0.92, 0.8]) * rng.uniform(150.0, 250.0)
    sun_width = 0.0015  # 1 - cos(angle) scale of the lobe

    theta = (np.arange(height) + 0.5) / height * math.pi
    phi = ((np.arange(width) + 0.5) / width - 0.5) * 2.0 * math.pi
    T, P = np.meshgrid(theta, phi, indexing="ij")
    d = np.stack([np.sin(T) * np.sin(P), np.cos(T), -np.sin(T) * np.cos(P)], axis=-1)
    up = d[..., 1]
    sky_t = np.sqrt(np.clip(up, 0.0, 1.0))[..., None]
    sky = horizon * (1.0 - sky_t) + zenith * sky_t
    gnd_t = np.clip(-up * 4.0, 0.0, 1.0)[..., None]
    gnd = horizon * (1.0 - gnd_t) + ground * gnd_t
    img = np.where(up[..., None] >= 0.0, sky, gnd)
    cosg = d @ sun
    img = img + sun_color * np.exp((cosg - 1.0) / sun_width)[..., None]
    return img.astype(np.float32)


def uniform_env(value=1.0, width=64, height=32) -> np.ndarray:
    return np.full((height, width, 3), value, dtype=np.float32)


def upper_hemisphere_env(value=1.0, width=64, height=32) -> np.ndarray:
    """Radiance `value` for directions with +y component > 0, black below (height even)."""
    assert height % 2 == 0
    env = np.zeros((height, width, 3), dtype=np.float32)
    env[: height // 2] = value
    return env


# --------------------------------------------------------------------------------------------
# Config 1: Cornell-style box
# --------------------------------------------------------------------------------------------

def cornell_box(seed=0, width=64, height=64, spp=16, max_depth=4) -> Scene:
    """Unit box with five walls (front open), two rotated boxes and a ceiling quad light.

    10 wall triangles + 24 box triangles; the library adds 2 light triangles -> 36.
    """
    rng = _rng(seed)
    mats = np.stack([
        diffuse((0.75, 0.75, 0.75)),   # 0 white
        diffuse((0.10, 0.75, 0.10)),   # 1 green (x = 0, right-hand side of the image)
        diffuse((0.75, 0.10, 0.10)),   # 2 red (x = 1, left-hand side of the image)
    ])
    mb = _MeshBuilder()
    v = np.array([[0, 0, 0], [1, 0, 0], [1, 0, 1], [0, 0, 1],
                  [0, 1, 0], [1, 1, 0], [1, 1, 1], [0, 1, 1]], dtype=np.float64)
    # inward-facing walls (counter-clockwise seen from inside the box)
    walls = [
        ((0, 3, 2), (0, 2, 1), 0),  # floor y=0, normal +y
        ((4, 5, 6), (4, 6, 7), 0),  # ceiling y=1, normal -y
        ((3, 7, 6), (3, 6, 2), 0),  # back z=1, normal -z
        ((0, 4, 7), (0, 7, 3), 1),  # left x=0, normal +x
        ((1, 2, 6), (1, 6, 5), 2),  # right x=1, normal -x
    ]
    for t1, t2, m in walls:
        mb.add(v, [t1, t2], m)
    placements = [((0.33, 0.37), 1.0), ((0.66, 0.66), 2.0)]
    for (cx, cz), hmul in placements:
        s = rng.uniform(0.2, 0.35)
        h = s * hmul
        rot = rng.uniform(0.0, 0.5 * math.pi)
        jx, jz = rng.uniform(-0.04, 0.04, 2)
        bv, bt = _box_mesh((cx + jx, 0.5 * h, cz + jz), (s, h, s), rot)
        mb.add(bv, bt, 0)
    verts, idx, mid = mb.arrays()
    # v is shared by the wall entries: compact duplicates is unnecessary for correctness.
    light = quad_light((0.375, 1.0 - 1e-3, 0.375), (0.25, 0.0, 0.0), (0.0, 0.0, 0.25),
                       (15.0, 15.0, 15.0))
    cam = Camera((0.5, 0.5, -1.4), (0.5, 0.5, 0.5), (0.0, 1.0, 0.0), 40.0, width, height)
    return Scene("cornell", verts, idx, mid, mats, light[None, :], None, cam, spp, max_depth,
                 {"seed": seed})


def many_light_box(n_lights=64, seed=0, width=64, height=64, spp=16, max_depth=4) -> Scene:
    """The Cornell geometry lit by `n_lights` small quads instead of one: 60 % on the ceiling
    facing down, the rest on the two side walls facing in; side 0.03-0.07, radiance with a
    heavy (Pareto, shape 1.5) tail and random tints; lights on one wall do not overlap
    (they share its plane).  A few lights dominate each point and which ones depends on where
    the point is: many-light direct illumination."""
    base = cornell_box(seed=seed, width=width, height=height, spp=spp, max_depth=max_depth)
    rng = _rng(seed + 101)
    lights = []
    placed = {0: [], 1: [], 2: []}                        # squares already on each wall

    def free(wall, a, b, size):
        # lights on one wall share a plane: overlapping ones would hit at equal depth
        return all(a + size + 0.005 <= a2 or a2 + s2 + 0.005 <= a or b + size + 0.005 <= b2 or b2 + s2 + 0.005 <= b
                   for a2, b2, s2 in placed[wall])

    for _ in range(n_lights):
        size = rng.uniform(0.03, 0.07)
        tint = rng.uniform(0.4, 1.0, 3)
        L = tuple(3.0 * (rng.pareto(1.5) + 1.0) * tint / tint.max())
        where = rng.random()
        wall = 0 if where < 0.6 else (1 if where < 0.8 else 2)
        for _attempt in range(200):
            a, b = rng.uniform(0.05, 0.95 - size, 2)
            if free(wall, a, b, size):
                break
        else:
            continue                                      # the wall is full
        placed[wall].append((a, b, size))
        if where < 0.6:                                   # ceiling, normal -y
            lights.append(quad_light((a, 1.0 - 1e-3, b), (size, 0.0, 0.0), (0.0, 0.0, size), L))
        elif where < 0.8:                                 # wall x = 0, normal +x
            lights.append(quad_light((1e-3, a, b), (0.0, size, 0.0), (0.0, 0.0, size), L))
        else:                                             # wall x = 1, normal -x
            lights.append(quad_light((1.0 - 1e-3, a, b), (0.0, 0.0, size), (0.0, size, 0.0), L))
    return Scene("many_light_box", base.vertices, base.indices, base.material_ids, base.materials,
                 np.stack(lights), None, base.camera, spp, max_depth, {"seed": seed, "n_lights": n_lights})


# --------------------------------------------------------------------------------------------
# Config 2: synthetic CAD pushbutton (lathe of a seeded spline profile)
# --------------------------------------------------------------------------------------------

def _catmull_rom(points, n_samples):
    """Uniform Catmull-Rom spline through `points` (k, 2), sampled at n_samples parameters."""
    p = np.asarray(points, dtype=np.float64)
    k = p.shape[0]
    ext = np.concatenate([2 * p[:1] - p[1:2], p, 2 * p[-1:] - p[-2:-1]])
    s = np.linspace(0.0, k - 1, n_samples)
    seg = np.minimum(np.floor(s).astype(int), k - 2)
    t = (s - seg)[:, None]
    p0, p1, p2, p3 = ext[seg], ext[seg + 1], ext[seg + 2], ext[seg + 3]
    return 0.5 * ((2 * p1) + (-p0 + p2) * t + (2 * p0 - 5 * p1 + 4 * p2 - p3) * t * t
                  + (-p0 + 3 * p1 - 3 * p2 + p3) * t * t * t)


def _lathe(profile, n_angular):
    """Surface of revolution about +y. profile[0] must lie on the axis (r = 0).

    Returns vertices, triangles (outward normals for a profile that runs from the top
    centre outwards and down) and the profile-segment index of each triangle.
    """
    r, y = profile[:, 0], profile[:, 1]
    n_prof = profile.shape[0]
    phi = np.arange(n_angular) * (2.0 * math.pi / n_angular)
    cphi, sphi = np.cos(phi), np.sin(phi)
    top = np.array([[0.0, y[0], 0.0]])
    rings = np.stack([r[1:, None] * cphi[None, :],
                      np.broadcast_to(y[1:, None], (n_prof - 1, n_angular)),
                      r[1:, None] * sphi[None, :]], axis=-1).reshape(-1, 3)
    v = np.concatenate([top, rings])
    ring = lambda j: 1 + (j - 1) * n_angular  # noqa: E731  first vertex of profile point j>=1
    i = np.arange(n_angular)
    i1 = (i + 1) % n_angular
    tris, segs = [], []
    # fan at the axis: (top, ring1[i1], ring1[i]) faces +y for phi increasing towards +z
    fan = np.stack([np.zeros(n_angular, dtype=np.int64), ring(1) + i1, ring(1) + i], axis=1)
    tris.append(fan)
    segs.append(np.zeros(n_angular, dtype=np.int64))
    for j in range(1, n_prof - 1):
        a = ring(j) + i
        b = ring(j) + i1
        c = ring(j + 1) + i1
        d = ring(j + 1) + i
        tris.append(np.stack([a, b, c], axis=1))
        tris.append(np.stack([a, c, d], axis=1))
        segs.append(np.full(2 * n_angular, j, dtype=np.int64))
    return v, np.concatenate(tris), np.concatenate(segs)


def _pushbutton_profile(rng, n_profile):
    ctrl = np.array([
        [0.00, 1.00], [0.22, 0.985], [0.40, 0.94], [0.50, 0.86],   # rounded cap
        [0.52, 0.70], [0.52, 0.45], [0.53, 0.36],                  # cylinder
        [0.66, 0.33], [0.74, 0.26], [0.75, 0.12], [0.70, 0.02],    # bezel
    ])
    jitter = rng.uniform(-0.03, 0.03, ctrl.shape)
    jitter[0, 0] = 0.0
    prof = _catmull_rom(ctrl + jitter, n_profile + 1)
    prof[0, 0] = 0.0
    prof[:, 0] = np.maximum(prof[:, 0], 0.0)
    prof[1:, 0] = np.maximum(prof[1:, 0], 1e-3)
    return prof


PUSHBUTTON_MATERIALS = None


def _pushbutton_materials():
    return np.stack([
        openpbr(base_color=(0.92, 0.92, 0.94), base_metalness=1.0, specular_roughness=0.2),  # 0 metal
        openpbr(base_color=(0.8, 0.05, 0.05), specular_roughness=0.3, specular_ior=1.5,
                coat_weight=1.0, coat_roughness=0.05, coat_ior=1.5),                          # 1 red plastic
        diffuse((0.5, 0.5, 0.5)),                                                             # 2 grey
    ])


def pushbutton_fuzz(**kw) -> Scene:
    """The pushbutton with its red coated plastic turned into velvet: the same red base and
    coat under a fuzz layer (weight 1, roughness 0.5, pale pink fibres)."""
    sc = pushbutton(**kw)
    mats = np.array(sc.materials, dtype=np.float32).copy()
    mats[1] = openpbr(base_color=(0.8, 0.05, 0.05), specular_roughness=0.3, specular_ior=1.5, coat_weight=1.0,
                      coat_roughness=0.05, coat_ior=1.5, fuzz_weight=1.0, fuzz_color=(1.0, 0.85, 0.85),
                      fuzz_roughness=0.5)
    return Scene("pushbutton_fuzz", sc.vertices, sc.indices, sc.material_ids, mats, sc.lights, sc.env, sc.camera,
                 sc.spp, sc.max_depth)


def pushbutton(seed=0, n_profile=250, n_angular=400, ground=(50, 100), width=1920, height=1080,
               spp=256, max_depth=8, env_size=(512, 256), with_light=True) -> Scene:
    """Config 2: lathe of a seeded Catmull-Rom profile (cap, cylinder, bezel) on a ground grid.

    With the defaults: 400 + 249*800 = 199,600 lathe triangles + 10,000 ground triangles.
    """
    rng = _rng(seed)
    prof = _pushbutton_profile(rng, n_profile)
    v, t, seg = _lathe(prof, n_angular)
    frac = seg / max(n_profile - 1, 1)
    mat = np.where(frac < 0.40, 1, 0)             # cap: red coated plastic, rest: metal
    mb = _MeshBuilder()
    mb.add(v, t, mat)
    if ground is not None and ground[0] * ground[1] > 0:
        gv, gt = _grid_plane(-4.0, 4.0, -4.0, 4.0, ground[0], ground[1], y=0.0)
        mb.add(gv, gt, 2)
    verts, idx, mid = mb.arrays()
    lights = (quad_light((-1.6, 3.2, -1.2), (1.0, 0.0, 0.0), (0.0, 0.0, 1.0), (9.0, 8.5, 8.0))[None, :]
              if with_light else np.zeros((0, N_LIGHT_FLOATS), np.float32))
    env = analytic_sky(env_size[0], env_size[1], seed) if env_size is not None else None
    cam = _frame_camera((-0.8, 0.0, -0.8), (0.8, 1.05, 0.8), (1.1, 0.85, -1.5), 35.0, width, height,
                        margin=0.7)
    return Scene("pushbutton", verts, idx, mid, _pushbutton_materials(), lights, env, cam, spp,
                 max_depth, {"seed": seed, "n_profile": n_profile, "n_angular": n_angular})


def pushbutton_lod(target_tris, seed=0, width=512, height=512, spp=100, max_depth=5) -> Scene:
    """Pushbutton tessellated to about `target_tris` triangles (Table 1/2 shaped LODs).

    The mesh is the lathe alone plus a 2-triangle ground quad; the angular count is four
    times the profile count, the same aspect the default tessellation has.
    """
    # tris = n_ang * (2 n_prof - 1) + 2 with n_ang = 1.6 n_prof  ->  solve for n_prof
    lathe = max(target_tris - 2, 64)
    n_prof = max(int(round(math.sqrt(lathe / 3.2))), 4)
    n_ang = max(int(round(lathe / (2 * n_prof - 1))), 8)
    sc = pushbutton(seed=seed, n_profile=n_prof, n_angular=n_ang, ground=(1, 1), width=width,
                    height=height, spp=spp, max_depth=max_depth)
    sc.name = f"pushbutton_lod{target_tris}"
    return sc


# --------------------------------------------------------------------------------------------
# Config 3: heavy scene (displaced icospheres)
# --------------------------------------------------------------------------------------------

def icosphere(level: int):
    """Unit icosphere by `level` 1:4 subdivisions with shared edge midpoints (20*4^level tris)."""
    t = (1.0 + math.sqrt(5.0)) / 2.0
    v = np.array([[-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0], [0, -1, t], [0, 1, t],
                  [0, -1, -t], [0, 1, -t], [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1]],
                 dtype=np.float64)
    f = np.array([[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11], [1, 5, 9],
                  [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8], [3, 9, 4], [3, 4, 2],
                  [3, 2, 6], [3, 6, 8], [3, 8, 9], [4, 9, 5], [2, 4, 11], [6, 2, 10],
                  [8, 6, 7], [9, 8, 1]], dtype=np.int64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    for _ in range(level):
        e = np.concatenate([f[:, [0, 1]], f[:, [1, 2]], f[:, [2, 0]]])
        e_sorted = np.sort(e, axis=1)
        key = e_sorted[:, 0] * (v.shape[0] + 1) + e_sorted[:, 1]
        uniq, inv = np.unique(key, return_inverse=True)
        a, b = uniq // (v.shape[0] + 1), uniq % (v.shape[0] + 1)
        mid = v[a] + v[b]
        mid /= np.linalg.norm(mid, axis=1, keepdims=True)
        base = v.shape[0]
        v = np.concatenate([v, mid])
        nf = f.shape[0]
        m01 = base + inv[:nf]
        m12 = base + inv[nf:2 * nf]
        m20 = base + inv[2 * nf:]
        f = np.concatenate([
            np.stack([f[:, 0], m01, m20], 1), np.stack([f[:, 1], m12, m01], 1),
            np.stack([f[:, 2], m20, m12], 1), np.stack([m01, m12, m20], 1)])
    return v, f


def _value_noise(p, table, perm):
    """Trilinear value noise on the integer lattice with smoothstep weights."""
    n = perm.shape[0]
    pi = np.floor(p).astype(np.int64)
    pf = p - pi
    w = pf * pf * (3.0 - 2.0 * pf)
    out = np.zeros(p.shape[0])
    for dx in (0, 1):
        for dy in (0, 1):
            for dz in (0, 1):
                h = perm[(perm[(perm[(pi[:, 0] + dx) % n] + pi[:, 1] + dy) % n] + pi[:, 2] + dz) % n]
                wx = w[:, 0] if dx else 1.0 - w[:, 0]
                wy = w[:, 1] if dy else 1.0 - w[:, 1]
                wz = w[:, 2] if dz else 1.0 - w[:, 2]
                out += wx * wy * wz * table[h]
    return out


def fbm(p, rng, octaves=5, base_freq=2.0):
    """Fractional Brownian motion of value noise, normalised to about [-1, 1]."""
    table = rng.uniform(-1.0, 1.0, 256)
    perm = rng.permutation(256)
    out = np.zeros(p.shape[0])
    amp, freq, norm = 1.0, base_freq, 0.0
    for _ in range(octaves):
        out += amp * _value_noise(p * freq, table, perm)
        norm += amp
        amp *= 0.5
        freq *= 2.0
    return out / norm


def heavy_scene(seed=0, level=7, n_instances=16, width=1920, height=1080, spp=64, max_depth=12,
                env_size=(512, 256), plane=(1, 1)) -> Scene:
    """Config 3: displaced icospheres (fBm amplitude 0.15 r) scattered on a ground plane.

    Instances are flattened into one mesh; each gets its own material row, drawn from
    glass (IOR 1.5, transmission 1, smooth), rough metal (roughness U[0.05, 0.8]) and
    coated diffuse (coat roughness 0.1).
    """
    rng = _rng(seed)
    sv, sf = icosphere(level)
    grid = int(math.ceil(math.sqrt(n_instances)))
    spacing = 2.6
    mb = _MeshBuilder()
    mats = []
    lo = np.array([np.inf] * 3)
    hi = -lo
    for i in range(n_instances):
        gx, gz = i % grid, i // grid
        r = rng.uniform(0.6, 1.0)
        cx = (gx - 0.5 * (grid - 1)) * spacing + rng.uniform(-0.4, 0.4)
        cz = (gz - 0.5 * (grid - 1)) * spacing + rng.uniform(-0.4, 0.4)
        disp = fbm(sv * 1.0 + rng.uniform(-50, 50, 3), rng)
        v = sv * (r * (1.0 + 0.15 * disp))[:, None]
        cy = r * 1.18
        v = v + np.array([cx, cy, cz])
        kind = int(rng.integers(0, 3))
        if kind == 0:
            m = openpbr(base_color=(1.0, 1.0, 1.0), specular_roughness=0.0, specular_ior=1.5,
                        transmission_weight=1.0)
        elif kind == 1:
            c = rng.uniform(0.55, 0.95, 3)
            m = openpbr(base_color=tuple(c), base_metalness=1.0,
                        specular_roughness=float(rng.uniform(0.05, 0.8)))
        else:
            c = rng.uniform(0.1, 0.8, 3)
            m = openpbr(base_color=tuple(c), specular_roughness=0.4, coat_weight=1.0,
                        coat_roughness=0.1, coat_ior=1.5)
        mats.append(m)
        mb.add(v, sf, len(mats) - 1)
        lo = np.minimum(lo, v.min(0))
        hi = np.maximum(hi, v.max(0))
    mats.append(diffuse((0.45, 0.45, 0.45)))
    ext = 0.5 * spacing * grid + 2.0
    gv, gt = _grid_plane(-ext, ext, -ext, ext, plane[0], plane[1], y=0.0)
    mb.add(gv, gt, len(mats) - 1)
    verts, idx, mid = mb.arrays()
    env = analytic_sky(env_size[0], env_size[1], seed)
    cam = _frame_camera(lo, hi, (0.9, 1.0, -1.4), 35.0, width, height, margin=0.95)
    return Scene("heavy", verts, idx, mid, np.stack(mats), np.zeros((0, N_LIGHT_FLOATS), np.float32),
                 env, cam, spp, max_depth, {"seed": seed, "level": level, "n_instances": n_instances})


# --------------------------------------------------------------------------------------------
# Config 4: batch of uneven scenes
# --------------------------------------------------------------------------------------------

BATCH_RESOLUTIONS = ((256, 256), (512, 512), (1024, 768), (1920, 1080))


def batch_specs(n_scenes=64, seed=0, min_tris=1_000, max_tris=500_000):
    """Deterministic list of (kind, target_tris, width, height, spp, max_depth, seed)."""
    rng = _rng(seed + 104729)
    specs = []
    for i in range(n_scenes):
        kind = "pushbutton" if rng.uniform() < 0.5 else "heavy"
        tris = int(math.exp(rng.uniform(math.log(min_tris), math.log(max_tris))))
        w, h = BATCH_RESOLUTIONS[int(rng.integers(0, len(BATCH_RESOLUTIONS)))]
        spp = int(rng.integers(1, 33))
        specs.append(dict(kind=kind, tris=tris, width=w, height=h, spp=spp, max_depth=8,
                          seed=seed * 1000 + i))
    return specs


def scene_from_spec(spec) -> Scene:
    """Build one batch scene; triangle counts land near (not exactly on) `tris`."""
    w, h = spec["width"], spec["height"]
    if spec["kind"] == "pushbutton":
        sc = pushbutton_lod(spec["tris"], seed=spec["seed"], width=w, height=h)
    else:
        # 20 * 4^level triangles per instance; pick level and instance count to match
        target = spec["tris"]
        level = 0
        while level < 7 and 20 * 4 ** (level + 1) * 2 <= target:
            level += 1
        n_inst = int(min(max(round(target / (20 * 4 ** level)), 1), 16))
        sc = heavy_scene(seed=spec["seed"], level=level, n_instances=n_inst, width=w, height=h)
    sc.spp = spec["spp"]
    sc.max_depth = spec["max_depth"]
    return sc


# --------------------------------------------------------------------------------------------
# Small analytic test scenes (white furnace, diffuse plane under a sky, plane under a quad)
# --------------------------------------------------------------------------------------------

def furnace_sphere(level=2, displace=0.0, seed=0, albedo=1.0, width=32, height=32,
                   spp=16, max_depth=8, env_value=1.0) -> Scene:
    """Closed (optionally fBm-displaced, hence concave) icosphere of radius 1 with a
    Lambertian albedo under a uniform environment, seen from outside."""
    v, f = icosphere(level)
    if displace > 0.0:
        rng = _rng(seed)
        v = v * (1.0 + displace * fbm(v * 1.3, rng, octaves=3, base_freq=1.5))[:, None]
    mats = diffuse((albedo, albedo, albedo))[None, :]
    cam = Camera((0.0, 0.6, -3.2), (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), 45.0, width, height)
    return Scene("furnace", v.astype(np.float32), f.astype(np.uint32),
                 np.zeros(f.shape[0], np.uint32), mats, np.zeros((0, N_LIGHT_FLOATS), np.float32),
                 uniform_env(env_value), cam, spp, max_depth, {"level": level})


def plane_under_sky(albedo=0.5, width=16, height=16, spp=64, max_depth=1) -> Scene:
    """Large Lambertian plane y = 0 under a sky of radiance 1 on the upper hemisphere."""
    v, t = _grid_plane(-50.0, 50.0, -50.0, 50.0, 1, 1)
    mats = diffuse((albedo, albedo, albedo))[None, :]
    cam = Camera((0.0, 2.0, 0.0), (0.3, 0.0, 1.0), (0.0, 1.0, 0.0), 30.0, width, height)
    return Scene("plane_sky", v.astype(np.float32), t.astype(np.uint32),
                 np.zeros(t.shape[0], np.uint32), mats, np.zeros((0, N_LIGHT_FLOATS), np.float32),
                 upper_hemisphere_env(1.0), cam, spp, max_depth, {})


def plane_with_quad(albedo=0.8, radiance=5.0, width=24, height=24, spp=256, max_depth=1) -> Scene:
    """Lambertian plane y = 0 lit by a 1 x 0.6 quad light at height 1.2 facing down; the
    camera looks at the plane away from the light, with a narrow field of view."""
    v, t = _grid_plane(-20.0, 20.0, -20.0, 20.0, 1, 1)
    mats = diffuse((albedo, albedo, albedo))[None, :]
    light = quad_light((-0.5, 1.2, -0.3), (1.0, 0.0, 0.0), (0.0, 0.0, 0.6),
                       (radiance, radiance, radiance))
    cam = Camera((0.4, 0.9, 1.6), (0.3, 0.0, 0.6), (0.0, 1.0, 0.0), 12.0, width, height)
    return Scene("plane_quad", v.astype(np.float32), t.astype(np.uint32),
                 np.zeros(t.shape[0], np.uint32), mats, light[None, :], None, cam, spp,
                 max_depth, {})


def emissive_sphere_interior(albedo=0.5, emission=0.5, level=2, width=16, height=16, spp=64,
                             max_depth=200) -> Scene:
    """Camera inside a closed icosphere whose inward-facing surface is Lambertian (albedo
    rho) and emits L_e on its inner side; the radiance everywhere inside is L_e/(1 - rho)."""
    v, f = icosphere(level)
    f = f[:, [0, 2, 1]]  # inward-facing winding
    mats = openpbr(base_color=(albedo, albedo, albedo), specular_weight=0.0,
                   emission_luminance=emission)[None, :]
    cam = Camera((0.05, -0.1, 0.02), (0.3, 0.2, 1.0), (0.0, 1.0, 0.0), 60.0, width, height)
    return Scene("emissive_interior", v.astype(np.float32), f.astype(np.uint32),
                 np.zeros(f.shape[0], np.uint32), mats, np.zeros((0, N_LIGHT_FLOATS), np.float32),
                 None, cam, spp, max_depth, {"level": level})
