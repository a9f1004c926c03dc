"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This module holds input generation only -- grids, rays, jitter, targets, MLP initial weights and
an analytic ground-truth scene -- and none of the rendering arithmetic of the method.  Both the
FP64 oracle and the CUDA path consume what it produces; neither is imported here.

The paper's datasets (Synthetic-NeRF and the others, Sec. 5.1) are not available, so these
generators stand in for them with the same shapes: an object inside the unit box, 800 x 800
inward-facing views on the upper hemisphere at radius 4 with focal 1111, grids of 32^3 to 256^3,
12 feature channels and batches of 8192 rays (Sec. 5.2, Supp. A).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

BOX_MIN = (-1.0, -1.0, -1.0)
BOX_MAX = (1.0, 1.0, 1.0)


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


# ----------------------------------------------------------------------------------------------
# Rays
# ----------------------------------------------------------------------------------------------

def sphere_rays(n: int, seed: int, radius: float = 4.0, jitter_sd: float = 0.1):
    """Origins uniform on a sphere of the given radius, directions normalise(-o/radius + N(0, sd^2))."""
    g = rng(seed)
    o = g.normal(size=(n, 3))
    o = o / np.linalg.norm(o, axis=1, keepdims=True) * radius
    d = -o / radius + g.normal(scale=jitter_sd, size=(n, 3))
    d = d / np.linalg.norm(d, axis=1, keepdims=True)
    return o.astype(np.float32), d.astype(np.float32)


def blob_rays(n: int, seed: int, radius: float = 4.0, blob_radius: float = 0.3):
    """Origins uniform on a sphere, each ray aimed at a uniform point inside a central ball."""
    g = rng(seed)
    o = g.normal(size=(n, 3))
    o = o / np.linalg.norm(o, axis=1, keepdims=True) * radius
    tgt = g.normal(size=(n, 3))
    tgt = tgt / np.linalg.norm(tgt, axis=1, keepdims=True) * blob_radius * g.uniform(size=(n, 1)) ** (1 / 3)
    d = tgt - o
    d = d / np.linalg.norm(d, axis=1, keepdims=True)
    return o.astype(np.float32), d.astype(np.float32)


@dataclass
class CameraRig:
    """Inward-facing pinhole cameras on the upper hemisphere (z up), looking at the origin."""
    c2w: np.ndarray      # [V, 3, 4] camera-to-world (OpenGL axes: x right, y up, -z forward)
    height: int
    width: int
    focal: float


def hemisphere_rig(n_views: int, seed: int, radius: float = 4.0, height: int = 800, width: int = 800,
                   focal: float = 1111.0, min_elev_deg: float = 5.0) -> CameraRig:
    g = rng(seed)
    c2w = np.zeros((n_views, 3, 4))
    for v in range(n_views):
        az = g.uniform(0.0, 2 * np.pi)
        el = np.deg2rad(g.uniform(min_elev_deg, 85.0))
        pos = radius * np.array([np.cos(el) * np.cos(az), np.cos(el) * np.sin(az), np.sin(el)])
        fwd = -pos / np.linalg.norm(pos)
        right = np.cross(fwd, np.array([0.0, 0.0, 1.0]))
        right /= np.linalg.norm(right)
        up = np.cross(right, fwd)
        c2w[v, :, 0] = right
        c2w[v, :, 1] = up
        c2w[v, :, 2] = -fwd
        c2w[v, :, 3] = pos
    return CameraRig(c2w=c2w, height=height, width=width, focal=focal)


def pixel_rays(rig: CameraRig, views, rows, cols):
    """World-space origin and (unnormalised) direction through pixel centres."""
    views = np.asarray(views); rows = np.asarray(rows); cols = np.asarray(cols)
    x = (cols + 0.5 - rig.width * 0.5) / rig.focal
    y = -(rows + 0.5 - rig.height * 0.5) / rig.focal
    dc = np.stack([x, y, -np.ones_like(x)], axis=-1)
    R = rig.c2w[views, :, :3]
    d = np.einsum("nij,nj->ni", R, dc)
    o = rig.c2w[views, :, 3]
    return o.astype(np.float32), d.astype(np.float32)


def random_pixel_rays(rig: CameraRig, n: int, seed: int, views=None):
    """n rays through uniformly drawn pixels of uniformly drawn views (a training batch)."""
    g = rng(seed)
    vpool = np.arange(rig.c2w.shape[0]) if views is None else np.asarray(views)
    v = vpool[g.integers(0, len(vpool), size=n)]
    r = g.integers(0, rig.height, size=n)
    c = g.integers(0, rig.width, size=n)
    o, d = pixel_rays(rig, v, r, c)
    return o, d, (v, r, c)


def jitter(n: int, seed: int):
    """Per-ray training jitter p ~ U[0, 1) (Supp. A)."""
    return rng(seed).uniform(0.0, 1.0, size=n).astype(np.float32)


def targets(n: int, seed: int):
    return rng(seed).uniform(0.0, 1.0, size=(n, 3)).astype(np.float32)


# ----------------------------------------------------------------------------------------------
# Grids
# ----------------------------------------------------------------------------------------------

def normal_grid(shape, channels: int, sd: float, seed: int):
    g = rng(seed)
    full = tuple(shape) + ((channels,) if channels > 1 else ())
    return g.normal(scale=sd, size=full).astype(np.float32)


def lattice_points(res: int):
    """Coordinates of an align-corners lattice of res points over [-1, 1]."""
    return np.linspace(BOX_MIN[0], BOX_MAX[0], res)


def sphere_density(res: int, centres, radii, value: float, background: float = 0.0):
    """Nearest-voxel rasterisation of balls: lattice points inside any ball get `value`."""
    ax = lattice_points(res).astype(np.float32)
    X, Y, Z = np.meshgrid(ax, ax, ax, indexing="ij")
    out = np.full((res, res, res), background, dtype=np.float32)
    for c, r in zip(centres, radii):
        inside = (X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2 <= r * r
        out[inside] = value
    return out


def random_spheres(n: int, seed: int, lo=-0.7, hi=0.7, rmin=0.1, rmax=0.3):
    g = rng(seed)
    return g.uniform(lo, hi, size=(n, 3)), g.uniform(rmin, rmax, size=n)


def binary_image(height: int, width: int, seed: int, n_shapes: int = 24):
    """A binary image ({0, 1} float32, [height, width]) standing in for the target of the
    image-fitting toy (Sec. 3, Fig. exdv_poc): the union of seeded discs, rotated rectangles and thin
    strokes -- large occupied and free regions with sharp, curved and straight boundaries."""
    g = rng(seed)
    y, x = np.meshgrid((np.arange(height) + 0.5) / height, (np.arange(width) + 0.5) / width, indexing="ij")
    img = np.zeros((height, width), dtype=bool)
    for _ in range(n_shapes):
        kind = g.integers(3)
        cy, cx = g.uniform(0.05, 0.95, size=2)
        if kind == 0:
            r = g.uniform(0.03, 0.15)
            img |= (y - cy) ** 2 + (x - cx) ** 2 < r * r
        else:
            th = g.uniform(0, np.pi)
            a, b = (g.uniform(0.04, 0.2), g.uniform(0.02, 0.1)) if kind == 1 else (g.uniform(0.1, 0.35),
                                                                                   g.uniform(0.002, 0.008))
            u = (x - cx) * np.cos(th) + (y - cy) * np.sin(th)
            v = -(x - cx) * np.sin(th) + (y - cy) * np.cos(th)
            img |= (np.abs(u) < a) & (np.abs(v) < b)
    return img.astype(np.float32)


def smooth_features(res: int, channels: int, seed: int, n_waves: int = 4, max_freq: float = 2.0):
    """Per channel, the mean of n_waves random low-frequency sinusoids: values in [-1, 1]."""
    g = rng(seed)
    ax = lattice_points(res).astype(np.float32)
    X, Y, Z = np.meshgrid(ax, ax, ax, indexing="ij")
    out = np.zeros((res, res, res, channels), dtype=np.float32)
    for ch in range(channels):
        acc = np.zeros((res, res, res), dtype=np.float32)
        for _ in range(n_waves):
            k = g.uniform(-max_freq, max_freq, size=3) * np.pi
            ph = g.uniform(0, 2 * np.pi)
            acc += np.sin(k[0] * X + k[1] * Y + k[2] * Z + ph).astype(np.float32)
        out[..., ch] = acc / n_waves
    return out


# ----------------------------------------------------------------------------------------------
# MLP weights
# ----------------------------------------------------------------------------------------------

def mlp_weights(in_dim: int, hidden: int, out_dim: int, seed: int, n_hidden_layers: int = 2):
    """U(+-1/sqrt(fan_in)) weights, row-major [in][out]; biases U(+-1/sqrt(fan_in)), output bias 0."""
    g = rng(seed)
    dims = [in_dim] + [hidden] * n_hidden_layers + [out_dim]
    out = {}
    for i in range(len(dims) - 1):
        bound = 1.0 / np.sqrt(dims[i])
        out[f"w{i + 1}"] = g.uniform(-bound, bound, size=(dims[i], dims[i + 1])).astype(np.float32)
        if i == len(dims) - 2:
            out[f"b{i + 1}"] = np.zeros(dims[i + 1], dtype=np.float32)
        else:
            out[f"b{i + 1}"] = g.uniform(-bound, bound, size=dims[i + 1]).astype(np.float32)
    return out


def proposal_weights(in_dim: int, width: int, seed: int):
    """Proposal MLP in -> width -> width -> width -> 1, keys w0..w3 / b0..b3."""
    m = mlp_weights(in_dim, width, 1, seed, n_hidden_layers=3)
    return {f"w{i}": m[f"w{i + 1}"] for i in range(4)} | {f"b{i}": m[f"b{i + 1}"] for i in range(4)}


# ----------------------------------------------------------------------------------------------
# Workload recipes
# ----------------------------------------------------------------------------------------------

def coarse_case(seed: int = 0, res: int = 32, n_rays: int = 4096):
    """32^3 density and RGB grids, N(0, 0.1^2); 4096 rays from the radius-4 sphere; U[0,1] targets."""
    dens = normal_grid((res,) * 3, 1, 0.1, seed)
    rgb = normal_grid((res,) * 3, 3, 0.1, seed + 1)
    o, d = sphere_rays(n_rays, seed + 2)
    tgt = targets(n_rays, seed + 3)
    return dict(density=dens, rgb=rgb, rays_o=o, rays_d=d, target=tgt)


def fine_scene(seed: int = 0, res: int = 160, feat_dim: int = 12, n_spheres: int = 8,
               value: float = 50.0):
    """Density: n_spheres balls of `value` (0 outside); features: smooth random albedo."""
    c, r = random_spheres(n_spheres, seed)
    dens = sphere_density(res, c, r, value)
    feat = smooth_features(res, feat_dim, seed + 1)
    return dens, feat


def fine_batch(n_rays: int, seed: int, rig_seed: int = 1234, n_views: int = 100):
    rig = hemisphere_rig(n_views, rig_seed)
    o, d, _ = random_pixel_rays(rig, n_rays, seed)
    return o, d, jitter(n_rays, seed + 7), targets(n_rays, seed + 11)


# ----------------------------------------------------------------------------------------------
# Analytic ground-truth scene (stand-in for a Synthetic-NeRF object): ray-cast primitives
# ----------------------------------------------------------------------------------------------

@dataclass
class AnalyticScene:
    kind: np.ndarray       # [P] 0 = sphere, 1 = axis-aligned box
    centre: np.ndarray     # [P, 3]
    size: np.ndarray       # [P, 3] sphere: radius in [0]; box: half extents
    albedo: np.ndarray     # [P, 3]
    spec: np.ndarray       # [P] specular weight
    shininess: np.ndarray  # [P]
    light: np.ndarray      # [3] unit direction towards the light


def analytic_scene(seed: int = 0, n_prims: int = 20) -> AnalyticScene:
    """n_prims seeded spheres / boxes of size 0.1-0.4 inside [-0.8, 0.8]^3 with Lambert albedo and a
    Blinn-Phong specular lobe."""
    g = rng(seed)
    kind = g.integers(0, 2, size=n_prims)
    size = np.zeros((n_prims, 3))
    size[:, 0] = g.uniform(0.1, 0.4, size=n_prims)
    box = kind == 1
    size[box] = g.uniform(0.08, 0.3, size=(int(box.sum()), 3))
    ext = np.where(kind == 0, size[:, 0], size.max(axis=1))
    centre = g.uniform(-0.8 + ext[:, None] * 0.5, 0.8 - ext[:, None] * 0.5, size=(n_prims, 3))
    light = np.array([0.4, 0.3, 0.87])
    return AnalyticScene(kind=kind, centre=centre, size=size, albedo=g.uniform(0.1, 0.95, size=(n_prims, 3)),
                         spec=g.uniform(0.0, 0.6, size=n_prims), shininess=g.uniform(8.0, 64.0, size=n_prims),
                         light=light / np.linalg.norm(light))


def render_analytic(scene: AnalyticScene, rays_o, rays_d, bg=(1.0, 1.0, 1.0)):
    """Ray-cast the primitives (torch, on the tensors' device): nearest hit, Lambert + ambient
    + Blinn-Phong highlight, background colour where nothing is hit.  Returns [N, 3] in [0, 1]."""
    import torch
    dev = rays_o.device
    o = rays_o.to(torch.float32)
    d = rays_d.to(torch.float32)
    d = d / d.norm(dim=-1, keepdim=True)
    N = o.shape[0]
    t_best = torch.full((N,), float("inf"), device=dev)
    nrm = torch.zeros((N, 3), device=dev)
    pid = torch.full((N,), -1, dtype=torch.long, device=dev)
    for i in range(len(scene.kind)):
        c = torch.tensor(scene.centre[i], dtype=torch.float32, device=dev)
        if scene.kind[i] == 0:
            r = float(scene.size[i, 0])
            oc = o - c
            b = (oc * d).sum(-1)
            disc = b * b - ((oc * oc).sum(-1) - r * r)
            hit = disc > 0
            sq = torch.sqrt(torch.clamp(disc, min=0.0))
            t = -b - sq
            t = torch.where(t > 1e-4, t, -b + sq)
            hit &= t > 1e-4
            n = (o + t[:, None] * d - c) / r
        else:
            h = torch.tensor(scene.size[i], dtype=torch.float32, device=dev)
            inv = 1.0 / torch.where(d.abs() < 1e-12, torch.full_like(d, 1e-12), d)
            t1 = (c - h - o) * inv
            t2 = (c + h - o) * inv
            tmin = torch.minimum(t1, t2).amax(-1)
            tmax = torch.maximum(t1, t2).amin(-1)
            hit = (tmax > torch.clamp(tmin, min=1e-4))
            t = torch.where(tmin > 1e-4, tmin, tmax)
            p = o + t[:, None] * d - c
            q = (p / h).abs()
            ax = q.argmax(-1)
            n = torch.zeros_like(p)
            n.scatter_(1, ax[:, None], torch.sign(p.gather(1, ax[:, None])))
        better = hit & (t < t_best)
        t_best = torch.where(better, t, t_best)
        nrm = torch.where(better[:, None], n, nrm)
        pid = torch.where(better, torch.full_like(pid, i), pid)
    out = torch.tensor(bg, dtype=torch.float32, device=dev).expand(N, 3).clone()
    hitm = pid >= 0
    if bool(hitm.any()):
        idx = pid[hitm]
        alb = torch.tensor(scene.albedo, dtype=torch.float32, device=dev)[idx]
        spw = torch.tensor(scene.spec, dtype=torch.float32, device=dev)[idx]
        shn = torch.tensor(scene.shininess, dtype=torch.float32, device=dev)[idx]
        L = torch.tensor(scene.light, dtype=torch.float32, device=dev)
        n = nrm[hitm]
        n = n / n.norm(dim=-1, keepdim=True).clamp(min=1e-12)
        v = -d[hitm]
        hv = L + v
        hv = hv / hv.norm(dim=-1, keepdim=True).clamp(min=1e-12)
        diff = torch.clamp((n * L).sum(-1), min=0.0)
        spec = torch.clamp((n * hv).sum(-1), min=0.0) ** shn
        col = alb * (0.25 + 0.75 * diff[:, None]) + (spw * spec)[:, None]
        out[hitm] = torch.clamp(col, 0.0, 1.0)
    return out


def rig_rays_torch(rig: CameraRig, device):
    """All pixel rays of every view of a rig as flat [V*H*W, 3] tensors (origins, directions)."""
    import torch
    H, W = rig.height, rig.width
    cols = torch.arange(W, device=device, dtype=torch.float32)
    rows = torch.arange(H, device=device, dtype=torch.float32)
    yy, xx = torch.meshgrid(rows, cols, indexing="ij")
    dc = torch.stack([(xx + 0.5 - W * 0.5) / rig.focal, -(yy + 0.5 - H * 0.5) / rig.focal,
                      -torch.ones_like(xx)], dim=-1).reshape(-1, 3)
    c2w = torch.tensor(rig.c2w, dtype=torch.float32, device=device)
    d = torch.einsum("vij,nj->vni", c2w[:, :, :3], dc).reshape(-1, 3)
    o = c2w[:, :, 3][:, None, :].expand(-1, H * W, 3).reshape(-1, 3)
    return o.contiguous(), d.contiguous()
