"""Seeded synthetic inputs for FastConv and the time-to-contact pipeline.

This module only *generates* inputs and closed-form ground truth; it holds none
of the method's arithmetic (no convolution, no derivative stencil, no sums, no
solve).  Both the FP64 oracle (``oracle/``) and the CUDA path take their inputs
from here, so they always see identical bytes.

Scenes follow the perspective model of Sec. V-A (Eqs. pp_start, ppcombined): a
pinhole camera with focal length ``f`` pixels looks along +Z (image x to the
right = +X, image y downward = +Y) and translates with constant velocity ``T``
(scene units per frame) towards a textured plane ``n . X = d``.  Pixel (i, j)
has its centre at x = j - (W-1)/2, y = i - (H-1)/2 relative to the principal
point.  A pixel is point-sampled at its centre: the ray (x/f, y/f, 1) is cut
with the plane and the analytic texture is evaluated at the hit point.

Ground truth (Sec. I and Eq. final_TTC): the time to contact is the time until
the optical centre reaches the plane, ``(d - n . c(t)) / (n . T)`` frames, and
the focus of expansion is the image of the direction of motion,
``f (Tx/Tz, Ty/Tz)`` pixels from the principal point.

The renderer uses torch float64 so that it runs on the host (tests) or on a
device (large benchmark videos) with the same code.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np
import torch

__all__ = [
    "PlaneScene",
    "fronto_parallel_scene",
    "tilted_plane_scene",
    "render",
    "render_sequence",
    "ground_truth",
    "uniform_array",
    "normal_array",
    "gaussian_kernel",
    "uneven_pair_sizes",
    "ramp_sequence",
]


@dataclasses.dataclass
class PlaneScene:
    """A camera translating towards a textured plane."""

    H: int
    W: int
    f: float                 # focal length, pixels
    n: np.ndarray            # (3,) unit plane normal, n_z > 0
    d: float                 # plane offset: n . X = d
    c0: np.ndarray           # (3,) camera centre at t = 0
    T: np.ndarray            # (3,) camera velocity, scene units per frame
    e1: np.ndarray           # (3,) orthonormal basis of the plane
    e2: np.ndarray
    tex_k: np.ndarray        # (m, 2) spatial frequencies, cycles per scene unit
    tex_phi: np.ndarray      # (m,) phases
    tex_a: np.ndarray        # (m,) amplitudes, sum |a| <= 0.5
    quantize: bool           # True: uint8 round-half-even(255 E); False: float32 E


def _plane_basis(n: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    a = np.array([1.0, 0.0, 0.0]) if abs(n[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    e1 = a - n * float(n @ a)
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(n, e1)
    return e1, e2


def _texture(rng: np.random.Generator, m: int, pmin: float, pmax: float,
             f: float, depth: float, amp_total: float):
    """m random-phase sinusoids whose image periods at ``depth`` lie in [pmin, pmax] px."""
    periods_px = np.exp(rng.uniform(math.log(pmin), math.log(pmax), size=m))
    periods_scene = periods_px * depth / f
    ang = rng.uniform(0.0, 2.0 * math.pi, size=m)
    k = np.stack([np.cos(ang), np.sin(ang)], axis=1) / periods_scene[:, None]
    phi = rng.uniform(0.0, 2.0 * math.pi, size=m)
    w = rng.uniform(0.5, 1.0, size=m)
    a = amp_total * w / w.sum()
    return k, phi, a


def fronto_parallel_scene(H: int = 128, W: int = 128, seed: int = 0, Z0: float = 10.0,
                          speed: float = 0.1, f: Optional[float] = None, m: int = 8,
                          pmin: float = 4.0, pmax: float = 32.0,
                          quantize: bool = False) -> PlaneScene:
    """Camera moving along the optical axis towards a fronto-parallel plane at Z0.

    Ground-truth TTC at time t is Z0/speed - t frames; the FOE is the principal point.
    """
    rng = np.random.default_rng(seed)
    f = float(W if f is None else f)
    n = np.array([0.0, 0.0, 1.0])
    e1, e2 = _plane_basis(n)
    k, phi, a = _texture(rng, m, pmin, pmax, f, Z0, 0.475)
    return PlaneScene(H=H, W=W, f=f, n=n, d=Z0, c0=np.zeros(3), T=np.array([0.0, 0.0, speed]),
                      e1=e1, e2=e2, tex_k=k, tex_phi=phi, tex_a=a, quantize=quantize)


def tilted_plane_scene(H: int = 1080, W: int = 1920, seed: int = 0, Z0: float = 20.0,
                       speed: float = 0.05, tilt_deg: float = 20.0, cone_deg: float = 15.0,
                       m: int = 64, pmin: float = 4.0, pmax: float = 64.0,
                       f: Optional[float] = None, quantize: bool = True) -> PlaneScene:
    """Band-limited-noise plane tilted ``tilt_deg`` about a random in-plane axis.

    The plane passes through (0, 0, Z0); the camera direction of motion is uniform
    on the spherical cap within ``cone_deg`` of +Z and its Z speed is ``speed``.
    """
    rng = np.random.default_rng(seed)
    f = float(W if f is None else f)
    alpha = rng.uniform(0.0, 2.0 * math.pi)
    axis = np.array([math.cos(alpha), math.sin(alpha), 0.0])
    th = math.radians(tilt_deg)
    z = np.array([0.0, 0.0, 1.0])
    # Rodrigues rotation of +Z about the in-plane axis
    n = z * math.cos(th) + np.cross(axis, z) * math.sin(th) + axis * float(axis @ z) * (1 - math.cos(th))
    n /= np.linalg.norm(n)
    d = float(n @ np.array([0.0, 0.0, Z0]))
    cos_max = math.cos(math.radians(cone_deg))
    cz = rng.uniform(cos_max, 1.0)
    ph = rng.uniform(0.0, 2.0 * math.pi)
    sz = math.sqrt(max(0.0, 1.0 - cz * cz))
    direction = np.array([sz * math.cos(ph), sz * math.sin(ph), cz])
    T = direction * (speed / cz)
    e1, e2 = _plane_basis(n)
    k, phi, a = _texture(rng, m, pmin, pmax, f, Z0, 0.48)
    return PlaneScene(H=H, W=W, f=f, n=n, d=d, c0=np.zeros(3), T=T, e1=e1, e2=e2,
                      tex_k=k, tex_phi=phi, tex_a=a, quantize=quantize)


def render(scene: PlaneScene, t: float, device="cpu") -> torch.Tensor:
    """Frame at time t: uint8 (H, W) if ``scene.quantize`` else float32 (H, W)."""
    dt = torch.float64
    H, W, f = scene.H, scene.W, scene.f
    x = (torch.arange(W, dtype=dt, device=device) - (W - 1) / 2.0) / f
    y = (torch.arange(H, dtype=dt, device=device) - (H - 1) / 2.0) / f
    yy, xx = torch.meshgrid(y, x, indexing="ij")
    c = scene.c0 + t * scene.T
    n = scene.n
    denom = n[0] * xx + n[1] * yy + n[2]
    s = (scene.d - float(n @ c)) / denom
    p0 = scene.d * n
    X = c[0] + s * xx - p0[0]
    Y = c[1] + s * yy - p0[1]
    Z = c[2] + s - p0[2]
    u = X * scene.e1[0] + Y * scene.e1[1] + Z * scene.e1[2]
    v = X * scene.e2[0] + Y * scene.e2[1] + Z * scene.e2[2]
    E = torch.full_like(u, 0.5)
    two_pi = 2.0 * math.pi
    for (kx, ky), ph, a in zip(scene.tex_k, scene.tex_phi, scene.tex_a):
        E += float(a) * torch.sin(two_pi * (float(kx) * u + float(ky) * v) + float(ph))
    if scene.quantize:
        q = torch.round(E.clamp(0.0, 1.0) * 255.0)       # round half to even
        return q.to(torch.uint8)
    return E.to(torch.float32)


def render_sequence(scene: PlaneScene, T: int, device="cpu", t0: float = 0.0) -> torch.Tensor:
    """T consecutive frames, shape (T, H, W)."""
    out = torch.empty((T, scene.H, scene.W),
                      dtype=torch.uint8 if scene.quantize else torch.float32, device=device)
    for i in range(T):
        out[i] = render(scene, t0 + i, device)
    return out


def ground_truth(scene: PlaneScene, t: float) -> tuple[float, float, float]:
    """(TTC in frames, FOE x, FOE y in pixels from the principal point) at time t."""
    c = scene.c0 + t * scene.T
    ttc = (scene.d - float(scene.n @ c)) / float(scene.n @ scene.T)
    foe_x = scene.f * scene.T[0] / scene.T[2]
    foe_y = scene.f * scene.T[1] / scene.T[2]
    return ttc, foe_x, foe_y


def ramp_sequence(H: int, W: int, Z0: float, speed: float, a: float, b: float, c: float,
                  f: float, T: int = 2) -> np.ndarray:
    """Fronto-parallel plane with the linear texture a X + b Y + c, float64 frames.

    Brightness at pixel offset (x, y) and time t is (Z0 - speed t)(a x + b y)/f + c,
    which is trilinear in (x, y, t).
    """
    x = np.arange(W, dtype=np.float64) - (W - 1) / 2.0
    y = np.arange(H, dtype=np.float64) - (H - 1) / 2.0
    yy, xx = np.meshgrid(y, x, indexing="ij")
    frames = np.empty((T, H, W), dtype=np.float64)
    for t in range(T):
        Z = Z0 - speed * t
        frames[t] = Z * (a * xx + b * yy) / f + c
    return frames


def uniform_array(shape, seed: int, dtype=np.float32) -> np.ndarray:
    return np.random.default_rng(seed).random(shape, dtype=np.float64).astype(dtype)


def normal_array(shape, seed: int, dtype=np.float32) -> np.ndarray:
    return np.random.default_rng(seed).standard_normal(shape).astype(dtype)


def gaussian_kernel(k: int, ndim: int = 2, dtype=np.float32) -> np.ndarray:
    """Normalised k^ndim Gaussian, sigma = k/6, centred at (k-1)/2."""
    sigma = k / 6.0
    g = np.exp(-0.5 * ((np.arange(k) - (k - 1) / 2.0) / sigma) ** 2)
    out = g
    for _ in range(ndim - 1):
        out = np.multiply.outer(out, g)
    return (out / out.sum()).astype(dtype)


def uneven_pair_sizes(n: int, seed: int, wmin=160, wmax=1920, hmin=120, hmax=1080):
    """Seeded (H, W, Z0, speed) for a batch of frame pairs of uneven sizes."""
    rng = np.random.default_rng(seed)
    W = rng.integers(wmin, wmax + 1, size=n)
    H = rng.integers(hmin, hmax + 1, size=n)
    Z0 = rng.uniform(5.0, 50.0, size=n)
    sp = rng.uniform(0.01, 0.2, size=n)
    return [(int(h), int(w), float(z), float(s)) for h, w, z, s in zip(H, W, Z0, sp)]


# camera streams for the serving workload: 16 streams each of 320x240, 640x480,
# 1280x720 and 1920x1080 (H, W)
CAMERA_CLASSES = ((240, 320), (480, 640), (720, 1280), (1080, 1920))


def camera_streams(per_class: int = 16, classes=CAMERA_CLASSES, seed: int = 0):
    """Seeded stream specs [(sid, H, W, scene_seed, Z0, speed)], classes interleaved."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(per_class):
        for H, W in classes:
            sid = len(out)
            out.append((sid, H, W, int(seed * 1000003 + sid), float(rng.uniform(10.0, 40.0)),
                        float(rng.uniform(0.02, 0.1))))
    return out


def poisson_arrivals(n_streams: int, fps: float, duration_s: float, seed: int):
    """Frame arrival times of independent streams: exponential inter-arrival times of
    mean 1/fps, each stream starting at a random phase.  Returns a time-sorted list of
    (t_seconds, stream, seq)."""
    rng = np.random.default_rng(seed)
    ev = []
    for s in range(n_streams):
        t = float(rng.uniform(0.0, 1.0 / fps))
        seq = 0
        while t < duration_s:
            ev.append((t, s, seq))
            seq += 1
            t += float(rng.exponential(1.0 / fps))
    ev.sort()
    return ev
