"""Seeded synthetic stereo inputs for the halfway-domain scene-flow solve.

This module only renders images. It holds none of the solver's arithmetic, so
both the FP64 CPU oracle and the CUDA path can be fed from it without sharing
any part of the method.

Image convention (the paper's four captured images I_c^t, Section 3.1):
index 0 = I_0^0 (left, previous), 1 = I_1^0 (right, previous),
2 = I_0^1 (left, current), 3 = I_1^1 (right, current).
Intensities are float32 in about [0, 1] (monochrome, Section 3.1) plus
additive Gaussian noise that is not clamped.

Generators
----------
``plane_quadruple``  a fronto-parallel textured plane seen by a rectified rig
    with a known integer disparity and a known integer translation between
    the two time steps, made by integer crops of one noise texture. The true
    halfway fields are then known in closed form.
``SceneVideo``       a stereo video of 3-6 value-noise textured planes and
    spheres at depths that give a stated disparity range, with per-object
    rigid motion and a smooth sinusoidal non-rigid texture flow, ray cast with
    a pinhole rig (focal length = image width, baseline 0.1, right camera at
    +baseline on the x axis).
``batch_sizes``      the seeded size mix of a batch of uneven sequences.

Value noise: 4 octaves, base period 32 px, lacunarity 2, gain 0.5, lattice
values uniform in [0, 1) from the SplitMix64 finaliser (Steele, Lea and Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014), smoothstep
interpolation; the weighted octave mean stays in [0, 1].
"""

from __future__ import annotations

import math

import numpy as np

__all__ = [
    "value_noise",
    "plane_quadruple",
    "SceneVideo",
    "batch_sizes",
    "random_quadruple",
]

_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_GOLD = np.uint64(0x9E3779B97F4A7C15)
_KX = np.uint64(0xD1B54A32D192ED03)
_KY = np.uint64(0xABC98388FB8FAC03)
_KO = np.uint64(0x8CB92BA72F3D8DD7)


def _mix64(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _lattice(seed: int, octave: int, ix: np.ndarray, iy: np.ndarray) -> np.ndarray:
    """Uniform [0,1) value at integer lattice points (counter-based, seeded)."""
    with np.errstate(over="ignore"):
        base = _mix64(np.full(ix.shape, seed, dtype=np.uint64) * _GOLD + np.uint64(octave) * _KO)
        h = base ^ (ix.astype(np.int64).view(np.uint64) * _KX)
        h = _mix64(h)
        h = h ^ (iy.astype(np.int64).view(np.uint64) * _KY)
        h = _mix64(h)
    return (h >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def value_noise(u: np.ndarray, v: np.ndarray, seed: int, octaves: int = 4,
                period: float = 32.0, lacunarity: float = 2.0, gain: float = 0.5) -> np.ndarray:
    """Seeded fractal value noise at real coordinates (u, v), in [0, 1]."""
    u = np.asarray(u, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    total = np.zeros(np.broadcast(u, v).shape)
    amp, norm, per = 1.0, 0.0, float(period)
    for o in range(octaves):
        fu, fv = u / per, v / per
        iu, iv = np.floor(fu), np.floor(fv)
        tu, tv = fu - iu, fv - iv
        su, sv = tu * tu * (3.0 - 2.0 * tu), tv * tv * (3.0 - 2.0 * tv)
        iu = iu.astype(np.int64)
        iv = iv.astype(np.int64)
        v00 = _lattice(seed, o, iu, iv)
        v10 = _lattice(seed, o, iu + 1, iv)
        v01 = _lattice(seed, o, iu, iv + 1)
        v11 = _lattice(seed, o, iu + 1, iv + 1)
        n = (v00 * (1 - su) + v10 * su) * (1 - sv) + (v01 * (1 - su) + v11 * su) * sv
        total += amp * n
        norm += amp
        amp *= gain
        per /= lacunarity
    return total / norm


def _add_noise(imgs: np.ndarray, sigma: float, rng: np.random.Generator) -> np.ndarray:
    if sigma > 0:
        imgs = imgs + sigma * rng.standard_normal(imgs.shape)
    return imgs.astype(np.float32)


def plane_quadruple(width: int = 160, height: int = 120, disparity: int = 8,
                    motion: tuple[int, int] = (2, -1), sigma: float = 0.01,
                    seed: int = 1, pad: int = 16) -> np.ndarray:
    """Four images of one fronto-parallel textured plane, by integer crops.

    Right image: I_1(x) = T(x + (disparity, 0)) (right camera at +baseline).
    Second time step: the content moves by ``motion``: I_c^1(x) = I_c^0(x - motion).
    Returns float32 [4, height, width] in the module's image order.
    """
    d = int(disparity)
    vx, vy = int(motion[0]), int(motion[1])
    if max(abs(d) + abs(vx), abs(vy)) > pad:
        raise ValueError("shifts exceed the texture padding")
    ys, xs = np.mgrid[0:height + 2 * pad, 0:width + 2 * pad]
    tex = value_noise(xs.astype(np.float64), ys.astype(np.float64), seed)

    def crop(dx: int, dy: int) -> np.ndarray:
        return tex[pad + dy:pad + dy + height, pad + dx:pad + dx + width]

    imgs = np.stack([crop(0, 0), crop(d, 0), crop(-vx, -vy), crop(d - vx, -vy)])
    return _add_noise(imgs, sigma, np.random.default_rng(seed))


def random_quadruple(width: int, height: int, seed: int, sigma: float = 0.0) -> np.ndarray:
    """Four independent noise textures (no geometric relation); for unit tests."""
    ys, xs = np.mgrid[0:height, 0:width].astype(np.float64)
    imgs = np.stack([value_noise(xs, ys, seed * 16 + c, period=8.0) for c in range(4)])
    return _add_noise(imgs, sigma, np.random.default_rng(seed))


class _Obj:
    __slots__ = ("kind", "seed", "u0", "v0", "disp0", "du", "dv", "ddisp", "size",
                 "tilt", "rot0", "rot_rate", "flow_amp", "flow_lambda", "flow_rate", "aspect")


class SceneVideo:
    """Seeded stereo video of value-noise textured planes and spheres.

    Pinhole rig: focal length f = width px, principal point at the image centre,
    left camera at the origin, right camera at (+b, 0, 0) with b = 0.1, both
    looking down +Z (rectified). A point at depth Z has disparity f*b/Z.

    Objects: a background plane that fills the view plus 2-5 foreground
    objects (tilted textured rectangles and spheres). Each object's centre
    moves in image and disparity space at a constant seeded velocity whose
    image part is at most ``max_motion`` px per frame; rectangles also turn
    about their normal and spheres about their vertical axis. A sinusoidal
    texture-coordinate flow A*sin(2*pi*(v/lambda + omega*t)) adds smooth
    non-rigid motion. Frame f of the video is the quadruple at times (f, f+1).
    """

    def __init__(self, width: int = 640, height: int = 480, n_frames: int = 30,
                 seed: int = 100, disparity: tuple[float, float] = (5.0, 40.0),
                 max_motion: float = 12.0, sigma: float = 0.01, baseline: float = 0.1):
        self.width, self.height, self.n_frames = int(width), int(height), int(n_frames)
        self.seed, self.sigma, self.baseline = int(seed), float(sigma), float(baseline)
        self.f = float(width)
        self.cx, self.cy = (width - 1) / 2.0, (height - 1) / 2.0
        self.dmin, self.dmax = float(disparity[0]), float(disparity[1])
        self.max_motion = float(max_motion)
        rng = np.random.default_rng(self.seed)
        n_obj = int(rng.integers(3, 7))
        objs = []
        bg = _Obj()
        bg.kind, bg.seed = "bg", self.seed * 64 + 0
        bg.u0, bg.v0 = self.cx, self.cy
        bg.disp0 = self.dmin + 0.05 * (self.dmax - self.dmin) * rng.random()
        ang = rng.random() * 2 * math.pi
        sp = 0.25 * self.max_motion * rng.random()
        bg.du, bg.dv, bg.ddisp = sp * math.cos(ang), sp * math.sin(ang), 0.0
        bg.size, bg.tilt, bg.aspect = 0.0, (0.0, 0.0), 1.0
        bg.rot0, bg.rot_rate = 0.0, 0.0
        bg.flow_amp, bg.flow_lambda, bg.flow_rate = 0.0, 1.0, 0.0
        objs.append(bg)
        for k in range(1, n_obj):
            o = _Obj()
            o.kind = "sphere" if rng.random() < 0.4 else "rect"
            o.seed = self.seed * 64 + k
            o.u0 = rng.uniform(0.15, 0.85) * width
            o.v0 = rng.uniform(0.15, 0.85) * height
            o.disp0 = rng.uniform(self.dmin + 0.15 * (self.dmax - self.dmin), self.dmax)
            ang = rng.random() * 2 * math.pi
            sp = self.max_motion * rng.uniform(0.2, 0.7)
            o.du, o.dv = sp * math.cos(ang), sp * math.sin(ang)
            o.ddisp = rng.uniform(-0.5, 0.5) * self.max_motion / 12.0
            o.size = rng.uniform(0.10, 0.28) * height
            o.aspect = rng.uniform(0.6, 1.6)
            o.tilt = (rng.uniform(-0.35, 0.35), rng.uniform(-0.35, 0.35))
            o.rot0 = rng.uniform(0, 2 * math.pi)
            # turn slowly enough that the rim moves by at most ~0.25 max_motion px
            o.rot_rate = rng.uniform(-1, 1) * 0.25 * self.max_motion / max(o.size, 1.0)
            o.flow_amp = rng.uniform(0.3, 1.5) * width / 640.0
            o.flow_lambda = rng.uniform(40.0, 120.0) * width / 640.0
            o.flow_rate = rng.uniform(-0.05, 0.05)
            objs.append(o)
        # far to near is irrelevant (z-buffered), but keep a stable order
        self.objects = objs

    # -- geometry ---------------------------------------------------------------
    def _centre(self, o: _Obj, t: float) -> tuple[np.ndarray, float]:
        disp = max(o.disp0 + o.ddisp * t, 0.5 * self.dmin)
        z = self.f * self.baseline / disp
        u = o.u0 + o.du * t
        v = o.v0 + o.dv * t
        c = np.array([(u - self.cx) * z / self.f, (v - self.cy) * z / self.f, z])
        return c, z

    def _render_camera(self, t: float, cam: int) -> np.ndarray:
        h, w = self.height, self.width
        ys, xs = np.mgrid[0:h, 0:w].astype(np.float64)
        ox = self.baseline * cam
        dx = (xs - self.cx) / self.f
        dy = (ys - self.cy) / self.f
        zbuf = np.full((h, w), np.inf)
        tu = np.zeros((h, w))
        tv = np.zeros((h, w))
        owner = np.full((h, w), -1, dtype=np.int64)
        for k, o in enumerate(self.objects):
            c, z0 = self._centre(o, t)
            px_per_unit = self.f / z0
            if o.kind == "bg":
                # fronto-parallel infinite plane Z = z0
                zhit = np.full((h, w), z0)
                X = ox + zhit * dx
                Y = zhit * dy
                a = (X - c[0]) * px_per_unit
                b = (Y - c[1]) * px_per_unit
                hit = np.ones((h, w), dtype=bool)
            elif o.kind == "rect":
                n = np.array([o.tilt[0], o.tilt[1], -1.0])
                n /= np.linalg.norm(n)
                # ray P = (ox,0,0) + s*(dx,dy,1); plane n.(P - c) = 0
                denom = n[0] * dx + n[1] * dy + n[2]
                s = (n @ c - n[0] * ox) / denom
                X = ox + s * dx
                Y = s * dy
                Z = s
                # in-plane axes, turned by the object's angle
                e1 = np.cross(np.array([0.0, 1.0, 0.0]), n)
                e1 /= np.linalg.norm(e1)
                e2 = np.cross(n, e1)
                ang = o.rot0 + o.rot_rate * t
                ca, sa = math.cos(ang), math.sin(ang)
                r1, r2 = ca * e1 + sa * e2, -sa * e1 + ca * e2
                qx, qy, qz = X - c[0], Y - c[1], Z - c[2]
                a = (qx * r1[0] + qy * r1[1] + qz * r1[2]) * px_per_unit
                b = (qx * r2[0] + qy * r2[1] + qz * r2[2]) * px_per_unit
                half = o.size
                hit = (s > 0) & (np.abs(a) < half * o.aspect) & (np.abs(b) < half)
                zhit = Z
            else:  # sphere
                r = o.size / px_per_unit
                # |(ox,0,0) + s*d - c|^2 = r^2 with d = (dx,dy,1)
                dd = dx * dx + dy * dy + 1.0
                mx, my, mz = ox - c[0], -c[1], -c[2]
                bq = 2.0 * (mx * dx + my * dy + mz)
                cq = mx * mx + my * my + mz * mz - r * r
                disc = bq * bq - 4.0 * dd * cq
                hit = disc > 0
                sq = np.sqrt(np.where(hit, disc, 0.0))
                s = (-bq - sq) / (2.0 * dd)
                hit &= s > 0
                X = ox + s * dx
                Y = s * dy
                Z = s
                qx, qy, qz = X - c[0], Y - c[1], Z - c[2]
                lon = np.arctan2(qx, -qz) + (o.rot0 + o.rot_rate * t)
                lat = np.arcsin(np.clip(qy / r, -1.0, 1.0))
                a = lon * o.size
                b = lat * o.size
                zhit = Z
            # smooth non-rigid texture flow
            if o.flow_amp > 0:
                a = a + o.flow_amp * np.sin(2 * math.pi * (b / o.flow_lambda + o.flow_rate * t))
            closer = hit & (zhit < zbuf)
            zbuf = np.where(closer, zhit, zbuf)
            tu = np.where(closer, a, tu)
            tv = np.where(closer, b, tv)
            owner = np.where(closer, k, owner)
        img = np.zeros((h, w))
        for k, o in enumerate(self.objects):
            m = owner == k
            if m.any():
                img[m] = value_noise(tu[m] + 1000.0, tv[m] + 1000.0, o.seed)
        return img

    def render(self, t: int) -> np.ndarray:
        """Noisy left and right images at integer time ``t``: float32 [2, H, W]."""
        imgs = np.stack([self._render_camera(float(t), 0), self._render_camera(float(t), 1)])
        rng = np.random.default_rng([self.seed, int(t)])
        return _add_noise(imgs, self.sigma, rng)

    def frames(self, n: int | None = None) -> np.ndarray:
        """All quadruples: float32 [n, 4, H, W]; frame f pairs times f and f+1."""
        n = self.n_frames if n is None else int(n)
        times = [self.render(t) for t in range(n + 1)]
        out = np.empty((n, 4, self.height, self.width), dtype=np.float32)
        for f in range(n):
            out[f, 0], out[f, 1] = times[f][0], times[f][1]
            out[f, 2], out[f, 3] = times[f + 1][0], times[f + 1][1]
        return out


def batch_sizes(n: int = 64, seed: int = 4000) -> list[tuple[int, int]]:
    """Seeded uniform draw of n sizes from {320x240, 640x480, 960x540, 1280x720}."""
    choices = [(320, 240), (640, 480), (960, 540), (1280, 720)]
    rng = np.random.default_rng(seed)
    return [choices[int(i)] for i in rng.integers(0, len(choices), size=n)]
