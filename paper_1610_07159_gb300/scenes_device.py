"""Device (PyTorch, FP64) rendering of the seeded stereo videos of ``scenes``.

The same scenes as ``scenes.SceneVideo`` (its objects, camera rig and value
noise), rendered with tensor operations on a CUDA device so that tens of
thousands of training quadruples for the warm-start network can be made in
seconds. Like ``scenes`` it holds none of the solver's arithmetic. The images
before noise agree with the host renderer to FP64 rounding (tested); the
additive Gaussian noise comes from a seeded device generator, so the noisy
images follow the same distribution but not the same draws.

The value-noise lattice hash is SplitMix64 on unsigned 64-bit words; here the
words live in int64 tensors, whose multiplication and XOR give the same bits,
and logical right shifts are arithmetic shifts with the sign bits masked off.
"""

from __future__ import annotations

import math

import torch

from .scenes import SceneVideo

_U64 = 1 << 64


def _s64(c: int) -> int:
    """An unsigned 64-bit constant as the int64 with the same bits."""
    return c - _U64 if c >= 1 << 63 else c


_M1 = _s64(0xBF58476D1CE4E5B9)
_M2 = _s64(0x94D049BB133111EB)
_GOLD = _s64(0x9E3779B97F4A7C15)
_KX = _s64(0xD1B54A32D192ED03)
_KY = _s64(0xABC98388FB8FAC03)
_KO = _s64(0x8CB92BA72F3D8DD7)


def _srl(z: torch.Tensor, k: int) -> torch.Tensor:
    return (z >> k) & ((1 << (64 - k)) - 1)


def _mix64(z: torch.Tensor) -> torch.Tensor:
    z = (z ^ _srl(z, 30)) * _M1
    z = (z ^ _srl(z, 27)) * _M2
    return z ^ _srl(z, 31)


def _wrap(v: int) -> int:
    v &= _U64 - 1
    return _s64(v)


def _lattice(seed: int, octave: int, ix: torch.Tensor, iy: torch.Tensor) -> torch.Tensor:
    base = _mix64(torch.full_like(ix, _wrap(seed * _GOLD + octave * _KO)))
    h = base ^ (ix * _KX)
    h = _mix64(h)
    h = h ^ (iy * _KY)
    h = _mix64(h)
    return _srl(h, 11).to(torch.float64) * (1.0 / 9007199254740992.0)


def value_noise(u: torch.Tensor, v: torch.Tensor, seed: int, octaves: int = 4, period: float = 32.0,
                lacunarity: float = 2.0, gain: float = 0.5) -> torch.Tensor:
    total = torch.zeros_like(u)
    amp, norm, per = 1.0, 0.0, float(period)
    for o in range(octaves):
        fu, fv = u / per, v / per
        iu, iv = torch.floor(fu), torch.floor(fv)
        tu, tv = fu - iu, fv - iv
        su, sv = tu * tu * (3.0 - 2.0 * tu), tv * tv * (3.0 - 2.0 * tv)
        iu = iu.to(torch.int64)
        iv = iv.to(torch.int64)
        v00 = _lattice(seed, o, iu, iv)
        v10 = _lattice(seed, o, iu + 1, iv)
        v01 = _lattice(seed, o, iu, iv + 1)
        v11 = _lattice(seed, o, iu + 1, iv + 1)
        n = (v00 * (1 - su) + v10 * su) * (1 - sv) + (v01 * (1 - su) + v11 * su) * sv
        total = total + amp * n
        norm += amp
        amp *= gain
        per /= lacunarity
    return total / norm


def render_cameras(video: SceneVideo, views, device, dtype=torch.float64) -> torch.Tensor:
    """Noise-free images [K, H, W] of the views [(t, cam), ...], rendered
    together (one tensor operation per object and step for all views)."""
    K = len(views)
    h, w = video.height, video.width

    def col(vals):  # per-view scalars as a [K, 1, 1] tensor
        return torch.tensor(vals, dtype=dtype, device=device).view(K, 1, 1)

    ys, xs = torch.meshgrid(torch.arange(h, dtype=dtype, device=device), torch.arange(w, dtype=dtype, device=device),
                            indexing="ij")
    ox = col([video.baseline * cam for _, cam in views])
    dx = ((xs - video.cx) / video.f).expand(K, h, w)
    dy = ((ys - video.cy) / video.f).expand(K, h, w)
    zbuf = torch.full((K, h, w), math.inf, dtype=dtype, device=device)
    tu = torch.zeros((K, h, w), dtype=dtype, device=device)
    tv = torch.zeros((K, h, w), dtype=dtype, device=device)
    owner = torch.full((K, h, w), -1, dtype=torch.int64, device=device)
    for k, o in enumerate(video.objects):
        cz = [video._centre(o, float(t)) for t, _ in views]
        c0, c1, c2 = col([c[0] for c, _ in cz]), col([c[1] for c, _ in cz]), col([c[2] for c, _ in cz])
        ppu = col([video.f / z0 for _, z0 in cz])
        if o.kind == "bg":
            zhit = c2.expand(K, h, w)
            X = ox + zhit * dx
            Y = zhit * dy
            a = (X - c0) * ppu
            b = (Y - c1) * ppu
            hit = torch.ones((K, h, w), dtype=torch.bool, device=device)
        elif o.kind == "rect":
            nrm = [o.tilt[0], o.tilt[1], -1.0]
            ln = math.sqrt(sum(x * x for x in nrm))
            n = [x / ln for x in nrm]
            denom = n[0] * dx + n[1] * dy + n[2]
            s = (n[0] * c0 + n[1] * c1 + n[2] * c2 - n[0] * ox) / denom
            X = ox + s * dx
            Y = s * dy
            Z = s
            # e1 = (0, 1, 0) x n, e2 = n x e1
            e1 = [n[2], 0.0, -n[0]]
            l1 = math.sqrt(sum(x * x for x in e1))
            e1 = [x / l1 for x in e1]
            e2 = [n[1] * e1[2] - n[2] * e1[1], n[2] * e1[0] - n[0] * e1[2], n[0] * e1[1] - n[1] * e1[0]]
            angs = [o.rot0 + o.rot_rate * float(t) for t, _ in views]
            ca, sa = col([math.cos(x) for x in angs]), col([math.sin(x) for x in angs])
            r1 = [ca * e1[i] + sa * e2[i] for i in range(3)]
            r2 = [-sa * e1[i] + ca * e2[i] for i in range(3)]
            qx, qy, qz = X - c0, Y - c1, Z - c2
            a = (qx * r1[0] + qy * r1[1] + qz * r1[2]) * ppu
            b = (qx * r2[0] + qy * r2[1] + qz * r2[2]) * ppu
            half = o.size
            hit = (s > 0) & (a.abs() < half * o.aspect) & (b.abs() < half)
            zhit = Z
        else:  # sphere
            r = o.size / ppu
            dd = dx * dx + dy * dy + 1.0
            mx, my, mz = ox - c0, -c1, -c2
            bq = 2.0 * (mx * dx + my * dy + mz)
            cq = mx * mx + my * my + mz * mz - r * r
            disc = bq * bq - 4.0 * dd * cq
            hit = disc > 0
            sq = torch.sqrt(torch.where(hit, disc, torch.zeros_like(disc)))
            s = (-bq - sq) / (2.0 * dd)
            hit = hit & (s > 0)
            X = ox + s * dx
            Y = s * dy
            Z = s
            qx, qy, qz = X - c0, Y - c1, Z - c2
            lon = torch.atan2(qx, -qz) + col([o.rot0 + o.rot_rate * float(t) for t, _ in views])
            lat = torch.asin(torch.clamp(qy / r, -1.0, 1.0))
            a = lon * o.size
            b = lat * o.size
            zhit = Z
        if o.flow_amp > 0:
            a = a + o.flow_amp * torch.sin(2 * math.pi * (b / o.flow_lambda + col([o.flow_rate * float(t) for t, _ in views])))
        closer = hit & (zhit < zbuf)
        zbuf = torch.where(closer, zhit, zbuf)
        tu = torch.where(closer, a, tu)
        tv = torch.where(closer, b, tv)
        owner = torch.where(closer, torch.full_like(owner, k), owner)
    img = torch.zeros((K, h, w), dtype=dtype, device=device)
    for k, o in enumerate(video.objects):
        m = owner == k
        img = torch.where(m, value_noise(tu + 1000.0, tv + 1000.0, o.seed).to(dtype), img)
    return img


def render_camera(video: SceneVideo, t: float, cam: int, device) -> torch.Tensor:
    """Noise-free image of camera ``cam`` at time ``t`` (FP64 [H, W])."""
    return render_cameras(video, [(t, cam)], device)[0]


def frames(video: SceneVideo, n: int, device, noise_seed: int | None = None, dtype=torch.float64) -> torch.Tensor:
    """Quadruples [n, 4, H, W] (float32 on device): frame f pairs times f and f + 1.
    dtype is the rendering precision (FP64 matches the host renderer; FP32 is
    faster and differs by FP32 rounding of the texture coordinates)."""
    views = [(float(t), cam) for t in range(n + 1) for cam in (0, 1)]
    clean = render_cameras(video, views, device, dtype).view(n + 1, 2, video.height, video.width).to(torch.float64)
    g = torch.Generator(device=device)
    g.manual_seed(video.seed if noise_seed is None else int(noise_seed))
    e = torch.randn(clean.shape, generator=g, device=device, dtype=torch.float64)
    noisy = (clean + video.sigma * e).to(torch.float32)
    out = torch.empty((n, 4, video.height, video.width), dtype=torch.float32, device=device)
    out[:, 0:2] = noisy[0:n]
    out[:, 2:4] = noisy[1:n + 1]
    return out


def stereo_pair_quadruple(video: SceneVideo, device, t: float = 0.0, noise_seed: int | None = None,
                          dtype=torch.float32) -> torch.Tensor:
    """A stereo-only quadruple [4, H, W] (float32 on device): the stereo pair
    of time t used at both times (L, R, L, R), as in the paper's experiments on
    still stereo pairs, where the motion and difference flows vanish."""
    clean = render_cameras(video, [(float(t), 0), (float(t), 1)], device, dtype).to(torch.float64)
    g = torch.Generator(device=device)
    g.manual_seed(video.seed if noise_seed is None else int(noise_seed))
    noisy = (clean + video.sigma * torch.randn(clean.shape, generator=g, device=device, dtype=torch.float64))
    pair = noisy.to(torch.float32)
    return torch.stack([pair[0], pair[1], pair[0], pair[1]])
