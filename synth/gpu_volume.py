"""GPU twin of synth.volume for bulk training data.

Same definition as synth/synth.c (Gaussian blobs with SplitMix64-drawn
parameters + smoothstep value noise on hashed lattices, min-max normalised,
uint16 = round(v * 65535)), evaluated with torch in float32 on the device.
Values match the C generator to float32 rounding, not bit for bit; these
volumes only feed the training of the learned-gamma model and are never
compared against the CPU oracle.
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
M1 = np.uint64(0xBF58476D1CE4E5B9)
M2 = np.uint64(0x94D049BB133111EB)


def _mix(x):
    """SplitMix64 output function applied to x + golden gamma (numpy uint64, wrapping)."""
    with np.errstate(over="ignore"):
        z = (np.asarray(x, dtype=np.uint64) + GAMMA).astype(np.uint64)
        z = ((z ^ (z >> np.uint64(30))) * M1).astype(np.uint64)
        z = ((z ^ (z >> np.uint64(27))) * M2).astype(np.uint64)
        return z ^ (z >> np.uint64(31))


def _stream(seed, n):
    """First n outputs of the sequential SplitMix64 stream seeded with `seed`."""
    with np.errstate(over="ignore"):
        states = (np.uint64(seed) + GAMMA * np.arange(1, n + 1, dtype=np.uint64)).astype(np.uint64)
    # the stream's k-th output is the output function of seed + k * gamma, i.e. _mix(seed + (k - 1) * gamma)
    with np.errstate(over="ignore"):
        z = states
        z = ((z ^ (z >> np.uint64(30))) * M1).astype(np.uint64)
        z = ((z ^ (z >> np.uint64(27))) * M2).astype(np.uint64)
        return z ^ (z >> np.uint64(31))


def _u53(h):
    return (np.asarray(h, dtype=np.uint64) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def _hash4(seed, a, b, c):
    h = _mix(np.uint64(seed))
    h = _mix(h ^ np.asarray(a, dtype=np.uint64))
    h = _mix(h ^ np.asarray(b, dtype=np.uint64))
    return _mix(h ^ np.asarray(c, dtype=np.uint64))


def volume(dims, n_blobs: int, octaves: int, seed: int, device="cuda", noise_amp: float = 0.1,
           base_freq: float = 4.0):
    """uint16 volume (as a torch.int16 tensor of shape (Z, Y, X)) on `device`."""
    import torch

    X, Y, Z = (int(d) for d in dims)
    r = _u53(_stream(seed, 6 * n_blobs)).reshape(n_blobs, 6)
    cen = torch.tensor(r[:, 0:3], dtype=torch.float32, device=device)
    sig = torch.tensor(0.03 + 0.12 * r[:, 3:6], dtype=torch.float32, device=device)

    def axis(n, a):
        u = torch.arange(n, dtype=torch.float32, device=device) / (n - 1)
        d = u[None, :] - cen[:, a:a + 1]
        return torch.exp(-d * d / (2 * sig[:, a:a + 1] ** 2))

    gx, gy, gz = axis(X, 0), axis(Y, 1), axis(Z, 2)
    vol = torch.einsum("bz,by,bx->zyx", gz, gy, gx) if n_blobs else torch.zeros((Z, Y, X), device=device)
    amp = 1.0
    for o in range(octaves):
        f = int(base_freq * (1 << o) + 0.5)
        ii = np.arange(f + 1, dtype=np.uint64)
        k3, j3, i3 = np.meshgrid(ii, ii, ii, indexing="ij")
        lat = _u53(_hash4(np.uint64(seed) ^ np.uint64(0x6e6f697365), np.uint64(o), i3 | (j3 << np.uint64(21)), k3))
        L = torch.tensor(lat, dtype=torch.float32, device=device)

        def idx(n):
            u = torch.arange(n, dtype=torch.float32, device=device) / (n - 1) * f
            i = torch.clamp(torch.floor(u), max=f - 1)
            t = u - i
            return i.long(), t * t * (3 - 2 * t)

        ix, sx = idx(X)
        iy, sy = idx(Y)
        iz, sz = idx(Z)
        acc = torch.zeros((Z, Y, X), dtype=torch.float32, device=device)
        for dz in (0, 1):
            wz = (sz if dz else 1 - sz)[:, None, None]
            for dy in (0, 1):
                wy = (sy if dy else 1 - sy)[None, :, None]
                for dx in (0, 1):
                    wx = (sx if dx else 1 - sx)[None, None, :]
                    acc += wz * wy * wx * L[(iz + dz)[:, None, None], (iy + dy)[None, :, None], (ix + dx)[None, None, :]]
        vol += noise_amp * amp * acc
        amp *= 0.5
    lo, hi = vol.min(), vol.max()
    v = (vol - lo) / torch.clamp(hi - lo, min=1e-30)
    u = torch.floor(v * 65535.0 + 0.5).clamp(0, 65535).to(torch.int32)
    return (u - 65536 * (u > 32767).int()).to(torch.int16)  # the uint16 bit pattern
