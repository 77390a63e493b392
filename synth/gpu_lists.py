"""GPU twin of synth.lists_compact / synth.one_list for full-size workloads.

Bit-identical to synth/synth.c: SplitMix64 in torch int64 arithmetic
(multiplication wraps mod 2^64; right shifts are masked to act as logical
shifts), draws as exact 24-bit floats, sorting, and single float
multiplications for the premultiplied colour.  Used to build device-resident
inputs too large to generate on the host; any pixel can be regenerated on the
host with synth.one_list for the oracle.
"""
from __future__ import annotations

import numpy as np

_G = np.uint64(0x9E3779B97F4A7C15).astype(np.int64).item()
_M1 = np.uint64(0xBF58476D1CE4E5B9).astype(np.int64).item()
_M2 = np.uint64(0x94D049BB133111EB).astype(np.int64).item()


def _i64(x: int) -> int:
    return np.uint64(x & 0xFFFFFFFFFFFFFFFF).astype(np.int64).item()


def _srl(z, s):
    """logical right shift of an int64 tensor"""
    return (z >> s) & ((1 << (64 - s)) - 1)


def mix(z):
    """SplitMix64 output function of z + golden gamma (torch int64, elementwise)."""
    z = z + _G
    z = (z ^ _srl(z, 30)) * _M1
    z = (z ^ _srl(z, 27)) * _M2
    return z ^ _srl(z, 31)


def _mix_scalar(x: int) -> int:
    with np.errstate(over="ignore"):
        z = (np.uint64(x & 0xFFFFFFFFFFFFFFFF) + np.uint64(0x9E3779B97F4A7C15)).astype(np.uint64)
        z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)).astype(np.uint64)
        z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)).astype(np.uint64)
        return int(z ^ (z >> np.uint64(31)))


def _u24(h):
    import torch

    return _srl(h, 40).to(torch.float32) * (1.0 / 16777216.0)


def list_keys(seed: int, req: int, set_: int, pixels):
    """synth_hash4(seed, (req << 32) | set, pixel, 0x6c697374) for an int64 tensor of pixel indices."""
    import torch

    h = _mix_scalar(seed)
    h = _mix_scalar(h ^ ((req << 32) | set_))
    z = mix(pixels.to(torch.int64) ^ _i64(h))
    return mix(z ^ 0x6c697374)


def lengths(seed, req, set_, pixels, n_s, dense=False):
    """List lengths: n_s when dense, else the key's hash mod (n_s + 1)."""
    import torch

    if dense:
        return torch.full(pixels.shape, n_s, dtype=torch.int32, device=pixels.device)
    key = list_keys(seed, req, set_, pixels)
    return _mod_u64(mix(key ^ 0x4c454e47), n_s + 1)


def _mod_u64(z, m, m_tensor=None):
    """unsigned 64-bit z mod m (m small, or the int64 tensor m_tensor) for an int64 tensor holding the bits of z"""
    import torch

    hi = _srl(z, 32)
    lo = z & 0xFFFFFFFF
    if m_tensor is not None:
        m = m_tensor
        r32 = torch.remainder(torch.full_like(m, 1 << 32), m)
        return ((torch.remainder(hi, m) * r32 + torch.remainder(lo, m)) % m).to(torch.int32)
    return ((torch.remainder(hi, m) * ((1 << 32) % m) + torch.remainder(lo, m)) % m).to(torch.int32)


def lists(seed, req, set_, pixels, n_s, dense=False):
    """(counts int32 [P], fb float32 [P, n_s, 2], rgba float32 [P, n_s, 4]); slots past a list's length are 0."""
    import torch

    P = pixels.shape[0]
    dev = pixels.device
    cnt = lengths(seed, req, set_, pixels, n_s, dense)
    key = list_keys(seed, req, set_, pixels)
    j = torch.arange(2 * n_s, dtype=torch.int64, device=dev)
    t = _u24(mix(key[:, None] + (2 * j[None, :] + 1)))
    valid = j[None, :] < (2 * cnt[:, None]).long()
    t = torch.where(valid, t, torch.full_like(t, 2.0))  # beyond the list: sort last
    t, _ = torch.sort(t, dim=1)
    fb = t.view(P, n_s, 2)
    i = torch.arange(n_s, dtype=torch.int64, device=dev)
    kc = mix(key[:, None] ^ (0x636f6c6f + 8 * i[None, :]))
    A = _u24(kc)
    r, g, b = _u24(mix(kc + 1)), _u24(mix(kc + 2)), _u24(mix(kc + 3))
    rgba = torch.stack([A * r, A * g, A * b, A], dim=-1)
    keep = (i[None, :] < cnt[:, None].long())
    fb = torch.where(keep[..., None], fb, torch.zeros_like(fb))
    rgba = torch.where(keep[..., None], rgba, torch.zeros_like(rgba))
    return cnt, fb, rgba


def pool_picks(seed, req, set_, pixels, n_s, runs):
    """(n int32, first record index int64 = run * 64 + start) of pooled lists; twin of synth.pool_pick."""
    import torch

    n = lengths(seed, req, set_, pixels, n_s, dense=False)
    key = list_keys(seed, req, set_, pixels)
    run = _mod_u64_big(mix(key ^ 0x706f6f6c), runs)
    start = _mod_u64(mix(key ^ 0x73747274), None, m_tensor=(64 - n + 1).to(torch.int64))
    return n, run * 64 + start.to(torch.int64)


def _mod_u64_big(z, m):
    """unsigned 64-bit z mod m for m < 2^31 (int64 result)"""
    import torch

    hi = _srl(z, 32)
    lo = z & 0xFFFFFFFF
    return (torch.remainder(hi, m) * ((1 << 32) % m) + torch.remainder(lo, m)) % m


def pool(seed, runs, chunk=1 << 19, device="cuda"):
    """Record pool of the pooled lists: (fb float32 [runs * 64, 2], rgba float32 [runs * 64, 4]); run r is
    one_list(seed, POOL_REQ, 0, r, 64, dense=True)."""
    import torch

    from synth import POOL_REQ, POOL_RUN

    fb = torch.empty((runs * POOL_RUN, 2), dtype=torch.float32, device=device)
    rgba = torch.empty((runs * POOL_RUN, 4), dtype=torch.float32, device=device)
    for r0 in range(0, runs, chunk):
        r1 = min(runs, r0 + chunk)
        pix = torch.arange(r0, r1, dtype=torch.int64, device=device)
        _, f, c = lists(seed, POOL_REQ, 0, pix, POOL_RUN, dense=True)
        fb[r0 * POOL_RUN:r1 * POOL_RUN] = f.reshape(-1, 2)
        rgba[r0 * POOL_RUN:r1 * POOL_RUN] = c.reshape(-1, 4)
    return fb, rgba


def dense_set(seed, req, set_, npix, n_s, chunk=1 << 20, device="cuda"):
    """Dense compact lists of one (request, set) over pixels [0, npix): (counts int32 [npix],
    offsets int64 [npix + 1] = p * n_s, fb float32 [npix * n_s, 2], rgba float32 [npix * n_s, 4])."""
    import torch

    counts = torch.full((npix,), n_s, dtype=torch.int32, device=device)
    offsets = torch.arange(npix + 1, dtype=torch.int64, device=device) * n_s
    fb = torch.empty((npix * n_s, 2), dtype=torch.float32, device=device)
    rgba = torch.empty((npix * n_s, 4), dtype=torch.float32, device=device)
    for p0 in range(0, npix, chunk):
        p1 = min(npix, p0 + chunk)
        pix = torch.arange(p0, p1, dtype=torch.int64, device=device)
        _, f, c = lists(seed, req, set_, pix, n_s, dense=True)
        fb[p0 * n_s:p1 * n_s] = f.reshape(-1, 2)
        rgba[p0 * n_s:p1 * n_s] = c.reshape(-1, 4)
    return counts, offsets, fb, rgba


def pack_f16(fb, rgba, chunk=1 << 24):
    """16-byte records {float32 f, float32 b, float16 R, G, B, tau} as int32 [n, 4]: premultiplied colour
    and the optical depth tau = -log2(1 - A) (+inf for A = 1), computed in float32 (1 - A is exact for
    A in [0, 1]) and rounded to nearest even."""
    import torch

    n = fb.shape[0]
    out = torch.empty((n, 4), dtype=torch.int32, device=fb.device)
    for i0 in range(0, n, chunk):
        i1 = min(n, i0 + chunk)
        c = rgba[i0:i1].clone()
        c[:, 3] = -torch.log2(1.0 - c[:, 3])
        out[i0:i1, 0:2] = fb[i0:i1].view(torch.int32)
        out[i0:i1, 2:4] = c.to(torch.float16).contiguous().view(torch.int32)
    return out
