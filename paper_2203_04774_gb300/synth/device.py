"""Device-side generation of the large seeded inputs (torch on CUDA).

Same draws as the host generators: the splitmix64 counter stream of
``synth.counter_u64`` (computed here with wrapping int64 arithmetic, logical
shifts emulated by masks) and the same inverse-CDF search over the same
float64 cumulative weights, so ``chung_lu_device(...)`` equals
``chung_lu(...)`` element for element.  Used for graphs too large to build
on the host (the 2-billion-edge Chung-Lu workload).
"""
from __future__ import annotations

import numpy as np

from . import GAMMA, _stream_key, chung_lu_weights

_MASK = (1 << 64) - 1


def _s64(x: int) -> int:
    """Two's-complement int64 value of a uint64 constant."""
    x &= _MASK
    return x - (1 << 64) if x >= (1 << 63) else x


def _lsr(x, k: int):
    """Logical right shift of an int64 tensor."""
    return (x >> k) & ((1 << (64 - k)) - 1)


def mix64_t(z):
    z = (z ^ _lsr(z, 30)) * _s64(0xBF58476D1CE4E5B9)
    z = (z ^ _lsr(z, 27)) * _s64(0x94D049BB133111EB)
    return z ^ _lsr(z, 31)


def counter_uniform_t(seed: int, stream: int, count: int, start: int, device):
    import torch
    key = _s64(int(_stream_key(seed, stream)))
    i = torch.arange(start + 1, start + count + 1, dtype=torch.int64, device=device)
    z = mix64_t(i * _s64(GAMMA) + key)
    return _lsr(z, 11).to(torch.float64) * (1.0 / (1 << 53))


def chung_lu_device(n: int, avg_deg: float, gamma: float, seed: int, device="cuda",
                    block: int = 1 << 26):
    """Chung-Lu edge list on the device: int32 tensor [M, 2] holding uint32 ids."""
    import torch
    w = chung_lu_weights(n, avg_deg, gamma)
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    cdf_t = torch.from_numpy(cdf).to(device)
    del w, cdf
    m = int(round(n * avg_deg / 2.0))
    out = torch.empty((m, 2), dtype=torch.int32, device=device)
    for col in (0, 1):
        for s in range(0, m, block):
            c = min(block, m - s)
            u = counter_uniform_t(seed, col, c, s, device)
            idx = torch.searchsorted(cdf_t, u, right=True)
            idx.clamp_(max=n - 1)
            out[s:s + c, col] = idx.to(torch.int32)
            del u, idx
    return out
