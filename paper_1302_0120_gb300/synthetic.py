"""Seeded synthetic inputs: spot-pattern stimulation targets and initial phases.

The paper benchmarks on bright spots on a dark background (Sec. IV, Fig. 3);
no dataset is involved. This module renders such targets and draws initial
phases from a seeded PCG64 generator. It holds none of the method's
arithmetic, so both the CUDA path and the CPU oracle may be fed from it.

Recipe (stated once, used everywhere):
  * Spots are isotropic Gaussians of width ``sigma`` (1.5 px) truncated at a
    toroidal distance of ``4 sigma`` (6 px); overlapping spots combine by max.
  * Spot centres are integer pixels drawn uniformly on the torus, rejected when
    closer than ``4 sigma + 1`` (7 px) to the zero-frequency pixel, so that no
    spot touches DC.
  * Arrays are laid out ``[ny, nx]`` in DFT order (zero frequency at [0, 0]),
    float32, intensity >= 0.
  * Initial phases are uniform in [0, 2 pi), float32.
"""

from __future__ import annotations

import numpy as np

SIGMA = 1.5
CUTOFF = 4.0 * SIGMA  # 6 px
DC_CLEARANCE = CUTOFF + 1.0  # 7 px


def _torus_dist2(dy, dx, ny, nx):
    dy = np.minimum(np.abs(dy) % ny, ny - np.abs(dy) % ny)
    dx = np.minimum(np.abs(dx) % nx, nx - np.abs(dx) % nx)
    return dy * dy + dx * dx


def spot_centres(rng: np.random.Generator, nspots: int, ny: int, nx: int) -> np.ndarray:
    """``nspots`` integer centres (y, x) on the torus, none within 7 px of DC."""
    out = []
    guard = 0
    while len(out) < nspots:
        guard += 1
        if guard > 1000 * (nspots + 10):
            raise RuntimeError("could not place spots away from DC")
        y = int(rng.integers(0, ny))
        x = int(rng.integers(0, nx))
        if _torus_dist2(np.array(y), np.array(x), ny, nx) < DC_CLEARANCE ** 2:
            continue
        out.append((y, x))
    return np.asarray(out, dtype=np.int64).reshape(-1, 2)


def render_spots(centres: np.ndarray, amps, ny: int, nx: int, sigma: float = SIGMA) -> np.ndarray:
    """Render max-combined truncated Gaussian spots into a float32 [ny, nx] array."""
    img = np.zeros((ny, nx), dtype=np.float64)
    r = int(np.floor(4.0 * sigma))
    d = np.arange(-r, r + 1)
    dy, dx = np.meshgrid(d, d, indexing="ij")
    d2 = (dy * dy + dx * dx).astype(np.float64)
    keep = d2 <= (4.0 * sigma) ** 2
    amps = np.broadcast_to(np.asarray(amps, dtype=np.float64), (len(centres),))
    for (cy, cx), a in zip(centres, amps):
        val = a * np.exp(-d2 / (2.0 * sigma * sigma))
        yy = (cy + dy) % ny
        xx = (cx + dx) % nx
        cur = img[yy[keep], xx[keep]]
        img[yy[keep], xx[keep]] = np.maximum(cur, val[keep])
    return img.astype(np.float32)


def spot_target(seed: int, ny: int, nx: int, nspots: int, amp_range=(1.0, 1.0)) -> np.ndarray:
    """A spot-pattern target intensity (float32, DFT order) from ``seed``.

    ``amp_range=(1, 1)`` gives unit peaks; ``(0.5, 1)`` draws peaks uniformly.
    """
    rng = np.random.default_rng(seed)
    c = spot_centres(rng, nspots, ny, nx)
    lo, hi = amp_range
    a = np.full(nspots, lo) if lo == hi else rng.uniform(lo, hi, size=nspots)
    return render_spots(c, a, ny, nx)


def random_phase(seed: int, ny: int, nx: int) -> np.ndarray:
    """Uniform initial phase in [0, 2 pi), float32, from its own seeded stream."""
    rng = np.random.default_rng([seed, 0x5EED])
    return (rng.random((ny, nx)) * (2.0 * np.pi)).astype(np.float32)


def siemens_star(ny: int, nx: int, spokes: int = 36, radius_frac: float = 0.4) -> np.ndarray:
    """The resolution target of Sec. IV: a Siemens star with ``spokes`` dark
    and ``spokes`` lit sectors inside a disc of radius ``radius_frac * min(ny, nx)``,
    centred on the grid centre and then moved to DFT order (centre at [0, 0]).
    Intensity 1 (lit) or 0, float32."""
    y = (np.arange(ny) - ny // 2)[:, None].astype(np.float64)
    x = (np.arange(nx) - nx // 2)[None, :].astype(np.float64)
    r = np.hypot(x, y)
    th = np.arctan2(y, x)
    star = (np.sin(spokes * th) > 0) & (r < radius_frac * min(ny, nx))
    return np.fft.ifftshift(star.astype(np.float32))


def laser_amplitude(ny: int, nx: int, waist_frac: float = 0.45, floor: float = 0.01) -> np.ndarray:
    """A Gaussian beam profile on the SLM (the amplitude p of the SLM set S),
    exp(-(r / w)^2) with w = waist_frac * size along each axis, plus a floor;
    float32 [ny, nx]."""
    y = (np.arange(ny) - ny / 2)[:, None] / (waist_frac * ny)
    x = (np.arange(nx) - nx / 2)[None, :] / (waist_frac * nx)
    return (np.exp(-(x * x + y * y)) + floor).astype(np.float32)


def neuron_positions(seed: int, count: int, ny: int, nx: int) -> np.ndarray:
    """A fixed set of ``count`` neuron positions for request streams."""
    rng = np.random.default_rng([seed, 0xCE11])
    return spot_centres(rng, count, ny, nx)


# Named workloads: grid, spot count, peak range, iterations.
WORKLOADS = {
    "spots64": dict(ny=64, nx=64, nspots=5, amp_range=(1.0, 1.0), iters=20),
    "spots512": dict(ny=512, nx=512, nspots=50, amp_range=(0.5, 1.0), iters=100),
    "spots1024": dict(ny=1024, nx=1024, nspots=50, amp_range=(0.5, 1.0), iters=100),
}


def mixed_batch(seed: int, count: int = 64, sizes=(256, 512, 1024), spots=(10, 200)):
    """``count`` masks of mixed size: each size drawn uniformly from ``sizes``
    and each spot count uniformly from ``spots[0]..spots[1]``; peaks U[0.5, 1].
    Returns a list of ``(I, phi0)``."""
    rng = np.random.default_rng([seed, 0xB47C])
    out = []
    for k in range(count):
        n = int(sizes[int(rng.integers(0, len(sizes)))])
        ns = int(rng.integers(spots[0], spots[1] + 1))
        out.append((spot_target(1000 * seed + k, n, n, ns, (0.5, 1.0)), random_phase(1000 * seed + k, n, n)))
    return out


def workload(name: str, seed: int = 0):
    """Return ``(I, phi0, iters)`` for a named workload."""
    w = WORKLOADS[name]
    I = spot_target(seed, w["ny"], w["nx"], w["nspots"], w["amp_range"])
    phi0 = random_phase(seed, w["ny"], w["nx"])
    return I, phi0, w["iters"]
