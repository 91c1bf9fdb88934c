"""Seeded synthetic trajectories and signals.

These stand in for the LAMMPS trajectories of Sec. 2.1 (SPC/E water with 6720
to 26880 molecules, 3500 frames; a 2x10^6-point pressure-tensor series), which
are not available.  Nothing here computes an MSD, a correlation or an
integral: the module only draws inputs.  Both the CUDA path and the FP64
oracle are fed the same float32 arrays made here.

Recipes (all draws from one seeded generator per call; base seed 1708086,
instance i of a batch uses base + i):

* positions: start uniform in [0, box)^3, plus a Gaussian random walk with
  step sigma per axis per frame, summed in FP64 and cast to float32 once.
  With ``sites_per_molecule=3`` atoms 3m, 3m+1, 3m+2 share molecule m's walk
  and carry fixed site offsets uniform in [-0.1, 0.1) nm (rigid 3-site
  molecules; the last molecule may have fewer sites).
* velocities: exact discretisation of an Ornstein-Uhlenbeck process per axis,
  phi = exp(-gamma), v_0 ~ N(0, sigma^2), v_{t+1} = phi v_t +
  sigma sqrt(1 - phi^2) xi_t.  Stationary, with C(tau) = 3 sigma^2 phi^tau.
* flux: the same recursion with a given phi and unit variance, shape
  [T][1][3] (three off-diagonal pressure components).
* constant velocity: x_t = x_0 + v t with x_0 and v multiples of 2^-10, so
  every value is exact in float32 for t up to a few thousand.
"""
from __future__ import annotations

import math

import numpy as np

BASE_SEED = 1708086


# ----------------------------------------------------------------- host (numpy)

def random_walk_positions(T: int, N: int, sigma: float, box: float, seed: int,
                          sites_per_molecule: int = 1,
                          site_offset: float = 0.1) -> np.ndarray:
    rng = np.random.default_rng(seed)
    nmol = -(-N // sites_per_molecule)
    start = rng.uniform(0.0, box, size=(nmol, 3))
    steps = rng.normal(0.0, sigma, size=(T, nmol, 3))
    steps[0] = 0.0
    walk = np.cumsum(steps, axis=0)
    walk += start[None]
    if sites_per_molecule > 1:
        offsets = rng.uniform(-site_offset, site_offset, size=(N, 3))
        mol = np.arange(N) // sites_per_molecule
        walk = walk[:, mol, :] + offsets[None]
    return np.ascontiguousarray(walk, dtype=np.float32)


def ou_velocities(T: int, N: int, gamma: float, sigma: float, seed: int) -> np.ndarray:
    from scipy.signal import lfilter
    rng = np.random.default_rng(seed)
    phi = math.exp(-gamma)
    kick = sigma * math.sqrt(1.0 - phi * phi)
    v = np.empty((T, N, 3), dtype=np.float64)
    v[0] = rng.normal(0.0, sigma, size=(N, 3))
    if T > 1:
        xi = rng.normal(0.0, 1.0, size=(T - 1, N, 3))
        # v[t] = phi v[t-1] + kick xi[t-1], started from v[0]
        v[1:] = lfilter([kick], [1.0, -phi], xi, axis=0, zi=(phi * v[0])[None])[0]
    return np.ascontiguousarray(v, dtype=np.float32)


def ar1_flux(T: int, phi: float, seed: int, ncomp_atoms: int = 1) -> np.ndarray:
    gamma = -math.log(phi)
    return ou_velocities(T, ncomp_atoms, gamma, 1.0, seed)


def constant_velocity(T: int, N: int, seed: int, vmax_units: int = 8,
                      x0_units: int = 4096) -> tuple[np.ndarray, np.ndarray]:
    """Dyadic x_t = x_0 + v t; returns (x[T][N][3] float32, v[N][3] float64)."""
    rng = np.random.default_rng(seed)
    q = 2.0 ** -10
    v = rng.integers(-vmax_units, vmax_units + 1, size=(N, 3)).astype(np.float64) * q
    x0 = rng.integers(-x0_units, x0_units + 1, size=(N, 3)).astype(np.float64) * q
    t = np.arange(T, dtype=np.float64)[:, None, None]
    x = x0[None] + v[None] * t
    x32 = x.astype(np.float32)
    if not np.array_equal(x32.astype(np.float64), x):
        raise ValueError("constant-velocity trajectory is not exact in float32")
    return x32, v


def batch_workload_shapes(count: int = 256, seed: int = BASE_SEED + 4):
    """Shapes of the uneven batching workload: instance i has N log-uniform in
    [64, 16384], T uniform in [500, 20000], tau_max = T // 4, stride 1; even
    instances are MSDs of random walks (sigma 0.01, 3 nm box), odd ones
    autocorrelations of OU velocities with gamma uniform in [0.01, 0.5].
    Returns a list of (kind, T, N, tau_max, stride, gamma); instance i's data
    is drawn with seed BASE_SEED + i."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        N = int(round(np.exp(rng.uniform(np.log(64), np.log(16384)))))
        Tn = int(rng.integers(500, 20001))
        gamma = float(rng.uniform(0.01, 0.5))
        out.append((i % 2, Tn, N, Tn // 4, 1, gamma))
    return out


def batch_instance_device(i: int, shape, device="cuda"):
    """Instance i of the batching workload drawn on the device (see
    batch_workload_shapes)."""
    kind, Tn, N, tm, s, gamma = shape
    if kind == 0:
        return random_walk_positions_device(Tn, N, 0.01, 3.0, BASE_SEED + i, device=device)
    return ou_velocities_device(Tn, N, gamma, 1.0, BASE_SEED + i, device=device)


# ------------------------------------------------------------- device (torch)

def _torch():
    import torch  # local import: the host generators above need no torch
    return torch


def random_walk_positions_device(T: int, N: int, sigma: float, box: float, seed: int,
                                 device="cuda", sites_per_molecule: int = 1,
                                 site_offset: float = 0.1, chunk_atoms: int = 8192):
    """Same recipe as ``random_walk_positions`` drawn with torch's device RNG.

    The numbers differ from the numpy version (another generator); the recipe
    is the same.  Summed in FP64 chunk by chunk over molecules, so the peak
    extra device memory is T * chunk_atoms * 3 doubles.
    """
    torch = _torch()
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    nmol = -(-N // sites_per_molecule)
    out = torch.empty((T, N, 3), dtype=torch.float32, device=device)
    offsets = None
    if sites_per_molecule > 1:
        offsets = (torch.rand((N, 3), generator=g, device=device, dtype=torch.float64)
                   * 2.0 - 1.0) * site_offset
    for m0 in range(0, nmol, chunk_atoms):
        m1 = min(nmol, m0 + chunk_atoms)
        start = torch.rand((m1 - m0, 3), generator=g, device=device, dtype=torch.float64) * box
        steps = torch.randn((T, m1 - m0, 3), generator=g, device=device, dtype=torch.float64) * sigma
        steps[0] = 0.0
        walk = torch.cumsum(steps, dim=0)
        walk += start[None]
        if sites_per_molecule > 1:
            a0 = m0 * sites_per_molecule
            a1 = min(N, m1 * sites_per_molecule)
            mol = torch.arange(a0, a1, device=device) // sites_per_molecule - m0
            out[:, a0:a1, :] = (walk[:, mol, :] + offsets[None, a0:a1]).to(torch.float32)
        else:
            out[:, m0:m1, :] = walk.to(torch.float32)
        del steps, walk
    return out


def ou_velocities_device(T: int, N: int, gamma: float, sigma: float, seed: int,
                         device="cuda"):
    """Exact OU recursion (see module docstring) with torch's device RNG.

    Frames are drawn in blocks of B: within a block
    v[k] = phi^k (phi v_prev + kick * sum_{j<=k} phi^-j xi[j]),
    with B small enough that phi^-B stays below 1e6.
    """
    torch = _torch()
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    phi = math.exp(-gamma)
    kick = sigma * math.sqrt(1.0 - phi * phi)
    out = torch.empty((T, N, 3), dtype=torch.float32, device=device)
    v = torch.randn((N, 3), generator=g, device=device, dtype=torch.float64) * sigma
    out[0] = v.to(torch.float32)
    B = int(max(1, min(512, math.floor(math.log(1e6) / max(gamma, 1e-12)))))
    for t0 in range(1, T, B):
        b = min(B, T - t0)
        xi = torch.randn((b, N, 3), generator=g, device=device, dtype=torch.float64)
        k = torch.arange(b, device=device, dtype=torch.float64)
        xi.mul_((phi ** (-k)).view(b, 1, 1))
        torch.cumsum(xi, dim=0, out=xi)
        xi.mul_(kick).add_(phi * v)
        xi.mul_((phi ** k).view(b, 1, 1))
        out[t0:t0 + b] = xi.to(torch.float32)
        v = xi[-1].clone()
        del xi
    return out
