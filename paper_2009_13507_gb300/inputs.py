"""Seeded synthetic inputs shared by the CUDA path's tests/benchmark and the oracle.

This module holds none of the method's arithmetic: it only draws random numbers
and lays out initial wave functions and instance tables, which both sides
receive as plain arrays.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): state += 0x9E3779B97F4A7C15,
then two xor-shift-multiply rounds; a double in [0, 1) is the top 53 bits
times 2^-53.

Initial states follow the workloads of the paper's 1D and 2D runs (Sec. 4:
Gaussian initial functions on grids x_i = (i - N/2) dx).
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int) -> np.ndarray:
    """n consecutive SplitMix64 outputs for the given 64-bit seed."""
    with np.errstate(over="ignore"):
        k = np.arange(1, n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, n: int) -> np.ndarray:
    """n doubles in [0, 1)."""
    return (splitmix64(seed, n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def grid_x(n: int, h: float) -> np.ndarray:
    """Grid coordinates x_i = (i - n//2) h, i = 0..n-1."""
    return (np.arange(n) - n // 2) * h


def _unit(psi: np.ndarray, cell: float) -> np.ndarray:
    return psi / np.sqrt(np.sum(np.abs(psi) ** 2) * cell)


def gaussian_jitter_1d(nx: int, dx: float, seed: int, amp: float = 1e-3, width: float = 1.0) -> np.ndarray:
    """[3][1][nx] complex128: exp(-x^2/(2 w^2)) in every component, times
    (1 + amp (u1 + i u2)) with u ~ U[-1, 1) per point and component; unit norm."""
    x = grid_x(nx, dx)
    u = uniform(seed, 2 * 3 * nx).reshape(2, 3, 1, nx) * 2.0 - 1.0
    g = np.exp(-x**2 / (2.0 * width**2))[None, None, :]
    psi = g * (1.0 + amp * (u[0] + 1j * u[1]))
    return _unit(psi.astype(np.complex128), dx)


def gaussian_phase_2d(nx: int, ny: int, dx: float, dy: float, seed: int, width: float = 1.0) -> np.ndarray:
    """[3][ny][nx] complex128: exp(-r^2/(2 w^2)) exp(i phi_j), phi_j ~ U[0, 2 pi) per component; unit norm."""
    x = grid_x(nx, dx)[None, :]
    y = grid_x(ny, dy)[:, None]
    phi = uniform(seed, 3) * 2.0 * np.pi
    g = np.exp(-(x**2 + y**2) / (2.0 * width**2))
    psi = g[None, :, :] * np.exp(1j * phi)[:, None, None]
    return _unit(psi.astype(np.complex128), dx * dy)


def random_state(shape, seed: int, cell: float, envelope: float = 0.0) -> np.ndarray:
    """Complex field with independent U[-1,1) real and imaginary parts per entry,
    optionally times a Gaussian envelope exp(-envelope * (i/n - 1/2)^2) per axis; unit norm."""
    shape = tuple(shape)
    n = int(np.prod(shape))
    u = uniform(seed, 2 * n).reshape((2,) + shape) * 2.0 - 1.0
    psi = u[0] + 1j * u[1]
    if envelope:
        for ax in range(1, len(shape)):
            m = shape[ax]
            t = (np.arange(m) + 0.5) / m - 0.5
            s = [1] * len(shape)
            s[ax] = m
            psi = psi * np.exp(-envelope * t**2).reshape(s)
    return _unit(psi.astype(np.complex128), cell)


def gaussian_target(nx: int, ny: int, dx: float, dy: float, seed: int) -> np.ndarray:
    """[ny][nx] float64 target density: a Gaussian of width w ~ U[0.8, 1.2] centred at
    (x0, y0) ~ U[-0.5, 0.5]^2 (y0 = 0 in 1D, ny = 1), normalised to unit integral."""
    u = uniform(seed, 3)
    w, x0, y0 = 0.8 + 0.4 * u[0], u[1] - 0.5, (u[2] - 0.5 if ny > 1 else 0.0)
    x = grid_x(nx, dx)[None, :]
    y = grid_x(ny, dy)[:, None] if ny > 1 else np.zeros((1, 1))
    rho = np.exp(-((x - x0) ** 2 + (y - y0) ** 2) / (w * w))
    return rho / (rho.sum() * dx * (dy if ny > 1 else 1.0))


def batch_table(seed: int, n1d: int = 32, n2d: int = 32):
    """Instance table of a batched workload: n1d 1D instances with nx ~ U{128..1024},
    n2d 2D instances n x n with n ~ U{128..384}; per instance
    (gamma, Omega, c0, c2) ~ U[0,1] x U[0,1] x U[1,100] x U[-2,2]."""
    m = n1d + n2d
    u = uniform(seed, 5 * m).reshape(m, 5)
    out = []
    for i in range(m):
        dim = 1 if i < n1d else 2
        if dim == 1:
            n = 128 + int(u[i, 0] * (1024 - 128 + 1))
        else:
            n = 128 + int(u[i, 0] * (384 - 128 + 1))
        out.append(dict(dim=dim, nx=n, ny=(n if dim == 2 else 1), gamma=float(u[i, 1]),
                        omega=float(u[i, 2]), c0=1.0 + 99.0 * float(u[i, 3]),
                        c2=-2.0 + 4.0 * float(u[i, 4])))
    return out


def vortex_state_2d(nx: int, ny: int, dx: float, dy: float, charges, width: float = 2.0,
                    amplitudes=(1.0, 1.0, 1.0)) -> np.ndarray:
    """[3][ny][nx] complex128 initial state with a vortex of angular momentum L_j
    imprinted in component j (Sec. 4's initial states): a Gaussian of the given
    width times (x + i y)^L for L > 0 and (x - i y)^|L| for L < 0, times
    amplitudes[j]; unit norm. E.g. charges (-1, 0, 1) for the polar and (0, 1, 2)
    for the ferromagnetic Rashba-coupled states."""
    x = grid_x(nx, dx)[None, :]
    y = grid_x(ny, dy)[:, None]
    g = np.exp(-(x**2 + y**2) / (2.0 * width**2))
    comps = []
    for L, a in zip(charges, amplitudes):
        z = x + 1j * y if L >= 0 else x - 1j * y
        comps.append(a * g * z ** abs(int(L)))
    psi = np.stack([np.broadcast_to(c, (ny, nx)) for c in comps]).astype(np.complex128)
    return _unit(psi, dx * dy)


def stripe_state_2d(nx: int, ny: int, dx: float, dy: float, gamma: float, width: float = 2.0) -> np.ndarray:
    """[3][ny][nx] complex128 stripe initial state (Sec. 4): a Gaussian times
    sin(gamma x) in the components +1 and -1 and cos(gamma x) in component 0; unit norm."""
    x = grid_x(nx, dx)[None, :]
    y = grid_x(ny, dy)[:, None]
    g = np.exp(-(x**2 + y**2) / (2.0 * width**2))
    s, c = g * np.sin(gamma * x), g * np.cos(gamma * x)
    psi = np.stack([s, c, s]).astype(np.complex128)
    return _unit(psi, dx * dy)
