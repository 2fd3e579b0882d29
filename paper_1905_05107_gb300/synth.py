"""Seeded synthetic snapshot matrices (inputs only, no POD arithmetic).

Both the CUDA path and the FP64 oracle consume the arrays made here; this
module holds none of the method's steps.  The paper's datasets (Faces, the
V_2D CFD velocities, the cropped and full Yale faces; Sec. 1) are not
available, so these stand in for them with the same shape class (tall, thin,
row-mean-centred snapshot matrices) and a spectrum that is known by
construction.

All randomness comes from ``numpy.random.default_rng(seed)`` (PCG64).  Every
matrix is column-major in the sense of the library: column j is snapshot j.
The arrays returned are C-contiguous (n, m) buffers viewed as (m, n) with
``.T``, i.e. Fortran order, so each snapshot is contiguous in memory.
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass
from typing import Optional

import numpy as np


def haar(rng: np.random.Generator, rows: int, cols: int) -> np.ndarray:
    """Haar-distributed orthonormal columns: Q of a Gaussian matrix with the
    sign of diag(R) made positive (Mezzadri 2007)."""
    G = rng.standard_normal((rows, cols))
    Q, R = np.linalg.qr(G, mode="reduced")
    d = np.sign(np.diag(R))
    d[d == 0] = 1.0
    return Q * d


def _finish(A64_t: np.ndarray, dtype, center: bool) -> np.ndarray:
    """A64_t is (n, m) FP64 (row j = snapshot j).  Mean-centre the rows of A
    (i.e. subtract, for every spatial index, its mean over snapshots), round
    to the storage dtype, return the (m, n) Fortran-ordered view."""
    if center:
        A64_t -= A64_t.mean(axis=0, keepdims=True)
    out = np.ascontiguousarray(A64_t, dtype=dtype)
    return out.T


def planted(m: int, n: int, sigma, noise: float, seed: int, dtype=np.float64,
            center: bool = True) -> np.ndarray:
    """A = U diag(sigma) V^T + noise * N(0, 1), U and V Haar, rows centred."""
    rng = np.random.default_rng(seed)
    sigma = np.asarray(sigma, dtype=np.float64)
    rho = sigma.size
    U = haar(rng, m, rho)
    V = haar(rng, n, rho)
    At = (V * sigma) @ U.T                      # (n, m)
    if noise > 0:
        At += noise * rng.standard_normal((n, m))
    return _finish(At, dtype, center)


def planted_large(m: int, n: int, sigma, noise: float, seed: int, dtype=np.float32,
                  block: int = 256, workers: Optional[int] = None) -> np.ndarray:
    """The recipe of ``planted`` for matrices too large for one generator to
    fill quickly: Haar U and V from ``default_rng(seed)``, A = U diag(sigma)
    V^T + noise * N(0, 1), rows centred in FP64, rounded to ``dtype``.  The
    noise of snapshot block b (columns [b block, (b + 1) block)) comes from
    its own generator ``default_rng([seed, 1, b])``, so blocks are filled by
    parallel threads and the result does not depend on the thread count.
    Holds one FP64 (n, m) buffer while it works."""
    rng = np.random.default_rng(seed)
    sigma = np.asarray(sigma, dtype=np.float64)
    U = haar(rng, m, sigma.size)
    V = haar(rng, n, sigma.size)
    At = np.empty((n, m), dtype=np.float64)
    nb = (n + block - 1) // block

    def fill_noise(b):
        part = At[b * block:min(n, (b + 1) * block)]
        if noise > 0:
            np.random.default_rng([seed, 1, b]).standard_normal(out=part)
            part *= noise
        else:
            part[...] = 0.0

    with ThreadPoolExecutor(max_workers=workers or os.cpu_count() or 1) as ex:
        list(ex.map(fill_noise, range(nb)))
    for b in range(nb):
        j0, j1 = b * block, min(n, (b + 1) * block)
        At[j0:j1] += (V[j0:j1] * sigma) @ U.T
    return _finish(At, dtype, True)


def planted_factors(m: int, n: int, sigma, seed: int):
    """The exact factors of ``planted(..., noise=0, center=False)``."""
    rng = np.random.default_rng(seed)
    sigma = np.asarray(sigma, dtype=np.float64)
    U = haar(rng, m, sigma.size)
    V = haar(rng, n, sigma.size)
    return U, sigma, V


@dataclass
class FlowModes:
    a: np.ndarray       # x wavenumbers
    b: np.ndarray       # y wavenumbers
    omega: np.ndarray   # temporal frequencies
    amp: np.ndarray     # amplitudes


def flow_modes(modes: int, seed: int, max_k: int = 40, max_omega: int = 200) -> FlowModes:
    rng = np.random.default_rng(seed)
    pairs = rng.choice(max_k * max_k, size=modes, replace=False)
    a = pairs // max_k + 1
    b = pairs % max_k + 1
    omega = rng.choice(max_omega, size=modes, replace=False) + 1
    amp = np.arange(1, modes + 1, dtype=np.float64) ** -1.5
    return FlowModes(a=a, b=b, omega=omega, amp=amp)


def flow(grid: int, n: int, modes: int, noise: float, seed: int, dtype=np.float32,
         center: bool = True, max_k: int = 40, max_omega: int = 200) -> np.ndarray:
    """Flow-like snapshots on a grid x grid periodic mesh:
    A[(p, q), s] = sum_j amp_j sin(a_j x_p + omega_j t_s) cos(b_j y_q) + noise,
    x_p = 2 pi p / grid, y_q = 2 pi q / grid, t_s = 2 pi s / n, row index
    p * grid + q.  Distinct integer wavenumbers below grid/2 and distinct
    integer frequencies below n/2 make every term orthogonal on the mesh, so
    the noiseless spectrum is amp_j * sqrt(m n / 8), each value twice."""
    fm = flow_modes(modes, seed, max_k, max_omega)
    rng = np.random.default_rng(seed + 1)
    x = 2 * np.pi * np.arange(grid) / grid
    ts = 2 * np.pi * np.arange(n) / n
    # sin(a x + w t) cos(b y) = sin(a x) cos(b y) cos(w t) + cos(a x) cos(b y) sin(w t)
    sx = np.sin(np.outer(x, fm.a))              # (grid, modes)
    cx = np.cos(np.outer(x, fm.a))
    cy = np.cos(np.outer(x, fm.b))
    Fs = (sx[:, None, :] * cy[None, :, :]).reshape(grid * grid, modes)
    Fc = (cx[:, None, :] * cy[None, :, :]).reshape(grid * grid, modes)
    Gc = np.cos(np.outer(ts, fm.omega)) * fm.amp
    Gs = np.sin(np.outer(ts, fm.omega)) * fm.amp
    At = Gc @ Fs.T + Gs @ Fc.T                  # (n, m)
    if noise > 0:
        At += noise * rng.standard_normal(At.shape)
    return _finish(At, dtype, center)


def flow_spectrum(grid: int, n: int, modes: int, seed: int, max_k: int = 40,
                  max_omega: int = 200) -> np.ndarray:
    """Closed-form singular values of the noiseless ``flow`` matrix, sorted."""
    fm = flow_modes(modes, seed, max_k, max_omega)
    m = grid * grid
    s = np.repeat(fm.amp * np.sqrt(m * n / 8.0), 2)
    return np.sort(s)[::-1]


# ----------------------------------------------------------------------------
# The workloads used by the tests and the benchmark
# ----------------------------------------------------------------------------
SEED_DATA = 0x19050510
SEED_SAMPLING = 0x5107


@dataclass
class Workload:
    name: str
    m: int
    n: int
    k: int
    c: int
    dtype: type
    tol: float
    description: str


PLANTED_SMALL = Workload(
    "planted-2000x500-f64", 2000, 500, 10, 20, np.float64, 1e-8,
    "planted sigma_i = 10^(-i/8), i < 40, Haar U (2000x40) and V (500x40), "
    "N(0, 1e-6^2) noise, rows centred, FP64; k=10, c=20")

FLOW_316 = Workload(
    "flow-316x316x2000-f32", 316 * 316, 2000, 20, 40, np.float32, 1e-8,
    "60 separable sin(a x + w t) cos(b y) modes on a 316x316 grid, 2000 "
    "snapshots, amplitudes j^-1.5, N(0, 1e-3^2) noise, rows centred, FP32; "
    "k=20, c=40")


def make_planted_small(seed: int = SEED_DATA + 1, dtype=np.float64) -> np.ndarray:
    sigma = 10.0 ** (-np.arange(40) / 8.0)
    return planted(2000, 500, sigma, 1e-6, seed, dtype)


def make_flow_316(seed: int = SEED_DATA + 2, dtype=np.float32, grid: int = 316,
                  n: int = 2000) -> np.ndarray:
    return flow(grid, n, 60, 1e-3, seed, dtype)


DIFF_C4 = Workload(
    "planted-200000x1000-f32-diff", 200_000, 1000, 16, 32, np.float32, 1e-8,
    "planted sigma_i = 1 - 0.05 (i - 1) for i = 1..16 (gaps 0.05), then "
    "0.1 exp(-(i - 17) / 10) for i = 17..64; Haar U (200000x64), V (1000x64); "
    "no noise, rows centred, FP32; k=16, c=32")


def diff_sigma() -> np.ndarray:
    i = np.arange(1, 65, dtype=np.float64)
    return np.where(i <= 16, 1.0 - 0.05 * (i - 1), 0.1 * np.exp(-(i - 17) / 10.0))


def make_diff_c4(seed: int = SEED_DATA + 4, dtype=np.float32, m: int = 200_000, n: int = 1000) -> np.ndarray:
    """The differentiation workload (sizes reducible for quick cases)."""
    return planted(m, n, diff_sigma(), 0.0, seed, dtype)


PRECISION_C3 = Workload(
    "planted-1000000x4000-f32", 1_000_000, 4000, 50, 100, np.float32, 1e-8,
    "planted sigma_i = exp(-i/15), i = 0..199, Haar U (1e6x200) and V "
    "(4000x200), N(0, 1e-4^2) noise, rows centred, FP32; k=50, c=100")


def precision_sigma() -> np.ndarray:
    return np.exp(-np.arange(200, dtype=np.float64) / 15.0)


def make_precision_c3(seed: int = SEED_DATA + 3, dtype=np.float32, m: int = 1_000_000,
                      n: int = 4000) -> np.ndarray:
    """The 16 GB precision workload (sizes reducible for quick cases)."""
    return planted_large(m, n, precision_sigma(), 1e-4, seed, dtype)


def diff_loss_weights(k: int, m: int, seed: int = SEED_DATA + 40):
    """Seeded w ~ U(0.5, 1.5)^k and g ~ N(0, I_m) of the loss sum w_i (u_i^T g)^2."""
    rng = np.random.default_rng(seed)
    return rng.uniform(0.5, 1.5, k), rng.standard_normal(m)
