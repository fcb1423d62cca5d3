"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds input generators only: point clouds and the dissimilarity
matrices computed from them.  It contains none of the k-medoids arithmetic
(no TD, BUILD or SWAP step), so both the CUDA path and the FP64 oracle may
draw their inputs from it.

The paper's own data sets (OR-Library, 100 plant leaves, optdigits, MNIST;
Sec. 4.2) are not available here.  These generators stand in for them with
Gaussian mixtures and uniform clouds of the sizes the workloads below name:

* ``manhattan_1000``  n=1000 2-D integer coordinates uniform in [0,1000),
                      Manhattan distances as an int32 matrix, k=10.
* ``gmm_20000``       n=20000, d=16, 100 isotropic clusters, centres uniform
                      in [-10,10]^16, sigma=1, equal weights; Euclidean f32.
* ``gmm_50000``       n=50000, d=32, 200 clusters, centres uniform in
                      [-10,10]^32, sigma_j ~ U[0.5,2], weights Dirichlet(1).
* ``features_200000`` n=200000, d=128 bf16 features, 200 clusters with
                      centres ~ N(0, 4I), sigma=1, equal weights.
* batched             instances with n ~ U[200,4000], d=8 uniform [0,1)^8,
                      k ~ U[5,50]; CLARA points: n=1e6, d=32, 100 clusters.
* ``bichromatic_*``   facility placement (the paper's Outlook): n consumers
                      from a 2-D Gaussian mixture (households around towns),
                      m candidate locations uniform over the same square;
                      an m x n rectangular matrix d(consumer, location)
                      (exact integer Manhattan, or FP64 Euclidean rounded
                      once to FP32), rows = locations.

Every distance is computed in FP64 from the coordinates by the direct
difference formula, rounded once to FP32 (or taken exactly for the integer
Manhattan case), then mirrored so the matrix is bitwise symmetric with a
zero diagonal.  Rows may be padded to a stride ``ld`` (a multiple of 4
elements); padding columns hold zeros and are never read as distances.
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 1000


def rng_for(tag, extra: int = 0) -> np.random.Generator:
    """numpy PCG64 stream for workload ``tag`` (an int index, or any value
    whose repr names the input)."""
    if not isinstance(tag, (int, np.integer)):
        txt = repr(tag)
        tag = sum((i + 1) * ord(ch) for i, ch in enumerate(txt)) % 99991
    return np.random.Generator(np.random.PCG64(SEED_BASE + int(tag) +
                                               1_000_003 * int(extra)))


def round_up(x: int, m: int) -> int:
    return (x + m - 1) // m * m


# ---------------------------------------------------------------- points --

def int_coords(n: int, dim: int = 2, hi: int = 1000, seed=1) -> np.ndarray:
    return rng_for(seed).integers(0, hi, size=(n, dim)).astype(np.int64)


def gmm_points(n: int, d: int, n_centers: int, *, seed=2,
               center_box: float | None = 10.0, center_std: float | None = None,
               sigma=1.0, sigma_range=None, dirichlet: bool = False,
               return_labels: bool = False):
    """Gaussian mixture in FP64.  Centres uniform in [-box, box]^d, or
    N(0, center_std^2 I); per-cluster sigma fixed or uniform in sigma_range;
    weights equal or Dirichlet(1).  Points come in random order."""
    g = rng_for(seed)
    if center_std is not None:
        centers = g.normal(0.0, center_std, size=(n_centers, d))
    else:
        centers = g.uniform(-center_box, center_box, size=(n_centers, d))
    if sigma_range is not None:
        sig = g.uniform(sigma_range[0], sigma_range[1], size=n_centers)
    else:
        sig = np.full(n_centers, float(sigma))
    if dirichlet:
        w = g.dirichlet(np.ones(n_centers))
    else:
        w = np.full(n_centers, 1.0 / n_centers)
    z = g.choice(n_centers, size=n, p=w)
    X = centers[z] + sig[z, None] * g.standard_normal(size=(n, d))
    return (X, z) if return_labels else X


def uniform_points(n: int, d: int, *, seed=5, extra: int = 0) -> np.ndarray:
    return rng_for(seed, extra).random(size=(n, d))


# -------------------------------------------------------------- matrices --

def manhattan_int32(X: np.ndarray, ld: int | None = None) -> np.ndarray:
    """Exact integer L1 distances as int32, shape (n, ld)."""
    X = np.asarray(X, dtype=np.int64)
    n = X.shape[0]
    ld = round_up(n, 4) if ld is None else ld
    D = np.zeros((n, ld), dtype=np.int32)
    for i0 in range(0, n, 512):
        blk = np.abs(X[i0:i0 + 512, None, :] - X[None, :, :]).sum(-1)
        D[i0:i0 + 512, :n] = blk.astype(np.int32)
    return D


def euclidean_f32(X: np.ndarray, ld: int | None = None) -> np.ndarray:
    """FP64 Euclidean distances, rounded to FP32, mirrored (CPU)."""
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    ld = round_up(n, 4) if ld is None else ld
    D = np.zeros((n, ld), dtype=np.float32)
    for i0 in range(0, n, 256):
        diff = X[i0:i0 + 256, None, :] - X[None, :, :]
        D[i0:i0 + 256, :n] = np.sqrt((diff * diff).sum(-1)).astype(np.float32)
    core = D[:, :n]
    upper = np.triu(core, 1)
    core[:] = upper + upper.T
    return D


def euclidean_f32_torch(X: np.ndarray, device, ld: int | None = None,
                        block: int = 256):
    """The same recipe evaluated with torch on ``device`` (for matrices too
    large to build on the host): FP64 direct differences, one rounding to
    FP32, then the upper triangle mirrored onto the lower one."""
    import torch
    Xt = torch.as_tensor(np.asarray(X, dtype=np.float64), device=device)
    n = Xt.shape[0]
    ld = round_up(n, 4) if ld is None else ld
    D = torch.zeros((n, ld), dtype=torch.float32, device=device)
    for i0 in range(0, n, block):
        diff = Xt[i0:i0 + block, None, :] - Xt[None, :, :]
        D[i0:i0 + block, :n] = torch.sqrt((diff * diff).sum(-1)).float()
        del diff
    # mirror: D[j, i] := D[i, j] for i < j, in square tiles
    T = 4096
    for i0 in range(0, n, T):
        i1 = min(n, i0 + T)
        for j0 in range(i0, n, T):
            j1 = min(n, j0 + T)
            blk = D[i0:i1, j0:j1]
            if j0 == i0:
                up = torch.triu(blk, 1)
                blk.copy_(up + up.T)
            else:
                D[j0:j1, i0:i1] = blk.T
    return D


def cross_manhattan_int32(L: np.ndarray, C: np.ndarray, ld: int | None = None) -> np.ndarray:
    """Exact integer L1 distances between rows L (locations) and C
    (consumers) as int32, shape (len(L), ld)."""
    L = np.asarray(L, dtype=np.int64)
    C = np.asarray(C, dtype=np.int64)
    m, n = L.shape[0], C.shape[0]
    ld = round_up(n, 4) if ld is None else ld
    D = np.zeros((m, ld), dtype=np.int32)
    for i0 in range(0, m, 512):
        D[i0:i0 + 512, :n] = np.abs(L[i0:i0 + 512, None, :] - C[None, :, :]).sum(-1)
    return D


def cross_euclidean_f32(L: np.ndarray, C: np.ndarray, ld: int | None = None) -> np.ndarray:
    """FP64 Euclidean distances between rows L and C, rounded once to FP32,
    shape (len(L), ld)."""
    L = np.asarray(L, dtype=np.float64)
    C = np.asarray(C, dtype=np.float64)
    m, n = L.shape[0], C.shape[0]
    ld = round_up(n, 4) if ld is None else ld
    D = np.zeros((m, ld), dtype=np.float32)
    for i0 in range(0, m, 256):
        diff = L[i0:i0 + 256, None, :] - C[None, :, :]
        D[i0:i0 + 256, :n] = np.sqrt((diff * diff).sum(-1)).astype(np.float32)
    return D


def cross_euclidean_f32_torch(L: np.ndarray, C: np.ndarray, device, ld: int | None = None,
                              block: int = 512):
    """cross_euclidean_f32 evaluated with torch on ``device``: FP64 direct
    differences, one rounding to FP32, shape (len(L), ld)."""
    import torch
    Lt = torch.as_tensor(np.asarray(L, dtype=np.float64), device=device)
    Ct = torch.as_tensor(np.asarray(C, dtype=np.float64), device=device)
    m, n = Lt.shape[0], Ct.shape[0]
    ld = round_up(n, 4) if ld is None else ld
    D = torch.zeros((m, ld), dtype=torch.float32, device=device)
    for i0 in range(0, m, block):
        diff = Lt[i0:i0 + block, None, :] - Ct[None, :, :]
        D[i0:i0 + block, :n] = torch.sqrt((diff * diff).sum(-1)).float()
        del diff
    return D


def bichromatic_points(m: int, n: int, *, towns: int = 40, seed=11, integer: bool = False):
    """(locations (m, 2), consumers (n, 2)): consumers from a mixture of
    ``towns`` Gaussian clusters (centres uniform in [0, 1000)^2, sigma
    U[10, 60]), locations uniform over the square; integer coordinates when
    ``integer``."""
    g = rng_for(("bichromatic", seed))
    centres = g.uniform(0.0, 1000.0, size=(towns, 2))
    sig = g.uniform(10.0, 60.0, size=towns)
    z = g.integers(0, towns, size=n)
    C = np.clip(centres[z] + sig[z, None] * g.standard_normal(size=(n, 2)), 0.0, 999.0)
    L = g.uniform(0.0, 1000.0, size=(m, 2))
    if integer:
        return np.floor(L).astype(np.int64), np.floor(C).astype(np.int64)
    return L, C


# -------------------------------------------------------------- workloads --

def bichromatic_100000(m: int = 20000, n: int = 100000):
    """Facility placement: n = 100000 consumers around 200 towns, m = 20000
    candidate locations uniform over the square (float coordinates)."""
    return bichromatic_points(m, n, towns=200, seed=100000)


def manhattan_1000(n: int = 1000):
    """Integer workload: (D int32 (n, ld), k=10)."""
    return manhattan_int32(int_coords(n, 2, 1000, seed=1)), 10


def gmm_20000_points(n: int = 20000, d: int = 16, n_centers: int = 100):
    return gmm_points(n, d, n_centers, seed=2, center_box=10.0, sigma=1.0)


def gmm_50000_points(n: int = 50000, d: int = 32, n_centers: int = 200):
    return gmm_points(n, d, n_centers, seed=3, center_box=10.0,
                      sigma_range=(0.5, 2.0), dirichlet=True)


def features_200000(n: int = 200000, d: int = 128, n_centers: int = 200):
    """bf16-representable features (returned as float32 holding bf16 values)
    of the 200-cluster mixture with centres ~ N(0, 4I), sigma = 1."""
    X = gmm_points(n, d, n_centers, seed=4, center_std=2.0, sigma=1.0)
    return to_bf16_values(X)


def to_bf16_values(X: np.ndarray) -> np.ndarray:
    """Round FP64 values to the nearest bf16 (ties to even), returned as
    float32 arrays whose low 16 bits are zero."""
    f = np.asarray(X, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def batched_specs(count: int = 512, n_lo: int = 200, n_hi: int = 4000,
                  k_lo: int = 5, k_hi: int = 50, seed=5):
    """(n_i, k_i) pairs for the batched workload, n ~ U[n_lo, n_hi],
    k ~ U[k_lo, k_hi] (integers, inclusive)."""
    g = rng_for(seed)
    ns = g.integers(n_lo, n_hi + 1, size=count)
    ks = g.integers(k_lo, k_hi + 1, size=count)
    ks = np.minimum(ks, ns)
    return [(int(a), int(b)) for a, b in zip(ns, ks)]


def batched_instance_points(i: int, n: int, d: int = 8) -> np.ndarray:
    return uniform_points(n, d, seed=5, extra=i + 1)


def batched_points(specs, d: int = 8, seed=5):
    """float32 points of every instance, concatenated, and the first row of
    each instance (uniform in [0,1)^d)."""
    parts = [uniform_points(n, d, seed=seed, extra=i + 1).astype(np.float32)
             for i, (n, _) in enumerate(specs)]
    offs = np.cumsum([0] + [p.shape[0] for p in parts])[:-1].astype(np.int64)
    return np.concatenate(parts, axis=0), offs


def clara_points(n: int = 1_000_000, d: int = 32, n_centers: int = 100):
    """float32 points of the 100-cluster mixture (centres U[-10,10]^d,
    sigma = 1, equal weights)."""
    return gmm_points(n, d, n_centers, seed=6, center_box=10.0,
                      sigma=1.0).astype(np.float32)


def clara_samples(n: int, samples: int, size: int, seed=7) -> np.ndarray:
    """CLARA subsamples: `samples` rows of `size` distinct point indices,
    each drawn uniformly without replacement and sorted (int32)."""
    g = rng_for(seed)
    return np.stack([np.sort(g.choice(n, size=size, replace=False))
                     for _ in range(samples)]).astype(np.int32)
