"""Seeded synthetic inputs shaped like the paper's embedding workloads.

This module holds no part of the method: it only draws input matrices.  It is
shared by the tests, the benchmark and the oracle checks; neither the oracle
nor the CUDA library imports it.

Recipe: z_ij ~ N(0, 1); y_j = sqrt(lambda_j) z_j with a power-law spectrum
lambda_j = j^-alpha (lambda_1 = 1); x = Q_data y with Q_data a seeded Haar
orthogonal d x d matrix.  After PCA the variances decay as a long tail and each
coordinate is near-normal with mean about 0, the structure the paper reports
for its datasets (Sec. 4.1 variance figure, Sec. 4.2 value distribution).
Seeds: data 1, data rotation 2, queries 3 (the method's own rotations use a
separate seed inside the fit).
"""
from __future__ import annotations

import torch

SEED_DATA = 1
SEED_ROT = 2
SEED_QUERY = 3


def spectrum(d: int, alpha: float) -> torch.Tensor:
    j = torch.arange(1, d + 1, dtype=torch.float64)
    return j.pow(-alpha)


def data_rotation(d: int, seed: int = SEED_ROT) -> torch.Tensor:
    """Seeded Haar rotation of the data (FP64, CPU)."""
    g = torch.Generator(device="cpu").manual_seed(seed)
    G = torch.randn(d, d, generator=g, dtype=torch.float64)
    Q, R = torch.linalg.qr(G)
    s = torch.sign(torch.diagonal(R))
    s[s == 0] = 1.0
    return Q * s


def power_law(n: int, d: int, alpha: float, seed: int = SEED_DATA,
              rot_seed: int = SEED_ROT, device="cpu", chunk: int = 1 << 17,
              out: torch.Tensor | None = None) -> torch.Tensor:
    """n x d float32 rows drawn as above, generated on `device` in row chunks
    (each chunk has its own derived seed, so a row depends only on its index
    range's chunk and the seeds)."""
    dev = torch.device(device)
    Q = data_rotation(d, rot_seed)
    sq = spectrum(d, alpha).sqrt()
    # fold the spectrum into the rotation: x = z diag(sqrt(lambda)) Q^T
    M = (sq[:, None] * Q.T).to(torch.float32).to(dev)
    X = out if out is not None else torch.empty(n, d, dtype=torch.float32, device=dev)
    prev_tf32 = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        for ci, i in enumerate(range(0, n, chunk)):
            m = min(chunk, n - i)
            g = torch.Generator(device=dev).manual_seed(seed * 1000003 + ci)
            z = torch.randn(m, d, generator=g, dtype=torch.float32, device=dev)
            torch.matmul(z, M, out=X[i:i + m])
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev_tf32
    return X


def queries(nq: int, d: int, alpha: float, device="cpu") -> torch.Tensor:
    return power_law(nq, d, alpha, seed=SEED_QUERY, device=device)


# The workloads: (name, n, d, alpha, avg_bits, rounds, queries)
WORKLOADS = {
    "c1_d128": dict(n=10_000, d=128, alpha=1.0, avg_bits=4.0, rounds=6, nq=100),
    "c2_d960": dict(n=1_000_000, d=960, alpha=0.8, avg_bits=4.0, rounds=6, nq=10_000),
    "c3_d1536": dict(n=1_000_000, d=1536, alpha=0.6, avg_bits=2.0, rounds=6, nq=1000),
    "c4_d3072": dict(n=500_000, d=3072, alpha=0.5, avg_bits=1.0, rounds=6, nq=1000),
    "c4_d3072_8b": dict(n=500_000, d=3072, alpha=0.5, avg_bits=8.0, rounds=6, nq=1000),
}
