"""Seeded synthetic inputs shared by the CUDA path, the oracle, tests and bench.

This module draws random numbers and lays them out; it holds none of the
method's arithmetic (no assembly, factorisation, network or solver step).
Both sides consume the arrays it returns, so no generator or libm difference
can leak between them.

Workload recipe (stand-in for the paper's STAND structural-analysis matrices,
which are not available): a unit cube of N^3 trilinear hex elements, Poisson
ratio 0.3, per-element Young modulus E_e = exp(sigma * g_e) with g_e ~ N(0,1),
the z = 0 face clamped, right-hand side b ~ U[-1, 1], x0 = 0.
"""
import numpy as np

# Stream tags keep the draws of one seed independent of each other.
_TAG_E, _TAG_B, _TAG_Z, _TAG_W, _TAG_SIGMA = 11, 23, 37, 41, 53

H = 32                      # hidden width of every MLP
N_GRAPHNORM = 27            # gamma[9], beta[9], alpha[9]
N_EDGE = H * 20 + H + H + 1  # W1[H][20], b1[H], W2[H], b2
N_NODE = H * 11 + H + 9 * H + 9  # W3[H][11], b3[H], W4[9][H], b4[9]
N_PARAMS = N_GRAPHNORM + 3 * N_EDGE + 2 * N_NODE


def fem_sizes(N: int):
    """(n, nnz(A), nnz(L), levels) of the clamped N^3 hex system (closed forms)."""
    n = 3 * N * (N + 1) ** 2
    nnz = 9 * (3 * N + 1) ** 2 * (3 * N - 2)
    return n, nnz, (nnz + n) // 2, 21 * N - 9


def material_field(N: int, seed: int, sigma: float = 1.0) -> np.ndarray:
    """Per-element Young modulus, element id ex + N*(ey + N*ez), float64."""
    rng = np.random.default_rng([seed, _TAG_E])
    g = rng.standard_normal(N ** 3)
    return np.exp(sigma * g)


def rhs(n: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng([seed, _TAG_B])
    return rng.uniform(-1.0, 1.0, n)


def training_sigma(seed: int, lo: float = 0.5, hi: float = 2.0) -> float:
    rng = np.random.default_rng([seed, _TAG_SIGMA])
    return float(rng.uniform(lo, hi))


def probes(m: int, n: int, seed: int, kind: str = "gaussian") -> np.ndarray:
    """m probe vectors of length n (float32), Gaussian or Rademacher."""
    rng = np.random.default_rng([seed, _TAG_Z])
    if kind == "gaussian":
        return rng.standard_normal((m, n), dtype=np.float32)
    if kind == "rademacher":
        return (rng.integers(0, 2, (m, n)) * 2 - 1).astype(np.float32)
    raise ValueError(kind)


def param_slices():
    """Name -> (offset, shape) of the flat GNN parameter vector."""
    out = {}
    off = 0

    def put(name, shape):
        nonlocal off
        out[name] = (off, shape)
        off += int(np.prod(shape))

    put("gn_gamma", (9,))
    put("gn_beta", (9,))
    put("gn_alpha", (9,))
    for l in range(3):
        put(f"W1_{l}", (H, 20))
        put(f"b1_{l}", (H,))
        put(f"W2_{l}", (H,))
        put(f"b2_{l}", (1,))
        if l < 2:
            put(f"W3_{l}", (H, 11))
            put(f"b3_{l}", (H,))
            put(f"W4_{l}", (9, H))
            put(f"b4_{l}", (9,))
    assert off == N_PARAMS
    return out


def gnn_init(seed: int, out_scale: float = 1.0) -> np.ndarray:
    """Random initial GNN parameters (float64): Glorot-uniform weights, zero
    biases, GraphNorm gamma = 1, beta = 0, alpha = 1. out_scale multiplies the
    last edge layer (W2 of block 2) so a small value starts near L_IC."""
    rng = np.random.default_rng([seed, _TAG_W])
    theta = np.zeros(N_PARAMS)
    for name, (off, shape) in param_slices().items():
        size = int(np.prod(shape))
        if name == "gn_gamma" or name == "gn_alpha":
            theta[off:off + size] = 1.0
        elif name.startswith("W"):
            fan_out, fan_in = (shape[0], shape[1]) if len(shape) == 2 else (1, shape[0])
            lim = np.sqrt(6.0 / (fan_in + fan_out))
            w = rng.uniform(-lim, lim, size)
            if name == "W2_2":
                w *= out_scale
            theta[off:off + size] = w
    return theta
