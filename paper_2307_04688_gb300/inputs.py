"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module holds random-number generation and the recipes that turn draws
into workload inputs. It holds none of the Chebyshev method's arithmetic:
no nodes, no polynomial evaluation, no fit. Both the CUDA path and the CPU
oracle receive the arrays made here as plain inputs.

Generator: SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014). Output k of a stream seeded with s is
mix(s + (k+1)*0x9E3779B97F4A7C15 mod 2^64). Uniforms take the top 53 bits,
u = (z >> 11) * 2^-53 in [0, 1). Normals use Box-Muller on consecutive
uniform pairs (u1, u2): r = sqrt(-2 ln(1 - u1)), first the cos branch
r cos(2 pi u2), then the sin branch r sin(2 pi u2). Draws are taken in
row-major order over a multi-index (last mode fastest).

The game parameters are drawn uniformly within +-30 % of nominal values. The
paper fixes beta = phi = 1, A = 0.5, c = 0.5 and the neighbour matrices of its
2-, 3- and 4-player examples (Section 4); it states no discount rate, so the
nominal rho = 0.5 is a reading, recorded with every result.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


class SplitMix64:
    """Counter-form SplitMix64 stream; every draw advances the counter by one."""

    def __init__(self, seed: int):
        self.state = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
        self.count = 0

    def next_u64(self, size: int) -> np.ndarray:
        k = np.arange(self.count + 1, self.count + 1 + size, dtype=np.uint64)
        self.count += size
        with np.errstate(over="ignore"):
            z = self.state + k * _GOLDEN
            z = (z ^ (z >> np.uint64(30))) * _M1
            z = (z ^ (z >> np.uint64(27))) * _M2
            z = z ^ (z >> np.uint64(31))
        return z

    def uniform(self, size: int) -> np.ndarray:
        z = self.next_u64(size)
        return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)

    def normal(self, size: int) -> np.ndarray:
        pairs = (size + 1) // 2
        u = self.uniform(2 * pairs).reshape(pairs, 2)
        r = np.sqrt(-2.0 * np.log1p(-u[:, 0]))
        t = 2.0 * np.pi * u[:, 1]
        out = np.empty((pairs, 2))
        out[:, 0] = r * np.cos(t)
        out[:, 1] = r * np.sin(t)
        return out.reshape(-1)[:size]


def decaying_coeffs(rng: SplitMix64, d: int, n: int, ratio: float) -> np.ndarray:
    """c_k = N(0,1) * ratio^(k_1+...+k_d), row-major, shape (n,)*d."""
    g = rng.normal(n ** d).reshape((n,) * d)
    k = np.indices((n,) * d).sum(axis=0)
    return g * ratio ** k


def uniform_grid(m: int) -> np.ndarray:
    """m equispaced points x_i = -1 + 2 i / (m - 1) on [-1, 1]."""
    return -1.0 + 2.0 * np.arange(m) / (m - 1)


def small_fit_workload(seed: int = 0, n: int = 17, n_grid: int = 129, n_points: int = 10000):
    """d=2 workload: coefficients 0.5^(k1+k2) N(0,1), a 129x129 grid, 10,000 points."""
    rng = SplitMix64(seed)
    c = decaying_coeffs(rng, 2, n, 0.5)
    pts = -1.0 + 2.0 * rng.uniform(n_points * 2).reshape(n_points, 2)
    return {"coeffs": c, "grid": [uniform_grid(n_grid)] * 2, "points": pts}


def tensor_grid_workload(seed: int = 1, d: int = 4, n: int = 33, m: int = 64):
    """d=4, n=33 coefficients 0.7^|k|_1 N(0,1) with a 64^4 uniform tensor grid."""
    rng = SplitMix64(seed)
    c = decaying_coeffs(rng, d, n, 0.7)
    return {"coeffs": c, "grid": [uniform_grid(m)] * d}


# ---- pollution game parameters -------------------------------------------

NOMINAL = {"A": 0.5, "phi": 1.0, "beta": 1.0, "c": 0.5, "rho": 0.5, "k": 1.0, "m": 1.0}


def neighbour_matrix(J: int, k: float = 1.0) -> np.ndarray:
    """Neighbour matrices of the paper's J = 2, 3, 4 examples (Section 4), times k.

    Rows sum to zero (diagonal = minus the number of neighbours). The printed
    3-player matrix has row 2 as [1, -2, 0]; the text says player 2 borders
    players 1 and 3, so row 2 is read as [1, -2, 1].
    """
    if J == 1:
        K = np.zeros((1, 1))
    elif J == 2:
        K = np.array([[-1.0, 1.0], [1.0, -1.0]])
    elif J == 3:
        K = np.array([[-1.0, 1.0, 0.0], [1.0, -2.0, 1.0], [0.0, 1.0, -1.0]])
    elif J == 4:
        K = np.array([[-1.0, 1.0, 0.0, 0.0], [1.0, -3.0, 1.0, 1.0],
                      [0.0, 1.0, -2.0, 1.0], [0.0, 1.0, 1.0, -2.0]])
    else:
        raise ValueError("J must be 1..4")
    return K * k


def game_params(J: int = 3, A=None, phi=None, beta=None, c=None, rho=None, k=None, m=None, gamma=None):
    """A parameter dict with the paper's nominal values for anything not given. gamma (J x J,
    default zero) is the emission-interaction coupling u_i sum_{l != i} gamma_il u_l of the
    dynamics, zero in the paper's examples."""
    def vec(v, name):
        v = NOMINAL[name] if v is None else v
        return np.broadcast_to(np.asarray(v, dtype=np.float64), (J,)).copy()
    kk = NOMINAL["k"] if k is None else float(k)
    return {"J": J, "K": neighbour_matrix(J, kk), "m": NOMINAL["m"] if m is None else float(m),
            "A": vec(A, "A"), "beta": vec(beta, "beta"), "phi": vec(phi, "phi"),
            "c": vec(c, "c"), "rho": NOMINAL["rho"] if rho is None else float(rho),
            "gamma": np.zeros((J, J)) if gamma is None else np.asarray(gamma, dtype=np.float64).reshape(J, J)}


def draw_game_params(rng: SplitMix64, J: int = 3, spread: float = 0.3):
    """Draw (A_1..A_J, phi_1..phi_J, rho, k), each nominal * (1 + spread (2U - 1))."""
    u = rng.uniform(2 * J + 2)
    f = 1.0 + spread * (2.0 * u - 1.0)
    return game_params(J, A=NOMINAL["A"] * f[:J], phi=NOMINAL["phi"] * f[J:2 * J],
                       rho=NOMINAL["rho"] * f[2 * J], k=NOMINAL["k"] * f[2 * J + 1])


def game_param_vector(p) -> np.ndarray:
    """The 2J+2 drawn quantities (A, phi, rho, k) of a parameter dict, as a vector."""
    J = p["J"]
    k = -p["K"][0, 0] if J > 1 else 0.0
    return np.concatenate([p["A"], p["phi"], [p["rho"], k]])


def single_game_workload(seed: int = 2, J: int = 3):
    """One J-player game with parameters drawn within +-30 % of nominal."""
    return draw_game_params(SplitMix64(seed), J)


def batched_game_workload(seed: int = 2, count: int = 1024, J: int = 3, sizes=(9, 17, 33)):
    """`count` games: per instance, n from sizes by floor(len(sizes) U), then its parameters."""
    rng = SplitMix64(seed)
    out = []
    for _ in range(count):
        n = sizes[min(int(rng.uniform(1)[0] * len(sizes)), len(sizes) - 1)]
        out.append((n, draw_game_params(rng, J)))
    return out


def surrogate_workload(seed: int = 3, count: int = 22000, J: int = 3):
    """`count` parameter draws for the learned warm start (first 20,000 train, rest test)."""
    rng = SplitMix64(seed)
    return [draw_game_params(rng, J) for _ in range(count)]
