"""PDE data of eq. (1.1) for the synthetic workloads (input generator, no method arithmetic).

Each problem gives, as vectorised functions of (x, y, z):
  kappa > 0, c >= 0, f, an optional convection field beta, the Dirichlet data u_D, the
  Neumann vector field g_N (eq. 1.1d: -q.nu = g_N.nu), and, where known, the exact u and
  q = -kappa grad u used to manufacture f.
The boundary split is a predicate on the cube's six planes.

Workloads (unit cube, s^3 subcubes x 6 Kuhn tetrahedra):
  cube4_k1          s=4,  k=1, kappa=c=tau=1, Dirichlet everywhere, u = sin(pi x)sin(pi y)sin(pi z)
  cube16_k3         s=16, k=3, kappa = 1 + 0.5 sin(2 pi x) cos(2 pi y), c = 1 + x^2,
                    u = (1 + x^2 + y z) exp(0.5 x - y + z), Dirichlet on x=0, x=1, Neumann elsewhere
  cube48_k2_conv    s=48 (jitter 0.2 h, seed 0), k=2, beta = (y, -x, 0.5 z),
                    kappa = 1 + 0.5 sin(2 pi z), c = 1, u = sin sin sin, Dirichlet everywhere
  cube32_k2_grf     s=32, k=2, kappa = exp(g) with g a seeded Gaussian random field, c = 1,
                    f = 1, u_D = 0, Dirichlet everywhere
Any of them can be re-instantiated at another s or k (tests use small s).
"""

from dataclasses import dataclass, field, replace
from typing import Callable, Optional

import numpy as np

PI = np.pi


@dataclass
class Problem:
    name: str
    s: int
    k: int
    kappa: Callable
    c: Callable
    f: Callable
    uD: Callable
    gN: Optional[Callable] = None
    beta: Optional[Callable] = None
    u: Optional[Callable] = None
    q: Optional[Callable] = None  # exact flux -kappa grad u, returns (qx, qy, qz)
    dirichlet_planes: tuple = ((0, 0.0), (0, 1.0), (1, 0.0), (1, 1.0), (2, 0.0), (2, 1.0))
    tau: float = 1.0
    jitter: float = 0.0
    seed: int = 0
    extra: dict = field(default_factory=dict)

    def classify(self, ax, val):
        return "D" if (ax, val) in self.dirichlet_planes else "N"

    def at(self, s=None, k=None):
        """Same PDE data on another mesh size or degree."""
        return replace(self, s=self.s if s is None else s, k=self.k if k is None else k)


# ---------------------------------------------------------------- sin sin sin, kappa const
def _sss(x, y, z):
    return np.sin(PI * x) * np.sin(PI * y) * np.sin(PI * z)


def _sss_grad(x, y, z):
    sx, sy, sz = np.sin(PI * x), np.sin(PI * y), np.sin(PI * z)
    cx, cy, cz = np.cos(PI * x), np.cos(PI * y), np.cos(PI * z)
    return PI * cx * sy * sz, PI * sx * cy * sz, PI * sx * sy * cz


def sinsinsin(name, s, k, kappa0=1.0, c0=1.0):
    """-div(kappa0 grad u) + c0 u = f with u = sin(pi x) sin(pi y) sin(pi z)."""
    def q(x, y, z):
        gx, gy, gz = _sss_grad(x, y, z)
        return -kappa0 * gx, -kappa0 * gy, -kappa0 * gz

    return Problem(
        name=name, s=s, k=k,
        kappa=lambda x, y, z: np.full(np.shape(x), kappa0),
        c=lambda x, y, z: np.full(np.shape(x), c0),
        f=lambda x, y, z: (3 * PI**2 * kappa0 + c0) * _sss(x, y, z),
        uD=_sss, u=_sss, q=q,
        gN=lambda x, y, z: tuple(-v for v in q(x, y, z)),
    )


# ---------------------------------------------------- polynomial x exponential, variable kappa
def _pe_u(x, y, z):
    return (1 + x**2 + y * z) * np.exp(0.5 * x - y + z)


def _pe_grad(x, y, z):
    g = 1 + x**2 + y * z
    E = np.exp(0.5 * x - y + z)
    return (2 * x + 0.5 * g) * E, (z - g) * E, (y + g) * E


def _pe_lap(x, y, z):
    g = 1 + x**2 + y * z
    E = np.exp(0.5 * x - y + z)
    return (2 + 2 * x + 2 * y - 2 * z + 2.25 * g) * E


def _k2_kappa(x, y, z):
    return 1 + 0.5 * np.sin(2 * PI * x) * np.cos(2 * PI * y)


def _k2_kappa_grad(x, y, z):
    return (PI * np.cos(2 * PI * x) * np.cos(2 * PI * y),
            -PI * np.sin(2 * PI * x) * np.sin(2 * PI * y),
            np.zeros(np.shape(x)))


def _k2_c(x, y, z):
    return 1 + x**2


def _k2_q(x, y, z):
    kap = _k2_kappa(x, y, z)
    gx, gy, gz = _pe_grad(x, y, z)
    return -kap * gx, -kap * gy, -kap * gz


def _k2_f(x, y, z):
    # f = c u + div q = c u - kappa lap u - grad kappa . grad u
    kap = _k2_kappa(x, y, z)
    kx, ky, kz = _k2_kappa_grad(x, y, z)
    gx, gy, gz = _pe_grad(x, y, z)
    return _k2_c(x, y, z) * _pe_u(x, y, z) - kap * _pe_lap(x, y, z) - (kx * gx + ky * gy + kz * gz)


def _k2_gN(x, y, z):
    # -q.nu = g_N.nu with q = -kappa grad u  =>  g_N = kappa grad u
    return tuple(-v for v in _k2_q(x, y, z))


def cube16_k3(s=16, k=3):
    return Problem(
        name="cube16_k3", s=s, k=k, kappa=_k2_kappa, c=_k2_c, f=_k2_f,
        uD=_pe_u, gN=_k2_gN, u=_pe_u, q=_k2_q,
        dirichlet_planes=((0, 0.0), (0, 1.0)),
    )


# ------------------------------------------------------------------------- convection
def _k3_beta(x, y, z):
    return y, -x, 0.5 * z


def _k3_kappa(x, y, z):
    return 1 + 0.5 * np.sin(2 * PI * z)


def _k3_q(x, y, z):
    kap = _k3_kappa(x, y, z)
    gx, gy, gz = _sss_grad(x, y, z)
    return -kap * gx, -kap * gy, -kap * gz


def _k3_f(x, y, z):
    # conservative form: div(q + beta u) + c u = f, q = -kappa grad u, div beta = 0.5
    kap = _k3_kappa(x, y, z)
    kz = PI * np.cos(2 * PI * z)
    gx, gy, gz = _sss_grad(x, y, z)
    u = _sss(x, y, z)
    lap = -3 * PI**2 * u
    bx, by, bz = _k3_beta(x, y, z)
    return -kap * lap - kz * gz + 0.5 * u + (bx * gx + by * gy + bz * gz) + 1.0 * u


def cube48_k2_conv(s=48, k=2):
    return Problem(
        name="cube48_k2_conv", s=s, k=k, kappa=_k3_kappa,
        c=lambda x, y, z: np.ones(np.shape(x)), f=_k3_f, uD=_sss, u=_sss, q=_k3_q,
        beta=_k3_beta, tau=2.5, jitter=0.2, seed=0,
    )


# ---------------------------------------------------------------- Gaussian random field
GRF_M = 128
GRF_SIGMA = 1.0
GRF_ELL = 0.2
GRF_FREQ_SEED = 12345


def grf_frequencies(M=GRF_M, ell=GRF_ELL, seed=GRF_FREQ_SEED):
    """Frequencies omega_m ~ N(0, ell^-2 I), drawn once."""
    return np.random.default_rng(seed).normal(0.0, 1.0 / ell, size=(M, 3))


def grf_sample(sample_id, M=GRF_M):
    """Amplitudes (xi_m, eta_m) ~ N(0,1) of one field, seeded by its id: shape [2M]."""
    return np.random.default_rng(1_000_003 + int(sample_id)).normal(size=2 * M)


def grf_field(amps, omega=None, sigma=GRF_SIGMA):
    """g(x) = sigma M^-1/2 sum_m (xi_m cos(omega_m.x) + eta_m sin(omega_m.x))."""
    if omega is None:
        omega = grf_frequencies()
    M = omega.shape[0]
    xi, eta = amps[:M], amps[M:]

    def g(x, y, z):
        x = np.asarray(x, dtype=np.float64)
        ph = (np.multiply.outer(x, omega[:, 0]) + np.multiply.outer(y, omega[:, 1])
              + np.multiply.outer(z, omega[:, 2]))
        return sigma / np.sqrt(M) * (np.cos(ph) @ xi + np.sin(ph) @ eta)

    return g


def cube32_k2_grf(sample_id=0, s=32, k=2):
    g = grf_field(grf_sample(sample_id))
    zero = lambda x, y, z: np.zeros(np.shape(x))  # noqa: E731
    return Problem(
        name="cube32_k2_grf", s=s, k=k, kappa=lambda x, y, z: np.exp(g(x, y, z)),
        c=lambda x, y, z: np.ones(np.shape(x)), f=lambda x, y, z: np.ones(np.shape(x)),
        uD=zero, extra={"sample_id": sample_id},
    )


# ---------------------------------------------------------------- batch of 64 problems
def batch_problems(nprob=64, seed=4):
    """64 independent cube problems: s ~ U{8..24}, k ~ U{1..4}, kappa = 10^U(-1,1), c ~ U[0,5]."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(nprob):
        s = int(rng.integers(8, 25))
        k = int(rng.integers(1, 5))
        kap = float(10 ** rng.uniform(-1, 1))
        c0 = float(rng.uniform(0, 5))
        out.append(sinsinsin(f"batch{i}", s, k, kappa0=kap, c0=c0))
    return out


PROBLEMS = {
    "cube4_k1": lambda: sinsinsin("cube4_k1", 4, 1),
    "cube16_k3": cube16_k3,
    "cube48_k2_conv": cube48_k2_conv,
    "cube32_k2_grf": cube32_k2_grf,
}


def get_problem(name, **kw):
    return PROBLEMS[name](**kw) if kw else PROBLEMS[name]()
