"""Seeded synthetic inputs shared by the CUDA path, the oracle and the tests.

This module generates *inputs* only -- element vertex coordinates, random
right-hand sides on the global nodes, analytic source and initial fields --
and holds none of the method's arithmetic (no quadrature, no derivative
matrix, no geometric factors, no gather-scatter).  The paper's flow cases
(Table 1: turbulent pipe, Taylor-Green vortex, Rayleigh-Benard; N = 7) have
no public meshes here, so box meshes with the shapes described below stand in
for them.

Vertex layout: verts[e, v, a], element e = ex + nx*(ey + ny*ez), vertex
v = vx + 2*vy + 4*vz, coordinate a in (x, y, z).
Random numbers: numpy.random.Generator(PCG64(seed)).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Bitmask of Dirichlet box faces: bit 2a = low face of axis a, bit 2a+1 = high.
ALL_FACES = 0b111111
Y_FACES = 0b001100


def _grid_1d(n: int, lo: float, hi: float, tanh_beta: float = 0.0) -> np.ndarray:
    """n+1 vertex positions on [lo, hi]; with beta > 0 clustered toward both
    ends by y_j = tanh(beta (2j/n - 1)) / tanh(beta) mapped onto [lo, hi]."""
    s = np.arange(n + 1, dtype=np.float64) / n
    if tanh_beta > 0.0:
        s = 0.5 * (np.tanh(tanh_beta * (2.0 * s - 1.0)) / math.tanh(tanh_beta) + 1.0)
    return lo + (hi - lo) * s


def box_vertices(nel, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), tanh_beta=(0.0, 0.0, 0.0),
                 perturb_amp: float = 0.0, seed: int = 0, jitter: float = 0.0) -> np.ndarray:
    """Vertices of an nx x ny x nz box of hexahedra, shape (E, 8, 3).

    perturb_amp > 0 moves every vertex by perturb_amp * h * b(v) * s(v), with h
    the (uniform) element size of each axis, b = 64 x(1-x) y(1-y) z(1-z) in
    box-normalised coordinates (zero on the boundary, so the box stays a box)
    and s a product of sines with seeded phases:
        s = (sin 2pi(y+f1) sin 2pi(z+f2), sin 2pi(z+f3) sin 2pi(x+f4),
             sin 2pi(x+f5) sin 2pi(y+f6)).
    jitter > 0 then moves every vertex, boundary ones included, by i.i.d.
    U[-jitter, jitter] * h per axis (small general hexahedra for tests).
    """
    nx, ny, nz = (int(a) for a in nel)
    gx = _grid_1d(nx, lo[0], hi[0], tanh_beta[0])
    gy = _grid_1d(ny, lo[1], hi[1], tanh_beta[1])
    gz = _grid_1d(nz, lo[2], hi[2], tanh_beta[2])
    X, Y, Z = np.meshgrid(gx, gy, gz, indexing="ij")  # [ix, iy, iz]
    P = np.stack([X, Y, Z], axis=-1)
    if perturb_amp > 0.0:
        rng = np.random.Generator(np.random.PCG64(seed))
        ph = rng.random(6)
        L = np.array([hi[a] - lo[a] for a in range(3)])
        h = L / np.array([nx, ny, nz], dtype=np.float64)
        q = (P - np.asarray(lo)) / L  # normalised coordinates in [0, 1]
        b = 64.0 * np.prod(q * (1.0 - q), axis=-1)
        tp = 2.0 * math.pi
        s = np.stack([
            np.sin(tp * (q[..., 1] + ph[0])) * np.sin(tp * (q[..., 2] + ph[1])),
            np.sin(tp * (q[..., 2] + ph[2])) * np.sin(tp * (q[..., 0] + ph[3])),
            np.sin(tp * (q[..., 0] + ph[4])) * np.sin(tp * (q[..., 1] + ph[5])),
        ], axis=-1)
        P = P + perturb_amp * h * b[..., None] * s
    if jitter > 0.0:
        rng = np.random.Generator(np.random.PCG64(seed + 7919))
        h = np.array([(hi[a] - lo[a]) / n for a, n in enumerate((nx, ny, nz))])
        P = P + jitter * h * rng.uniform(-1.0, 1.0, size=P.shape)
    E = nx * ny * nz
    verts = np.empty((nz, ny, nx, 8, 3))
    for v in range(8):
        vx, vy, vz = v & 1, (v >> 1) & 1, (v >> 2) & 1
        sub = P[vx:vx + nx, vy:vy + ny, vz:vz + nz]  # [ex, ey, ez, 3]
        verts[:, :, :, v, :] = np.transpose(sub, (2, 1, 0, 3))
    return verts.reshape(E, 8, 3)


def global_dims(N: int, nel, periodic) -> tuple[int, int, int]:
    """Global node counts per axis of the box numbering (I = ex*N + i ...)."""
    return tuple(int(nel[a]) * N + (0 if periodic[a] else 1) for a in range(3))


def global_masked(N: int, nel, periodic, faces: int) -> np.ndarray:
    """Boolean flags over the global nodes (I fastest) that lie on a Dirichlet
    face of the box (topology only)."""
    G = global_dims(N, nel, periodic)
    I, J, K = np.meshgrid(np.arange(G[0]), np.arange(G[1]), np.arange(G[2]), indexing="ij")
    idx = (I, J, K)
    m = np.zeros(G, dtype=bool)
    for a in range(3):
        if periodic[a]:
            continue
        if (faces >> (2 * a)) & 1:
            m |= idx[a] == 0
        if (faces >> (2 * a + 1)) & 1:
            m |= idx[a] == G[a] - 1
    return np.transpose(m, (2, 1, 0)).reshape(-1)  # I fastest


def random_rhs_global(N: int, nel, periodic, faces: int, seed: int = 0) -> np.ndarray:
    """i.i.d. U[-1, 1] on the global nodes, zero on Dirichlet nodes, shifted to
    zero mean over the free nodes.  Global index I + Gx (J + Gy K)."""
    G = global_dims(N, nel, periodic)
    rng = np.random.Generator(np.random.PCG64(seed))
    b = rng.uniform(-1.0, 1.0, size=G[0] * G[1] * G[2])
    m = global_masked(N, nel, periodic, faces)
    free = ~m
    b[free] -= b[free].mean()
    b[m] = 0.0
    return b


def manufactured_u(x, y, z):
    """Exact solution u* = sin(pi x) sin(pi y) sin(pi z) on the unit cube."""
    return np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z)


def manufactured_f(x, y, z):
    """Source f = -lap u* = 3 pi^2 sin(pi x) sin(pi y) sin(pi z)."""
    return 3.0 * np.pi ** 2 * manufactured_u(x, y, z)


def tgv_velocity(x, y, z):
    """Taylor-Green vortex initial velocity on [0, 2pi]^3."""
    return (np.sin(x) * np.cos(y) * np.cos(z),
            -np.cos(x) * np.sin(y) * np.cos(z),
            np.zeros_like(x))


def tgv_pressure(x, y, z):
    """Exact initial pressure of the Taylor-Green vortex (up to a constant)."""
    return (np.cos(2 * x) + np.cos(2 * y)) * (np.cos(2 * z) + 2.0) / 16.0


@dataclass
class BoxCase:
    """A synthetic box problem: topology, vertices and right-hand-side recipe."""
    name: str
    N: int
    nel: tuple
    periodic: tuple
    faces: int
    lo: tuple = (0.0, 0.0, 0.0)
    hi: tuple = (1.0, 1.0, 1.0)
    tanh_beta: tuple = (0.0, 0.0, 0.0)
    perturb_amp: float = 0.0
    seed: int = 0
    jitter: float = 0.0
    rhs: str = "random"  # "random" | "manufactured"
    extra: dict = field(default_factory=dict)

    @property
    def E(self) -> int:
        return int(np.prod(self.nel))

    @property
    def nloc(self) -> int:
        return self.E * (self.N + 1) ** 3

    @property
    def n_paper(self) -> int:
        """The paper's DOF count n = E N^3 (Table 1)."""
        return self.E * self.N ** 3

    def vertices(self) -> np.ndarray:
        return box_vertices(self.nel, self.lo, self.hi, self.tanh_beta, self.perturb_amp,
                            self.seed, self.jitter)

    def rhs_global(self) -> np.ndarray:
        return random_rhs_global(self.N, self.nel, self.periodic, self.faces, self.seed)


def cube_manufactured(nel: int = 4, N: int = 7) -> BoxCase:
    """Unit cube, nel^3 undeformed elements, Dirichlet on all faces, source
    from u* = sin(pi x) sin(pi y) sin(pi z)."""
    return BoxCase("cube_manufactured", N, (nel, nel, nel), (0, 0, 0), ALL_FACES, rhs="manufactured")


def channel(nel: int = 32, N: int = 7, beta: float = 2.0, seed: int = 0) -> BoxCase:
    """Channel-like box [0, 2pi] x [-1, 1] x [0, pi], tanh wall-normal
    stretching in y, periodic in x and z, Dirichlet walls in y."""
    return BoxCase("channel", N, (nel, nel, nel), (1, 0, 1), Y_FACES,
                   lo=(0.0, -1.0, 0.0), hi=(2 * math.pi, 1.0, math.pi),
                   tanh_beta=(0.0, beta, 0.0), seed=seed)


def deformed_cube(nel: int = 64, N: int = 7, amp: float = 0.05, seed: int = 0) -> BoxCase:
    """Unit cube with smoothly perturbed interior vertices, Dirichlet on all faces."""
    return BoxCase("deformed_cube", N, (nel, nel, nel), (0, 0, 0), ALL_FACES,
                   perturb_amp=amp, seed=seed)


def tgv_box(nel: int = 32, N: int = 7) -> BoxCase:
    """Fully periodic [0, 2pi]^3 box for the Taylor-Green vortex."""
    tp = 2 * math.pi
    return BoxCase("tgv", N, (nel, nel, nel), (1, 1, 1), 0, hi=(tp, tp, tp), rhs="tgv")


def batched_cases(nsolve: int = 64, seed: int = 0, emin: int = 8 ** 3, emax: int = 40 ** 3,
                  orders=(5, 7, 9)) -> list[BoxCase]:
    """Independent deformed-box Poisson problems of uneven size: E ~ U{emin..emax},
    nx = ny = floor(cbrt E), nz = round(E / nx^2), N ~ U(orders)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for s in range(nsolve):
        E = int(rng.integers(emin, emax + 1))
        N = int(rng.choice(np.asarray(orders)))
        nx = int(math.floor(round(E ** (1.0 / 3.0), 9)))
        nz = max(1, int(round(E / (nx * nx))))
        out.append(BoxCase(f"batched_{s}", N, (nx, nx, nz), (0, 0, 0), ALL_FACES,
                           perturb_amp=0.05, seed=int(rng.integers(0, 2 ** 31))))
    return out


def mlp_init(n_in: int, n_hidden: int, n_out: int, seed: int = 0) -> dict:
    """Seeded initial parameters of the element-local network (He-uniform
    weights, the output layer scaled by 0.01 so that training starts near the
    zero correction; zero biases), FP32: W1 [H, I], b1 [H], W2 [H, H], b2 [H],
    W3 [O, H], b3 [O]."""
    rng = np.random.Generator(np.random.PCG64(seed))

    def he(o, i):
        lim = math.sqrt(6.0 / i)
        return rng.uniform(-lim, lim, size=(o, i)).astype(np.float32)

    return {"W1": he(n_hidden, n_in), "b1": np.zeros(n_hidden, np.float32),
            "W2": he(n_hidden, n_hidden), "b2": np.zeros(n_hidden, np.float32),
            "W3": he(n_out, n_hidden) * np.float32(0.01), "b3": np.zeros(n_out, np.float32)}
