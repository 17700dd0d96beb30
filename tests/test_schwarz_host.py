"""Host logic of the hybrid Schwarz set-up, without a GPU: the library's 1-D
fast-diagonalisation problems against the oracle's assembly (oracle/
schwarz.py: extended_1d) and scipy's generalised eigensolver, and the local-
solve kernel's line tables (every line exactly once per pass; no bank shared
within a 32-lane group where the strides allow it)."""
from collections import Counter

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import schwarz as sw
from paper_2405_05640_gb300 import binding, build, inputs


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()


@pytest.mark.parametrize("N", [2, 3, 5, 7, 9])
@pytest.mark.parametrize("flags", [0b0011, 0b0001, 0b0010, 0b0111, 0b1011, 0b0000])
def test_fdm_1d_matches_oracle_assembly(N, flags):
    h, hL, hR = 0.37, 0.21, 0.58
    hasL, hasR, dirL, dirR = bool(flags & 1), bool(flags & 2), bool(flags & 4), bool(flags & 8)
    A, B, _ = sw.extended_1d(N, h, hL, hR, hasL, hasR, dirL, dirR)
    S, lam = binding.schwarz_fdm_1d(N, h, hL, hR, flags)
    scale = np.abs(A).max()
    # A S = B S Lambda and S^T B S = I
    assert np.abs(A @ S - B @ S @ np.diag(lam)).max() <= 1e-11 * scale
    assert np.abs(S.T @ B @ S - np.eye(N + 3)).max() <= 1e-11
    np.testing.assert_allclose(np.sort(lam), sla.eigh(A, B, eigvals_only=True), rtol=1e-11,
                               atol=1e-11 * np.abs(lam).max())


def test_fdm_1d_argument_checks():
    with pytest.raises(binding.SemError) as ei:
        binding.schwarz_fdm_1d(1, 1.0, 1.0, 1.0, 3)
    assert ei.value.status == binding.SEM_ERR_UNSUPPORTED
    with pytest.raises(binding.SemError) as ei:
        binding.schwarz_fdm_1d(5, 0.0, 1.0, 1.0, 3)
    assert ei.value.status == binding.SEM_ERR_INVALID_ARG
    with pytest.raises(binding.SemError) as ei:
        binding.schwarz_fdm_1d(5, 1.0, 1.0, 1.0, 16)
    assert ei.value.status == binding.SEM_ERR_INVALID_ARG


@pytest.mark.parametrize("N", range(2, 10))
def test_line_tables_deal_every_line_once(N):
    ne = N + 3
    tab, pj, pk = binding.schwarz_line_table(N)
    lpt = -(-ne * ne // 32)
    assert tab.shape == (3, 32 * lpt)
    assert pj >= ne and pk >= pj * ne
    # the K passes keep the natural order (their global accesses coalesce)
    assert tab[2][:ne * ne].tolist() == list(range(ne * ne)) and (tab[2][ne * ne:] == -1).all()
    for ax in range(3):
        ids = tab[ax][tab[ax] >= 0]
        assert sorted(ids.tolist()) == list(range(ne * ne)), ax
        # bank spread of each 32-lane group
        worst = 0
        for q in range(lpt):
            g = tab[ax][32 * q:32 * (q + 1)]
            g = g[g >= 0]
            c1, c2 = g % ne, g // ne
            base = pj * c1 + pk * c2 if ax == 0 else (c1 + pk * c2 if ax == 1 else c1 + pj * c2)
            if len(base):
                worst = max(worst, max(Counter((base % 32).tolist()).values()))
        if N in (3, 4, 6, 7):  # strides chosen so that no bank holds more than LPT line starts
            assert worst == 1, (N, ax, worst)


COARSE_CASES = [
    inputs.channel(3, 7),
    inputs.deformed_cube(3, 5),
    inputs.BoxCase("x1_periodic", 4, (1, 3, 2), (1, 0, 1), inputs.Y_FACES),
    inputs.BoxCase("x2_periodic", 3, (2, 2, 3), (1, 1, 0), 0b110000, jitter=0.1, seed=3),
]


@pytest.mark.parametrize("case", COARSE_CASES, ids=[c.name for c in COARSE_CASES])
def test_coarse_stencil_equals_oracle_trilinear_operator(case):
    """The coarse level's assembled 27-point stencil (the set-up's own code,
    run on the host) against the oracle's N = 1 operator on the same
    vertices, assembled column by column: entries, Dirichlet rows/columns,
    periodic aliases (one and two elements across a periodic direction) and
    the inverse diagonal."""
    import oracle
    V = case.vertices()
    mc = oracle.Mesh(1, case.nel, case.periodic, case.faces, V)
    sten, cdinv = binding.schwarz_coarse_operator(case.nel, case.periodic, case.faces, mc.G)
    nel, per = case.nel, case.periodic
    nv = [n + (0 if p else 1) for n, p in zip(nel, per)]
    nvt = nv[0] * nv[1] * nv[2]

    def vid(vx, vy, vz):
        if per[0] and vx == nel[0]:
            vx = 0
        if per[1] and vy == nel[1]:
            vy = 0
        if per[2] and vz == nel[2]:
            vz = 0
        return vx + nv[0] * (vy + nv[1] * vz)

    # the library's vertex numbering against the oracle's global nodes
    to_g = np.full(nvt, -1)
    for e in range(mc.E):
        ex, ey, ez = e % nel[0], (e // nel[0]) % nel[1], e // (nel[0] * nel[1])
        for c in range(8):
            v = vid(ex + (c & 1), ey + ((c >> 1) & 1), ez + (c >> 2))
            g = mc.gid[e * 8 + c]
            assert to_g[v] in (-1, g)
            to_g[v] = g
    assert (to_g >= 0).all() and len(set(to_g.tolist())) == nvt == mc.nglob
    # dense library operator
    A = np.zeros((nvt, nvt))
    for v in range(nvt):
        vx, vy, vz = v % nv[0], (v // nv[0]) % nv[1], v // (nv[0] * nv[1])
        for o in range(27):
            ox, oy, oz = o % 3 - 1, (o // 3) % 3 - 1, o // 9 - 1
            c = []
            for w, d, n, p in ((vx, ox, nv[0], per[0]), (vy, oy, nv[1], per[1]), (vz, oz, nv[2], per[2])):
                w = w + d
                if p:
                    w %= n
                c.append(w if 0 <= w < n else -1)
            if min(c) < 0:
                assert sten[o, v] == 0
                continue
            A[to_g[v], to_g[c[0] + nv[0] * (c[1] + nv[1] * c[2])]] += sten[o, v]
    # dense oracle operator, Dirichlet rows and columns removed
    first = np.zeros(mc.nglob, dtype=np.int64)
    first[mc.gid[::-1]] = np.arange(mc.nloc)[::-1]
    free = mc.apply_mask(np.ones(mc.nloc))[first] != 0
    Ao = np.zeros((mc.nglob, mc.nglob))
    for c in range(mc.nglob):
        if not free[c]:
            continue
        eg = np.zeros(mc.nglob)
        eg[c] = 1.0
        Ao[:, c] = mc.apply(eg[mc.gid])[first]
    Ao[~free, :] = 0.0
    scale = np.abs(Ao).max()
    assert np.abs(A - Ao).max() <= 2e-6 * scale
    dg = np.diag(Ao)
    ref = np.where(free, 1.0 / np.where(free, dg, 1.0), 0.0)
    np.testing.assert_allclose(cdinv[np.argsort(to_g)], ref, rtol=2e-6, atol=0)
