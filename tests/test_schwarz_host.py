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
from paper_2405_05640_gb300 import binding, build


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
