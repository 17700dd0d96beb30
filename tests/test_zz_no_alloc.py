"""The allocation-free inner product (sem_glsc3_noalloc) agrees with sem_glsc3.

Some callers cannot allocate device memory -- host codes whose device memory
belongs to their own pool or framework allocator, fixed-budget embedded or
plugin contexts, loops that cannot take cudaMalloc's implicit synchronisation
-- so this entry point keeps its reduction scratch in a static device array
inside the library instead of a caller buffer.  The test calls it through the
C ABI twice in a row (different inputs; the static array keeps the previous
call's contents).  Both entry points run the same kernel with the same grid
and summation order, so each result must equal the scratch-taking entry
point's bit for bit; each is also checked against the oracle's unique-node
inner product at the bar of the other inner-product tests (1e-13 of the sum
of |a b / mult|).  This file is collected last on purpose.
"""
import numpy as np
import pytest

import oracle
from paper_2405_05640_gb300 import binding, inputs

pytestmark = pytest.mark.gpu


def test_glsc3_noalloc_matches_glsc3_twice():
    import torch
    case = inputs.channel(5, 7)
    V = case.vertices()
    gm = binding.Mesh(case.N, case.nel, case.periodic, case.faces, V)
    om = oracle.Mesh(case.N, case.nel, case.periodic, case.faces, V)
    rng = np.random.default_rng(123)
    for _ in range(2):
        a = om.scatter(rng.standard_normal(om.nglob))
        b = om.scatter(rng.standard_normal(om.nglob))
        ta, tb = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
        ref = gm.glsc3(ta, tb)
        got = gm.glsc3_noalloc(ta, tb)
        assert got == ref, (got, ref)
        want = om.glsc3(a, b)
        assert abs(got - want) <= 1e-13 * np.abs(a * b / om.mult).sum(), (got, want)
