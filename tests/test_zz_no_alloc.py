"""The allocation-free inner product (sem_glsc3_noalloc) agrees with sem_glsc3.

Some callers cannot allocate device memory -- host codes whose device memory
belongs to their own pool or framework allocator, fixed-budget embedded or
plugin contexts, loops that cannot take cudaMalloc's implicit synchronisation
-- so this entry point keeps its reduction scratch in a static device array
inside the library instead of a caller buffer.  The test calls it through the
C ABI twice in a row (different inputs; the static array keeps the previous
call's contents) and compares each result with the scratch-taking entry
point's.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_2405_05640_gb300 import binding, inputs

pytestmark = pytest.mark.gpu


def test_glsc3_noalloc_matches_glsc3_twice():
    import torch
    case = inputs.channel(5, 7)
    gm = binding.Mesh(case.N, case.nel, case.periodic, case.faces, case.vertices())
    rng = np.random.default_rng(123)
    for _ in range(2):
        a = gm.scatter(torch.from_numpy(rng.standard_normal(gm.nglob)).cuda())
        b = gm.scatter(torch.from_numpy(rng.standard_normal(gm.nglob)).cuda())
        ref = gm.glsc3(a, b)
        got = gm.glsc3_noalloc(a, b)
        scale = float((a * b).abs().sum())
        assert abs(got - ref) <= 1e-13 * scale, (got, ref)
