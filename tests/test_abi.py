"""The C-ABI library loads on a machine without a GPU and exports every
function include/sem.h declares; host-side argument checks need no GPU."""
import ctypes
import os
import re

import pytest

from paper_2405_05640_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(sem_[a-z0-9_]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    build.build()
    return binding.lib()


def test_header_declares_the_boundary():
    d = _declared()
    for name in ("sem_mesh_create", "sem_ax", "sem_dssum", "sem_pcg_solve"):
        assert name in d


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing
    # and the binding marshals every declared entry point
    assert not (_declared() - set(binding.exported_names())), _declared() - set(binding.exported_names())


def test_host_side_argument_checks(lib):
    assert lib.sem_version().startswith(b"sem_gb300")
    d = binding.MeshDesc()
    d.N = 0
    d.nel[:] = [1, 1, 1]
    assert lib.sem_mesh_workspace_bytes(ctypes.byref(d)) == 0
    assert lib.sem_mesh_create(ctypes.byref(d), None, 0, None, ctypes.byref(ctypes.c_void_p())) == \
        binding.SEM_ERR_UNSUPPORTED
    d.N = 7
    d.nel[:] = [0, 1, 1]
    assert lib.sem_mesh_workspace_bytes(ctypes.byref(d)) == 0  # empty mesh rejected
    d.nel[:] = [2, 2, 2]
    assert lib.sem_mesh_workspace_bytes(ctypes.byref(d)) == 0  # NULL vertices rejected
    assert lib.sem_ax(None, None, None, 0, None) == binding.SEM_ERR_INVALID_ARG
    assert lib.sem_status_string(binding.SEM_ERR_NAN) == b"NaN or Inf in right-hand side"


def test_workspace_size_accounts_for_all_arrays(lib):
    import numpy as np
    from paper_2405_05640_gb300 import inputs
    case = inputs.channel(4, 7)
    V = np.ascontiguousarray(case.vertices())
    d = binding.MeshDesc()
    d.N = 7
    d.nel[:] = list(case.nel)
    d.periodic[:] = list(case.periodic)
    d.dirichlet_faces = case.faces
    d.vertices = V.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    n = lib.sem_mesh_workspace_bytes(ctypes.byref(d))
    nloc = case.nloc
    # G (6 per point) + B + mult + minv + dinv in FP64, at least
    assert n >= 8 * nloc * 10
    d.geom_flags = binding.SEM_GEOM_F32
    assert lib.sem_mesh_workspace_bytes(ctypes.byref(d)) >= n + 4 * nloc * 8


def test_schwarz_and_solver_option_host_checks(lib):
    """The hybrid Schwarz entry points reject bad arguments before any
    device work (no GPU needed)."""
    assert lib.sem_schwarz_workspace_bytes(None, None) == 0
    out = ctypes.c_void_p()
    assert lib.sem_schwarz_create(None, None, None, 0, None, ctypes.byref(out)) == binding.SEM_ERR_INVALID_ARG
    assert out.value is None
    assert lib.sem_schwarz_apply(None, None, None, 3, 1e-2, None) == binding.SEM_ERR_INVALID_ARG
    assert lib.sem_schwarz_problems(None) == -1
    assert lib.sem_schwarz_destroy(None) == binding.SEM_OK
    # the solver options carry the Schwarz handle, its coarse settings, the
    # double-float outer-residual switch and the intermediate multigrid level
    # at the end of the struct
    names = [f[0] for f in binding.PcgOpts._fields_]
    assert names[-9:] == ["schwarz", "coarse_iters", "coarse_tol", "outer_pair", "schwarz_mid", "mid_weight",
                          "inner_adapt", "krylov", "gmres_restart"]
    assert lib.sem_schwarz_mid_work_bytes(None) == 0
    assert lib.sem_schwarz_apply3(None, None, 0.15, None, None, 3, 1e-2, None, 0, None) == \
        binding.SEM_ERR_INVALID_ARG


def _header_struct(name):
    """(field, C type class) of `typedef struct { ... } name;` in sem.h, in
    declaration order."""
    text = open(os.path.join(ROOT, "include", "sem.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    m = re.search(r"typedef struct \{([^{}]*)\}\s*" + name + r"\s*;", text)
    assert m, name
    out = []
    for decl in m.group(1).split(";"):
        decl = " ".join(decl.split())
        if not decl:
            continue
        kind = "ptr" if "*" in decl else decl.split()[0]
        pieces = decl.replace("*", " ").split(",")
        out.append((pieces[0].split()[-1], kind))
        out += [(p.strip(), kind) for p in pieces[1:]]
    return out


@pytest.mark.parametrize("cname,pyname", [("sem_pcg_opts", "PcgOpts"), ("sem_pcg_stats", "PcgStats")])
def test_option_and_stats_structs_match_the_header(cname, pyname):
    """The binding's ctypes layouts follow the header field by field (name,
    order and type), so a field added to the C struct cannot shift the
    ones after it."""
    kinds = {"double": ctypes.c_double, "int": ctypes.c_int, "ptr": ctypes.c_void_p}
    want = [(n, kinds[k]) for n, k in _header_struct(cname)]
    got = list(getattr(binding, pyname)._fields_)
    assert got == want
