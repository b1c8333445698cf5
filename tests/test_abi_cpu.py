"""The C-ABI library loads, exports every symbol include/lbm.h declares, and checks its
arguments on the host (no GPU needed for any of these)."""
import ctypes
import re
from pathlib import Path

import numpy as np
import pytest

import oracle as O
from paper_2407_12263_gb300 import build as cuda_build
from paper_2407_12263_gb300 import lbm

ROOT = Path(__file__).resolve().parent.parent


@pytest.fixture(scope="module")
def lib():
    cuda_build.build()
    return lbm.load()


def _declared_functions():
    names = []
    for h in (ROOT / "include").glob("*.h"):
        text = re.sub(r"/\*.*?\*/", "", h.read_text(), flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[a-z_ ]+\**\s*\**(lbm_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = _declared_functions()
    assert len(names) >= 14
    for name in names:
        assert hasattr(lib, name), name
    assert {s[0] for s in lbm.SIGNATURES} >= set(names)


def _declared_arity():
    """Number of parameters of every lbm_* prototype in include/*.h (comments stripped)."""
    out = {}
    for h in (ROOT / "include").glob("*.h"):
        text = re.sub(r"/\*.*?\*/", "", h.read_text(), flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[a-z_ ]+\**\s*\**(lbm_\w+)\s*\(([^;{]*?)\)\s*;", text, flags=re.M | re.S):
            params = m.group(2).strip()
            out[m.group(1)] = 0 if params in ("", "void") else params.count(",") + 1
    return out


def _declared_return_types():
    out = {}
    for h in (ROOT / "include").glob("*.h"):
        text = re.sub(r"/\*.*?\*/", "", h.read_text(), flags=re.S)
        for m in re.finditer(r"^\s*((?:const\s+)?[a-z_ ]+?\s*\**)\s*(lbm_\w+)\s*\(", text, flags=re.M):
            out[m.group(2)] = " ".join(m.group(1).replace("*", " * ").split())
    return out


def test_binding_return_types_match_the_headers():
    want = {"int": ctypes.c_int, "void": None, "const char *": ctypes.c_char_p, "long long": ctypes.c_longlong,
            "double": ctypes.c_double}
    declared = _declared_return_types()
    for name, restype, _ in lbm.SIGNATURES:
        c_type = declared[name]
        if c_type.endswith("*") and c_type != "const char *":
            assert restype is ctypes.c_void_p, (name, c_type, restype)  # a handle
        else:
            assert restype is want[c_type], (name, c_type, restype)


def test_binding_argument_counts_match_the_headers():
    """Every signature the ctypes binding declares takes as many arguments as the C prototype."""
    arity = _declared_arity()
    assert len(arity) >= 14
    for name, _, argtypes in lbm.SIGNATURES:
        assert name in arity, name
        assert len(argtypes) == arity[name], (name, len(argtypes), arity[name])


def test_library_is_built_for_sm_103a():
    assert "arch=compute_103a,code=sm_103a" in " ".join(cuda_build.ARCH)
    assert lbm.library_path().exists()


@pytest.mark.parametrize("Q", [9, 19])
def test_lattice_tables_match_documented_order_and_oracle(lib, Q):
    d, e, w = lbm.lbm_lattice_tables(Q)
    do, eo, to = O.lattice(Q)
    assert d == do
    np.testing.assert_array_equal(e, eo)
    np.testing.assert_allclose(w, to, rtol=0, atol=1e-16)


def _create(**over):
    args = dict(grid=(8, 8, 8), lattice=19, tau_f=0.8, tau_g=0.8, M=0.02, xi=4.0, sigma=1e-3,
                rho_ratio=1.0, mu_ratio=1.0, body_force=(0.0, 0.0, 0.0))
    args.update(over)
    return lbm.lbm_create(**args)


@pytest.mark.parametrize("over", [
    dict(lattice=7), dict(grid=(2, 8, 8)), dict(grid=(8, 2, 8)), dict(grid=(8, 8, 2)),
    dict(lattice=9, grid=(8, 8, 2)), dict(grid=(8, 8, 70000)), dict(grid=(2048, 2048, 1024)),
    dict(tau_f=0.0), dict(tau_f=float("nan")), dict(M=0.0, tau_g=0.0), dict(M=-1.0, tau_g=-1.0),
    dict(xi=1.5), dict(xi=float("inf")), dict(sigma=-1e-3), dict(rho_ratio=0.0), dict(mu_ratio=-2.0),
    dict(body_force=(0.0, float("nan"), 0.0)), dict(lattice=9, grid=(8, 8, 1), body_force=(0.0, 0.0, 1e-5)),
])
def test_create_rejects_invalid_arguments(lib, over):
    with pytest.raises(lbm.LBMError) as exc:
        _create(**over)
    assert exc.value.status == lbm.LBM_EINVAL
    assert lbm.lbm_last_error(None) != "no error"


@pytest.mark.parametrize("field,value", [("scheme", 5), ("storage", 3), ("storage", -1), ("walls", 8), ("walls", -1), ("courant", 0.0),
                                         ("courant", 1.5), ("graph_steps", 1), ("graph_steps", 3),
                                         ("graph_steps", -2)])
def test_create_rejects_invalid_options(lib, field, value):
    o = lbm.lbm_default_opts()
    setattr(o, field, value)
    with pytest.raises(lbm.LBMError) as exc:
        _create(opts=o)
    assert exc.value.status == lbm.LBM_EINVAL


def test_default_options(lib):
    o = lbm.lbm_default_opts()
    assert (o.scheme, o.storage, o.courant, o.walls, o.graph_steps) == (0, 0, 0.997, 0, 32)
    assert o.stream is None


def test_null_handle_calls_fail_cleanly(lib):
    assert lib.lbm_step(None, 1) == lbm.LBM_EINVAL
    assert lib.lbm_mass(None, None, None) == lbm.LBM_EINVAL
    assert lib.lbm_launch_count(None) == 0
    assert lib.lbm_surrogate_reserve(None, 2) == lbm.LBM_EINVAL
    lib.lbm_destroy(None)
    out = ctypes.c_void_p()
    assert lib.lbm_create(ctypes.byref(out), None, 19, 0.8, 0.8, 0.02, 4.0, 1e-3, 1.0, 1.0, None, None) == lbm.LBM_EINVAL
    assert lib.lbm_create(None, None, 19, 0.8, 0.8, 0.02, 4.0, 1e-3, 1.0, 1.0, None, None) == lbm.LBM_EINVAL


def test_product_path_does_not_import_the_oracle():
    pkg = ROOT / "paper_2407_12263_gb300"
    for src in list(pkg.rglob("*.py")) + list(pkg.rglob("*.cu")) + list(pkg.rglob("*.cuh")) + list(pkg.rglob("*.h")):
        text = src.read_text()
        assert "import oracle" not in text and "from oracle" not in text and "lbm_oracle" not in text, src


def _case(**over):
    c = dict(grid=(8, 8, 8), lattice=19, tau_f=0.8, tau_g=0.8, M=0.02, xi=4.0, sigma=1e-3)
    c.update(over)
    return lbm.make_case(**c)


@pytest.mark.parametrize("cases,opts", [
    ([], None),
    ([_case(), _case(lattice=9, grid=(8, 8, 1))], None),
    ([_case(storage=4)], None),
    ([_case(storage=-1)], None),
    ([_case(grid=(2, 8, 8))], None),
    ([_case()], dict(graph_steps=3)),
    ([_case()], dict(graph_steps=-2)),
])
def test_batch_create_rejects_invalid_arguments(lib, cases, opts):
    o = None
    if opts:
        o = lbm.lbm_batch_default_opts()
        for k, v in opts.items():
            setattr(o, k, v)
    with pytest.raises(lbm.LBMError) as exc:
        lbm.lbm_batch_create(cases, o)
    assert exc.value.status == lbm.LBM_EINVAL
    assert lbm.lbm_batch_last_error(None) != "no error"


def test_batch_null_calls_fail_cleanly(lib):
    assert lib.lbm_batch_step(None, 1) == lbm.LBM_EINVAL
    assert lib.lbm_batch_tune(None, 1) == lbm.LBM_EINVAL
    assert lib.lbm_batch_case(None, 0) is None
    assert lib.lbm_batch_case_config(None, 0, None, None, None) == lbm.LBM_EINVAL
    assert lib.lbm_batch_set_config(None, 0, None, 0) == lbm.LBM_EINVAL
    assert lib.lbm_batch_launch_count(None) == 0
    lib.lbm_batch_destroy(None)
    o = lbm.lbm_batch_default_opts()
    assert (o.stream, o.graph_steps) == (None, 32)


def test_rising_bubble_recipe_matches_its_groups():
    """The seeded batch recipe: grid and radius rules, ranges, and the Eotvos and Morton numbers
    recomputed from the lattice parameters."""
    from paper_2407_12263_gb300 import inputs as I
    cases = I.rising_bubble_cases()
    assert len(cases) == 256
    assert cases == I.rising_bubble_cases()  # seeded
    for c in cases:
        s = c["grid"][0]
        assert s in (32, 48, 64, 96) and c["grid"][1] == s and c["grid"][2] in (s, 2 * s)
        assert c["R"] == s / 8 and c["walls"] == 7
        assert 2 <= c["rho_ratio"] <= 10 and 1 <= c["mu_ratio"] <= 10
        D, g, drho = 2 * c["R"], -c["body_force"][2], c["rho_ratio"] - 1
        eta2 = c["tau_f"] / 3.0
        eta1 = eta2 * c["mu_ratio"]
        assert drho * g * D * D / c["sigma"] == pytest.approx(c["Eo"], rel=1e-12)
        assert g * eta1 ** 4 * drho / (c["rho_ratio"] ** 2 * c["sigma"] ** 3) == pytest.approx(c["Mo"], rel=1e-12)
        assert 1 <= c["Eo"] <= 50 and 1e-5 <= c["Mo"] <= 1e-1
        assert np.sqrt(g * D) == pytest.approx(c["U"], rel=1e-12) and 0.04 <= c["U"] <= 0.1


@pytest.mark.parametrize("Q,grid,storage,pair", [
    (19, (128, 128, 128), 0, 8), (19, (37, 21, 19), 1, 4), (19, (8, 8, 8), 2, 4), (19, (9, 7, 5), 0, 8), (19, (9, 7, 5), 1, 4),
    (9, (64, 64, 1), 0, 8), (9, (45, 39, 1), 1, 4),
])
def test_state_bytes_is_the_documented_layout(lib, Q, grid, storage, pair):
    """8 B of zeroth moments per cell (padded to a multiple of 16 B for FP32 storage) plus Q - 1
    moving pairs of 8 B (FP32) or 4 B (16-bit) per cell."""
    n = grid[0] * grid[1] * grid[2]
    moments = (8 * n + 15) // 16 * 16 if storage == 0 else 8 * n
    assert lbm.lbm_state_bytes(Q, grid, storage) == moments + (Q - 1) * pair * n


def test_state_bytes_rejects_invalid_arguments(lib):
    assert lbm.lbm_state_bytes(7, (8, 8, 8), 0) == 0
    assert lbm.lbm_state_bytes(19, (8, 8, 8), 3) == 0
    assert lbm.lbm_state_bytes(19, (0, 8, 8), 0) == 0
    assert lbm.lbm_state_bytes(19, (2048, 2048, 1024), 0) == 0


def test_projection_workspace_and_argument_checks(lib):
    """Host-side checks of lbm_project_solenoidal: its workspace size is the twiddles (padded to
    256 bytes) plus three complex FP32 planes, and invalid calls return LBM_EINVAL before any
    launch (NULL pointers, extents outside 1 .. 512)."""
    from paper_2407_12263_gb300 import lbm
    assert lbm.lbm_project_workspace_bytes((64, 64, 64)) == 1536 + 3 * 64 ** 3 * 8
    assert lbm.lbm_project_workspace_bytes((9, 7, 5)) == 256 + 3 * 9 * 7 * 5 * 8
    for bad in ((0, 4, 4), (4, 4, 513), (-1, 2, 2)):
        assert lbm.lbm_project_workspace_bytes(bad) == -1
    assert lbm.lbm_project_solenoidal(0, (4, 4, 4), 0, 1 << 20, None) == lbm.LBM_EINVAL
    assert lbm.lbm_project_solenoidal(16, (4, 4, 600), 16, 1 << 30, None) == lbm.LBM_EINVAL
