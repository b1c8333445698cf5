"""The dimensionless-groups helper (inputs.lattice_parameters): every group it is given is
recovered from the lattice parameters it returns, by the definitions in its docstring, and the
named workloads carry the groups they are quoted at."""
import math

import pytest

from paper_2407_12263_gb300 import inputs as I

CS2 = 1.0 / 3.0


def _groups(p, L0, U, D=None):
    rho1 = p["rho_ratio"]
    eta2 = p["tau_f"] * CS2           # rho2 = 1
    eta1 = p["mu_ratio"] * eta2
    return dict(Re=rho1 * U * L0 / eta1, Ca=eta1 * U / p["sigma"],
                We=rho1 * U * U * (L0 if D is None else D) / p["sigma"], Cn=p["xi"] / L0, Pe=U * L0 / p["M"])


@pytest.mark.parametrize("rho_ratio,mu_ratio", [(1.0, 1.0), (3.0, 1.0), (10.0, 10.0), (0.5, 4.0)])
def test_groups_are_recovered(rho_ratio, mu_ratio):
    L0, U = 128.0, 0.03
    p = I.lattice_parameters(L0, U, Re=400.0, rho_ratio=rho_ratio, mu_ratio=mu_ratio, Ca=0.2, Cn=0.05, Pe=50.0)
    g = _groups(p, L0, U)
    for k, v in dict(Re=400.0, Ca=0.2, Cn=0.05, Pe=50.0).items():
        assert g[k] == pytest.approx(v, rel=1e-13), k
    p2 = I.lattice_parameters(L0, U, Re=400.0, rho_ratio=rho_ratio, mu_ratio=mu_ratio, We=12.0, D=32.0)
    assert _groups(p2, L0, U, D=32.0)["We"] == pytest.approx(12.0, rel=1e-13)
    assert p2["xi"] == 4.0 and p2["M"] == 0.02  # the defaults when Cn and Pe are not given


def test_exactly_one_surface_tension_group():
    with pytest.raises(ValueError):
        I.lattice_parameters(64, 0.04, 100.0)
    with pytest.raises(ValueError):
        I.lattice_parameters(64, 0.04, 100.0, Ca=0.1, We=5.0)


def test_rayleigh_taylor_workload_groups():
    """128 x 128 x 512 box: At = 0.5, Re = 256 with fluid 1, U = sqrt(g W) = 0.04, Ca = 1."""
    w = I.WORKLOADS["rayleigh_taylor_128x128x512"]
    W = w["grid"][0]
    rho1 = w["rho_ratio"]
    assert (rho1 - 1.0) / (rho1 + 1.0) == pytest.approx(0.5, rel=1e-14)
    U = math.sqrt(-w["body_force"][2] * W)
    assert U == pytest.approx(0.04, rel=1e-14)
    g = _groups(w, W, U)
    assert g["Re"] == pytest.approx(256.0, rel=1e-13) and g["Ca"] == pytest.approx(1.0, rel=1e-13)


def test_taylor_green_workload_groups():
    """256^3: u0 = 0.04, Re = 1000 on L0, We = 20 on D = 2R = L0/4."""
    w = I.WORKLOADS["taylor_green_256"]
    g = _groups(w, 256, w["u0"], D=2 * w["R"])
    assert g["Re"] == pytest.approx(1000.0, rel=1e-13) and g["We"] == pytest.approx(20.0, rel=1e-13)
    assert w["R"] == 32.0
