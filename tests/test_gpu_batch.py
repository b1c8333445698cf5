"""Batches of independent cases advanced by one launch per step (lbm_batch_*).

Every cell of a batch runs the same code as the single-case kernel, so each case must give the
same bits as its own handle advanced by lbm_step: the tests compare populations with exact
equality. The single-case path is itself compared with the FP64 oracle elsewhere; one test
here also compares a batch case with the oracle directly.
"""
import numpy as np
import pytest

import oracle as O
from paper_2407_12263_gb300 import build as cuda_build
from paper_2407_12263_gb300 import inputs as I
from paper_2407_12263_gb300 import lbm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    cuda_build.build()
    lbm.load()


CASE_KEYS = ("grid", "lattice", "tau_f", "tau_g", "M", "xi", "sigma", "rho_ratio", "mu_ratio", "body_force", "walls")


def _mixed_cases():
    """Uneven grids, periodic and walled, density and viscosity ratios, gravity, 16-bit storage."""
    base = dict(lattice=19, tau_f=0.8, tau_g=0.8, M=0.02, xi=4.0, sigma=1e-3, rho_ratio=1.0, mu_ratio=1.0,
                body_force=(0.0, 0.0, 0.0), walls=0, storage=0)
    specs = [dict(grid=(20, 14, 11)),
             dict(grid=(33, 17, 9), rho_ratio=3.0, mu_ratio=2.0, body_force=(1e-5, 0.0, -2e-5), walls=4),
             dict(grid=(16, 16, 16), storage=lbm.LBM_STORAGE_FP16, walls=7, rho_ratio=2.0, body_force=(0, 0, -1e-5)),
             dict(grid=(48, 48, 24), tau_f=0.3, sigma=5e-3),
             dict(grid=(12, 40, 8), storage=lbm.LBM_STORAGE_BF16, walls=3, mu_ratio=4.0),
             dict(grid=(9, 7, 5), courant=1.0),
             dict(grid=(32, 32, 32), sigma=2e-3)]  # rows of whole warps: dedicated launches by default
    out = []
    for s in specs:
        c = dict(base)
        c.update(s)
        out.append(c)
    return out


def _fields(c, seed):
    phi0 = I.multi_droplet_phi(c["grid"], seed=seed, count=2, r_range=(2.0, 4.0), xi=3.0)
    u0 = I.smooth_velocity(c["grid"], seed=seed + 1, amplitude=0.01)
    return phi0, u0


def _make_batch(cases, **kw):
    structs = [lbm.make_case(**{k: c[k] for k in CASE_KEYS}, storage=c.get("storage", 0),
                             courant=c.get("courant", 0.0)) for c in cases]
    return lbm.Batch(structs, **kw)


def _single(c):
    return lbm.Lattice(c["grid"], c["lattice"], **{k: c[k] for k in CASE_KEYS[2:]},
                       storage=c.get("storage", 0), courant=c.get("courant", 0.997), graph_steps=0)


def _init_pair(cases, **kw):
    batch = _make_batch(cases, **kw)
    singles = []
    for k, c in enumerate(cases):
        phi0, u0 = _fields(c, 100 + k)
        batch.case(k).init_phi(phi0, u0)
        s = _single(c)
        s.init_phi(phi0, u0)
        singles.append(s)
    return batch, singles


def _assert_same(batch, singles):
    for k, s in enumerate(singles):
        fb, gb = batch.case(k).get_pops()
        fs, gs = s.get_pops()
        np.testing.assert_array_equal(fb, fs, err_msg=f"case {k} f")
        np.testing.assert_array_equal(gb, gs, err_msg=f"case {k} g")


@pytest.mark.parametrize("graph_steps", [0, 4])
def test_batch_equals_single_handles_bit_for_bit(graph_steps):
    cases = _mixed_cases()
    batch, singles = _init_pair(cases, graph_steps=graph_steps)
    m0 = [batch.case(k).mass()[0] for k in range(len(cases))]
    batch.step(11)
    for s in singles:
        s.step(11)
    _assert_same(batch, singles)
    assert [batch.case(k).mass()[0] for k in range(len(cases))] == m0
    assert batch.launch_count > 0 and batch.launch_count % 11 == 0


def test_batch_follows_steps_of_a_single_case():
    """A case advanced on its own between batch steps stays consistent (the batch rebuilds its
    table from the handles' buffers)."""
    cases = _mixed_cases()[:3]
    batch, singles = _init_pair(cases, graph_steps=2)
    batch.step(5)
    batch.case(1).step(3)
    batch.step(4)
    for k, s in enumerate(singles):
        s.step(5 + 4 + (3 if k == 1 else 0))
    _assert_same(batch, singles)


def test_default_forms():
    """Without tuning: dedicated launches for rows of whole warps (nx a multiple of 32, at least
    2^15 cells), group launches of tiles 2^a x 8 x 128/(8 2^a) otherwise."""
    cases = _mixed_cases()
    batch = _make_batch(cases)
    for k, c in enumerate(cases):
        tile, storage, dedicated = batch.config(k)
        nx = c["grid"][0]
        assert dedicated == (nx % 32 == 0 and np.prod(c["grid"]) >= 32768)
        assert tile[0] * tile[1] * tile[2] == 128
        if nx >= 8:
            assert nx % tile[0] == 0 or tile[0] == 8


def test_tuner_keeps_the_state_and_picks_valid_tiles():
    cases = _mixed_cases()
    batch, singles = _init_pair(cases)
    batch.step(3)
    before = [batch.case(k).get_pops() for k in range(len(cases))]
    batch.tune(trial_steps=2)
    for k in range(len(cases)):
        after = batch.case(k).get_pops()
        np.testing.assert_array_equal(before[k][0], after[0])
        np.testing.assert_array_equal(before[k][1], after[1])
        tile, storage, dedicated = batch.config(k)
        assert tile[0] * tile[1] * tile[2] == 128 and tile[0] >= 8 or cases[k]["grid"][0] < 8
        assert storage == cases[k]["storage"]
    batch.step(6)
    for s in singles:
        s.step(9)
    _assert_same(batch, singles)


@pytest.mark.parametrize("dedicated", [False, True])
def test_forms_set_by_hand_give_the_same_bits(dedicated):
    """Every case in group launches with odd tile shapes, or every case in dedicated launches,
    graph-replayed: still the bits of the single handles."""
    cases = _mixed_cases()
    batch, singles = _init_pair(cases, graph_steps=4)
    shapes = [(8, 4, 4), (16, 1, 8), (8, 16, 1), (32, 4, 1), (8, 2, 8), (16, 8, 1), (8, 8, 2)]
    for k in range(len(cases)):
        batch.set_config(k, shapes[k], dedicated)
        assert batch.config(k)[0] == shapes[k] and batch.config(k)[2] == dedicated
    batch.step(9)
    for s in singles:
        s.step(9)
    _assert_same(batch, singles)
    with pytest.raises(lbm.LBMError) as e:
        batch.set_config(0, (16, 16, 1))
    assert e.value.status == lbm.LBM_EINVAL
    with pytest.raises(lbm.LBMError) as e:
        batch.set_config(0, (12, 2, 2))
    assert e.value.status == lbm.LBM_EINVAL


def test_auto_storage_is_chosen_before_init_and_used():
    c = dict(_mixed_cases()[1])
    c["storage"] = lbm.LBM_STORAGE_AUTO
    cases = [c, dict(c, grid=(24, 24, 24))]
    batch = _make_batch(cases)
    batch.tune(trial_steps=2)
    chosen = [batch.config(k)[1] for k in range(2)]
    assert all(s in (0, 1, 2) for s in chosen)
    singles = []
    for k, cc in enumerate(cases):
        phi0, u0 = _fields(cc, 300 + k)
        batch.case(k).init_phi(phi0, u0)
        s = _single(dict(cc, storage=chosen[k]))
        s.init_phi(phi0, u0)
        singles.append(s)
    batch.step(7)
    for s in singles:
        s.step(7)
    _assert_same(batch, singles)


def test_batch_case_against_the_oracle():
    """A walled bubble case of the rising-bubble recipe, advanced in a batch with a second
    case, against the FP64 oracle (the FP32 bounds of the parity tests). It starts from a
    uniform pressure under gravity, like the Rayleigh-Taylor box, whose top-wall transient makes
    the trajectory follow rounding after a few tens of steps, so the comparison is at step 10."""
    bc = dict(I.rising_bubble_cases(n=1, seed=7, sizes=(32,), heights=(1,))[0])
    cases = [bc, dict(_mixed_cases()[0])]
    batch = _make_batch(cases)
    phi0 = I.bubble_phi(bc)
    batch.case(0).init_phi(phi0)
    phi1, u1 = _fields(cases[1], 5)
    batch.case(1).init_phi(phi1, u1)
    ref = O.Oracle(19, bc["grid"], bc["tau_f"], bc["tau_g"], bc["M"], bc["xi"], bc["sigma"], bc["rho_ratio"],
                   bc["mu_ratio"], bc["body_force"], walls=bc["walls"])
    ref.init_phi(phi0)
    batch.step(10)
    ref.step(10)
    (phi_g, p_g, u_g), (phi_o, p_o, u_o) = batch.case(0).moments(), ref.moments()
    assert np.abs(phi_g - phi_o).max() <= 1e-4
    assert np.linalg.norm(u_g - u_o) / np.linalg.norm(u_o) <= 1e-3
    assert np.abs(p_g - p_o).max() <= 1e-6


def test_batch_errors_and_ownership():
    cases = _mixed_cases()[:2]
    batch = _make_batch(cases)
    with pytest.raises(lbm.LBMError) as e:
        batch.step(1)
    assert e.value.status == lbm.LBM_ESTATE
    with pytest.raises(lbm.LBMError) as e:
        batch.tune(0)
    assert e.value.status == lbm.LBM_EINVAL
    with pytest.raises(lbm.LBMError) as e:
        batch.step(-1)
    assert e.value.status == lbm.LBM_EINVAL
    with pytest.raises(lbm.LBMError):
        lbm.lbm_batch_case(batch.b, 2)
    for k, c in enumerate(cases):
        batch.case(k).init_phi(_fields(c, k)[0])
    lbm.lbm_destroy(batch.case(0).h)  # a batch case: left to the batch
    batch.step(2)
    assert np.isfinite(batch.case(0).moments()[0]).all()
    batch.close()


def test_full_batch_of_rising_bubbles_in_the_benchmarked_configuration():
    """The 256 seeded rising-bubble cases of the batched workload at full size, FP32, in the
    default forms and with the graph-replayed step the benchmark times (32-step graphs after a
    whole graph of warm-up): after 36 steps every case keeps its sum phi exactly, eight sampled
    cases (group and dedicated forms) equal their own handles advanced alone bit for bit, and
    one more step of a sampled case matches the FP64 oracle started from the batch's state
    (the one-step bound of the parity tests, 2e-7, scaled by the populations' size where the
    density ratio makes them larger than 1)."""
    cases = I.rising_bubble_cases()
    assert len(cases) == 256
    structs = [lbm.make_case(**{k: c[k] for k in CASE_KEYS}, storage=lbm.LBM_STORAGE_FP32) for c in cases]
    batch = lbm.Batch(structs)
    for k, c in enumerate(cases):
        batch.case(k).init_phi(I.bubble_phi(c))
    sums = [batch.case(k).mass()[0] for k in range(len(cases))]
    batch.step(32)
    batch.step(36)
    assert [batch.case(k).mass()[0] for k in range(len(cases))] == sums
    forms = set()
    for k in range(0, 256, 32):
        c = cases[k]
        forms.add(batch.config(k)[2])
        s = lbm.Lattice(c["grid"], 19, **{key: c[key] for key in CASE_KEYS[2:]})
        s.init_phi(I.bubble_phi(c))
        s.step(68)
        fb, gb = batch.case(k).get_pops()
        fs, gs = s.get_pops()
        np.testing.assert_array_equal(fb, fs, err_msg=f"case {k} f")
        np.testing.assert_array_equal(gb, gs, err_msg=f"case {k} g")
        s.close()
    assert forms == {True, False}  # both forms among the samples
    k = 96
    c = cases[k]
    ref = O.Oracle(19, c["grid"], c["tau_f"], c["tau_g"], c["M"], c["xi"], c["sigma"], c["rho_ratio"], c["mu_ratio"],
                   c["body_force"], walls=c["walls"])
    f0, g0 = batch.case(k).get_pops()
    ref.set_pops(f0, g0)
    batch.case(k).step(1)
    ref.step(1)
    (fb, gb), (fo, go) = batch.case(k).get_pops(), ref.get_pops()
    np.testing.assert_allclose(fb, fo, rtol=0, atol=2e-7 * max(1.0, np.abs(fo).max()))
    np.testing.assert_allclose(gb, go, rtol=0, atol=2e-7 * max(1.0, np.abs(go).max()))
    batch.close()
