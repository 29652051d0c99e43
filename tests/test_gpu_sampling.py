"""GPU rejection sampling of Voronoi sites (Sect. 2.4) against the oracle, through the C ABI: the
sites (positions and order) and the number of proposals must be identical, bit for bit."""
import numpy as np
import pytest

from helpers import to_gpu
from oracle.physics import lte_alpha_S
from oracle.sampling import rejection_sample
from synth import make_atmosphere
from synth.atmosphere import regular_fields

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2306_01041_gb300 as rt
    return rt


def _box(atm):
    return (0.0, atm.Lx, 0.0, atm.Ly, atm.zmin, atm.zmax)


def _check(rt, f, z, box, n, seed):
    f = np.ascontiguousarray(f, dtype=np.float32)
    xyz, nprop = rt.sample_sites(to_gpu(f), z, box, n, seed)
    ref, nref = rejection_sample(f, z, box, n, seed)
    got = xyz.cpu().numpy()
    assert nprop == nref
    assert np.array_equal(got, ref), np.abs(got - ref).max()
    return nprop


@pytest.mark.parametrize("seed", [5, 2 ** 63 + 11])
def test_density_target(rt, seed):
    """Sites following rho^0.3 of the synthetic atmosphere on a 32 x 32 x 48 mesh (mesh heights
    cell-centred, so proposals near the walls take the clamped end planes)."""
    atm = make_atmosphere(0)
    f, (x, y, z, dx, dy) = regular_fields(32, 32, 48, atm)
    target = (f["rho"] ** 0.3).reshape(48, 32, 32)
    _check(rt, target, z, _box(atm), 20000, seed)


def test_continuum_opacity_target_over_several_batches(rt):
    """The 500 nm continuum opacity (the paper's alpha_cont target) on a 24 x 24 x 64 mesh,
    floored at 1e-3 of its maximum: about one proposal in 83 is kept, so 60 000 sites come from
    more than one batch of 2^22 proposals."""
    atm = make_atmosphere(1)
    f, (x, y, z, dx, dy) = regular_fields(24, 24, 64, atm)
    a, _ = lte_alpha_S(f["T"], f["rho"], atm.kappa0, 500e-9)
    target = np.maximum(a / a.max(), 1e-3).reshape(64, 24, 24)
    nprop = _check(rt, target, z, _box(atm), 60000, seed=77)
    assert nprop > 2 ** 22


def test_constant_target_keeps_every_proposal(rt):
    z = np.linspace(-0.5, 2.5, 5)
    box = (0.0, 6.0, 0.0, 6.0, -0.5, 2.5)
    assert _check(rt, np.full((5, 3, 4), 2.0), z, box, 999, seed=3) == 999


def test_bad_targets_are_refused(rt):
    z = np.linspace(0.0, 1.0, 4)
    box = (0.0, 1.0, 0.0, 1.0, 0.0, 1.0)
    for f in (np.zeros((4, 2, 2)), np.full((4, 2, 2), -1.0)):
        with pytest.raises(rt.RTError):
            rt.sample_sites(to_gpu(np.asarray(f, np.float32)), z, box, 10, 1)
