"""The seeded input generators (paper_1307_2665_gb300/inputs.py) against the
recipes they implement: the workloads' coefficient fields, the boundary data
and the sampling helpers.  They hold none of the method's arithmetic."""
import numpy as np
import pytest

from paper_1307_2665_gb300 import hps
from paper_1307_2665_gb300 import inputs as I
from paper_1307_2665_gb300.build import build

UNIT = (0.0, 1.0, 0.0, 1.0)
SKEW = (-0.3, 0.9, 0.1, 1.7)


@pytest.fixture(scope="module", autouse=True)
def _built():
    build()


@pytest.mark.parametrize("fn", [I.convection_diffusion, I.gaussian_bump_helmholtz,
                                lambda x, y: I.random_smooth_operator(3, x, y)])
def test_leaf_grid_sampling_equals_pointwise_sampling(fn):
    """The tensor-product evaluation used for large grids gives the same values
    as evaluating the field at every node of hps_cheb_nodes."""
    nx, ny, p = 3, 2, 8
    xy = hps.hps_cheb_nodes(SKEW, nx, ny, p)
    xs = xy[:nx, 0, :, 0].reshape(-1)
    ys = xy[::nx, :, 0, 1].reshape(-1)
    grid = I.sample_on_leaf_grid(fn, xs, ys, nx, ny, p)
    point = fn(xy[..., 0], xy[..., 1])
    for k in I.COEFF_NAMES:
        if point.get(k) is None:
            assert grid[k] is None
        else:
            ref = np.broadcast_to(point[k], (nx * ny, p, p))
            assert np.array_equal(grid[k], ref), k


@pytest.mark.parametrize("dom", [UNIT, SKEW])
def test_fourier_data_is_continuous_around_the_boundary(dom):
    """f is a periodic function of the counter-clockwise arclength, so the two
    sides meeting at each corner agree there (the corner averaging of Step 1
    assumes continuous data)."""
    x0, x1, y0, y1 = dom
    e = 1e-9
    pairs = [((x1 - e, y0), (x1, y0 + e)), ((x1, y1 - e), (x1 - e, y1)),
             ((x0 + e, y1), (x0, y1 - e)), ((x0, y0 + e), (x0 + e, y0))]
    for seed in (0, 5):
        for a, b in pairs:
            fa = I.fourier_boundary(seed, np.array([a[0]]), np.array([a[1]]), dom)
            fb = I.fourier_boundary(seed, np.array([b[0]]), np.array([b[1]]), dom)
            assert abs(fa[0] - fb[0]) < 1e-5


def test_fourier_data_seeds_and_bank():
    bxy = hps.hps_boundary_nodes_grid(UNIT, 4, 3, 6)
    x, y = bxy[:, 0], bxy[:, 1]
    f0 = I.fourier_boundary(0, x, y, UNIT)
    assert np.array_equal(f0, I.fourier_boundary(0, x, y, UNIT))  # reproducible
    assert not np.allclose(f0, I.fourier_boundary(1, x, y, UNIT))  # seeds differ
    bank = I.fourier_boundary_bank(0, x, y, UNIT, 3)
    assert bank.shape == (3, len(x))
    np.testing.assert_allclose(bank[0], f0, rtol=0, atol=1e-12)  # first row = one draw of 40
    s = I.boundary_arclength(x, y, UNIT)
    assert np.all(np.diff(s) > 0) and s[0] > 0 and s[-1] < 4.0  # Gamma order: counter-clockwise


def test_smooth_fields_have_the_stated_scales():
    """Each field's maximum modulus on the 129 x 129 grid of [0,1]^2 is 1, so
    c11, c22 = 1 + 0.5 field, c12 = 0.2 field, c1, c2 = +-50 field reach their
    stated bounds there; c = 0."""
    g = np.linspace(0.0, 1.0, 129)
    gx, gy = np.meshgrid(g, g)
    for seed in (0, 7):
        assert np.max(np.abs(I.smooth_field(seed, gx, gy))) == pytest.approx(1.0, abs=1e-14)
        co = I.random_smooth_operator(seed, gx, gy)
        assert np.max(np.abs(co["c11"] - 1.0)) == pytest.approx(0.5, abs=1e-13)
        assert np.max(np.abs(co["c22"] - 1.0)) == pytest.approx(0.5, abs=1e-13)
        assert np.max(np.abs(co["c12"])) == pytest.approx(0.2, abs=1e-13)
        assert np.max(np.abs(co["c1"])) == pytest.approx(50.0, abs=1e-11)
        assert np.max(np.abs(co["c2"])) == pytest.approx(50.0, abs=1e-11)
        assert co["c"] is None
        assert not np.allclose(co["c11"], co["c22"])  # independent fields


def test_workload_coefficients():
    """Convection-diffusion: c1 = -100 cos(4 pi y), c2 = 100 sin(4 pi x), unit
    diffusion, no c12 or c.  Variable-speed Helmholtz: c = -80^2 (1 - 0.5
    exp(-|x - (0.5, 0.5)|^2 / 0.02)), so -3200 at the centre."""
    x = np.array([0.1, 0.37, 0.9])
    y = np.array([0.2, 0.55, 0.05])
    cd = I.convection_diffusion(x, y)
    np.testing.assert_allclose(cd["c1"], -100 * np.cos(4 * np.pi * y), rtol=1e-15)
    np.testing.assert_allclose(cd["c2"], 100 * np.sin(4 * np.pi * x), rtol=1e-15)
    assert np.all(cd["c11"] == 1) and np.all(cd["c22"] == 1)
    assert cd["c12"] is None and cd["c"] is None
    hz = I.gaussian_bump_helmholtz(np.array([0.5, 0.0]), np.array([0.5, 0.0]))
    assert hz["c"][0] == pytest.approx(-3200.0, rel=1e-15)
    assert hz["c"][1] == pytest.approx(-6400.0 * (1 - 0.5 * np.exp(-25.0)), rel=1e-15)
    assert hz["c1"] is None and hz["c2"] is None and hz["c12"] is None


def test_section_9_2_convection_is_divergence_free():
    """Section 9.2 calls the diffusion-convection field divergence free: with
    c1 a function of y alone and c2 of x alone, d c1/dx + d c2/dy = 0."""
    h = 1e-6
    rng = np.random.default_rng(0)
    x, y = rng.uniform(0, 1, 20), rng.uniform(0, 1, 20)
    d = (I.paper_diffusion_convection(x + h, y)["c1"] - I.paper_diffusion_convection(x - h, y)["c1"]
         + I.paper_diffusion_convection(x, y + h)["c2"]
         - I.paper_diffusion_convection(x, y - h)["c2"]) / (2 * h)
    assert np.max(np.abs(d)) < 1e-6
    assert np.max(np.abs(I.paper_diffusion_convection(x, y)["c1"])) > 1e3
