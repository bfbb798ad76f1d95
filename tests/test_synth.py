"""Properties of the seeded synthetic inputs (transducer kernel, phantom, noise)."""
import math

import numpy as np

import synth


def test_eir_is_normalised_odd_derivative():
    g = synth.workload("tiny_16x16x24_T64_k7_N8_P2").geom
    v = synth.eir_taps(g)
    assert len(v) % 2 == 1
    assert np.max(np.abs(v)) == 1.0
    np.testing.assert_allclose(v, -v[::-1], atol=1e-15)  # derivative of a Gaussian: odd


def test_kernel_arrivals_centre_on_focus_and_fit_window():
    prob = synth.workload("tiny_16x16x24_T64_k7_N8_P2")
    g = prob.geom
    K = synth.transducer_kernel(g)
    assert K.shape == g.k_shape()
    nz = np.abs(K) > 0
    t_any = np.where(nz.any(axis=(0, 1, 2)))[0]
    assert t_any.min() > 0 and t_any.max() < g.T - 1  # no arrival clipped at the record edges
    # on axis, the shallowest depth arrives earlier than the deepest one
    r = g.r
    first = lambda j: np.where(nz[j, r, r])[0].min()
    assert first(0) < first(g.Z - 1)
    # the two depths straddling the focal plane put their arrivals around T/2
    mid = [g.Z // 2 - 1, g.Z // 2]
    for j in mid:
        ts = np.where(nz[j, r, r])[0]
        assert ts.min() <= g.T // 2 + 2 and ts.max() >= g.T // 2 - 2


def test_kernel_is_seeded_and_asymmetric():
    g = synth.workload("tiny_16x16x24_T64_k7_N8_P2").geom
    a = synth.transducer_kernel(g, seed=0)
    b = synth.transducer_kernel(g, seed=0)
    c = synth.transducer_kernel(g, seed=1)
    np.testing.assert_array_equal(a, b)
    assert np.abs(a - c).max() > 0
    # random aperture points break the dx <-> dy symmetry
    assert np.abs(a - a.transpose(0, 2, 1, 3)).max() > 0


def test_phantom_ranges_and_species():
    prob = synth.workload("tiny_16x16x24_T64_k7_N8_P2")
    c = synth.tube_phantom(prob.geom, prob.tubes, seed=0, per_species=True)
    assert c.shape == prob.geom.c_shape()
    assert c.min() == 0.0 and c.max() <= 1.0
    vals = c[c > 0]
    assert vals.min() >= 0.5
    for p in range(prob.geom.P):
        assert (c[p] > 0).any()


def test_noise_sigma_matches_snr():
    rng = np.random.default_rng(0)
    clean = rng.standard_normal(10000) * 3.0
    s = synth.noise_sigma(clean, 20.0)
    assert math.isclose(s * s, np.mean(clean ** 2) / 100.0, rel_tol=1e-12)


def test_batch_shapes_are_in_range():
    shapes = synth.batch_shapes(16, seed=0)
    assert len(shapes) == 16
    for pr in shapes:
        g = pr.geom
        assert g.X in (32, 48, 64, 96, 128) and 48 <= g.Z <= 128
        assert 128 <= g.T <= 512 and g.T % 16 == 0
        assert 20 <= g.N <= 80 and g.N % 10 == 0 and g.P in (2, 3)
        assert g.k % 2 == 1 and 11 <= g.k <= 31


def test_spr_image_is_a_seeded_beam_narrowest_at_the_focus():
    g = synth.matched_time_grid(synth.workload("medium_64x64x64_T256_k15_N40_P2").geom)
    assert abs(g.c_mm_per_us * g.dt_us - g.dz_mm) < 1e-15
    a, b = synth.spr_image(g, seed=2), synth.spr_image(g, seed=2)
    assert np.array_equal(a, b) and not np.array_equal(a, synth.spr_image(g, seed=3))
    r = g.r
    # on-axis amplitude peaks at the focal plane; off-axis energy spreads away from it
    axis = a[:, r, r]
    mid = (g.Z - 1) / 2.0
    centre = axis[int(mid) - 2:int(mid) + 3].mean()
    assert centre > 2.0 * axis[0] and centre > 2.0 * axis[-1]
    width = (a * (np.arange(-r, r + 1)[None, None, :] ** 2)).sum(axis=(1, 2)) / a.sum(axis=(1, 2))
    assert width[0] > width[int(mid)] and width[-1] > width[int(mid)]
    assert np.all(a > 0)
