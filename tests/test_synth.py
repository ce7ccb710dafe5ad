"""Seeded input generators: published SplitMix64 outputs and moments."""
import numpy as np

import synth


def test_splitmix64_reference_outputs():
    # first outputs of SplitMix64 from seed 0 (Steele, Lea & Flood 2014 reference code)
    z = synth.splitmix64(0, 2)
    assert int(z[0]) == 0xE220A8397B1DCDAF
    assert int(z[1]) == 0x6E789E6AA1B965F4
    np.testing.assert_array_equal(synth.splitmix64(5, 4, offset=3), synth.splitmix64(5, 7)[3:])


def test_uniform_and_normal_moments():
    u = synth.uniform(1, 200000)
    assert u.min() >= -1.0 and u.max() < 1.0
    assert abs(u.mean()) < 5e-3 and abs(u.var() - 1 / 3) < 5e-3
    g = synth.normal(2, 200000)
    assert abs(g.mean()) < 1e-2 and abs(g.var() - 1.0) < 1e-2


def test_correlated_field_normalised_and_smooth():
    f = synth.correlated_field(4, (20, 20, 20), 8.0)
    assert abs(f.mean()) < 1e-12 and abs(f.std() - 1.0) < 1e-12
    lag1 = np.mean(f[:, :, 1:] * f[:, :, :-1])
    assert lag1 > 0.9          # correlation length 8 cells


def test_workloads_shapes():
    w = synth.convdiff_2d_64()
    assert w.n == 4096 and w.s == 4
    B = synth.rhs_block(w)
    assert B.shape == (4096, 4) and B.flags.c_contiguous
    w3 = synth.convdiff_3d(16, 3)
    D = synth.diffusion_field(w3)
    assert D.shape == (16, 16, 16) and np.all(D > 0)


def test_request_stream_is_seeded_and_poisson():
    a = synth.request_stream(5, 2000, rate=40.0)
    b = synth.request_stream(5, 2000, rate=40.0)
    assert a == b
    t = np.array([r["arrival"] for r in a])
    assert np.all(np.diff(t) >= 0.0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() - 1 / 40.0) < 0.1 / 40.0          # exponential mean 1/rate
    assert abs(np.median(gaps) - np.log(2) / 40.0) < 0.15 / 40.0
    assert {r["n"] for r in a} == {32, 48, 64, 96, 128}
    assert {r["s"] for r in a} == {2, 4, 8, 16}
    assert {r["precision"] for r in a} == {"fp32", "fp64"}
