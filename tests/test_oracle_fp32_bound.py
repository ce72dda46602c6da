"""Pins of the oracle parts that set or check reduced-precision tolerances,
and of the kinetic half of the Eq. 15 stress (no GPU).

- ``forces_on`` (the one-particle-at-a-time LJ sums used for sampled
  particles of boxes too large for a full oracle step) equals the rows of
  ``forces``, on its cell-list path and on its all-pairs path.
- ``band_pairs`` finds exactly the pairs within the band of the cut-off that a
  numpy minimum-image enumeration finds, with the Eq. 9 pair force.
- ``force_error_bound`` covers, on every particle, the error of an
  independent numpy float32 evaluation of the same reference-relative
  arithmetic (tests/fp32_model.py), and is not much looser than needed: the
  worst float32 separation error seen reaches at least a quarter of the
  bound's separation term u (6P + 2r), and the L2 norm of the bound stays
  within 100 times that of the float32 error (25-60 measured).
- The kinetic part of Eq. 15, -(1/V) sum m (v_x - v_s(z)) v_z with v_s of
  Eq. 1, against a hand-computed value for particles too far apart to
  interact (lab-frame velocities in place of peculiar ones change it).
"""
import math

import numpy as np
import pytest

import oracle
import synth
from fp32_model import f32_forces, ordered_pairs, separation_errors

U = 2.0 ** -24


def _jittered(n, rho, seed, amp=0.12):
    pos, box = synth.lj_box(n, rho, seed)
    g = np.random.default_rng(seed)
    return np.mod(pos + g.uniform(-amp, amp, pos.shape), box), box


@pytest.mark.parametrize("n, frac", [(864, 0.37), (500, 0.0)])
def test_forces_on_equals_rows_of_forces(n, frac):
    """n = 864 at rho 0.8442 gives L = 10.1 >= 3 rc: the cell-list path;
    n = 500 at rho 0.9 gives L = 8.2 < 3 rc: the all-pairs path."""
    rho = 0.8442 if n == 864 else 0.9
    pos, box = _jittered(n, rho, 7)
    p = oracle.params(box, 0.3, 2.5)
    dX = frac * box
    _, F, _, _ = oracle.forces(p, dX, pos)
    idx = np.random.default_rng(3).choice(n, 97, replace=False)
    Fo = oracle.forces_on(p, dX, pos, idx)
    assert np.abs(Fo - F[idx]).max() <= 1e-12 * np.abs(F).max()
    assert np.abs(F[idx]).max() > 1.0


def test_band_pairs_match_a_numpy_enumeration():
    pos, box = _jittered(1372, 0.8442, 11)
    p = oracle.params(box, 0.5, 2.5)
    dX = 0.61 * box
    band = 2e-3
    ij, f, inside = oracle.band_pairs(p, dX, pos, band)
    i, j, d, _ = ordered_pairs(pos, box, dX, 2.5 + band)
    r = np.linalg.norm(d, axis=1)
    m = np.abs(r - 2.5) <= band
    want = {(int(a), int(b)): d[k] for k, (a, b) in enumerate(zip(i, j)) if m[k]}
    got = {(int(a), int(b)): k for k, (a, b) in enumerate(ij)}
    assert set(got) == set(want) and len(want) > 20
    for key, k in got.items():
        dd = want[key]
        r2 = float(dd @ dd)
        s6 = r2 ** -3
        np.testing.assert_allclose(f[k], 24.0 * (2 * s6 * s6 - s6) / r2 * dd, rtol=1e-12)
        assert inside[k] == (r2 < 6.25)


@pytest.mark.parametrize("n, seed, frac, drift", [(1372, 5, 0.37, 0.15), (2048, 9, 0.0, 0.0),
                                                  (864, 13, 0.93, 0.15)])
def test_rounding_bound_covers_a_float32_evaluation(n, seed, frac, drift):
    pos, box = _jittered(n, 0.8442, seed)
    rc, skin = 2.5, 0.3
    dX = frac * box
    p = oracle.params(box, 0.2, rc)
    _, F, _, _ = oracle.forces(p, dX, pos)
    F32, _, _, P = f32_forces(pos, box, dX, rc, rc + skin, drift=drift, seed=seed)
    err = np.linalg.norm(F32 - F, axis=1)
    B = oracle.force_error_bound(p, dX, pos, None, U, P)
    assert np.all(err <= B), int(np.argmax(err / B))
    ratio = np.linalg.norm(B) / np.linalg.norm(err)
    assert ratio <= 100.0, ratio
    # the separation term itself: covered on every pair, and reached within 4x
    se, r, P2 = separation_errors(pos, box, dX, rc, rc + skin, drift=drift, seed=seed)
    assert P2 == P
    t = se / (math.sqrt(3.0) * U * (6.0 * P + 2.0 * r))
    assert t.max() <= 1.0 and t.max() * math.sqrt(3.0) >= 0.25, t.max()


def test_rounding_bound_admits_a_pair_at_the_cut_off():
    """A pair a hair inside rc: the strict test may go either way in FP32, so
    the bound holds the whole pair force there."""
    box = 12.0
    rc = 2.5
    pos = np.array([[3.0, 4.0, 5.0], [3.0 + rc * (1 - 1e-9), 4.0, 5.0]])
    p = oracle.params(box, 0.0, rc)
    B = oracle.force_error_bound(p, 0.0, pos, None, U, 1.6)
    s6 = rc ** -6
    f_rc = abs(24.0 * (2 * s6 * s6 - s6) / rc)
    assert B[0] >= f_rc and B[1] >= f_rc
    pos[1, 0] = 3.0 + rc * 0.99          # well inside: only rounding terms
    B2 = oracle.force_error_bound(p, 0.0, pos, None, U, 1.6)
    assert B2[0] < 1e-3 * f_rc


def test_kinetic_stress_closed_form():
    """Four particles more than rc apart, no thermostat: the Eq. 15 tensor's
    xz element is -(1/V) sum m (v_x - v_s(z)) v_z, with v_s(z) = shear (z -
    Lz/2) (Eq. 1), at the start and after free flight."""
    box = np.array([12.0, 11.0, 10.0])
    gd = 0.4
    pos = np.array([[1.0, 1.0, 1.0], [7.0, 6.0, 2.5], [2.0, 8.0, 8.0], [8.0, 2.0, 6.5]])
    vel = np.array([[0.3, -0.2, 0.5], [-0.1, 0.4, -0.3], [0.7, 0.0, 0.2], [-0.5, 0.1, -0.6]])
    p = oracle.params(box, gd, 2.5, thermostat=0, xi=0.0, dt=0.01)
    V = float(np.prod(box))

    def closed(r, v):
        vs = gd * (r[:, 2] - 0.5 * box[2])
        return -float(np.sum((v[:, 0] - vs) * v[:, 2])) / V

    st = oracle.State(p, pos, vel)
    S, _, _ = st.observe()
    assert S[0, 2] == pytest.approx(closed(pos, vel), rel=1e-14, abs=1e-16)
    lab = -float(np.sum(vel[:, 0] * vel[:, 2])) / V
    assert abs(lab - closed(pos, vel)) > 0.2 * abs(closed(pos, vel))   # v_s matters
    # the free flight keeps the particles apart for 60 steps
    assert st.run(60, sample_every=60) == oracle.OK
    assert st.samples.nsamples == 1
    assert st.samples.sxz_sum == pytest.approx(closed(st.pos, st.vel), rel=1e-13, abs=1e-16)
    assert np.allclose(st.vel, vel)
