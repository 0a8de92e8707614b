"""The Sec. 4 drivers (``paper_1808_06787_gb300.scenarios``) on the GPU.

* Sec. 4.1 through the driver: the errors of Table I.
* Sec. 4.2 (200 x 200): xi_2 at x = 0.72 falls to 0.1581 at about t = 0.2; the
  probe shows the sequence the paper describes for species 2 -- reverse
  diffusion (-J_2 d(xi_2)/dx < 0) up to t_1, osmotic diffusion at t_1 and t_2
  (d(xi_2)/dx = 0 with J_2 != 0), reverse diffusion again up to t_3 and a
  diffusion barrier at t_3 (J_2 = 0 with d(xi_2)/dx != 0); the probe series
  equals the FP64 oracle's (1D copy of the x-only problem) to 1e-12.
* Sec. 4.3 (200 x 200): the bottom-half average of xi_2 peaks at t* = 0.35 h;
  the two halves' averages always mean the equilibria 0.2575 and 0.497.
"""

import numpy as np
import pytest

pytestmark = [pytest.mark.gpu, pytest.mark.usefixtures("oracle_lib")]

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_erf_driver_reproduces_table_I():
    import theory as th

    from paper_1808_06787_gb300 import scenarios as sc

    Pn = th.golden_numbers()
    for relax, tag in (("magic", "mrt"), ("srt", "srt")):
        r = sc.erf_binary(relax=relax)
        for i, t in enumerate((1, 5, 20)):
            assert r["t"][i] == pytest.approx(t, abs=1e-9)
            assert r["E_xi1"][i] == pytest.approx(Pn["erf.%s.Ex.t%d" % (tag, t)], rel=3e-3)
            assert r["E_J1"][i] == pytest.approx(Pn["erf.%s.EJ.t%d" % (tag, t)], rel=3e-3)


@pytest.fixture(scope="module")
def duncan_toor():
    from paper_1808_06787_gb300 import scenarios as sc

    return sc.duncan_toor(t_end=0.4, samples=400)


def test_duncan_toor_minimum_of_xi2(duncan_toor):
    import theory as th

    Pn = th.golden_numbers()
    d = duncan_toor
    i = int(np.argmin(d["xi"][:, 1]))
    assert abs(d["xi"][i, 1] - Pn["duncan_toor.xi2_min"]) < 5e-4
    assert abs(d["t"][i] - Pn["duncan_toor.t_min"]) < 0.02
    # xi_1 rises towards its equilibrium 0.4 without cross effects (D12 = D13)
    assert np.all(np.diff(d["xi"][:, 0]) >= 0.0)
    np.testing.assert_allclose(d["xi"].sum(axis=1), 1.0, rtol=0, atol=1e-13)


def test_duncan_toor_reverse_osmotic_barrier_sequence(duncan_toor):
    d = duncan_toor
    t, J2, g2 = d["t"][1:], d["J"][1:, 1], d["neg_grad"][1:, 1]
    reverse = J2 * g2 < 0.0  # -J_2 d(xi_2)/dx < 0
    change = np.flatnonzero(np.diff(reverse.astype(int)) != 0)
    assert reverse[0]  # reverse diffusion from the start
    assert len(change) == 3
    # the first two changes are zeros of the gradient with J_2 != 0 (osmotic),
    # the third a zero of J_2 with a gradient (barrier)
    for c, kind in zip(change, ("osmotic", "osmotic", "barrier")):
        if kind == "osmotic":
            assert np.sign(g2[c]) != np.sign(g2[c + 1]) and np.sign(J2[c]) == np.sign(J2[c + 1])
        else:
            assert np.sign(J2[c]) != np.sign(J2[c + 1]) and np.sign(g2[c]) == np.sign(g2[c + 1])
    assert t[change[0]] < t[change[1]] < t[change[2]] < 0.4


def test_duncan_toor_probe_matches_the_oracle(duncan_toor):
    import oracle
    import synthetic as sy

    d = duncan_toor
    nx = d["X"].size
    steps = np.round(d["t"] / d["dt"]).astype(np.int64)[::20]
    D = sy.D_from_pairs(3, {(1, 2): 0.1, (1, 3): 0.1, (2, 3): 0.1 * 0.168 / 0.833})
    _, snaps = oracle.run("D2Q5", D, sy.duncan_toor_1d(nx), int(steps[-1]),
                          bc=("noflux", "noflux") + ("periodic",) * 4, snapshots=steps)
    for k, s in enumerate(snaps):
        probe = [np.interp(0.72, d["X"], s[i, 0, 0]) for i in range(3)]
        np.testing.assert_allclose(d["xi"][20 * k], probe, rtol=0, atol=1e-12)


def test_loschmidt_peak_time_and_conservation():
    import theory as th

    from paper_1808_06787_gb300 import scenarios as sc

    Pn = th.golden_numbers()
    r = sc.loschmidt(t_end_hours=0.6, samples=300)
    i = int(np.argmax(r["bottom"][:, 1]))
    assert abs(r["hours"][i] - Pn["loschmidt.t_peak_hours"]) <= 0.005
    # bottom xi_2 rises then falls, top xi_2 mirrors it (cross effects)
    assert r["bottom"][i, 1] > r["bottom"][0, 1] and r["bottom"][i, 1] > r["bottom"][-1, 1]
    mean = 0.5 * (r["bottom"] + r["top"])
    np.testing.assert_allclose(mean[:, 0], Pn["loschmidt.xi1_eq"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(mean[:, 1], Pn["loschmidt.xi2_eq"], rtol=0, atol=1e-12)
