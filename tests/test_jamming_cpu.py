"""Host-side fit of the jamming blow-up law (Eq. blowup, mu ~ c |t - t*|^-beta)
used by paper_1912_04501_gb300.jamming: on samples of the law itself with
the parameters the paper reports for Examples 4 and 5, the fit recovers
them; a window too short to fit is refused."""
import numpy as np
import pytest

pytest.importorskip("scipy")


@pytest.mark.parametrize("c,tstar,beta,window", [(2.187, 0.458, 2.431, (0.40, 0.44)),
                                                  (12.16, 0.472, 1.31, (0.40, 0.45))])
def test_fit_recovers_the_power_law(c, tstar, beta, window):
    from paper_1912_04501_gb300.jamming import fit_blowup
    t = np.arange(0.0, window[1] + 1e-12, 5e-4)
    mu = c * (tstar - t) ** (-beta)
    f = fit_blowup(t, mu, window)
    assert abs(f["beta"] - beta) < 1e-6 and abs(f["t_star"] - tstar) < 1e-8 and abs(f["c"] / c - 1) < 1e-5
    assert f["rel_residual"] < 1e-8
    # 1% multiplicative noise: the exponent within a few per cent
    rng = np.random.default_rng(0)
    g = fit_blowup(t, mu * (1 + 0.01 * rng.standard_normal(t.size)), window)
    assert abs(g["beta"] - beta) < 0.1 * beta


def test_fit_needs_points():
    from paper_1912_04501_gb300.jamming import fit_blowup
    with pytest.raises(ValueError):
        fit_blowup([0.41, 0.42], [1.0, 2.0], (0.4, 0.44))
