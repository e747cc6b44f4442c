"""Exp 1 of Sec. 4.1, shortened to 200 assimilation steps: the bootstrap filter collapses
onto one particle and loses the truth, while the filter with adaptive tempering and PCN
jittering keeps a spread ensemble that tracks it (the qualitative result of the paper's
Exp 1 figures).  N = 150, Matern noise (eta = 1, k = 3, kappa = 1), sigma = 0.05."""
import numpy as np
import pytest

from workloads import get_config
from tests.helpers import gpu_model

pytestmark = pytest.mark.gpu


def test_exp1_bootstrap_collapses_and_tempering_tracks():
    from paper_2402_06927_gb300 import twin
    cfg = get_config("exp1_f64")
    g = gpu_model(cfg)
    T = 200
    out = twin.exp1(g, cfg, T)
    b, t = out["bootstrap"]["series"], out["tempering_jittering"]["series"]
    late = slice(T // 2, T)
    print("initial", out["initial"], "bootstrap", b[late].mean(axis=0), "tempered", t[late].mean(axis=0),
          "stages", np.mean(out["tempering_jittering"]["stages"]), "min RES/EMRE", np.min(t[:, 2] / t[:, 0]),
          "collapsed", np.sum(b[:, 2] < 1e-9))
    # every filter starts from the same spread-out ensemble, far from the truth
    assert out["initial"][0] > 1.0
    # the bootstrap ensemble degenerates to copies of one particle, again and again (the
    # model noise spreads the copies apart between collapses)
    assert np.sum(b[:, 2] < 1e-9) >= 2
    assert b[late, 2].mean() < 0.75 * t[late, 2].mean()
    # tempering and jittering keep the ensemble spread at every step, and closer to the truth
    assert np.min(t[:, 2] / t[:, 0]) > 0.1
    assert t[late, 0].mean() < 0.9 * b[late, 0].mean()
    assert 3 <= np.mean(out["tempering_jittering"]["stages"]) <= 15


def test_exp2_half_domain_observations():
    # Exp 2 (only [0, L/2] observed), 200 steps: the tempered and jittered ensemble keeps its
    # spread and its mean follows the truth on the observed half, much closer than on the
    # other half and closer than the bootstrap ensemble's mean there
    from paper_2402_06927_gb300 import twin
    cfg = get_config("exp1_f64")
    g = gpu_model(cfg)
    T = 200
    out = twin.exp2(g, cfg, T)
    b, t = out["bootstrap"]["series"], out["tempering_jittering"]["series"]
    hv = out["tempering_jittering"]["halves"]
    late = slice(T // 2, T)
    print("bootstrap", b[late].mean(axis=0), "tempered", t[late].mean(axis=0), "halves", hv[late].mean(axis=0),
          "bootstrap halves", out["bootstrap"]["halves"][late].mean(axis=0),
          "stages", np.mean(out["tempering_jittering"]["stages"]), "collapsed", np.sum(b[:, 2] < 1e-9))
    hb = out["bootstrap"]["halves"]
    assert np.min(t[:, 2] / t[:, 0]) > 0.1
    assert hv[late, 0].mean() < hv[late, 1].mean() / 3
    assert hv[late, 0].mean() < hb[late, 0].mean()
