"""What the trained surface surrogate gains over the method without learning.

The no-learning foil predicts the surface displacement as the indenter's
penetration into the undeformed surface, Gaussian-smoothed, pointing down;
its one parameter (the smoothing width) is fitted on training trajectories.
The trained network (the committed parameters) and the foil are scored by the
same per-frame error -- RMS over the pixels of |u_pred - u_IMPM| divided by
the trajectory's press depth -- on held-out trajectories that the batched
IMPM simulates here.  The stated margin: the network's median error is at
most 60 % of the foil's, and so is its mean.
"""
import os

import numpy as np
import pytest

from paper_2405_02914_gb300 import inputs as I
from paper_2405_02914_gb300 import surrogate as G

pytestmark = pytest.mark.gpu

WEIGHTS = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2405_02914_gb300",
                       "weights", "surrogate_pad64.npz")
MARGIN = 0.6


def test_trained_network_beats_the_no_learning_foil():
    assert os.path.exists(WEIGHTS), "the trained parameters are committed with the package"
    params, _ = G.load_params(WEIGHTS)
    train = G.generate(I.surrogate_scenes(2, seed=0))           # the foil's fit (training split)
    sigma = G.fit_foil(train)
    held = G.generate(I.surrogate_scenes(4, seed=1))            # held-out split
    e_net = G.frame_errors(G.predict(params, held), held)
    e_foil = G.frame_errors(G.foil(held, sigma), held)
    print("held-out frames %d: network median %.4f mean %.4f, foil (sigma %.1f px) median %.4f mean %.4f"
          % (len(held), np.median(e_net), e_net.mean(), sigma, np.median(e_foil), e_foil.mean()))
    assert np.isfinite(e_net).all() and np.isfinite(e_foil).all()
    assert np.median(e_net) <= MARGIN * np.median(e_foil)
    assert e_net.mean() <= MARGIN * e_foil.mean()
