"""What the trained network (paper_2509_26361_gb300/data/mlp_curvature_params.npy,
made by ``python -m paper_2509_26361_gb300.learned train``) gains over height
functions alone, on a seeded grid of ellipsoids it was not trained on: a
smaller curvature error on the cells where height functions give a value, and
a value on the cells where they give none."""
import numpy as np
import pytest

from paper_2509_26361_gb300 import learned

pytestmark = pytest.mark.gpu


def test_trained_network_beats_height_functions_on_unseen_ellipsoids():
    mlp = learned.load_network()
    r = learned.evaluate(mlp, seed=44, n=128, count=16, amin=4.0, amax=16.0, repeats=1)
    mlp.close()
    # more accurate where height functions give a value
    assert r["rms_mlp_on_hf_cells"] < 0.9 * r["rms_hf"], r
    # and a value where they give none: every interface cell is covered
    assert r["hf_no_value"] > 0
    assert np.isfinite(r["rms_mlp"]) and r["rms_mlp"] < 0.05, r
    for b in r["bins"]:
        if b["hf_cells"] > 500:
            assert b["rms_mlp_on_hf_cells"] < b["rms_hf"], b
