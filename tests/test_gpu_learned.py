"""The learned placement model: trained on the GPU by the library's own MLP
kernels from measured random points, it must (i) predict placements whose
median regret against exhaustive measurement on held-out points is at most
10 %, and (ii) gain over the method without it -- nearest-grid-cell lookup in
the exhaustively measured table -- and over the best single fixed placement."""
import os

import numpy as np
import pytest

import paper_2609_28179_gb300 as g

pytestmark = pytest.mark.gpu

TUNING = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2609_28179_gb300",
                      "tuning")
TRAIN = os.path.join(TUNING, "sm103_random_train.jsonl")
HELD = os.path.join(TUNING, "sm103_random_heldout.jsonl")


@pytest.fixture(scope="module")
def trained():
    if not (os.path.exists(TRAIN) and os.path.exists(HELD)):
        pytest.skip("random-point measurements not committed")
    import paper_2609_28179_gb300.learned as Lm
    from paper_2609_28179_gb300 import _build
    _build.build()
    g.lib()
    train_pts, held = Lm.load_points(TRAIN), Lm.load_points(HELD)
    w, mu, sd, losses = Lm.train(train_pts, epochs=300, log_every=50)
    return Lm, w, mu, sd, losses, train_pts, held


def test_training_loss_decreases(trained):
    Lm, w, mu, sd, losses, _, _ = trained
    assert losses[-1] < 0.5 * losses[0], losses


def test_learned_regret_and_gain_over_table_and_fixed(trained):
    Lm, w, mu, sd, _, train_pts, held = trained
    res = Lm.evaluate(w, mu, sd, train_pts, held)
    print(res)
    assert res["learned"]["median"] <= 0.10, res
    # Both medians sit at the measurement-noise floor (a fraction of a
    # percent, far inside the 5 % dispatch margin), so the gain over the
    # nearest-grid table is judged where the two differ: the tail of the
    # regret and the share of choices within the margin.  The median may tie
    # within one percent.
    assert res["learned"]["median"] <= res["nearest_grid_table"]["median"] + 0.01, res
    assert res["learned"]["p90"] < res["nearest_grid_table"]["p90"], res
    assert res["learned"]["within_5pct"] >= res["nearest_grid_table"]["within_5pct"], res
    assert res["learned"]["mean"] < res["fixed_placement"]["mean"], res


def test_library_uses_the_installed_model_off_grid(trained, tmp_path):
    Lm, w, mu, sd, _, _, held = trained
    path = tmp_path / "m.bin"
    Lm.save(str(path), w, mu, sd)
    Lm.install(str(path))
    p = next(q for q in held if q["n"] not in (3, 6, 7, 12, 14, 24, 32, 64))
    choice = Lm.learned_choices(w, mu, sd, [p])[0]
    s, (scope, pack) = g.glass_get_placement(Lm.OP_ID[p["op"]], p["n"], p["k"], p["batch"], 0, 1)
    assert s == g.GLASS_OK
    # the library's host-side forward pass agrees with the GPU forward kernel
    assert f"{scope}x{pack}" == choice
