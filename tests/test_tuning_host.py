"""Host logic of the placement tuner (CPU): the selection rule and the
generated tables, which must be exactly what the committed GB300
measurements produce."""
import os

import pytest

from paper_2609_28179_gb300 import tune


def test_choose_prefers_fewer_resources_within_the_margin():
    meas = {(2, 1): {"us": 10.0}, (1, 4): {"us": 10.4}, (0, 8): {"us": 10.6}, (1, 1): {"us": 12.0}}
    assert tune.choose(meas) == (1, 4)          # 4 % slower than the best, a smaller scope
    meas[(0, 8)]["us"] = 10.49
    assert tune.choose(meas) == (0, 8)          # within 5 %: thread scope wins
    assert tune.choose({(2, 2): {"us": 5.0}, (2, 1): {"us": 5.2}}) == (2, 1)   # then the smaller pack
    assert tune.choose({(3, 1): {"us": 5.0}, (1, 1): {"us": 5.2}}) == (1, 1)   # the composition ranks last


@pytest.mark.parametrize("gen,inp,committed", [
    ("codegen", tune.GRID_FILE, tune.TABLE_H),
    ("riccati_codegen", tune.RICCATI_FILE, tune.RICCATI_H),
    ("robo_codegen", tune.ROBO_FILE, tune.ROBO_H),
    ("fp64_codegen", tune.F64_FILE, tune.F64_H),
])
def test_committed_tables_match_the_committed_measurements(gen, inp, committed, tmp_path):
    out = tmp_path / os.path.basename(committed)
    getattr(tune, gen)(inp, str(out))
    assert out.read_text() == open(committed).read()


def test_measurement_files_cover_the_grid():
    from paper_2609_28179_gb300.cells import OPS, SWEEP_B, TABLE_N
    cells = tune.load_grid()
    for op in OPS:
        for n in TABLE_N:
            for b in SWEEP_B:
                meas = cells[(op, n, b)]
                assert meas, (op, n, b)
                assert all(v["us"] > 0 for v in meas.values())
