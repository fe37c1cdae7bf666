"""The autotuner's choice logic on the host: prediction from the nearest
ladder point scaled by flops, the leaf-size cutoff, and the stability cap,
over a synthetic timing ladder (the GPU timing of the constructor is
bypassed; the plans are the library's own, compiled on the host)."""
import math

import pytest

from paper_1507_00687_gb300 import build as B

S, SS, W = ("strassen",), ("strassen", "strassen"), ("winograd",)


@pytest.fixture(scope="module")
def tuner():
    B.build()
    from paper_1507_00687_gb300 import api
    t = api.Autotuner.__new__(api.Autotuner)
    t.leaf, t.sizes, t.cutoff = "bf16", (512, 2048), 256
    t.candidates = ((), S, W, SS)
    t._plans = {c: api.Plan(list(c), "bf16") for c in t.candidates}
    # ms per product on the ladder (square sizes); absent = not timed
    t.table = {((), 512): 1.0, (S, 512): 1.2, (W, 512): 1.3,
               ((), 2048): 64.0, (S, 2048): 50.0, (W, 2048): 49.0, (SS, 2048): 52.0}
    return t


def test_prediction_nearest_point_scaled_by_flops(tuner):
    assert tuner.predict(S, 2048, 2048, 2048) == pytest.approx(50.0)
    # geometric mean 1625 is nearer 2048 than 512 in log distance
    assert tuner.predict(S, 1024, 1024, 4096) == pytest.approx(50.0 * 1024 * 1024 * 4096 / 2048**3)
    # geometric mean 645: the 512 point, scaled up
    g = (600 * 700 * 640)
    assert tuner.predict((), 600, 700, 640) == pytest.approx(1.0 * g / 512**3)
    # Strassen twice was timed only at 2048: that point serves every shape
    assert tuner.predict(SS, 512, 512, 512) == pytest.approx(52.0 / 64)
    # a candidate never timed predicts infinity
    assert math.isinf(tuner.predict(("winograd", "winograd"), 512, 512, 512))


def test_choice_fastest_among_fitting(tuner):
    assert tuner.choose(2048, 2048, 2048) == list(W)
    assert tuner.choose(512, 512, 512) == []  # classical fastest at the small size
    # Strassen twice would leave 128-wide leaf blocks at n = 512: below the cutoff
    assert not tuner._fits(SS, 512, 512, 512) and tuner._fits(SS, 2048, 2048, 2048)
    assert tuner._fits((), 8, 8, 8)  # the classical product always fits


def test_choice_under_stability_cap(tuner):
    from paper_1507_00687_gb300 import api
    rs, rw = (api.relative_instability(tuner._plans[c]) for c in (S, W))
    assert rs < rw  # Winograd's E = 18 against Strassen's 12, same k0 = 2
    # a cap between the two removes Winograd: Strassen is then fastest
    assert tuner.choose(2048, 2048, 2048, max_instability=(rs + rw) / 2) == list(S)
    # a cap below every fast rule leaves the classical product
    assert tuner.choose(2048, 2048, 2048, max_instability=min(rs, rw) / 2) == []
