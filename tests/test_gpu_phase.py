"""Phase-transition driver on the GPU (Sec. 5.1): a reduced sweep runs the
protocol (rho up from 0.01 until a point recovers nothing) through batched
decodes, and the 50 % point lands inside the swept range."""
import math

import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ccs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1508_01256_gb300 import build, ccs
    build.build()
    return ccs


def test_reduced_phase_transition(ccs):
    from paper_1508_01256_gb300 import phase
    res = phase.phase_transition(ccs, n=2 ** 12, d=7, deltas=[0.1, 0.3], per_point=3, seed=5)
    for r in res:
        assert r["recovered"] > 0 and r["decodes"] > r["recovered"]
        assert not math.isnan(r["rho_star"]) and 0.0 < r["rho_star"] < r["points"] * 0.01 + 0.01


def test_banded_signals_lower_the_transition(ccs):
    """Sec. 5.6: signals whose support mostly shares one value recover over a
    smaller range than dissociated ones."""
    from paper_1508_01256_gb300 import phase
    plain = phase.sweep_delta(ccs, 2 ** 12, 7, 0.3, per_point=4, seed=9)
    banded = phase.sweep_delta(ccs, 2 ** 12, 7, 0.3, per_point=4, seed=9, model="banded",
                               band=0.9)
    assert banded["rho_star"] < plain["rho_star"]
