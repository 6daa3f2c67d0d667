"""The learned Ca_cr proposal against plain bisection on real runs.

Two held-out matrix-viscoelastic triples of the study regime are searched
by both modes with full simulations on the GPU: every bracket end is a
full-run verdict (break-up flag within 30 emulsion times).  The proposal
network is the one trained on the study's collected runs
(results/ca_cr/proposal_net.npy; recipe in results/ca_cr/README.md).  Both
modes must find the same stable-to-broken transition (brackets that
intersect, widths <= 0.02) and the proposal must need fewer full runs."""
import os

import numpy as np
import pytest

from paper_1411_2181_gb300 import study

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
NET = os.path.join(ROOT, "results", "ca_cr", "proposal_net.npy")


@pytest.fixture(scope="module")
def net():
    from paper_1411_2181_gb300 import build
    build.build()
    from paper_1411_2181_gb300 import mlp
    n = mlp.MLP(max_batch=4096, bf16=True)
    n.set_params(np.load(NET))
    return n


def test_proposal_finds_the_bisection_transition_in_fewer_runs(net):
    from paper_1411_2181_gb300 import study_run
    triples = study_run.held_out_triples(16)[:2]
    sb, stb = study.search_bisect(triples)
    sm, stm = study.search_mlp(triples, net, delta=0.06)
    for b, m in zip(sb, sm):
        assert b.width <= 0.02 + 1e-12 and m.width <= 0.02 + 1e-12
        assert max(b.lo, m.lo) <= min(b.hi, m.hi) + 1e-12, (b.triple, (b.lo, b.hi), (m.lo, m.hi))
        assert abs(0.5 * (b.lo + b.hi) - 0.5 * (m.lo + m.hi)) <= 0.02
        # every bracket end is a full-run verdict: stable below, broken above
        for s in (b, m):
            if study.CA_MIN < 0.5 * (s.lo + s.hi) < study.CA_MAX:
                assert (s.lo, False) in s.history and (s.hi, True) in s.history
    assert stm["runs"] < stb["runs"], (stm["runs"], stb["runs"])
