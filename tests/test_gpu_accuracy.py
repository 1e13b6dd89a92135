"""The CUDA filter on the accuracy study's inputs: every decision and count
equals the oracle's, for the three variants of the study over each read
length's whole threshold sweep, so the study's rates hold for the GPU path."""
import pytest

from oracle import oracle as O
from paper_2103_14978_gb300 import gk, synth
from tests.gpu_helpers import GpuRun, assert_same, oracle_run, require_gpu

pytestmark = pytest.mark.gpu

VARIANTS = ((gk.GK_COUNT_RUNS4, 0, O.RUNS4, 0), (gk.GK_COUNT_POPCOUNT, 0, O.POPCOUNT, 0),
            (gk.GK_COUNT_RUNS4, gk.GK_FLAG_NO_EDGE_FIX, O.RUNS4, O.FLAG_NO_EDGE_FIX))


@pytest.mark.parametrize("m,e_max", [(100, 10), (150, 15), (250, 25)])
def test_study_inputs_gpu_equals_oracle(m, e_max):
    require_gpu()
    w = synth.accuracy_set(m, 2 * e_max, 3000, seed=synth.SEED_BASE + 5)
    run = GpuRun(w)
    for e in range(e_max + 1):
        for mode, flags, omode, oflags in VARIANTS:
            assert_same(run.filter(e=e, mode=mode, flags=flags), oracle_run(w, e, omode, oflags),
                        f"{m} bp e={e} mode={mode} flags={flags}")
