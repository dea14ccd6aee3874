"""The GPU heatbath (synth/heatbath_gpu.cu) reproduces the host generator bit
for bit: at small sizes against heatbath.c run in the same process, and at
512^2 and 1024^2 against the fingerprints stored with the tuned masses (the
fields the masses were tuned on were made by the host generator)."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    return torch


@pytest.mark.parametrize("L,sweeps,seed", [(16, 50, 7), (64, 1000, 64000), (96, 20, 3)])
def test_gpu_heatbath_bitwise_equal_to_host(cuda, L, sweeps, seed):
    Uh = synth.heatbath(L, L, synth.BETA, sweeps, seed)
    Ug = synth.heatbath_gpu(L, L, synth.BETA, sweeps, seed)
    assert np.array_equal(Uh.view(np.uint64), Ug.view(np.uint64))


def test_gpu_heatbath_rectangular_and_zero_beta(cuda):
    Uh = synth.heatbath(48, 32, 0.0, 5, 11)
    Ug = synth.heatbath_gpu(48, 32, 0.0, 5, 11)
    assert np.array_equal(Uh.view(np.uint64), Ug.view(np.uint64))


@pytest.mark.parametrize("L,config", [(512, 0), (512, 9), (1024, 0)])
def test_gpu_heatbath_matches_tuned_fingerprints(cuda, L, config):
    U = synth.heatbath_gpu(L, L, synth.BETA, synth.default_sweeps(L), synth.gauge_seed(L, config))
    assert synth.check_fingerprint(L, config, U)
