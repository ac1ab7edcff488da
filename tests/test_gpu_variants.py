"""Decoding ablation (Sec. IV-D1): the decode_mode toggles of the library against
the oracle's P_hat = f_ACT(f_NL(f_N(P))) followed by softmax and PSD."""
import numpy as np
import pytest

import oracle
from helpers import config_for, normwise, oracle_grid, run_gpu
from paper_2408_09066_gb300 import synth
from paper_2408_09066_gb300 import vsaogm as V

pytestmark = pytest.mark.gpu

ACTS = {V.ACT_ENTROPY: "entropy", V.ACT_RELU: "relu", V.ACT_TANH: "tanh",
        V.ACT_SIGMOID: "sigmoid", V.ACT_NONE: "none"}
MODES = [0, V.ACT_RELU, V.ACT_TANH, V.ACT_SIGMOID, V.ACT_NONE,
         V.MODE_NO_SQUARE | V.ACT_NONE, V.MODE_NO_NORM | V.MODE_NO_SQUARE | V.ACT_TANH,
         V.MODE_NO_NORM | V.ACT_SIGMOID, V.MODE_NO_SQUARE | V.ACT_ENTROPY,
         V.MODE_NO_NORM | V.MODE_NO_SQUARE | V.ACT_NONE]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2408_09066_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def case():
    wl = synth.small_scan(seed=55)
    cfg = config_for(wl)
    g = oracle_grid(cfg)
    nx, ny = oracle.draw_nu(cfg.seed, cfg.D, float(np.float32(cfg.length_scale)))
    om = oracle.memories(g, nx, ny, wl.xy, wl.labels, "tile")
    return wl, oracle.decode_map(g, nx, ny, om, "tile")


@pytest.mark.parametrize("mode", MODES)
def test_decode_mode_matches_oracle(case, mode):
    wl, P = case
    cfg = config_for(wl, decode_mode=mode)
    got = run_gpu(cfg, wl.xy, wl.labels)
    norm = not (mode & V.MODE_NO_NORM)
    square = not (mode & V.MODE_NO_SQUARE)
    act = ACTS[mode & 0xF0]
    pr1, pr0, ogm = oracle.decode_variant(P, norm, square, act, cfg.r_occ, cfg.r_emp)
    assert np.abs(got["occ"] - pr1).max() <= 1e-3
    assert np.abs(got["occ_query"] - pr1).max() <= 1e-3
    # vsaogm_decode returns f_NL(f_N(P)) under the same toggles
    ph = np.array(P)
    if norm:
        ph = np.stack([ph[c] / ph[c].max() if ph[c].max() > 0 else 0 * ph[c] for c in range(2)])
    if square:
        ph = ph * ph
    assert normwise(got["Phat"], ph) <= 1e-4


def test_unknown_mode_rejected():
    wl = synth.small_scan(seed=56)
    with pytest.raises(V.VsaogmError) as ei:
        V.Map(config_for(wl, decode_mode=0x50))
    assert ei.value.code == V.E_INVAL
