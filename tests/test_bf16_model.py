"""CPU checks of the BF16 operand-rounding model used by the tensor-core
tests: without rounding it must reproduce the FP64 oracle, and its BF16
rounding must be round-to-nearest-even."""
import math

import numpy as np

import bf16_model
import oracle
import synth


def test_rounding_matches_ties_to_even():
    # 1 + 2^-8 is halfway between BF16 neighbours 1 and 1 + 2^-7: ties to
    # the even significand (1); 1 + 3 * 2^-8 rounds up to 1 + 2^-6.
    x = np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, 1 + 2 ** -8 + 2 ** -20, -2.5, 3e38], np.float32)
    r = bf16_model.bf16_rn(x)
    assert list(r[:4]) == [1.0, 1.0, 1 + 2 ** -6, 1 + 2 ** -7]
    assert r[4] == -2.5
    assert np.all(np.abs(r - x) <= 2.0 ** -8 * np.abs(x))


def test_model_without_rounding_is_the_oracle():
    w = synth.TINY
    n = 512
    params = synth.random_params(w, 5)
    pos = synth.positions(5, n)
    uu = synth.uniform_rows(5, synth.S_DIR, 2, n)
    dirs = synth.sphere_dirs(uu[0], uu[1])
    raw = bf16_model.raw_outputs(w, params, pos, rounding=lambda a: np.asarray(a, np.float32),
                                 fp16_grid=False)
    got = bf16_model.density(w, raw, dirs)
    ref = oracle.eval_pdf64(w, params, pos, dirs)
    assert np.max(np.abs(got - ref) / np.maximum(ref, 1e-2 / (4 * math.pi))) < 1e-5
