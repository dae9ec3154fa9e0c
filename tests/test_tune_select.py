"""The autotuner's decision rule (pico_tune_select), on synthetic timing tables, without a GPU.

pico_autotune times candidates and hands the table to this pure host
function; these cases fix what it must choose: the Gram variant fastest at
the largest batch, the smallest batch from which on the Gram operator is
never slower than the column FFTs, and the largest probe batch within 3 % of
the lowest time per image.
"""
import math

import pytest

import paper_2605_09590_gb300 as pico
from paper_2605_09590_gb300 import build as pico_build


@pytest.fixture(scope="module", autouse=True)
def _lib():
    pico_build.build()
    pico.load_library()


def table(fft, g16=None, g16t=None, g8=None, batches=(16, 32, 64, 128, 256)):
    t = {"fft": dict(zip(batches, fft))}
    for name, row in (("gram16", g16), ("gram16_tmem", g16t), ("gram8", g8)):
        if row is not None:
            t[name] = dict(zip(batches, row))
    return t


def test_knee_like_table():
    # the measured knee operator: Gram wins from 32 on; 256 is the fastest batch
    t = table([8.37, 7.36, 7.05, 6.69, 6.52], [12.16, 6.56, 3.74, 2.32, 2.01], [11.74, 6.35, 3.65, 2.33, 2.02],
              [12.73, 6.78, 3.89, 2.39, 2.13])
    sel = pico.pico_tune_select(t, 256)
    assert sel == {"gram_min_batch": 32, "gram_kc": 16, "gram_a_tmem": 0, "probe_batch": 0}


def test_tensor_memory_variant_chosen_when_fastest_at_the_largest_batch():
    t = table([9, 9, 9, 9, 9], [5, 4, 3, 2.2, 2.1], [5, 4, 3, 2.2, 2.0], [5, 4, 3, 2.2, 2.3])
    sel = pico.pico_tune_select(t, 256)
    assert (sel["gram_kc"], sel["gram_a_tmem"]) == (16, 1)
    t = table([9, 9, 9, 9, 9], [5, 4, 3, 2.2, 2.1], [5, 4, 3, 2.2, 2.2], [5, 4, 3, 2.2, 1.9])
    assert pico.pico_tune_select(t, 256)["gram_kc"] == 8


def test_crossover_requires_every_larger_batch_to_favour_the_gram_operator():
    # Gram faster at 16 but slower at 32: the crossover is 64, not 16
    t = table([5, 4, 4, 4, 4], [4.5, 4.2, 3.9, 3, 2], [9] * 5, [9] * 5)
    assert pico.pico_tune_select(t, 256)["gram_min_batch"] == 64
    # never faster: the Gram operator is switched off
    t = table([1, 1, 1, 1, 1], [2, 2, 2, 2, 2], [3] * 5, [3] * 5)
    sel = pico.pico_tune_select(t, 256)
    assert sel["gram_min_batch"] == 257 and sel["probe_batch"] == 0


def test_probe_batch_is_the_largest_within_three_percent():
    # FFT-only context: 128 is 2 % slower than 64, 256 is 5 % slower
    t = table([3.0, 2.0, 1.00, 1.02, 1.05])
    sel = pico.pico_tune_select(t, 256, gram=False)
    assert sel["probe_batch"] == 128 and sel["gram_kc"] == 0 and sel["gram_min_batch"] == 257
    # the fastest batch is max_batch itself: probe_batch 0 (= max_batch)
    t = table([3.0, 2.0, 1.5, 1.2, 1.0])
    assert pico.pico_tune_select(t, 256, gram=False)["probe_batch"] == 0


def test_max_batch_between_the_fixed_sizes_and_missing_entries():
    # max_batch 100: batches 16, 32, 64 and 100 (the sixth column)
    t = {"fft": {16: 4.0, 32: 3.0, 64: 2.5, 100: 2.0}}
    assert pico.pico_tune_select(t, 100, gram=False)["probe_batch"] == 0
    t = {"fft": {16: 4.0, 32: 3.0, 64: 2.0, 100: 2.5}}
    assert pico.pico_tune_select(t, 100, gram=False)["probe_batch"] == 64
    # batches with no column-FFT time are ignored; a Gram row without times is not chosen
    t = {"fft": {16: 4.0, 32: math.nan, 64: 2.0}, "gram16": {16: 1.0, 64: 1.0}}
    sel = pico.pico_tune_select(t, 64)
    assert sel["gram_kc"] == 16 and sel["gram_min_batch"] == 16
    with pytest.raises(pico.PicoError):
        pico.pico_tune_select({"fft": {}}, 64)
