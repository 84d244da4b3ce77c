"""The C-ABI library without a GPU: it builds, loads, exports every symbol include/bsm.h declares,
and its host-side logic (parameter validation, vote tables) agrees with the oracle."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_1402_2020_gb300 import bsm, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1402_2020_gb300 import build

    build.build()
    return bsm.lib()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "bsm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bsm_[a-z_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "bsm_create" in names and "bsm_cost_aggregate_wta" in names
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(bsm.EXPORTED) == names
    nm = subprocess.run(["nm", "-D", "--defined-only", bsm.LIB_PATH], capture_output=True, text=True).stdout
    for n in names:
        assert re.search(rf"\bT {n}$", nm, flags=re.M), n


def test_status_strings(lib):
    assert bsm.bsm_status_string(0) == "ok"
    assert "timed out" in bsm.bsm_status_string(bsm.BSM_ERR_TIMEOUT)
    assert bsm.bsm_abi_version() == 3


def _params(**kw):
    pairs = kw.pop("pairs", synth.pair_table(256, 31, seed=1))
    return bsm.make_params(pairs, **kw)


def test_validate_params(lib):
    assert bsm.bsm_validate_params(_params()) == bsm.BSM_OK
    assert bsm.bsm_validate_params(_params(agg_window=1)) == bsm.BSM_OK
    assert bsm.bsm_validate_params(_params(pairs=synth.pair_table(64, 31, seed=2))) == bsm.BSM_OK
    bad = [
        dict(agg_window=4),
        dict(agg_window=0),
        dict(agg_window=17),  # 256 * 17^2 > 65535
        dict(mask_rank=257),
        dict(mask_rank=-1),
        dict(dmax=0),
        dict(lr_tol=-1),
        dict(vote_radius=40),
        dict(lambda_c=0),
        dict(window_S=11),  # offsets up to 15 exceed S/2
        dict(pairs=synth.pair_table(40, 31, seed=3)[:40]),  # n not a multiple of 32
    ]
    for kw in bad:
        assert bsm.bsm_validate_params(_params(**kw)) == bsm.BSM_ERR_INVALID_ARG, kw
    unsupported = [dict(pairs=synth.pair_table(768, 31, seed=4)), dict(agg_window=9, pairs=synth.pair_table(64, 31)),
                   dict(dmax=300), dict(pairs=synth.pair_table(96, 31, seed=5))]
    for kw in unsupported:
        assert bsm.bsm_validate_params(_params(**kw)) == bsm.BSM_ERR_UNSUPPORTED, kw
    # long descriptors: every power of two up to the paper's 4096, with n * W^2 <= 65535
    for n, win in ((512, 5), (1024, 7), (2048, 5), (4096, 3), (4096, 1)):
        assert bsm.bsm_validate_params(_params(pairs=synth.pair_table(n, 31, seed=n), agg_window=win)) == bsm.BSM_OK
    assert bsm.bsm_validate_params(_params(pairs=synth.pair_table(4096, 31, seed=6), agg_window=5)) == \
        bsm.BSM_ERR_INVALID_ARG
    assert bsm.bsm_validate_params(_params(pairs=synth.pair_table(8192, 31, seed=6), agg_window=1)) == \
        bsm.BSM_ERR_INVALID_ARG
    # mask modes: 0 (Eq. 8), 1 (no mask, Eq. 4), 2 (both views' masks, n >= 256)
    assert bsm.bsm_validate_params(_params(mask_mode=3)) == bsm.BSM_ERR_INVALID_ARG
    assert bsm.bsm_validate_params(_params(mask_mode=-1)) == bsm.BSM_ERR_INVALID_ARG
    assert bsm.bsm_validate_params(_params(mask_mode=1, mask_rank=5)) == bsm.BSM_ERR_INVALID_ARG
    assert bsm.bsm_validate_params(_params(mask_mode=1)) == bsm.BSM_OK
    assert bsm.bsm_validate_params(_params(mask_mode=2)) == bsm.BSM_OK
    assert bsm.bsm_validate_params(_params(mask_mode=2, pairs=synth.pair_table(128, 31, seed=8))) == \
        bsm.BSM_ERR_UNSUPPORTED
    with pytest.raises(bsm.BsmError) as e:
        bsm.bsm_server_create(_params(mask_mode=2))
    assert e.value.status == bsm.BSM_ERR_UNSUPPORTED
    # the server batches descriptors of up to 256 bits; it refuses longer ones before touching a device
    with pytest.raises(bsm.BsmError) as e:
        bsm.bsm_server_create(_params(pairs=synth.pair_table(512, 31, seed=7)))
    assert e.value.status == bsm.BSM_ERR_UNSUPPORTED
    # a NULL pair table
    p = _params()
    p.pairs = ctypes.POINTER(ctypes.c_int8)()
    assert bsm.bsm_validate_params(p) == bsm.BSM_ERR_INVALID_ARG


def test_create_rejects_bad_params_before_touching_the_gpu(lib):
    with pytest.raises(bsm.BsmError) as e:
        bsm.bsm_create(_params(agg_window=2))
    assert e.value.status == bsm.BSM_ERR_INVALID_ARG


@pytest.mark.parametrize("lc,le,R", [(9, 16, 15), (9, 16, 31), (5, 10, 3)])
def test_vote_tables_match_oracle(lib, orc, lc, le, R):
    Ec, Es = bsm.bsm_vote_tables(lc, le, 766, 2 * R * R + 1)
    oEc, oEs = orc.vote_tables(lc, le, R)
    assert (Ec == oEc).all() and (Es == oEs).all()


def test_vote_tables_reject_bad_args(lib):
    with pytest.raises(bsm.BsmError):
        bsm.bsm_vote_tables(0, 16, 766, 10)
