"""The C-ABI library builds, loads and exports every entry point declared in include/fairrank.h
(no GPU needed: only argument validation that happens before any CUDA call is exercised)."""
import ctypes as ct
import os
import re

import pytest

from paper_2406_10262_gb300 import build as frbuild
from paper_2406_10262_gb300 import fairrank as fr

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "fairrank.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fr_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    frbuild.build()
    return fr.lib()


def test_every_declared_symbol_is_exported(lib):
    syms = declared_symbols()
    assert len(syms) >= 18
    raw = ct.CDLL(fr.LIB_PATH)
    for s in syms:
        assert hasattr(raw, s), s


def test_config_defaults_and_columns(lib):
    cfg = fr.Config()
    lib.fr_config_default(ct.byref(cfg), 10, 20, 5, fr.PARAM_FULL_C)
    assert (cfg.n_users, cfg.n_items, cfg.n_slots) == (10, 20, 5)
    assert cfg.epsilon == 1.0 and cfg.sinkhorn_iters == 50 and cfg.warm_start == 1
    assert cfg.lr == 0.1 and cfg.beta1 == 0.9 and cfg.beta2 == 0.999 and cfg.adam_eps == 1e-8
    lib.fr_config_default(ct.byref(cfg), 10, 20, 5, fr.PARAM_ITEM)
    assert cfg.lr == 0.05
    assert fr.num_cols(20, 5) == 6 and fr.num_cols(5, 5) == 5


@pytest.mark.parametrize("field,value", [("n_users", 0), ("n_slots", 0), ("n_items", 3), ("epsilon", 0.0),
                                         ("sinkhorn_iters", 0), ("lr", -1.0), ("optimizer", 7),
                                         ("max_wait_polls", -2)])
def test_create_rejects_invalid_config_before_touching_the_device(lib, field, value):
    cfg = fr.Config()
    lib.fr_config_default(ct.byref(cfg), 4, 5, 4, fr.PARAM_FULL_C)
    setattr(cfg, field, value)
    h = ct.c_void_p()
    st = lib.fr_create(ct.byref(cfg), None, ct.byref(h))
    assert st == 1 and not h.value  # FR_EINVAL
    assert len(lib.fr_last_error(None)) > 0


def test_null_context_is_rejected(lib):
    assert lib.fr_step(None, 1, None) == 1
    assert lib.fr_impacts(None, None, None, None) == 1
    assert lib.fr_trace(None, 0, None, None, None) == 1


def batch_cfgs(lib, sizes, param=fr.PARAM_ITEM):
    cfgs = (fr.Config * len(sizes))()
    for j, (U, I, K) in enumerate(sizes):
        lib.fr_config_default(ct.byref(cfgs[j]), U, I, K, param)
    return cfgs


@pytest.mark.parametrize("sizes,param,fields,status", [
    ([(3, 50, 5), (0, 40, 5)], fr.PARAM_ITEM, {}, 1),                       # no consumers
    ([(3, 50, 5), (3, 4, 5)], fr.PARAM_ITEM, {}, 1),                        # K > |I|
    ([(3, 50, 5), (3, 40, 5)], fr.PARAM_ITEM, {1: {"param": fr.PARAM_FULL_C}}, 1),  # mixed params
    ([(3, 50, 5), (3, 40, 5)], fr.PARAM_ITEM, {1: {"epsilon": 0.5}}, 1),    # fields must match
    ([(3, 50, 5)], fr.PARAM_FULL_C, {0: {"rel_dtype": fr.BF16}}, 7),        # free costs: FP32 r
    ([(3, 50, 5)], fr.PARAM_ITEM, {0: {"grad_mode": fr.GRAD_UNROLLED}}, 7),  # implicit only
    ([(3, 4097, 20)], fr.PARAM_ITEM, {}, 7),                                 # per-item <= 4096 items
    ([(3, 50, 40)], fr.PARAM_ITEM, {}, 7),                                   # per-item <= 32 columns
])
def test_batch_create_rejects_before_touching_the_device(lib, sizes, param, fields, status):
    cfgs = batch_cfgs(lib, sizes, param)
    for j, f in fields.items():
        for k, v in f.items():
            setattr(cfgs[j], k, v)
    h = ct.c_void_p()
    assert lib.fr_batch_create(cfgs, len(sizes), None, ct.byref(h)) == status and not h.value
    assert len(lib.fr_batch_last_error(None)) > 0


def test_batch_create_rejects_null_arguments(lib):
    h = ct.c_void_p()
    cfgs = batch_cfgs(lib, [(3, 50, 5)])
    assert lib.fr_batch_create(cfgs, 1, None, None) == 1
    assert lib.fr_batch_create(None, 1, None, ct.byref(h)) == 1
    assert lib.fr_batch_create(cfgs, 0, None, ct.byref(h)) == 1


def test_missing_library_fails_loudly(monkeypatch):
    """No fallback: without the compiled library every entry point of the binding raises."""
    monkeypatch.setattr(fr, "_lib", None)
    monkeypatch.setattr(fr, "LIB_PATH", os.path.join(ROOT, "no-such-dir", "libfairrank.so"))
    with pytest.raises(RuntimeError, match="not built"):
        fr.lib()
    with pytest.raises(RuntimeError, match="not built"):
        fr.FairRank(4, 10, 3)
    with pytest.raises(RuntimeError, match="not built"):
        fr.FairRankBatch([(4, 10, 3)])
