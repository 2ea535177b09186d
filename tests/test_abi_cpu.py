"""The C-ABI library builds, loads without a GPU and exports every function
that include/hexval.h declares; host-side argument checks need no device."""
import ctypes
import os
import re

import pytest

from paper_1706_01613_gb300 import _build
from paper_1706_01613_gb300 import hexval as hv

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "hexval.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hexval_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return hv.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 8
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(hv.EXPORTS) == names


def test_default_config(lib):
    cfg = hv.default_config()
    assert cfg.struct_size == ctypes.sizeof(hv.Config)
    assert (cfg.precision, cfg.max_depth) == (hv.FP64, 8)
    assert cfg.max_batch == 1 << 24 and cfg.queue_capacity == 1 << 23
    assert cfg.exact_capacity == 1 << 16 and cfg.max_nodes == 1 << 24


def test_host_side_argument_errors(lib):
    null = ctypes.c_void_p()
    assert lib.hexval_check_soa(null, 10, null, null, null, null, null) == -1
    assert lib.hexval_check_indexed(null, 1, null, 1, null, null, null, null, null) == -1
    assert lib.hexval_status(null, null) == -1
    assert lib.hexval_destroy(null) == -1
    assert lib.hexval_create(None, ctypes.byref(ctypes.c_void_p())) == -1
    bad = hv.default_config()
    bad.max_depth = 16
    assert lib.hexval_create(ctypes.byref(bad), ctypes.byref(ctypes.c_void_p())) == -1
    bad = hv.default_config()
    bad.struct_size = 3
    assert lib.hexval_create(ctypes.byref(bad), ctypes.byref(ctypes.c_void_p())) == -1


def test_strerror(lib):
    for code, name in hv.CODES.items():
        assert lib.hexval_strerror(code).decode()
    assert lib.hexval_strerror(-99).decode() == "unknown code"


def test_binding_refuses_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(RuntimeError):
        hv.Validator()


def _header():
    text = open(os.path.join(ROOT, "include", "hexval.h")).read()
    return re.sub(r"/\*.*?\*/", "", text, flags=re.S)


def _enum_values(text):
    return {k: int(v, 0) for k, v in re.findall(r"\b(HEXVAL_\w+)\s*=\s*(-?\w+)", text)}


def test_binding_constants_match_the_header():
    """Option bits, profile phases and the statistics record of the binding
    are the header's."""
    vals = _enum_values(_header())
    assert vals["HEXVAL_OPT_PAIR32"] == hv.OPT_PAIR32
    assert vals["HEXVAL_OPT_PREFETCH"] == hv.OPT_PREFETCH
    assert vals["HEXVAL_OPT_DFREDO"] == hv.OPT_DFREDO
    assert vals["HEXVAL_OPT_NO_REPLAY"] == hv.OPT_NO_REPLAY
    assert vals["HEXVAL_OPT_LEVEL1"] == hv.OPT_LEVEL1
    assert vals["HEXVAL_OPT_PARTIAL64"] == hv.OPT_PARTIAL64
    assert len(hv.PHASES) == vals["HEXVAL_PH_COUNT"]
    for name, ph in (("nodes32", "NODES32"), ("bulk32", "BULK32"), ("bulk64", "BULK64"),
                     ("tail", "TAIL"), ("redo_df", "REDODF"), ("level1", "LEVEL1"),
                     ("redo_partial", "PARTIAL")):
        assert hv.PHASES.index(name) == vals["HEXVAL_PH_" + ph]
    body = re.search(r"typedef struct \{([^}]*)\} hexval_stats;", _header()).group(1)
    fields = re.findall(r"uint64_t\s+(\w+);", body)
    assert [f for f, _ in hv.Stats._fields_] == fields
    for code, name in hv.CODES.items():
        assert vals[name] == code


def test_options_outside_the_known_bits_are_refused(lib):
    bad = hv.default_config()
    bad.options = 64
    assert lib.hexval_create(ctypes.byref(bad), ctypes.byref(ctypes.c_void_p())) == -1
    bad = hv.default_config()  # two redos of the same escalation list
    bad.options = hv.OPT_DFREDO | hv.OPT_PARTIAL64
    assert lib.hexval_create(ctypes.byref(bad), ctypes.byref(ctypes.c_void_p())) == -1
    bad = hv.default_config()
    bad.reserved = 1
    assert lib.hexval_create(ctypes.byref(bad), ctypes.byref(ctypes.c_void_p())) == -1
    assert hv.default_config().spin_limit == 0  # the default budget
    for field, val in (("reserved2", 1), ("tail_warp_items", 0), ("tail_warp_items", 65)):
        bad = hv.default_config()
        setattr(bad, field, val)
        assert lib.hexval_create(ctypes.byref(bad), ctypes.byref(ctypes.c_void_p())) == -1


def test_placement_defaults():
    cfg = hv.default_config()
    assert (cfg.esc_in_pass, cfg.refine_in_pass, cfg.tail_warp_items) == (4096, 512, 8)


def test_copy_soa_range_refuses_bad_ranges(lib):
    """The range copy checks its range on the host and enqueues nothing on
    error (no device needed to see the refusal)."""
    buf = ctypes.create_string_buffer(24 * 8 * 10)
    p = ctypes.cast(buf, ctypes.c_void_p)
    assert lib.hexval_copy_soa_range(None, p, 10, 0, 5, None) == -1
    assert lib.hexval_copy_soa_range(p, p, 10, 6, 5, None) == -1
    assert lib.hexval_copy_soa_range(p, p, 10, -1, 5, None) == -1
    assert lib.hexval_copy_soa_range(p, p, 10, 3, 0, None) == 0  # empty: nothing to do


def test_prepared_nodes_refusals(lib):
    """The prepared-node entry points check their arguments on the host: no
    handle, no node array, or no prepared nodes is HEXVAL_E_ARG."""
    buf = ctypes.create_string_buffer(64)
    p = ctypes.cast(buf, ctypes.c_void_p)
    assert lib.hexval_prepare_nodes(None, 10, p, None) == -1
    assert lib.hexval_check_indexed_prepared(None, 10, p, p, None, None, None) == -1
