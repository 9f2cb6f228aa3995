"""The C-ABI library builds, loads and exports every entry point include/asicp.h declares
(no compute calls: these run without a GPU)."""
import ctypes
import json
import os
import re

import pytest

from paper_2412_08346_gb300 import asicp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header="asicp.h"):
    with open(os.path.join(ROOT, "include", header)) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(asicp_[a-z_]+)\s*\(", text)))


def test_header_symbols_are_exported():
    lib = asicp.load()
    names = _declared()
    assert "asicp_create" in names and "asicp_step" in names and len(names) >= 12
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/asicp.h but not exported"
    assert sorted(asicp.EXPORTED) == names


def test_proposal_header_symbols_are_exported():
    from paper_2412_08346_gb300 import proposal
    lib = asicp.load()
    names = _declared("asicp_proposal.h")
    assert "asicp_prop_create" in names and len(names) == 9
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/asicp_proposal.h but not exported"
    assert sorted(proposal.PROP_EXPORTED) == names
    from oracle import proposal as orc
    for P in (1, 3, 10):
        assert proposal.num_params(P) == orc.num_params(P)


def test_proposal_create_rejects_bad_sizes_without_touching_the_gpu():
    from paper_2412_08346_gb300 import proposal
    for args in ((0, 256, 4), (3, 8, 4), (3, 256, 0), (17, 256, 4)):
        with pytest.raises(asicp.AsicpError) as e:
            proposal.Proposal(*args)
        assert e.value.status == asicp.ASICP_ERR_INVALID_ARG


def test_defaults_follow_table1():
    with open(os.path.join(ROOT, "tests", "golden", "table1_parameters.json")) as f:
        t1 = json.load(f)
    cfg = asicp.asicp_config_default()
    assert cfg.eta_sgd == t1["sgd_learning_rate"]
    assert cfg.w_com == t1["cost_weights"]
    assert cfg.C_cycles == t1["annealing_cycles_C"] and cfg.p_exp == t1["annealing_exponent_p"]
    assert cfg.conv_tol == pytest.approx(t1["convergence_criterion_relative"])
    assert (cfg.k_stein, cfg.k_max - cfg.k_stein) == (t1["svgd_iterations"], t1["sgd_iterations"])
    assert cfg.schedule == 0 and cfg.bandwidth_mode == 0 and cfg.eta_svgd == 0.0


@pytest.mark.parametrize("field,value", [("P", 0), ("K", 0), ("K", 2048), ("k_stein", 99), ("k_max", -1),
                                         ("schedule", 3), ("C_cycles", 0.0), ("init_radius", -1.0)])
def test_create_rejects_bad_config_without_touching_the_gpu(field, value):
    cfg = asicp.asicp_config_default()
    setattr(cfg, field, value)
    with pytest.raises(asicp.AsicpError) as e:
        asicp.asicp_create(cfg)
    assert e.value.status == asicp.ASICP_ERR_INVALID_ARG


def test_null_context_is_an_error_not_a_crash():
    lib = asicp.load()
    assert lib.asicp_step(None, 0) == asicp.ASICP_ERR_INVALID_ARG
    assert lib.asicp_run(None, None) == asicp.ASICP_ERR_INVALID_ARG
    assert lib.asicp_set_object(None, None, 0, None, 0) == asicp.ASICP_ERR_INVALID_ARG
    assert lib.asicp_destroy(None) == asicp.ASICP_OK
    assert lib.asicp_last_error(None) == b"NULL context"
    out = ctypes.c_void_p()
    assert lib.asicp_create(None, ctypes.byref(out)) == asicp.ASICP_ERR_INVALID_ARG


def test_library_is_in_tree():
    assert os.path.commonpath([asicp.library_path(), ROOT]) == ROOT
