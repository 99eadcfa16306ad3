"""Fixtures under tests/golden/ that hold values the paper prints, each with
its citation, checked against the defaults of the library, the oracle and
the host-side basis and cubature construction (no GPU)."""
import inspect
import os

import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _parameters():
    out = {}
    with open(os.path.join(GOLDEN, "paper_parameters.txt")) as f:
        for line in f:
            if not line.strip() or line.startswith("#"):
                continue
            name, value, cite = line.split(None, 2)
            assert cite.startswith("Sec."), f"{name} has no citation"
            out[name] = float(value)
    return out


P = _parameters()


def test_partitioning_constants_follow_the_paper():
    from paper_2508_13386_gb300 import basis
    assert P["jump_penalty_min"] <= basis.JUMP_PENALTY <= P["jump_penalty_max"]
    assert basis.PRUNE_RATIO == P["imbalance_ratio"]
    assert basis.PRUNE_EVERY == P["prune_every"]
    assert basis.PRUNE_COUNT == P["prune_count"]


def test_cubature_tolerance_follows_the_paper():
    from paper_2508_13386_gb300 import cubature
    assert cubature.DEFAULT_TOL == P["cubature_rtol"]


def test_oracle_paper_mode_defaults_follow_the_paper():
    from oracle import newton, subspace
    pt = inspect.signature(newton.paper_timestep).parameters
    assert P["refine_cg_min"] <= pt["n_cg"].default <= P["refine_cg_max"]
    assert pt["tol"].default == P["newton_tol"]
    assert inspect.signature(subspace.subspace_direction_literal).parameters["rtol"].default == \
        P["subspace_pcg_rtol"]


def test_library_defaults_follow_the_paper():
    import paper_2508_13386_gb300 as mls
    from paper_2508_13386_gb300 import _lib
    try:
        lib = mls._get_lib()
    except OSError as e:                      # the library is built by build(); its absence is reported
        pytest.fail(f"libmls.so not loadable: {e}")
    import ctypes as C
    o = _lib.Options()
    assert lib.mls_default_options(C.byref(o)) == 0
    assert o.pcg_rtol == P["subspace_pcg_rtol"]
    assert P["refine_cg_min"] <= o.refine_iters <= P["refine_cg_max"]
    assert o.paper_tol == P["newton_tol"]
