"""The constants the paper fixes (tests/golden/paper_constants.json, each with
its passage) are the ones the oracle, the library's Python defaults and the
workloads use."""
import inspect
import json
import os

import numpy as np

from oracle.gauss_newton import FLOOR, fit_pose
from oracle.harmonic import harmonic_initialization
from oracle.projections import CLAMP
from workloads.meshes import sweater_shell

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))


def val(key):
    return GOLDEN[key]["value"]


def default(fn, name):
    return inspect.signature(fn).parameters[name].default


def test_every_constant_has_a_citation():
    for k, v in GOLDEN.items():
        if not k.startswith("_"):
            assert v["cite"].startswith(("Sec.", "Teaser", "Table")), k


def test_oracle_uses_the_papers_constants():
    assert CLAMP == val("volume_target_clamp")
    assert FLOOR == val("nonnegativity_floor")
    assert default(fit_pose, "gd_step") == val("gd_initial_step")
    assert default(fit_pose, "gn_step") == val("gn_initial_step")
    assert default(fit_pose, "floor") == val("nonnegativity_floor")
    assert tuple(default(harmonic_initialization, "ranks")) == tuple(val("harmonic_ranks"))


def test_library_defaults_use_the_papers_constants():
    # the binding's signatures only (no GPU needed to read them)
    import ast
    src = open(os.path.join(os.path.dirname(os.path.dirname(__file__)), "paper_2405_12484_gb300", "sim.py")).read()
    tree = ast.parse(src)
    defaults = {}
    for node in ast.walk(tree):
        if isinstance(node, ast.FunctionDef):
            args = node.args.args[-len(node.args.defaults):] if node.args.defaults else []
            defaults[node.name] = {a.arg: ast.literal_eval(d) for a, d in zip(args, node.args.defaults)
                                   if isinstance(d, (ast.Constant, ast.Tuple))}
    assert defaults["fit_pose"]["gd_step"] == val("gd_initial_step")
    assert defaults["fit_pose"]["gn_step"] == val("gn_initial_step")
    assert defaults["fit_pose"]["floor"] == val("nonnegativity_floor")
    assert defaults["fit_pose_reduced"]["floor"] == val("nonnegativity_floor")
    assert tuple(defaults["harmonic_initialization"]["ranks"]) == tuple(val("harmonic_ranks"))
    assert defaults["solver_opts"]["modes"] == val("normal_modes_per_domain")


def test_the_sweater_workload_matches_the_teaser():
    w = sweater_shell()
    assert abs(w.dt - val("sweater_time_step")) < 1e-15
    assert w.n_t == val("sweater_elements")
    assert np.isclose(1.0 / w.dt, 150.0)
