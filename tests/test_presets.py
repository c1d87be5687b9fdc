"""The Table 1 presets of the submitted algorithms (Sec. 4): subset counts as the divisor
of the number of views nearest 25 (24.2 for ALG3), preconditioner update epochs, step
rules and subset orders."""
import pytest

presets = pytest.importorskip("paper_2506_04976_gb300.presets")


def test_subset_counts():
    # 224 views (the large TOF workload): the rule gives 28, not the 25 used there
    assert presets.petric_subsets("ALG1", 224) == 28
    assert presets.petric_subsets("ALG3", 224) == 28
    # 216 views (the paper's simulated scanner, Sec. 3.1): 24 (27 is farther)
    assert presets.petric_subsets("ALG2", 216) == 24
    # 168 views: 24 for both targets
    assert presets.petric_subsets("ALG1", 168) == 24 and presets.petric_subsets("ALG3", 168) == 24
    # a tie (25 +- 3 with divisors 22 and 28 of 308) goes to the smaller divisor
    assert presets.petric_subsets("ALG1", 308) == 22
    # 312 views: 24 and 26 tie for 25 (the smaller wins); 24.2 picks 24 outright
    assert presets.petric_subsets("ALG3", 312) == 24 and presets.petric_subsets("ALG1", 312) == 24
    assert presets.petric_subsets("ALG1", 7) == 7
    with pytest.raises(ValueError):
        presets.petric_subsets("ALG4", 100)


def test_solver_settings():
    pet = presets.pet
    n = 24
    a1 = presets.petric_solver_kwargs("ALG1", n)
    a2 = presets.petric_solver_kwargs("ALG2", n)
    a3 = presets.petric_solver_kwargs("ALG3", n)
    assert a1["pc_iters"] == (0, n, 2 * n) and a2["pc_iters"] == (0, n, 3 * n, 5 * n) == a3["pc_iters"]
    assert a1["step_rule"] == pet.STEP_ALG1 and a2["step_rule"] == a3["step_rule"] == pet.STEP_ALG2
    assert a1["sampling"] == a2["sampling"] == pet.SAMPLE_PERM and a3["sampling"] == pet.SAMPLE_COFACTOR
    assert all(a["algo"] == pet.SVRG and a["precond_kind"] == 1 for a in (a1, a2, a3))
    assert a1["bb_until"] == 0 and a2["bb_until"] == a3["bb_until"] == 6 * n
    assert a2["tau0"] >= 3.0  # before the first BB step the Table 1 caps apply
    with pytest.raises(ValueError):
        presets.petric_solver_kwargs("ALG4", n)
