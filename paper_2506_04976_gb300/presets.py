"""Settings of the three algorithms submitted to the PETRIC challenge (Sec. 4, Table 1):
all use SVRG with the harmonic preconditioner of eq. 8; they differ in the number of
subsets, the subset order, the preconditioner update epochs and the stepsize rule.

    n = petric_subsets("ALG3", nview)
    plan = Plan(geom, n)
    solver = Solver(plan, **petric_solver_kwargs("ALG3", n), beta=..., gamma=..., eps=...)

Host-side parameter choice only; every iteration runs in the library's kernels.
"""
from __future__ import annotations

from . import binding as pet

_TARGET = {"ALG1": 25.0, "ALG2": 25.0, "ALG3": 24.2}
# preconditioner update epochs (1-based) of Table 1
_PC_EPOCHS = {"ALG1": (1, 2, 3), "ALG2": (1, 2, 4, 6), "ALG3": (1, 2, 4, 6)}


def petric_subsets(name: str, nview: int) -> int:
    """Number of subsets of Table 1: the divisor of the number of views closest to 25
    (ALG1, ALG2) or to 24.2 (ALG3); on a tie the smaller divisor."""
    if name not in _TARGET:
        raise ValueError(f"unknown algorithm {name!r} (ALG1, ALG2 or ALG3)")
    t = _TARGET[name]
    divisors = [d for d in range(1, nview + 1) if nview % d == 0]
    return min(divisors, key=lambda d: (abs(d - t), d))


def petric_solver_kwargs(name: str, nsubsets: int) -> dict:
    """Solver keyword arguments of Table 1 for `nsubsets` subsets: SVRG (snapshot every
    two epochs), harmonic preconditioner updated at the start of the listed epochs
    (epoch e starts at iteration (e - 1) n), the ALG1 piecewise steps or the BB steps
    capped as in ALG2/ALG3, subsets without replacement (ALG1, ALG2) or in cofactor order
    (ALG3).  The BB step is computed at the snapshot refreshes that end epochs 2, 4 and 6
    and kept afterwards; before the first one the caps themselves are the steps (tau0 = 3
    is above every cap)."""
    if name not in _TARGET:
        raise ValueError(f"unknown algorithm {name!r} (ALG1, ALG2 or ALG3)")
    n = int(nsubsets)
    alg1 = name == "ALG1"
    return dict(algo=pet.SVRG, omega=2, precond_kind=1, alpha=1.0,
                pc_iters=tuple((e - 1) * n for e in _PC_EPOCHS[name]),
                step_rule=pet.STEP_ALG1 if alg1 else pet.STEP_ALG2, tau0=1.0 if alg1 else 3.0,
                bb_until=0 if alg1 else 6 * n,
                sampling=pet.SAMPLE_COFACTOR if name == "ALG3" else pet.SAMPLE_PERM)
