"""The dependency structure the one-launch step (k_step) relies on, checked on the oracle's
P-ERK families (Eq. PartitionedRKSystem with the tableaux of Sec. 3.3 and 4.3): a stage state of
member r at stage i combines U, K_1 and K_{i-1} only, and K_{i-1} enters only where member r
evaluated stage i-1.  The kernel's waits (for K_{i-1}: stage i-1 of the element done; for K_1:
stage 0 done) therefore always target a stage the element computed, in an item dealt earlier,
and every element computes stage 0."""
import numpy as np
import pytest

from oracle.perk import perk2_family, perk3_family

FAMILIES = [("perk2", [4, 6, 10, 16]), ("perk2", [4, 8]), ("perk2", [6, 10, 16]), ("perk2", [2, 3]),
            ("perk3", [4, 8, 16]), ("perk3", [3, 4, 6]), ("perk3", [3, 8])]


@pytest.mark.parametrize("kind,E", FAMILIES)
def test_stage_states_couple_to_k1_and_the_previous_evaluated_stage(kind, E):
    fam = perk2_family(E) if kind == "perk2" else perk3_family(E)
    S = fam.S
    for r in range(fam.R):
        A = np.asarray(fam.A[r])
        assert fam.active(r, 0)                       # K_1 is evaluated by every member
        for i in range(1, S):
            row = A[i]
            others = [j for j in range(S) if j not in (0, i - 1) and row[j] != 0.0]
            assert not others, (kind, E, r, i, others)
            if row[i - 1] != 0.0 and i - 1 > 0:
                # K_{i-1} is read: the member evaluated stage i-1 (and stages stay evaluated to the
                # end, so it evaluates stage i too)
                assert fam.active(r, i - 1) and fam.active(r, i), (kind, E, r, i)
            if not fam.active(r, i):
                # a member that skips stage i contributes only U + dt c_i K_1 to neighbouring faces
                assert all(row[j] == 0.0 for j in range(1, S)), (kind, E, r, i)
        # evaluated stages after K_1 form one contiguous block ending at stage S
        evaluated = [i for i in range(1, S) if fam.active(r, i)]
        if evaluated:
            assert evaluated == list(range(evaluated[0], S)), (kind, E, r)
