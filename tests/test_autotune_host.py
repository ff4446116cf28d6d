"""The autotuner's selection rule (host logic, no GPU)."""
import pytest

from paper_2111_00110_gb300.autotune import Candidate, select


def C(g, o, ms, err):
    return Candidate(g, o, "separable", ms, err)


def test_fastest_within_target():
    cands = [C(32, 4, 1.0, 3e-2), C(32, 6, 1.5, 8e-3), C(64, 4, 2.0, 9e-3), C(64, 8, 4.0, 1e-4)]
    assert select(cands, 1e-2) == cands[1]
    assert select(cands, 1e-3) == cands[3]
    assert select(cands, 1.0) == cands[0]


def test_none_within_target_takes_the_most_accurate():
    cands = [C(32, 4, 1.0, 3e-2), C(32, 6, 0.5, 2e-2), C(64, 6, 2.0, 2e-2)]
    assert select(cands, 1e-3) == cands[1]   # most accurate, ties broken by time


def test_ties_in_time_prefer_accuracy():
    cands = [C(32, 6, 1.0, 5e-3), C(64, 4, 1.0, 1e-3)]
    assert select(cands, 1e-2) == cands[1]


def test_empty():
    with pytest.raises(ValueError):
        select([], 1e-2)


def test_batch_refinement_moves_fp32_forms_to_occupied_when_the_batch_is_faster():
    from paper_2111_00110_gb300.autotune import refine_batch
    cs = [Candidate(64, 6, "separable", 1.0, 5e-3, tile=32), Candidate(64, 8, "occupied", 2.0, 4e-3),
          Candidate(64, 6, "bf16", 0.5, 8e-3)]
    seen = []

    def timer(choice):
        seen.append([c.m2l for c in choice])
        return 10.0 if choice[0].m2l == "separable" else 8.0

    out, info = refine_batch(cs, timer)
    assert [c.m2l for c in out] == ["occupied", "occupied", "bf16"]   # mixed forms keep their own error
    assert out[0].tile == 0 and out[0].err == cs[0].err and out[0].order == 6
    assert info == {"per_instance_ms": 10.0, "occupied_ms": 8.0}
    out2, _ = refine_batch(cs, lambda choice: 8.0 if choice[0].m2l == "separable" else 10.0)
    assert out2 == cs
    out3, info3 = refine_batch([cs[1]], timer)   # nothing to move: no batch timed
    assert out3 == [cs[1]] and info3 == {} and len(seen) == 2


def test_candidates_carry_their_tile():
    a = Candidate(64, 6, "separable", 1.0, 5e-3, tile=32)
    b = Candidate(64, 6, "separable", 1.1, 5e-3)
    assert select([a, b], 1e-2).tile == 32 and b.tile == 0
