"""The Soft/Hard Pruning schedule (Sec. 4.2.2, 4.2.3, reading 28) as
iteration sets: Soft Prunes at 6k, 9k and 12k, each at an opacity reset of
the densification (every 3k before 15k), then Hard Prunes every 3k from 15k
to the end; the same pattern at the scaled counts the bench and the tests
run."""
from paper_2412_00578_gb300.prune import Schedule


def test_paper_schedule():
    sch = Schedule(scale=1.0)
    soft, resets, hard = sch.events(30_000)
    assert soft == {6_000, 9_000, 12_000}
    assert resets == {3_000, 6_000, 9_000, 12_000}
    assert soft <= resets  # every Soft Prune coincides with a reset
    assert hard == set(range(15_000, 30_001, 3_000))
    assert max(soft) < min(hard)
    assert sch.events(30_000, prune=False) == (set(), resets, set())


def test_scaled_schedules():
    for scale, total in ((0.1, 3_000), (0.02, 600)):
        sch = Schedule(scale=scale)
        soft, resets, hard = sch.events(total)
        assert soft == {round(x * scale) for x in (6_000, 9_000, 12_000)}
        assert soft <= resets and max(resets) < round(15_000 * scale)
        step = round(3_000 * scale)
        assert sorted(hard) == list(range(round(15_000 * scale), total + 1, step))
