"""Host logic of the learned form (no GPU): where its proposal window starts."""
import pytest


@pytest.mark.parametrize("every", [1, 7, 100])
def test_first_proposal_sweep_is_the_first_chunk_ending_past_start(every):
    from paper_2505_18508_gb300.learned import first_proposal_sweep
    for S in (0, 1, every - 1, every, 3 * every + 2, 350):
        for start in range(-2, S + every + 2):
            chunks = [k0 for k0 in range(0, S, every) if k0 + every > start]
            assert first_proposal_sweep(S, every, start) == (chunks[0] if chunks else S), (S, every, start)
