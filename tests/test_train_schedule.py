"""The annealing schedule of Methods "Variational annealing" (host logic)."""
import pytest

from paper_2606_22984_gb300.train import TrainConfig, Trainer, anneal_temperature


def test_schedule_warmup_levels_and_end():
    T0, nw, na, ne = 2.0, 10, 4, 3
    assert all(anneal_temperature(i, T0, nw, na, ne) == T0 for i in range(nw + 1))
    # lowered by T0 / n_anneal every n_eq steps after the warm-up
    assert anneal_temperature(nw + ne, T0, nw, na, ne) == pytest.approx(T0 - T0 / na)
    assert anneal_temperature(nw + ne - 1, T0, nw, na, ne) == T0
    # zero after n_warmup + n_eq * n_anneal steps, and it stays there
    total = nw + ne * na
    assert anneal_temperature(total, T0, nw, na, ne) == 0.0
    assert anneal_temperature(total + 50, T0, nw, na, ne) == 0.0
    seq = [anneal_temperature(i, T0, nw, na, ne) for i in range(total + 5)]
    assert all(a >= b for a, b in zip(seq, seq[1:]))
    assert len(set(seq)) == na + 1


def test_schedule_rejects_bad_arguments():
    with pytest.raises(ValueError):
        anneal_temperature(5, 1.0, 0, 0, 1)


def test_trainer_needs_exactly_one_temperature_rule():
    cfg = TrainConfig(B=8, steps=1)
    with pytest.raises(ValueError):
        Trainer.__init__(object.__new__(Trainer), None, None, cfg)
