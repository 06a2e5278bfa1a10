"""Host logic of the autotuner: coordinate descent over the launch-shape
axes keeps the fastest admissible candidate and skips rejected ones."""
from paper_2106_13465_gb300.autotune import coordinate_descent


def test_coordinate_descent_finds_the_separable_minimum():
    axes = {"a": [0, 1, 2, 3], "b": [0, 10, 20], "c": [5, 6]}
    target = {"a": 2, "b": 10, "c": 6}

    def cost(cfg):
        return sum(abs(cfg[k] - target[k]) for k in cfg) + 1.0

    cfg, best, trials = coordinate_descent(cost, axes)
    assert cfg == target and best == 1.0
    assert len(trials) == 1 + 3 + 2 + 1


def test_rejected_candidates_are_never_chosen():
    axes = {"a": [0, 1, 2]}

    def cost(cfg):
        return None if cfg["a"] == 2 else 10.0 - cfg["a"]

    cfg, best, _ = coordinate_descent(cost, axes)
    assert cfg == {"a": 1} and best == 9.0
