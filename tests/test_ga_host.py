"""Host-side rule of the global-alignment driver (no GPU): the Eq. 4
learning-rate choice from the median epipolar distance agrees with the
oracle's, on both sides of each boundary."""
from oracle import ga as OG
from paper_2509_25191_gb300 import ga


def test_learning_rate_rule_matches_the_oracle():
    for m in (0.0, 1.0, 2.4999, 2.5, 2.5001, 5.0, 7.4999, 7.5, 7.5001, 40.0, 1e6):
        assert ga.lr_rule(m) == OG.lr_rule(m), m
    assert (ga.lr_rule(2.4), ga.lr_rule(5.0), ga.lr_rule(8.0)) == ga.LRS
