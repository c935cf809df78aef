"""Check of an oracle follow-mode result, shared by the GPU parity tests.

The comparison rule: the GPU's selection may leave the oracle's only where
the two values that decide a step (the group's top errors for the argmax of
Alg. 1, or the group maximum and E* for its E > E* test) agree to 1e-6
relative.  Every such step is logged: the count and the largest relative gap
are printed with the test's output, and the gap is held to the band.
"""

TIE = 1e-6


def check_follow(f, label=""):
    s = f["stats"]
    print(f"\nfollow {label}: divergences {s['n_div']}, worst relative gap "
          f"{s['worst_rel_gap']:.3e}, rejected {s['n_fail']}")
    assert s["n_fail"] == 0, s
    assert s["worst_rel_gap"] <= TIE, s
    return s
