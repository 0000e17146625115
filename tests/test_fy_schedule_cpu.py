"""The parallel schedule of the GPU Fisher-Yates shuffle (n <= 65535), as a
plain-Python model of one warp: lane l holds step hi - l of the window and its
draw j; each round applies at once the longest leading run of steps whose
swaps touch pairwise distinct positions (a step with j != i allows runs of at
most hi - j steps; a draw repeated from an earlier step ends the run), then
shifts the window.  Whatever the draws, the result must equal the sequential
loop i = n-1 .. 1 of swap(p[i], p[j_i]), and every round must make progress."""
import numpy as np
import pytest


def sequential(n, draws):
    p = list(range(n))
    for i in range(n - 1, 0, -1):
        j = draws[i]
        p[i], p[j] = p[j], p[i]
    return p


def warp_schedule(n, draws):
    p = list(range(n))
    hi, rounds = n - 1, 0
    while hi >= 1:
        rounds += 1
        pos = [hi - lane for lane in range(32)]
        valid = [i >= 1 for i in pos]
        j = [draws[pos[l]] if valid[l] else -1 - l for l in range(32)]
        lim = [0 if not valid[l] else (32 if j[l] == pos[l] else hi - j[l]) for l in range(32)]
        for l in range(1, 32):                       # running minimum over lanes 0..l
            lim[l] = min(lim[l], lim[l - 1])
        take = [valid[l] and l < lim[l] and j[l] not in j[:l] for l in range(32)]
        k = 0
        while k < 32 and take[k]:
            k += 1
        assert k >= 1
        swaps = [(pos[l], j[l]) for l in range(k) if j[l] != pos[l]]
        touched = [x for s in swaps for x in s]
        assert len(touched) == len(set(touched))     # the run's swaps are disjoint
        old = {x: p[x] for x in touched}
        for a, b in swaps:
            p[a], p[b] = old[b], old[a]
        hi -= k
    return p, rounds


@pytest.mark.parametrize("n", [1, 2, 3, 5, 31, 32, 33, 64, 100, 1000, 4099])
def test_runs_of_disjoint_swaps_equal_the_sequential_shuffle(n):
    rng = np.random.default_rng(n)
    for _ in range(8 if n < 2000 else 2):
        draws = [0] + [int(rng.integers(0, i + 1)) for i in range(1, n)]
        got, rounds = warp_schedule(n, draws)
        assert got == sequential(n, draws)
        assert rounds <= max(n - 1, 0)


def test_adversarial_draws():
    # every step draws the position just below it, or itself: runs of length 1
    # and self-swaps must both come out as the sequential loop does
    for n in (40, 97):
        for draws in ([0] + [i - 1 for i in range(1, n)], [0] + list(range(1, n)),
                      [0] + [0] * (n - 1)):
            assert warp_schedule(n, draws)[0] == sequential(n, draws)
