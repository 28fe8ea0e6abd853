"""Pins of the oracle's comb population control against what the comb's
definition fixes (systematic resampling): conservation of the walker count,
n_i within one of W w_i / S (floor or ceiling), exact unbiasedness of the
copy numbers and of weighted estimates over the draw xi, and the special
cases of equal and of single non-zero weights."""
import numpy as np

from oracle.afqmc import Options, initial_state, slice_step, local_energy
from oracle.population import comb_counts, comb_pairs, population_control, scaled_weights
from oracle.ueg import UEG
from synthetic_inputs import WORKLOADS, gaussian_fields


def test_counts_conserve_and_stay_within_one_of_expectation():
    rng = np.random.default_rng(3)
    for W in (1, 7, 64, 1000):
        for _ in range(20):
            w = rng.exponential(size=W) * (rng.random(W) > 0.2)
            if w.sum() == 0:
                continue
            xi = rng.random()
            n = comb_counts(w, xi)
            assert n.sum() == W
            x = W * w / w.sum()
            assert np.all(n >= np.floor(x - 1e-9)) and np.all(n <= np.ceil(x + 1e-9))
            assert np.all(n[w == 0] == 0)


def test_copy_numbers_are_unbiased_over_the_draw():
    """E_xi[n_i] = W w_i / S exactly: the average over a uniform grid of xi
    is within 1/grid of it."""
    rng = np.random.default_rng(4)
    W, grid = 50, 4000
    w = rng.exponential(size=W)
    mean = np.mean([comb_counts(w, (g + 0.5) / grid) for g in range(grid)], axis=0)
    assert np.max(np.abs(mean - W * w / w.sum())) < 2.0 / grid


def test_special_cases():
    W = 16
    for xi in (0.0, 0.3, 0.999999):
        assert np.array_equal(comb_counts(np.ones(W), xi), np.ones(W, dtype=int))
        w = np.zeros(W)
        w[5] = 2.5
        n = comb_counts(w, xi)
        assert n[5] == W and n.sum() == W
    # extra copies of 1 (two), 5 and 7 fill the empty slots 0, 3, 4, 6 in order
    n = np.array([0, 3, 1, 0, 0, 2, 0, 2])
    assert comb_pairs(n) == [(1, 0), (1, 3), (5, 4), (7, 6)]


def test_pairs_fill_every_empty_slot():
    rng = np.random.default_rng(5)
    W = 40
    w = rng.exponential(size=W) * (rng.random(W) > 0.3)
    n = comb_counts(w, 0.37)
    pairs = comb_pairs(n)
    dst = [d for _, d in pairs]
    assert sorted(dst) == [i for i in range(W) if n[i] == 0]
    assert all(n[s] >= 2 for s, _ in pairs)
    assert dst == sorted(dst) and [s for s, _ in pairs] == sorted(s for s, _ in pairs)


def _states(W, slices=6):
    c = WORKLOADS["ueg_n2_m7"]
    s = UEG(c["N"], c["M"], c["rs"], c["theta"], c["dtau"])
    f = gaussian_fields(11, slices, W, s.N_alpha)
    states = [initial_state(s) for _ in range(W)]
    for k in range(1, slices + 1):
        states = [slice_step(s, st, f[k - 1, w], k, Options())[0] for w, st in enumerate(states)]
    return s, states


def test_weighted_estimate_is_unbiased_over_the_draw():
    """sum_i w_i O_i / W before the comb equals the average over xi of the
    combed sum_i w'_i O'_i / W (every walker then weighs S / W)."""
    s, states = _states(12)
    w, ref = scaled_weights(states)
    O = np.array([local_energy(s, st.G)[0].real for st in states])
    before = np.sum(w * O)
    grid = 2000
    acc = 0.0
    for g in range(grid):
        new, parent = population_control(states, (g + 0.5) / grid)
        wn = np.exp(np.array([st.logw.real for st in new]) - ref)
        assert np.allclose(wn, w.sum() / len(w))
        acc += np.sum(wn * O[parent])
    assert abs(acc / grid - before) < 5e-3 * abs(before)


def test_population_control_copies_states_and_weights():
    s, states = _states(10)
    states[3] = states[3].__class__(**{**states[3].__dict__, "alive": False})
    new, parent = population_control(states, 0.61)
    w, _ = scaled_weights(states)
    n = comb_counts(w, 0.61)
    assert parent[3] != 3                       # a dead walker's slot is refilled
    for i, p in enumerate(parent):
        assert n[p] >= 1 and np.array_equal(new[i].G, states[p].G) and new[i].alive
        assert new[i].logw == new[0].logw


# ------------------------------------------------------------------ pair branching
def test_pair_branch_conserves_weight_and_thresholds():
    from oracle.population import pair_branch_pairs
    rng = np.random.default_rng(9)
    for W in (8, 64, 500):
        w = rng.exponential(size=W) ** 2 * (rng.random(W) > 0.1)
        draws = rng.random(W // 2)
        pairs = pair_branch_pairs(w, draws)
        new = w.copy()
        for src, dst, nw in pairs:
            new[src] = new[dst] = nw
        assert abs(new.sum() - w.sum()) < 1e-12 * w.sum()          # total weight exact
        u = w / w.mean()
        for src, dst, _ in pairs:                                    # one heavy, one light
            assert (u[src] > 2 and u[dst] < 0.5) or (u[src] < 0.5 and u[dst] > 2)
        unpaired = set(range(W)) - {s for s, _, _ in pairs} - {d for _, d, _ in pairs}
        heavy_left = [i for i in unpaired if u[i] > 2]
        light_left = [i for i in unpaired if u[i] < 0.5]
        assert not (heavy_left and light_left)                       # no pairable walkers remain


def test_pair_branch_is_unbiased_over_the_draws():
    """The expected weight carried by each walker's state is unchanged."""
    from oracle.population import pair_branch_pairs
    rng = np.random.default_rng(10)
    W, grid = 30, 2000
    w = rng.exponential(size=W) ** 3
    acc = np.zeros(W)
    for g in range(grid):
        draws = np.full(W // 2, (g + 0.5) / grid)
        carried = w.copy()
        for src, dst, nw in pair_branch_pairs(w, draws):
            carried[dst] = 0.0
            carried[src] = 0.0
        for src, dst, nw in pair_branch_pairs(w, draws):
            carried[src] += 2 * nw                                   # two copies of src's state
        acc += carried
    assert np.max(np.abs(acc / grid - w)) < 2e-3 * w.max()


def test_leftover_tooth_never_revives_a_dead_walker():
    """With xi just below 1 the last tooth (W - 1 + xi) S / W rounds to S
    itself; it belongs to the last walker that carries weight, never to a
    dead walker in the last slot (a dead walker has weight 0 and, by the
    comb's definition, an empty interval)."""
    xi = np.nextafter(1.0, 0.0)
    rng = np.random.default_rng(0)
    cases = 0
    for _ in range(200):
        W = int(rng.integers(2, 50))
        w = rng.exponential(size=W)
        w[-1] = 0.0
        if W > 3:
            w[-2] = 0.0
        C = np.cumsum(w)
        if (W - 1 + xi) * (C[-1] / W) < C[-1]:
            continue
        cases += 1
        n = comb_counts(w, xi)
        assert n.sum() == W
        assert np.all(n[w == 0] == 0)
    assert cases > 20
