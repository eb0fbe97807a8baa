"""The online pools of Alg. 2 (Supp. "Online Frame Processing"): FIFO order of the local pool,
reservoir sampling of the global pool (every frame that leaves the local pool is kept with the
same probability |M_g| / (j + 1), checked statistically over many seeds), and the eta split
of a batch between the pools."""
import numpy as np

from paper_2503_12886_gb300.online import LocalGlobalSampler


def test_local_pool_is_fifo_and_global_fills_in_order():
    s = LocalGlobalSampler(150, 1000, 0.7, seed=1)
    for i in range(200):
        s.push(i)
    assert list(s.local) == list(range(50, 200))
    assert s.glob == list(range(50))
    for i in range(200, 1150):
        s.push(i)
    assert s.glob == list(range(1000)) and list(s.local) == list(range(1000, 1150))


def test_reservoir_keeps_every_frame_with_equal_probability():
    """local 100, global 20, 600 frames: the 500 frames that left the local pool are each in
    the global pool with probability 20/500 after the last push (Vitter's Algorithm R, indexed
    by the frame's own stream position). Inclusion counts over 600 seeds, in 10 bins of 50
    stream positions, each within 5 sigma of 600*50*0.04."""
    cap, loc, n, runs = 20, 100, 600, 600
    counts = np.zeros(n - loc)
    for seed in range(runs):
        s = LocalGlobalSampler(loc, cap, 0.7, seed=seed)
        for i in range(n):
            s.push(i)
        counts[np.asarray(s.glob)] += 1
    bins = counts.reshape(10, 50).sum(1)
    p = cap / (n - loc)
    mean = runs * 50 * p
    sd = np.sqrt(runs * 50 * p * (1 - p))
    assert np.all(np.abs(bins - mean) <= 5 * sd), (bins, mean, sd)
    assert counts.sum() == runs * cap


def test_batch_split_and_fill_in():
    s = LocalGlobalSampler(150, 1000, 0.7, seed=3)
    for i in range(3):
        s.push(i)
    assert sorted(s.sample(16)) == [0, 1, 2]                 # both pools short
    for i in range(3, 160):
        s.push(i)                                            # 10 frames in the global pool
    b = s.sample(16)
    assert len(b) == 16 and len(set(b)) == 16
    assert sum(x < 10 for x in b) == 5 and sum(x >= 10 for x in b) == 11
    for i in range(160, 1400):
        s.push(i)
    for _ in range(20):
        b = s.sample(16)
        loc = set(s.local)
        assert len(set(b)) == 16
        assert sum(x in loc for x in b) == 11                # round(0.7 * 16)
    s2 = LocalGlobalSampler(4, 100, 0.7, seed=5)
    for i in range(40):
        s2.push(i)
    assert sum(x in set(s2.local) for x in s2.sample(16)) == 4   # local short: global fills in


def test_runs_are_a_function_of_the_seed():
    def run(seed):
        s = LocalGlobalSampler(10, 30, 0.7, seed=seed)
        out = []
        for i in range(300):
            s.push(i)
            if i % 7 == 0:
                out.append(tuple(s.sample(8)))
        return out, list(s.glob)
    assert run(11) == run(11) and run(11) != run(12)
