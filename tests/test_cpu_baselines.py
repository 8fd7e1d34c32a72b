"""The benchmark's timed CPU references against the oracle (CPU only).

cpu_hss_omp runs the method's steps on all host cores with OpenMP; it must
give exactly the oracle's splitters, offsets, round statistics and output, so
that its time is the time of the same result.  std::sort is checked against
numpy's sort."""
import numpy as np
import pytest

import oracle
from paper_1803_01237_gb300 import inputs


@pytest.mark.parametrize("gen,N,p,eps,seed", [
    (inputs.uniform, 1 << 20, 64, 0.05, 1), (inputs.zipf, 300001, 13, 0.02, 3), (inputs.skew2, 100000, 7, 0.05, 2),
    (inputs.gauss_mix, 1 << 18, 128, 0.01, 4), (inputs.nested_clusters, 70000, 5, 0.05, 5),
    (inputs.uniform, 1000, 999, 0.05, 2), (inputs.uniform, 1 << 15, 1, 0.05, 1), (inputs.uniform, 7, 7, 0.05, 1)])
def test_omp_hss_equals_oracle(gen, N, p, eps, seed):
    keys = gen(N, seed)
    sk, ss, sp, off, out, rounds, z, rc = oracle.hss_omp(keys, p, eps, seed)
    ref = oracle.hss(keys, p, eps, seed)
    assert rc == ref.status and rounds == ref.rounds
    assert list(z) == [int(x) for x in ref.sample_size]
    assert np.array_equal(off, ref.offsets)
    assert np.array_equal(sk, ref.splitter_key) and np.array_equal(ss, ref.splitter_seg)
    assert np.array_equal(sp, ref.splitter_spos)
    assert np.array_equal(out, ref.out_keys)


def test_omp_uses_threads_and_std_sort_sorts():
    assert oracle.baseline_threads() >= 1
    keys = inputs.zipf(100000, 9)
    assert np.array_equal(oracle.std_sort(keys), np.sort(keys))
