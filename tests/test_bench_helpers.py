"""Host-side helpers of the benchmark: D and L from an LCP array (checked
against the oracle's Lemma 2.1 routine), and the sources a recorded traffic
figure is keyed to."""
import os
import sys

import numpy as np

import gen
import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_d_and_l_matches_oracle():
    import bench
    for s in (gen.url_set(3000, 5), gen.random_set(2000, 6, 0, 6, ord("a"), ord("c")), gen.dna_suffix_set(3000, 7)):
        _, lcp = oracle.sort(s.chars, s.offsets, s.max_len)
        assert bench.d_and_l(lcp) == tuple(int(x) for x in oracle.dl(lcp))
    assert bench.d_and_l(np.zeros(0, np.uint32)) == (0, 0)


def test_kernel_sources():
    import bench
    names = {os.path.basename(f) for f in bench.kernel_sources("big_scatter")}
    assert {"ss_big.cu", "ss_step.cuh", "ss_internal.cuh", "ss_kernels.h"} <= names
    assert "ss_host.cu" not in names  # host code does not change the kernel
    merge = {os.path.basename(f) for f in bench.kernel_sources("merge_round")}
    assert "ss_merge.cu" in merge and "ss_big.cu" not in merge
    every = {os.path.basename(f) for f in bench.kernel_sources(None)}
    assert {"ss_host.cu", "ss_big.cu", "ss_merge.cu"} <= every
    assert bench.source_hash("big_scatter") != bench.source_hash("merge_round")
