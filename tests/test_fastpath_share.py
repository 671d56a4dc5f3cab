"""The share of reaction-warps that the float-pair rate kernel's float32 path
takes on the benchmark's states, reproduced on the host: the oracle's gross
rates of each reaction, visited in the emitted kernel's class order, with
the kernel's running per-state scale (set by the first rate at 2^62, raised
when a rate lands above 2^96) and its rule (every state of a warp of 32
below 2^-40 of the scale's anchor).  On the 53/325 workload the path takes
about 90 % of the elementary, three-body and falloff reaction-warps."""
import re

import numpy as np

from paper_2411_02640_gb300 import kx, synth
from tests.gpu_common import oracle


def _order(src):
    """Reaction indices in the order of the emitted class loops."""
    heads = [tuple(map(int, t)) for t in re.findall(r"// class \d+: (\d+) reactions, (\d+) reactant and (\d+) product entries", src)]
    ncls = len(set(re.findall(r"kx_s(\d+)\[", src)))
    order = []
    for ci, (nrx, nre, npr) in enumerate(heads[:ncls]):
        vals = [int(v) for v in re.search(r"int kx_s%d\[\d+\] = \{(.*?)\};" % ci, src, re.S).group(1).split(",") if v.strip()]
        E = nre + npr
        P = (E + 1 + 3) // 4 * 4
        order += [vals[P * r + E] for r in range(nrx)]
    return order


def test_float32_share_on_the_benchmark_states(tmp_path):
    name = "gri_53_325"
    path = synth.mechanism_file(name, str(tmp_path))
    src = kx.Mechanism(path, cache_dir=str(tmp_path / "cache"), compile_only=1, lazy=1, rates_layout=1).kernel_source("wdot_fp64")
    order = _order(src)
    m = synth.mechanism(name)
    assert sorted(order) == list(range(len(m.reactions)))
    n = 32 * 64
    T, p, Y = synth.make_states(m.n_species, synth.STATE_SPECS[name], 0, n)
    g = oracle(name).reaction_gross(T, p, Y)
    with np.errstate(divide="ignore"):
        ex = np.floor(np.log2(np.where(g > 0, g, 2.0 ** -3000)))
    small = np.zeros((len(order), n), bool)
    for s in range(n):
        S = None
        for j, r in enumerate(order):
            if S is not None and ex[r, s] < S + 22:
                small[j, s] = True
            if S is None or ex[r, s] > S + 96:
                S = ex[r, s] - 62
    eligible = np.array([m.reactions[r].kind in ("elementary", "three_body", "falloff", "chem_act") for r in order])
    share = small.reshape(len(order), -1, 32).all(axis=2)[eligible].mean()
    print(f"\nfloat32 path: {share:.3f} of the eligible reaction-warps")
    assert 0.8 <= share <= 0.97
