"""Host-side check of the warp-cooperative production-rate kernel's gather
tables (no GPU): the emitted entry list, chunk and slot tables are read back
from the kernel source and the kernel's gather and combine steps are replayed
lane by lane in Python on random rates of progress; the result must be
wdot_k = sum_i nu_ki q_i for every species (up to float64 rounding of the
replay), every slot index must stay inside the per-state species region, and
every lane's chunk must be no longer than the table's chunk length."""
import re

import numpy as np
import pytest

from paper_2411_02640_gb300 import kx, synth
from tests import toys


def _array(src, name):
    m = re.search(r"__device__ const (?:int2|int) %s\[(\d+)\] = \{(.*?)\};" % name, src, re.S)
    assert m, name
    vals = [int(v) for v in re.findall(r"-?\d+", m.group(2))]
    return vals


def _nu(mech):
    ns, nr = mech.n_species, len(mech.reactions)
    nu = np.zeros((ns, nr))
    for i, r in enumerate(mech.reactions):
        for k, c in r.reactants:
            nu[k, i] -= c
        for k, c in r.products:
            nu[k, i] += c
    return nu


def _replay(src, ns, nr, q):
    G = int(re.search(r"const int gs = lane & (\d+);", src).group(1)) + 1
    svs = int(re.search(r"\[G\]\[(\d+)\]: \{ln \|C_k\|, mu_k\}", src).group(1))
    tab = np.array(_array(src, "kx_wtab")[:-1], dtype=np.int64) & 0xffffffff
    chs = _array(src, "kx_wchs")[:-1]
    ws = np.array(_array(src, "kx_wslot")).reshape(-1, 2)[:ns]
    nch = 32 // G
    assert len(chs) == nch and tab.size % nch == 0
    cl = tab.size // nch
    slots = {}
    for ch in range(nch):
        sl, acc = chs[ch], 0.0
        for j in range(cl):
            w = int(tab[j * nch + ch])
            r = w & 0x7fff
            coef = np.frombuffer(np.uint32(w & 0xffff0000).tobytes(), np.float32)[0]
            assert r < nr
            acc += float(coef) * q[r]
            if w & 0x8000:
                assert sl < 2 * svs, "slot outside the species region"
                slots[sl] = acc
                sl, acc = sl + 1, 0.0
        if ch + 1 < nch:
            assert sl == chs[ch + 1]
    out = np.zeros(ns)
    for k in range(ns):
        first, count = ws[k]
        out[k] = sum(slots[first + j] for j in range(count))
    return out


def _check(mech_obj, path, tmp_cache):
    m = kx.Mechanism(path, cache_dir=tmp_cache, compile_only=1, lazy=1)
    src = m.kernel_source("wdot_fp64_wc")
    assert "kx_wtab" in src
    ns, nr = mech_obj.n_species, len(mech_obj.reactions)
    rng = np.random.default_rng(3)
    q = rng.standard_normal(nr) * np.exp(rng.uniform(-20, 20, nr))
    want = _nu(mech_obj) @ q
    got = _replay(src, ns, nr, q)
    scale = np.abs(_nu(mech_obj)) @ np.abs(q)
    assert np.all(np.abs(got - want) <= 1e-13 * np.maximum(scale, 1e-300))


@pytest.mark.parametrize("name", ["h2o2_9_21", "gri_53_325", "large_160_900"])
def test_gather_tables_replay(name, tmp_path):
    _check(synth.mechanism(name), synth.mechanism_file(name, str(tmp_path)), str(tmp_path / "cache"))


def test_gather_tables_replay_every_reaction_kind(tmp_path):
    from tests.test_gpu_reaction_kinds import reactions
    mech, path = toys.toy("kinds", reactions(), str(tmp_path))
    _check(mech, path, str(tmp_path / "cache"))


@pytest.mark.parametrize("group", [1, 2, 4, 8, 16, 32])
def test_gather_tables_every_group_size(group, tmp_path):
    name = "h2o2_9_21"
    mech = synth.mechanism(name)
    path = synth.mechanism_file(name, str(tmp_path))
    m = kx.Mechanism(path, cache_dir=str(tmp_path / "cache"), compile_only=1, lazy=1, rates_group=group)
    src = m.kernel_source("wdot_fp64_wc")
    assert f"const int gs = lane & {group - 1};" in src
    rng = np.random.default_rng(group)
    q = rng.standard_normal(len(mech.reactions))
    got = _replay(src, mech.n_species, len(mech.reactions), q)
    np.testing.assert_allclose(got, _nu(mech) @ q, rtol=1e-12, atol=1e-12)


def _vjp_replay(src, mech_obj, af, ar, gx, ic):
    m = re.search(r"kx_vtab\[(\d+)\] = \{(.*?)\};", src, re.S)
    num = r"\(?([-+0-9.eE]+)f?\)?"
    entries = re.findall(r"\{(-?\d+),%s,%s,0\}" % (num, num), m.group(2))
    tab = [(int(w) & 0xffffffff, float(np.float32(c)) + float(np.float32(cl))) for w, c, cl in entries][:-1]
    svs = max(mech_obj.n_species + 1, (mech_obj.n_species + 33) // 2)
    chs = _array(src, "kx_vchs")[:-1]
    ws = np.array(_array(src, "kx_vslot")).reshape(-1, 2)[:mech_obj.n_species]
    tbr = [int(x) for x in re.search(r"// third-body slot -> reaction: \{([0-9,]*)\}", src).group(1).split(",") if x]
    assert sorted(tbr) == [i for i, r in enumerate(mech_obj.reactions) if r.uses_third_body()]
    nch = len(chs)
    cl = len(tab) // nch
    slots = {}
    for ch in range(nch):
        sl, acc = chs[ch], 0.0
        for j in range(cl):
            w, cf = tab[j * nch + ch]
            if cf != 0.0:
                r, kind, k = w & 0x3FFF, (w >> 14) & 3, (w >> 16) & 0x7FFF
                acc += cf * (gx[tbr[r]] if kind == 2 else (af[r] if kind == 0 else ar[r]) * ic[k])
            if w & 0x80000000:
                assert sl < 2 * svs, "slot outside the species vectors"
                slots[sl] = acc
                sl, acc = sl + 1, 0.0
    return np.array([sum(slots[f + j] for j in range(c)) for f, c in ws])


@pytest.mark.parametrize("name", ["h2o2_9_21", "gri_53_325"])
def test_vjp_gather_tables_replay(name, tmp_path):
    """The warp-cooperative adjoint's species-major entry list: replayed on
    random per-reaction terms, d/dC_k = sum_i (nu'_ki a c R_f,i + nu''_ki
    (-a c R_r,i)) / C_k + sum_i (eff_ki - eff_default,i) a (R_f - R_r)_i."""
    mech_obj = synth.mechanism(name)
    path = synth.mechanism_file(name, str(tmp_path))
    m = kx.Mechanism(path, cache_dir=str(tmp_path / "cache"), compile_only=1, lazy=1, vjp_layout=2)
    src = m.kernel_source("vjp")
    ns, nr = mech_obj.n_species, len(mech_obj.reactions)
    rng = np.random.default_rng(5)
    af, ar, gx, ic = rng.standard_normal(nr), rng.standard_normal(nr), rng.standard_normal(nr), rng.standard_normal(ns)
    want = np.zeros(ns)
    for i, r in enumerate(mech_obj.reactions):
        for k, c in r.reactants:
            want[k] += c * af[i] * ic[k]
        if r.reversible:
            for k, c in r.products:
                want[k] += c * ar[i] * ic[k]
        if r.uses_third_body():
            if r.collider is not None:
                want[r.collider] += gx[i]
            else:
                for k, e in r.efficiencies.items():
                    if e != r.default_eff:
                        want[k] += (e - r.default_eff) * gx[i]
    got = _vjp_replay(src, mech_obj, af, ar, gx, ic)
    # coefficients as float pairs: efficiency differences (0.7 - 1 and the like) to about 2^-48
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12)
