"""The FP64 C++/OpenMP CPU evaluation (oracle/cpu_eval.cpp), the benchmark's timed CPU baseline,
pinned element by element to the numpy oracle (oracle/qg_oracle.py), which the other oracle tests
pin to the paper.  The two share no code: different layout, loop order and adjoint arrangement (the
C++ side sums a period's adjoint solves before applying the reduced-Laplacian inverse, by the rank-1
identity of Eq. rank_correct)."""
import dataclasses

import numpy as np
import pytest

import oracle
import synth
from oracle import cpu_eval


def point(c, seed):
    return np.clip(synth.random_point(c, seed), *oracle.box(c))


def check(c, x, tol_el=1e-9):
    ref = oracle.evaluate(c, x)
    ev = cpu_eval.CpuOracle(c)
    obj, g, terms = ev.evaluate(x)
    ev.close()
    assert obj == pytest.approx(ref.obj, rel=1e-12)
    assert np.allclose(terms, list(ref.terms.values()), rtol=1e-12, atol=1e-12 * abs(ref.obj))
    floor = 1e-9 * np.max(np.abs(ref.grad))
    err = np.abs(g - ref.grad) / (np.abs(ref.grad) + floor)
    assert err.max() <= tol_el, (int(err.argmax()), float(err.max()))


@pytest.mark.parametrize("name,seed", [("tiny", 1), ("tiny", 2), ("mid", 3)])
def test_matches_the_numpy_oracle_at_random_points(name, seed):
    c = getattr(synth, name)()
    check(c, point(c, seed))


def test_matches_the_numpy_oracle_on_rt617_at_its_start():
    c = synth.rt617()
    check(c, synth.lp_start(c)[0])


def test_matches_with_other_eps_and_beta_and_a_single_period():
    c = dataclasses.replace(synth.mid(), eps=3e-2, beta=0.37)
    check(c, point(c, 5))
    t = synth.tiny()
    one = dataclasses.replace(t, T=1, dt=t.dt[:1], load_p=t.load_p[:1], load_q=t.load_q[:1],
                              reserve_req=t.reserve_req[:1])
    check(one, point(one, 6))


def test_without_outages():
    c = synth.tiny()
    c = dataclasses.replace(c, ctg=np.zeros(0, np.int32))
    check(c, point(c, 7))


def test_thread_count_does_not_change_the_bits():
    c = synth.mid()
    x = point(c, 8)
    ev = cpu_eval.CpuOracle(c)
    o1, g1, _ = ev.evaluate(x, threads=1)
    o4, g4, _ = ev.evaluate(x, threads=4)
    ev.close()
    assert o1 == o4 and np.array_equal(g1, g4)


def test_refuses_cases_outside_its_scope():
    c = synth.tiny()
    for other in (synth.with_transformers(c, 0.3, 4), synth.with_block_bids(c, 3, 0.3, 1), synth.with_commitment(c, 1)):
        with pytest.raises(ValueError):
            cpu_eval.CpuOracle(other)


# mistakes planted in a copy of the C++ source: the thermal term rated at s_ctg instead of s_max, the
# ramp limit without its d_t, the angle adjoint's sign at the to bus, the slack mean left out
PLANTS = [("const double u = (fr ? sf : st) - h.smax[m];", "const double u = (fr ? sf : st) - h.sctg[m];"),
          ("const double lim = h.ramp[k] * h.dt[t];", "const double lim = h.ramp[k];"),
          ("gtht[bb] -= gd;", "gtht[bb] += gd;"),
          ("gp[(size_t)t * G + k] += eta[h.gbus[k]] - mean;", "gp[(size_t)t * G + k] += eta[h.gbus[k]];")]


@pytest.mark.parametrize("old,new", PLANTS)
def test_a_planted_mistake_is_caught(tmp_path, old, new):
    import subprocess
    src = open(cpu_eval.SRC).read()
    assert src.count(old) == 1
    path = tmp_path / "planted.cpp"
    path.write_text(src.replace(old, new))
    lib = str(tmp_path / "libplanted.so")
    subprocess.run(["g++", "-O1", "-std=c++17", "-fopenmp", "-fPIC", "-shared", str(path), "-o", lib], check=True)
    c = synth.mid()
    # thermal overloads present, and period lengths other than one hour (the ramp limit scales by d_t)
    c = dataclasses.replace(c, s_max=0.6 * c.s_max, dt=0.5 + 0.25 * (np.arange(c.T) % 3))
    x = point(c, 9)
    x[:c.T * c.n_bus] = np.clip(x[:c.T * c.n_bus], 0.9, 1.1)
    ref = oracle.evaluate(c, x)
    ev = cpu_eval.CpuOracle(c, lib)
    obj, g, _ = ev.evaluate(x)
    ev.close()
    floor = 1e-9 * np.max(np.abs(ref.grad))
    err = np.max(np.abs(g - ref.grad) / (np.abs(ref.grad) + floor))
    assert abs(obj - ref.obj) > 1e-9 * abs(ref.obj) or err > 1e-6
