"""Population control at interior census times on the GPU (mc_run with census_times, through the
C ABI) against the CPU oracle and closed forms:

- FP64 replay: the event sequence of the logged histories (their copies included) and every counter
  equal the oracle's across all intervals;
- FP32: AZURV1 (c = 1.1) keeps the closed-form flux e^{0.1 t} while each census banks N e^{0.2}
  particles and splitting-roulette restores N; the 7-group pulse with census times matches the
  matrix exponential;
- event- and history-based runs give identical fixed-point tallies and counters;
- combing (pc_method "comb"): the same FP64 replay and closed forms, exactly N_b particles per batch
  restored at every census.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import closed_forms as CF
from paper_2305_07636_gb300 import mc
from paper_2305_07636_gb300 import problems as P

pytestmark = pytest.mark.gpu

THREADS = 16


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    if not _t.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    return _t


def exact_z(mg, sg, exact, rel_max=0.1):
    mg, sg, exact = (np.asarray(a, dtype=np.float64).ravel() for a in (mg, sg, exact))
    ok = (sg > 0) & (sg < rel_max * np.abs(mg))
    return (mg[ok] - exact[ok]) / sg[ok]


def balanced(c):
    started = c["source"] + c["secondary"] + c["ww_split"] + c["pc_copies"]
    ended = c["capture"] + c["production"] + c["leak"] + c["census"] + c["lost"] + c["ww_kill"] + c["pc_banked"]
    return started == ended


def test_pc_fp64_replays_the_oracle(torch):
    prob = P.azurv1(t_end=6.0, n_tbins=6)
    n, nlog, ct = 4000, 100, [2.0, 4.0]
    o = oracle.run_pc(prob, n, ct, 8, seed=91, threads=THREADS, log_first=0, log_count=nlog,
                      log_cap=4000 * nlog)
    p = mc.Problem(prob)
    p.run(n, 91, precision="fp64", n_batches=8, census_times=ct, log_first=0, log_count=nlog,
          log_capacity=4000 * nlog, bank_capacity=1 << 16)
    ev, eo = p.events(4000 * nlog), o.events
    assert len(ev) == len(eo) and len(ev) > nlog
    assert np.array_equal(ev["tag"], eo["tag"]) and np.array_equal(ev["k"], eo["k"])
    for f in ("kind", "outcome", "n_child", "cell", "g", "root"):
        assert np.array_equal(ev[f], eo[f]), f
    for f in ("x", "y", "z", "ux", "uy", "uz", "t", "w"):
        scale = np.maximum(np.maximum(np.abs(ev[f]), np.abs(eo[f])), 1.0)
        assert np.max(np.abs(ev[f] - eo[f]) / scale) <= 1e-9, f
    c = p.counters()
    for name in oracle.COUNTER_NAMES:
        assert c[name] == o.counters[name], name
    assert balanced(c) and c["pc_copies"] > 0
    p.close()


def test_pc_azurv1_fp32_closed_forms(torch):
    prob = P.azurv1()
    ct = np.arange(2.0, 20.0, 2.0)
    n = 4_096_000  # N e^{0.2} above 2^22 particles at every census: the default bank sizing
    p = mc.Problem(prob)
    p.run(n, 92, n_batches=256, census_times=ct)
    m, s = p.tally(0)
    z = exact_z(m, s, CF.infinite_time_bins(1.0, 0.6, 0.5, 1.0, prob["tallies"][0]["t"]))
    assert z.size >= 18 and np.all(np.abs(z) < 4), z
    c = p.counters()
    assert balanced(c)
    # every census banks about N e^{0.1 dt}; splitting-roulette restores about N
    assert abs(c["pc_banked"] / len(ct) / n / math.exp(0.2) - 1) < 0.01
    assert abs(c["pc_copies"] / len(ct) / n - 1) < 0.01
    p.close()


def test_pc_multigroup_pulse_fp32_expm(torch):
    prob = P.config2()
    mat, v, te = prob["materials"][0], prob["speed"], prob["tallies"][0]["t"]
    p = mc.Problem(prob)
    p.run(2_048_000, 93, n_batches=256, census_times=[1e-8, 1e-7, 1e-6, 1e-5, 1e-4])
    m, s = p.tally(0)
    z = exact_z(m.reshape(7, -1), s.reshape(7, -1), CF.multigroup_time_bins(mat, v, te))
    assert z.size >= 300 and np.all(np.abs(z) < 4), np.abs(z).max()
    assert balanced(p.counters())
    p.close()


def test_pc_identical_across_algorithms(torch):
    prob = P.azurv1(t_end=10.0, n_tbins=10)
    p = mc.Problem(prob)
    ref = None
    for alg in ("event", "history"):
        p.run(200_000, 94, census_times=[2.5, 5.0, 7.5], algorithm=alg)
        got = (p.tally_batches(0), {k: v for k, v in p.counters().items() if k != "iterations"})
        if ref is None:
            ref = got
        else:
            assert np.array_equal(got[0], ref[0]) and got[1] == ref[1]
    with pytest.raises(mc.McError) as e:
        p.run(1000, 1, census_times=[5.0, 2.0])
    assert e.value.code == mc.MC_ERR_INVALID
    p.close()


def test_comb_fp64_replays_the_oracle(torch):
    prob = P.azurv1(t_end=6.0, n_tbins=6)
    n, nlog, ct = 4000, 100, [2.0, 4.0]
    o = oracle.run_pc(prob, n, ct, 8, seed=95, threads=THREADS, log_first=0, log_count=nlog,
                      log_cap=4000 * nlog, method="comb")
    p = mc.Problem(prob)
    p.run(n, 95, precision="fp64", n_batches=8, census_times=ct, pc_method="comb", log_first=0,
          log_count=nlog, log_capacity=4000 * nlog, bank_capacity=1 << 16)
    ev, eo = p.events(4000 * nlog), o.events
    assert len(ev) == len(eo) and len(ev) > nlog
    for f in ("tag", "k", "kind", "outcome", "n_child", "cell", "g", "root"):
        assert np.array_equal(ev[f], eo[f]), f
    for f in ("x", "y", "z", "ux", "uy", "uz", "t", "w"):
        scale = np.maximum(np.maximum(np.abs(ev[f]), np.abs(eo[f])), 1.0)
        assert np.max(np.abs(ev[f] - eo[f]) / scale) <= 1e-9, f
    c = p.counters()
    for name in oracle.COUNTER_NAMES:
        assert c[name] == o.counters[name], name
    assert balanced(c) and c["pc_copies"] == len(ct) * n
    p.close()


def test_comb_azurv1_fp32_closed_forms(torch):
    prob = P.azurv1()
    ct = np.arange(2.0, 20.0, 2.0)
    n = 1_024_000
    p = mc.Problem(prob)
    p.run(n, 96, n_batches=256, census_times=ct, pc_method="comb")
    m, s = p.tally(0)
    z = exact_z(m, s, CF.infinite_time_bins(1.0, 0.6, 0.5, 1.0, prob["tallies"][0]["t"]))
    assert z.size >= 18 and np.all(np.abs(z) < 4), z
    c = p.counters()
    assert balanced(c) and c["pc_copies"] == len(ct) * n  # exactly N_b per batch at every census
    assert abs(c["pc_banked"] / len(ct) / n / math.exp(0.2) - 1) < 0.01
    p.close()


def test_comb_identical_across_algorithms_and_rejects_bad_method(torch):
    prob = P.azurv1(t_end=10.0, n_tbins=10)
    p = mc.Problem(prob)
    ref = None
    for alg in ("event", "history"):
        p.run(200_000, 97, census_times=[2.5, 5.0, 7.5], pc_method="comb", algorithm=alg)
        got = (p.tally_batches(0), {k: v for k, v in p.counters().items() if k != "iterations"})
        if ref is None:
            ref = got
        else:
            assert np.array_equal(got[0], ref[0]) and got[1] == ref[1]
    with pytest.raises(mc.McError) as e:
        p.run(1000, 1, census_times=[5.0], pc_method=2)
    assert e.value.code == mc.MC_ERR_INVALID
    p.close()
