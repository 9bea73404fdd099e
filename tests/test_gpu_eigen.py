"""k-eigenvalue power iteration on the GPU (mc_run_eigen, through the C ABI) against the CPU oracle
and the closed forms:

- FP64 replay: every cycle's fission-site count, the event sequence of the logged histories of every
  cycle and k of every cycle equal the oracle's (k to rounding: the track-length sums are exact
  integers of per-flight values that agree to the last bits).
- FP32 statistics: k and the tallies over the active cycles agree with the oracle within 4 sigma;
  the infinite-medium k and spectrum agree with the eigenpair of A^-1 F.
- Determinism: repeated runs, event- and history-based algorithms give identical k and tallies.
"""
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


def test_eigen_fp64_replays_the_oracle(torch):
    prob = P.pin_cell()
    n, ni, na, nlog = 3000, 3, 3, 200
    o = oracle.run_eigen(prob, n, ni, na, seed=81, threads=THREADS, log_first=0, log_count=nlog,
                         log_cap=2000 * nlog * (ni + na))
    p = mc.Problem(prob)
    k, sites, km, ke = p.run_eigen(n, ni, na, seed=81, precision="fp64", log_first=0, log_count=nlog,
                                   log_capacity=2000 * nlog * (ni + na))
    assert np.array_equal(sites, o.sites_cycle)
    assert np.allclose(k, o.k_cycle, rtol=1e-12, atol=0.0)
    ev, eo = p.events(2000 * nlog * (ni + na)), o.events
    assert len(ev) == len(eo) and len(ev) > nlog * (ni + na)
    assert np.array_equal(ev["tag"], eo["tag"]) and np.array_equal(ev["k"], eo["k"])
    for f in ("kind", "outcome", "n_child", "cell", "elem", "in_pin", "g"):
        assert np.array_equal(ev[f], eo[f]), f
    for f in ("x", "y", "z", "ux", "uy", "uz", "t", "w"):
        scale = np.maximum(np.maximum(np.abs(ev[f]), np.abs(eo[f])), 1.0)
        assert np.max(np.abs(ev[f] - eo[f]) / scale) <= 1e-9, f
    c = p.counters()
    for name in oracle.COUNTER_NAMES:
        assert c[name] == o.counters[name], name
    p.close()


def test_eigen_fp32_pin_cell_against_oracle(torch):
    prob = P.pin_cell()
    o = oracle.run_eigen(prob, 20000, 10, 40, seed=82, threads=THREADS)
    p = mc.Problem(prob)
    k, sites, km, ke = p.run_eigen(100_000, 10, 40, seed=83)
    assert abs(km - o.k_mean) < 4 * np.hypot(ke, o.k_std), (km, ke, o.k_mean, o.k_std)
    mg, sg = p.tally(0)
    mo, so = o.tallies[0]
    ok = (sg > 0) & (so > 0) & (sg < 0.1 * np.abs(mg)) & (so < 0.1 * np.abs(mo))
    z = (mg[ok] - mo[ok]) / np.sqrt(sg[ok] ** 2 + so[ok] ** 2)
    assert ok.sum() > 100 and np.all(np.abs(z) < 4), np.abs(z).max()
    assert np.all(np.abs(sites / (1e5 * k / np.concatenate([[1.0], k[:-1]])) - 1) < 0.02)
    p.close()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_eigen_infinite_media_closed_forms(torch, precision):
    p = mc.Problem(P.eigen_infinite_1g())
    k, sites, km, ke = p.run_eigen(200_000, 5, 30, seed=84, precision=precision)
    assert abs(km - 0.96) < 4 * ke
    m, s = p.tally(0)
    assert abs(m.ravel()[0] - 2.0) < 4 * s.ravel()[0]  # track length per history = 1 / Sigma_a
    p.close()
    prob = P.eigen_infinite_mg()
    k_exact, phi = CF.infinite_k(prob["materials"][0])
    p = mc.Problem(prob)
    k, sites, km, ke = p.run_eigen(200_000, 10, 30, seed=85, precision=precision)
    assert abs(km - k_exact) < 4 * ke, (km, ke, k_exact)
    b = p.tally_batches(0).reshape(30, 7)  # each active cycle's group flux
    spec = b / b.sum(axis=1, keepdims=True)
    z = (spec.mean(0) - phi) / (spec.std(0, ddof=1) / np.sqrt(30))
    assert np.all(np.abs(z) < 4), z
    p.close()


def test_eigen_runs_are_deterministic(torch):
    p = mc.Problem(P.pin_cell())
    ref = p.run_eigen(50_000, 3, 4, seed=86)
    tb = p.tally_batches(0)
    for alg in ("event", "history"):
        got = p.run_eigen(50_000, 3, 4, seed=86, algorithm=alg)
        assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1]), alg
        assert np.array_equal(p.tally_batches(0), tb), alg
    p.close()


def test_eigen_rejects_what_it_cannot_run(torch):
    p = mc.Problem(P.config2())  # time census, no production
    with pytest.raises(mc.McError) as e:
        p.run_eigen(1000, 1, 2, seed=1)
    assert e.value.code == mc.MC_ERR_INVALID
    p.close()
    p = mc.Problem(P.pin_cell())
    for kw in ({"implicit_capture": 1}, {"first_history": 5}):
        with pytest.raises(mc.McError) as e:
            p.run_eigen(1000, 1, 2, seed=1, **kw)
        assert e.value.code == mc.MC_ERR_INVALID
    with pytest.raises(mc.McError):
        p.run_eigen(1000, 1, 1, seed=1)  # one active cycle gives no error estimate
    p.close()
