"""The learned self-distance surrogate end to end: exact labels against the oracle, the
evaluation / fallback bookkeeping on the CPU, and on the GPU a short training run whose
network, with the exact fallback below the margin, answers faster than the exact path
alone without missing a near-collision configuration of the held-out set."""
import os

import numpy as np
import pytest

from paper_2407_02363_b300 import synth


def test_evaluate_fallback_and_missed_bookkeeping():
    from paper_2407_02363_b300.surrogate import evaluate
    exact = np.array([[0.20, 0.30], [0.04, 0.30], [0.06, 0.30], [0.30, 0.01]])
    pred = np.array([[0.21, 0.30], [0.07, 0.30], [0.045, 0.30], [0.30, 0.50]])
    valid = np.array([[True, True], [True, True], [True, True], [True, False]])
    r = evaluate(pred, exact, valid, margin=0.05)
    # row 1: exact 4 cm but predicted 7 cm -> missed; row 2 falls back; row 3's near
    # entry is masked so it is neither near nor a fallback
    assert r.fallback_rate == 0.25 and r.missed_rate == 0.25
    assert np.isclose(r.max_err_mm, 30.0)


def test_sphere_margins_are_safe_on_their_calibration_set_and_fall_back_less():
    """Per-sphere margins (5 cm + each sphere's largest validation error) never miss a
    near configuration of the set they were calibrated on, equal the single margin for the
    worst sphere, and send fewer configurations to the exact path when the other spheres
    are more accurate.  A margin set from the wrong sphere's errors does miss."""
    from paper_2407_02363_b300.surrogate import evaluate, sphere_margins
    rng = np.random.default_rng(7)
    n, m = 20000, 6
    exact = rng.uniform(0.0, 0.35, size=(n, m))
    scale = np.array([0.002, 0.004, 0.008, 0.016, 0.03, 0.06])      # sphere 5 is the worst
    pred = exact + rng.normal(0.0, 1.0, size=(n, m)) * scale
    valid = rng.random((n, m)) > 0.1
    margins = sphere_margins(pred, exact, valid)
    one = 0.05 + np.abs(pred - exact)[valid].max()
    assert np.isclose(margins.max(), one) and int(np.argmax(margins)) == 5
    err = np.where(valid, np.abs(pred - exact), 0.0).max(axis=0)
    assert np.allclose(margins, 0.05 + err)
    r_sph, r_one = evaluate(pred, exact, valid, margins), evaluate(pred, exact, valid, one)
    assert r_sph.missed_rate == 0.0 and r_one.missed_rate == 0.0
    assert r_sph.fallback_rate < r_one.fallback_rate
    assert np.isclose(r_sph.margin_m, one)
    # the worst sphere's margin taken from the best sphere's errors: its near entries slip
    wrong = margins.copy()
    wrong[5] = margins[0]
    assert evaluate(pred, exact, valid, wrong).missed_rate > 0.0
    # a sphere with no valid entry keeps the base margin
    v2 = valid.copy()
    v2[:, 2] = False
    assert np.isclose(sphere_margins(pred, exact, v2)[2], 0.05)


def _setup():
    chain = synth.make_chain(1234 + 4000, (1.28, 1.28, 1.28))
    spheres = synth.sphere_model(chain)
    return chain, spheres


@pytest.mark.gpu
def test_exact_labels_match_oracle():
    import oracle
    from paper_2407_02363_b300.surrogate import ExactSelfDistance
    chain, spheres = _setup()
    lab = ExactSelfDistance(chain, spheres, n_maps=8)
    q = synth.joint_states(1234 + 4000, 19)
    dist, stat = lab(q)
    links = synth.link_models(chain, 0.02)
    for i in range(len(q)):
        s = np.zeros((128, 128, 128), np.uint8)
        oracle.insert_links(s, (128, 128, 128), 0.02, (0, 0, 0), links, oracle.fk(chain, q[i]).astype(np.float32),
                            0b111)
        sq, ix = oracle.edt(s)
        r = oracle.query_spheres(sq, ix, (128, 128, 128), 0.02, (0, 0, 0), oracle.sphere_centres(chain, spheres, q[i]),
                                 spheres.radius)
        assert np.array_equal(stat[i], r["status"])
        assert np.array_equal(dist[i].view(np.uint32), r["dist"].view(np.uint32))
    lab.close()


@pytest.mark.gpu
def test_label_cache_reads_back_the_same_labels(tmp_path):
    from paper_2407_02363_b300.surrogate import ExactSelfDistance, cached_labels
    chain, spheres = _setup()
    lab = ExactSelfDistance(chain, spheres, n_maps=8)
    q = synth.joint_states(77, 12)
    path = str(tmp_path / "labels.npz")
    d1, s1 = cached_labels(lab, q, path)
    stamp = os.path.getmtime(path)
    d2, s2 = cached_labels(lab, q, path)
    assert os.path.getmtime(path) == stamp          # read back, not rewritten
    assert np.array_equal(d1, d2) and np.array_equal(s1, s2)
    d0, s0 = lab(q)
    assert np.array_equal(d0, d1) and np.array_equal(s0, s1)
    q2 = q.copy()
    q2[0, 0] += 0.1                                                 # other joint states: recomputed
    d3, _ = cached_labels(lab, q2, path)
    assert np.array_equal(d3, lab(q2)[0])
    lab.close()


@pytest.mark.gpu
def test_surrogate_trains_and_hybrid_beats_exact_safely():
    import torch

    from oracle import mlp as omlp
    from paper_2407_02363_b300 import surrogate as sg
    from paper_2407_02363_b300 import vedt as v
    chain, spheres = _setup()
    lab = sg.ExactSelfDistance(chain, spheres, n_maps=512)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
    net = v.MLP(65536)
    net.set_params(omlp.init_params(0).astype(np.float32))
    hist, r_va, margin, _, margins = sg.fit(lab, net, n_train=262144, n_val=8192, seed=1, steps=12000,
                                            log_every=4000)
    assert margins.shape == (24,) and np.all(margins <= margin + 1e-7) and np.all(margins >= 0.05)
    assert hist[-1][1] < 0.2 * hist[0][1], hist
    q_te = synth.joint_states(3, 8192)
    d_te, s_te = lab(q_te)
    p_te = sg.clip(sg.predict(net, dev(q_te)).cpu().numpy())
    r_te = sg.evaluate(p_te, sg.clip(d_te), lab.valid_mask(s_te), margin=margin)
    assert r_te.p99_err_mm < 45.0, r_te
    assert r_te.missed_rate == 0.0, r_te
    r_sph = sg.evaluate(p_te, sg.clip(d_te), lab.valid_mask(s_te), margin=margins)
    assert r_sph.missed_rate == 0.0 and r_sph.fallback_rate <= r_te.fallback_rate, (r_sph, r_te)
    # throughput: exact labels vs surrogate + exact fallback on the flagged fraction
    qd = dev(synth.joint_states(4, 65536))
    out = torch.empty((65536, 24), device="cuda")
    sur_qps = sg.throughput(lambda: net.forward(qd, out), 65536, reps=5)
    exact_qps = sg.throughput(lambda: lab(q_te[:1024]), 1024, reps=2, warmup=1)
    hybrid_qps = 1.0 / (1.0 / sur_qps + r_te.fallback_rate / exact_qps)
    assert sur_qps > 50 * exact_qps
    assert r_te.fallback_rate < 0.9 and hybrid_qps > 1.1 * exact_qps, (r_te, sur_qps, exact_qps, hybrid_qps)
    net.close()
    lab.close()
