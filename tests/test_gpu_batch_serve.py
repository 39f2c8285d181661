"""Graph replay, launch-shape tuning, multi-system batching and the serving
loop. Each is checked for the one property it must not break: a walker
step's results. Graph replay and batching run the same kernels with the same
Philox counters, so they must reproduce plain launches bit for bit; tuned
launch shapes change only FP32 summation order, so every shape must still
meet the reduced-precision tolerance against the FP64 oracle; a served run
must give the same results alone and in a mix."""
import numpy as np
import pytest

from gpu_helpers import compare_energy, compare_state
from oracle import afqmc as O
from synth import config_c1, small_system

pytestmark = pytest.mark.gpu

RTOL_REDUCED = 1e-4


@pytest.fixture(scope="session", autouse=True)
def built():
    from paper_1804_03310_gb300 import build
    build.build()


def ctx(system, **kw):
    from paper_1804_03310_gb300 import Afqmc
    return Afqmc.from_system(system, **kw)


def snapshot(c):
    w, lo = c.afqmc_weights()
    return dict(state=c.afqmc_get_state(), w=w, lo=lo, hist=c.afqmc_energy_history(),
                launches=c.afqmc_launch_count())


def assert_identical(a, b, label):
    assert a["state"] == b["state"], f"{label}: walker state differs"
    assert np.array_equal(a["w"], b["w"]), f"{label}: weights differ"
    assert np.array_equal(a["lo"].view(np.float64), b["lo"].view(np.float64)), label
    assert np.array_equal(a["hist"], b["hist"]), f"{label}: energy history differs"


def mixed_system(seed=5, M=20, n_up=4, n_dn=3, n_chol=30, W=48):
    return small_system(M=M, n_up=n_up, n_dn=n_dn, n_chol=n_chol, seed=seed,
                        n_walkers=W, dtau=0.01, l_sigma=0.05, ortho_every=2,
                        measure_every=10, pc_every=10)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32x3", "bf16x3"])
def test_graph_replay_is_bitwise_plain_launches(prec):
    s = mixed_system()
    g = ctx(s, precision=prec, graphs=True)
    p = ctx(s, precision=prec, graphs=False)
    # a mix of call lengths: remainders run as plain launches, whole periods
    # (10 steps) as graph replays
    for n in (7, 20, 3, 40, 1, 9):
        g.afqmc_propagate(n)
        p.afqmc_propagate(n)
    assert g.afqmc_graph_count() > 0
    assert p.afqmc_graph_count() == 0
    a, b = snapshot(g), snapshot(p)
    assert_identical(a, b, prec)
    assert a["launches"] == b["launches"]
    g.close()
    p.close()


def test_device_bytes_equal_the_footprint():
    from paper_1804_03310_gb300 import Inputs, afqmc_footprint
    for s, prec in ((mixed_system(), "tf32x3"), (mixed_system(M=13), "fp64"),
                    (small_system(M=12, n_up=3, n_dn=3, n_chol=9, n_det=7, seed=2,
                                  n_walkers=16), "fp32")):
        c = ctx(s, precision=prec)
        res, _ = afqmc_footprint(Inputs.from_system(s, precision=prec))
        assert c.afqmc_device_bytes() == res
        c.close()


def _variants(c0):
    t = c0.afqmc_get_tuning()
    out = []
    for xs in sorted({1, 2, t["xsplit"]}):
        for bn in (64, 128):
            for fused in (0, 1, 2):
                out.append(dict(xsplit=xs, bn_force_bias=bn, bn_one_body=bn, bn_energy=bn,
                                bn_half_step=bn, taylor_fused=fused))
    return out


def test_every_launch_shape_meets_the_tolerance():
    s = small_system(M=28, n_up=5, n_dn=4, n_chol=70, seed=6, n_walkers=24, dtau=0.01,
                     l_sigma=0.04, ortho_every=2, measure_every=5, pc_every=0)
    c0 = ctx(s, precision="tf32x3")
    variants = _variants(c0)
    c0.close()
    for v in variants:
        c = ctx(s, precision="tf32x3", autotune=False)
        c.afqmc_set_tuning(**v)
        assert c.afqmc_get_tuning() == v
        orc = O.OracleRun(s)
        for k in range(1, 7):
            c.afqmc_propagate(1)
            orc.step()
            compare_state(c, orc, rtol=RTOL_REDUCED, label=f"{v} step {k}")
        compare_energy(c, orc, rtol=RTOL_REDUCED, label=str(v))
        c.close()


def test_tuning_rejects_invalid_shapes():
    from paper_1804_03310_gb300 import AfqmcError
    s = mixed_system(M=68, n_chol=20, W=8)
    c = ctx(s, precision="tf32")
    with pytest.raises(AfqmcError):
        c.afqmc_set_tuning(taylor_fused=1)           # M > 64
    with pytest.raises(AfqmcError):
        c.afqmc_set_tuning(taylor_fused=2)           # M > 64
    with pytest.raises(AfqmcError):
        c.afqmc_set_tuning(taylor_fused=4)
    with pytest.raises(AfqmcError):
        c.afqmc_set_tuning(bn_energy=96)
    c.afqmc_set_tuning(taylor_fused=3)               # streamed operator: M > 64
    c.close()
    c = ctx(mixed_system(M=40, n_chol=20, W=8), precision="tf32")
    with pytest.raises(AfqmcError):
        c.afqmc_set_tuning(taylor_fused=3)           # M <= 64
    c.close()
    f = ctx(mixed_system(W=8), precision="fp64")
    assert f.afqmc_get_tuning()["xsplit"] == 1
    with pytest.raises(AfqmcError):
        f.afqmc_set_tuning(xsplit=2)
    f.close()


def batch_members():
    """Uneven systems: sizes, electron counts, n_chol, walkers, precisions
    and a multi-determinant trial."""
    return [
        (config_c1().replace(measure_every=10, pc_every=10), "fp64"),
        (mixed_system(seed=7, M=24, n_up=5, n_dn=5, n_chol=50, W=64), "tf32x3"),
        (mixed_system(seed=8, M=17, n_up=3, n_dn=2, n_chol=21, W=40), "fp32"),
        (small_system(M=14, n_up=3, n_dn=3, n_chol=12, seed=9, n_det=9, n_walkers=32,
                      dtau=0.01, l_sigma=0.05, ortho_every=2, measure_every=5,
                      pc_every=10), "tf32x3"),
    ]


def test_batch_matches_each_member_alone():
    from paper_1804_03310_gb300 import Batch
    members = batch_members()
    together = [ctx(s, precision=p) for s, p in members]
    alone = [ctx(s, precision=p) for s, p in members]
    b = Batch(together, steps_per_block=20)
    b.afqmc_batch_propagate(3)
    b.afqmc_batch_synchronize()
    assert b.afqmc_batch_launches() == 3
    for c in alone:
        c.afqmc_propagate(60)
    for i, (x, y) in enumerate(zip(together, alone)):
        assert_identical(snapshot(x), snapshot(y), f"member {i}")
    # members stay usable one by one between batch calls
    together[1].afqmc_propagate(5)
    alone[1].afqmc_propagate(5)
    b.afqmc_batch_propagate(1)
    for c in alone:
        c.afqmc_propagate(20)
    for i, (x, y) in enumerate(zip(together, alone)):
        assert_identical(snapshot(x), snapshot(y), f"member {i} after mixed calls")
    b.close()
    for c in together + alone:
        c.close()


def serve_inputs(seed, M, n_up, n_chol, W, prec="tf32x3", run_id=0):
    from paper_1804_03310_gb300 import Inputs
    s = small_system(M=M, n_up=n_up, n_dn=n_up, n_chol=n_chol, seed=seed, n_walkers=W,
                     dtau=0.005, l_sigma=0.05 * np.sqrt(10 / M), ortho_every=2,
                     measure_every=10, pc_every=10)
    return Inputs.from_system(s.replace(run_id=run_id), precision=prec)


def run_alone(inp, n_blocks, spb):
    from paper_1804_03310_gb300 import Server
    srv = Server()
    rid = srv.afqmc_server_submit(inp, n_blocks, spb)
    srv.afqmc_server_wait(rid, 300)
    out = srv.afqmc_server_poll(rid)
    srv.close()
    return out


def test_served_run_is_the_same_alone_and_in_a_mix():
    from paper_1804_03310_gb300 import Server
    target = serve_inputs(21, 24, 5, 60, 96, run_id=3)
    alone = run_alone(target, 4, 10)
    assert alone["state"] == "done", alone["message"]
    others = [serve_inputs(30 + k, M, n, G, W, prec, run_id=k)
              for k, (M, n, G, W, prec) in enumerate([(40, 8, 120, 128, "tf32x3"),
                                                       (20, 4, 50, 256, "fp32"),
                                                       (32, 6, 100, 64, "tf32")])]
    srv = Server()
    ids = [srv.afqmc_server_submit(others[0], 6, 10)]
    rid = srv.afqmc_server_submit(target, 4, 10)
    ids += [srv.afqmc_server_submit(o, 5, 10) for o in others[1:]]
    srv.afqmc_server_wait(-1, 600)
    mixed = srv.afqmc_server_poll(rid)
    st = srv.afqmc_server_stats()
    for i in ids:
        info = srv.afqmc_server_poll(i)
        assert info["state"] == "done", info["message"]
        assert info["blocks_done"] == info["n_blocks"]
    srv.close()
    assert mixed["state"] == "done"
    ea = np.array([b["e_mixed"] for b in alone["blocks"]])
    em = np.array([b["e_mixed"] for b in mixed["blocks"]])
    wa = np.array([b["weight_sum"] for b in alone["blocks"]])
    wm = np.array([b["weight_sum"] for b in mixed["blocks"]])
    assert np.all(np.isfinite(ea)) and len(ea) == 4
    # the stated tolerance; the run is in fact reproduced bit for bit
    assert np.max(np.abs(em - ea)) <= RTOL_REDUCED * np.max(np.abs(ea))
    assert np.max(np.abs(wm - wa)) <= RTOL_REDUCED * np.max(np.abs(wa))
    assert np.array_equal(ea, em) and np.array_equal(wa, wm)
    assert [b["step"] for b in mixed["blocks"]] == [10, 20, 30, 40]
    # the mix overlapped on the device
    assert st["max_active_seen"] >= 2
    assert st["completed"] == 4 and st["failed"] == 0
    assert np.isfinite(st["p50_ms"]) and st["p99_ms"] >= st["p50_ms"] > 0


def test_served_energy_matches_a_plain_context():
    from paper_1804_03310_gb300 import Afqmc
    inp = serve_inputs(41, 20, 4, 40, 64)
    served = run_alone(inp, 3, 10)
    c = Afqmc(inp)
    e = []
    for _ in range(3):
        c.afqmc_propagate(10)
        e.append(c.afqmc_energy_history()[-1, 1])
    c.close()
    assert np.array_equal(np.array(e), np.array([b["e_mixed"] for b in served["blocks"]]))


def test_admission_respects_the_hbm_budget():
    from paper_1804_03310_gb300 import Server, afqmc_footprint
    runs = [serve_inputs(50 + k, 24, 5, 48, 64) for k in range(4)]
    need = max(sum(afqmc_footprint(r)) for r in runs)
    min_res = min(afqmc_footprint(r)[0] for r in runs)
    budget = need + min_res // 2                  # room for one run at a time
    srv = Server(hbm_budget=budget)
    ids = [srv.afqmc_server_submit(r, 2, 10) for r in runs]
    srv.afqmc_server_wait(-1, 300)
    st = srv.afqmc_server_stats()
    infos = [srv.afqmc_server_poll(i) for i in ids]
    srv.close()
    assert all(i["state"] == "done" for i in infos)
    assert st["max_active_seen"] == 1
    assert st["peak_bytes"] <= budget
    # one at a time, in arrival order
    admits = [i["t_admit"] for i in infos]
    dones = [i["t_done"] for i in infos]
    assert admits == sorted(admits)
    assert all(admits[k + 1] >= dones[k] for k in range(3))


def test_oversized_run_fails_without_blocking_the_queue():
    from paper_1804_03310_gb300 import Server, afqmc_footprint
    small = serve_inputs(60, 16, 3, 20, 32)
    big = serve_inputs(61, 64, 12, 200, 512)
    budget = int(sum(afqmc_footprint(small)) * 2)
    srv = Server(hbm_budget=budget)
    rb = srv.afqmc_server_submit(big, 1, 10)
    rs = srv.afqmc_server_submit(small, 2, 10)
    srv.afqmc_server_wait(-1, 120)
    ib, is_ = srv.afqmc_server_poll(rb), srv.afqmc_server_poll(rs)
    srv.close()
    assert ib["state"] == "failed" and ib["status"] == 2 and "budget" in ib["message"]
    assert is_["state"] == "done"


# ------------------------------------------------------- correlated sampling
def cs_pair(run_ids=(0, 0), W=512, measure=10, pc=0):
    """Neutral (5+5) and cation (5+4) of the 10-orbital system, same
    Hamiltonian and orbitals; equal run_ids mean shared field draws. Without
    the comb (pc = 0) walker i of the neutral run and walker i of the cation
    run see the same fields at every step."""
    from synth import make_system
    kw = dict(M=10, n_chol=40, ham_seed=0, l_kind="dense", l_sigma=0.05, trial="eig",
              dtau=0.01, n_walkers=W, seed=17, ortho_every=5, measure_every=measure,
              pc_every=pc)
    neu = make_system("neutral", n_up=5, n_dn=5, run_id=run_ids[0], **kw)
    cat = make_system("cation", n_up=5, n_dn=4, run_id=run_ids[1], **kw)
    return neu, cat


def test_correlated_sampling_reduces_the_variance_of_the_difference():
    """Sec. V: with shared auxiliary-field paths the cation - neutral energy
    difference fluctuates far less than with independent paths."""
    out = {}
    for label, ids in (("cs", (3, 3)), ("independent", (3, 4))):
        neu, cat = cs_pair(ids)
        e = []
        for s in (neu, cat):
            with ctx(s, precision="fp64") as c:
                c.afqmc_propagate(600)
                e.append(c.afqmc_energy_history()[:, 1])
        d = (e[1] - e[0])[10:]           # after 1 Ha^-1
        out[label] = float(np.var(d))
    print("variance of the energy difference per measurement:", out)
    # measured ratio about 3.6 with 512 walkers (8 with 2048, in the bench):
    # the extra electron makes the paired walkers drift apart, so the
    # correlation decays within a few Ha^-1
    assert out["cs"] < 0.5 * out["independent"]


def test_server_admits_a_correlated_sampling_group_together():
    from paper_1804_03310_gb300 import AfqmcError, Inputs, Server
    neu, cat = cs_pair((5, 5), W=128, measure=10, pc=10)
    other = mixed_system(seed=3, W=64)
    srv = Server(max_active=8)
    a = srv.afqmc_server_submit(Inputs.from_system(neu, precision="fp64", cs_group=9,
                                                   cs_size=2), 2, 20)
    b = srv.afqmc_server_submit(Inputs.from_system(other, precision="fp64"), 2, 20)
    srv.afqmc_server_wait(b, 120)
    assert srv.afqmc_server_poll(a)["state"] == "queued"   # waits for its partner
    # a member that does not match the group is refused
    bad = cat.replace(seed=99)
    with pytest.raises(AfqmcError):
        srv.afqmc_server_submit(Inputs.from_system(bad, precision="fp64", cs_group=9,
                                                   cs_size=2), 2, 20)
    c = srv.afqmc_server_submit(Inputs.from_system(cat, precision="fp64", cs_group=9,
                                                   cs_size=2), 2, 20)
    srv.afqmc_server_wait(-1, 120)
    ia, ic = srv.afqmc_server_poll(a), srv.afqmc_server_poll(c)
    assert ia["state"] == ic["state"] == "done"
    assert ia["t_admit"] >= ic["t_submit"] and ic["t_admit"] >= ic["t_submit"]
    with pytest.raises(AfqmcError):           # the group is closed once admitted
        srv.afqmc_server_submit(Inputs.from_system(cat, precision="fp64", cs_group=9,
                                                   cs_size=2), 2, 20)
    # each member's blocks equal the same run alone
    for info, s in ((ia, neu), (ic, cat)):
        with ctx(s, precision="fp64") as alone:
            alone.afqmc_propagate(40)
            h = alone.afqmc_energy_history()
        got = [blk["e_mixed"] for blk in info["blocks"]]
        want = [h[h[:, 0] == blk["step"], 1][0] for blk in info["blocks"]]
        assert got == want
    srv.close()
