"""The persistent batched GNEB kernel: every image of every chain, all the
iterations of a call, in one cooperative launch with grid barriers between
the passes (Sec. GNEB, Appendix F; the batching of many chains of uneven
sizes in one launch).

* bit for bit the iterates of the one-launch-per-pass path, for chains of
  different lattices and image counts, climbing/falling images and
  energy-weighted springs, FP32 and FP64;
* a barrier wait that runs out (the poll limit set to 1) makes every block
  leave the kernel: the call returns, the status word reports SP_ERR_TIMEOUT,
  and the next call with the default limit computes the right result again.
"""
import numpy as np
import pytest
import torch

from paper_1901_11350_gb300 import binding as B
from paper_1901_11350_gb300 import build
from paper_1901_11350_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TIMEOUT = -5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    B.lib()


def _chains():
    out = []
    g = I.hexagonal(24, 20, periodic=(True, True), mu_s=2.0)
    h = dict(J=[1.0], dmi_kind="interfacial", D=[0.35], K=[0.08], Khat=[[0, 0, 1]], B=[0, 0, 1.2])
    r = I.site_positions(g)
    out.append((g, h, I.slerp_chain(I.ferromagnet(I.n_spins(g)), I.neel_skyrmion(r, r.mean(0), 4.0, np.pi), 9, r,
                                     r.mean(0))))
    g = I.square(13, 9, periodic=(True, False), mu_s=1.5)
    h = dict(J=[1.0, 0.1], dmi_kind="interfacial", D=[0.2], K=[0.2], Khat=[[0, 0, 1]], B=[0, 0, 0.5])
    out.append((g, h, I.slerp_chain(I.random_spins(117, 1), I.random_spins(117, 2), 5)))
    g = I.simple_cubic(8, 6, 5, periodic=(True, True, False))
    h = dict(J=[1.0, -0.2], dmi_kind="bulk", D=[0.2], K=[0.05], Khat=[[0, 0, 1]], B=[0, 0, 0.3])
    out.append((g, h, I.slerp_chain(I.ferromagnet(240), I.ferromagnet(240, (0, 0.2, -1)), 7)))
    return out


def _run(prec, persistent, n_iter, limit=0, **kw):
    chains = _chains()
    ctxs = [B.Context(g, h, prec) for g, h, _ in chains]
    ctxs[0].set_option("gneb_persistent", persistent)
    ctxs[0].set_option("wait_limit", limit)
    offs, Ms, off = [], [], 0
    for c, (_, _, ch0) in zip(ctxs, chains):
        offs.append(off)
        Ms.append(ch0.shape[0])
        off += ch0.shape[0] * ch0.shape[1]
    x = torch.cat([c.spins(ch0).reshape(-1, 4) for c, (_, _, ch0) in zip(ctxs, chains)])
    v = torch.zeros_like(x)
    out = []
    for n in n_iter:
        E, F = B.gneb_batch_step(ctxs, x, v, offs, Ms, n_iter=n, k_spring=0.7, dt=0.1, **kw)
        out.append((E.clone(), F.clone()))
    return ctxs, x, v, out


KINDS = {
    "climbing": dict(climbing=True),
    "kinds_and_weighted": dict(image_types=["normal", "climbing", "normal", "falling", "normal", "normal", "normal",
                                            "normal", "normal"] + ["normal", "falling", "normal", "climbing",
                                                                   "normal"] + ["normal"] * 7, energy_weight=0.4),
}


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("kind", list(KINDS))
def test_persistent_kernel_matches_the_per_pass_launches(prec, kind):
    _, xa, va, oa = _run(prec, 0, (1, 25, 8), **KINDS[kind])
    cb, xb, vb, ob = _run(prec, 1, (1, 25, 8), **KINDS[kind])
    assert torch.equal(xa, xb) and torch.equal(va, vb)
    for (Ea, Fa), (Eb, Fb) in zip(oa, ob):
        assert torch.equal(Ea, Eb) and torch.equal(Fa, Fb)
    assert cb[0].sync_status()[0] == 0


def test_a_barrier_wait_that_runs_out_reports_a_timeout():
    # reference: the per-pass launches
    _, xr, vr, orf = _run("f32", 0, (12,))
    # one poll per wait: the first block at a barrier gives up at once
    ctxs, x, v, _ = _run("f32", 1, (12,), limit=1)
    code, msg = ctxs[0].sync_status()  # returns: no block was left waiting
    assert code == TIMEOUT, (code, msg)
    assert ctxs[0].sync_status()[0] == 0
    # with the default limit the same context steps correctly again
    ctxs[0].set_option("wait_limit", 0)
    chains = _chains()
    offs, Ms, off = [], [], 0
    for (_, _, ch0) in chains:
        offs.append(off)
        Ms.append(ch0.shape[0])
        off += ch0.shape[0] * ch0.shape[1]
    x2 = torch.cat([c.spins(ch0).reshape(-1, 4) for c, (_, _, ch0) in zip(ctxs, chains)])
    v2 = torch.zeros_like(x2)
    E, F = B.gneb_batch_step(ctxs, x2, v2, offs, Ms, n_iter=12, k_spring=0.7, dt=0.1, climbing=True)
    assert ctxs[0].sync_status()[0] == 0
    assert torch.equal(x2, xr) and torch.equal(v2, vr)
    assert torch.equal(E, orf[0][0]) and torch.equal(F, orf[0][1])


def test_single_chain_call_takes_the_persistent_kernel_too():
    g, h, ch0 = _chains()[0]
    res = []
    for persistent in (0, 1):
        c = B.Context(g, h, "f64")
        c.set_option("gneb_persistent", persistent)
        x, v = c.spins(ch0), c.spins(np.zeros_like(ch0))
        E, F = c.gneb_step(x, v, n_iter=30, k_spring=1.0, dt=0.1)
        res.append((x, v, E, F))
    for a, b in zip(res[0], res[1]):
        assert torch.equal(a, b)


def test_autotune_picks_a_launch_mode_and_leaves_the_chains_alone():
    chains = _chains()
    ctxs = [B.Context(g, h, "f32") for g, h, _ in chains]
    offs, Ms, off = [], [], 0
    for (_, _, ch0) in chains:
        offs.append(off)
        Ms.append(ch0.shape[0])
        off += ch0.shape[0] * ch0.shape[1]
    x = torch.cat([c.spins(ch0).reshape(-1, 4) for c, (_, _, ch0) in zip(ctxs, chains)])
    v = torch.zeros_like(x)
    x0, v0 = x.clone(), v.clone()
    choice, t_pass, t_pers = B.gneb_batch_autotune(ctxs, x, v, offs, Ms, n_trial=20, k_spring=0.7, dt=0.1)
    print("GNEB batch autotune: per pass %.3f ms, persistent %.3f ms -> %s" % (
        t_pass, t_pers, "persistent" if choice else "per pass"))
    assert torch.equal(x, x0) and torch.equal(v, v0)
    assert choice == (1 if t_pers < t_pass else 0) == ctxs[0].get_option("gneb_persistent")
    assert t_pass > 0 and t_pers > 0
