"""Metropolis Monte Carlo on the GPU against the oracle's sweep, statistically.

The method's sweep (Sec. Monte Carlo) visits every spin once per iteration in
a random sequential order; the oracle does exactly that (a fresh random
permutation per sweep).  The GPU sweeps colour by colour (spins of one colour
never interact), which samples the same Boltzmann distribution but not the
same chain, so the two are compared through their equilibrium averages:
32 independent replicas per side, each thermalised with the adaptive cone
and then sampled with the cone fixed; per replica the time averages of the
energy E, the magnetisation m and the Binder cumulant U4 = 1 - <m^4>/(3<m^2>^2);
the replica means of GPU and oracle must agree within 4 combined standard
errors (72 comparisons in this file: at 4 sigma the chance of a false
alarm in the whole file is about 1%; at 3 sigma it would be about 20%).
The colour-ordered oracle (`order="coloured"`) is the bit-exact check of the
kernels' decomposition in test_gpu_parity.py.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1901_11350_gb300 import binding as B
from paper_1901_11350_gb300 import build
from paper_1901_11350_gb300 import inputs as I

pytestmark = pytest.mark.gpu

R = 32
NSIG = 4.0

CASES = {
    "sc4_dmi_field": (I.simple_cubic(4, 4, 4), dict(J=[1.0, -0.2], dmi_kind="bulk", D=[0.2], K=[0.1],
                                                    Khat=[[0, 0, 1]], B=[0, 0.3, 0.8]), 6.0, 500, 4000),
    "hex9_skyrmion_params": (I.hexagonal(9, 9, periodic=(True, True), mu_s=2.0),
                             dict(J=[1.0], dmi_kind="interfacial", D=[0.3], K=[0.05], Khat=[[0, 0, 1]],
                                  B=[0, 0, 1.0]), 6.0, 500, 4000),
    "hex6_open": (I.hexagonal(6, 5, periodic=(True, False), mu_s=3.0), dict(J=[1.0], B=[0.2, 0, 0.5]), 8.0, 500, 4000),
    "sc6_nn_dmi": (I.simple_cubic(6, 4, 4), dict(J=[1.0], dmi_kind="bulk", D=[0.25], K=[0.1], Khat=[[0, 0, 1]],
                                                 B=[0, 0.3, 0.8]), 10.0, 500, 4000),
    "sq6x5_open": (I.square(6, 5, periodic=(True, False), mu_s=2.0), dict(J=[1.0], B=[0, 0, 0.4]), 4.0, 500, 4000),
    "sc9x3x3_mod3": (I.simple_cubic(9, 3, 3), dict(J=[1.0], K=[0.1], Khat=[[0, 0, 1]], B=[0.2, 0, 0.5]),
                     12.0, 500, 4000),
    "sc5_mod5": (I.simple_cubic(5, 5, 5), dict(J=[1.0], dmi_kind="bulk", D=[0.2], B=[0, 0, 0.3]), 10.0, 500, 4000),
    # the Tc workload's smallest lattice close to its critical temperature
    "sc10_near_tc": (I.simple_cubic(10, 10, 10, periodic=(True, True, True), mu_s=2.0), dict(J=[1.0]),
                     16.5, 1000, 6000),
}

_oracle_cache = {}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    B.lib()


def _starts(N):
    return np.stack([I.random_spins(N, 1000 + r) for r in range(R)])


def _observables(st):
    st = np.asarray(st)
    n = st[:, 5]
    m, m2, m4, E = st[:, 0] / n, st[:, 1] / n, st[:, 2] / n, st[:, 3] / n
    return {"E": E, "m": m, "U4": 1.0 - m4 / (3.0 * m2 * m2)}


def _oracle_obs(name):
    if name not in _oracle_cache:
        g, h, T, n_th, n_s = CASES[name]
        o = oracle.System(g, h)
        x0 = _starts(o.N)
        x, cone, _ = o.mc(x0, [T] * R, n_th, seed=11, target_accept=0.5, sample=False)
        _, _, st = o.mc(x, [T] * R, n_s, seed=11, sweep0=n_th, target_accept=0.0, sample=True, cone=cone)
        _oracle_cache[name] = _observables(st)
    return _oracle_cache[name]


@pytest.mark.parametrize("prec,resident", [("f64", 1), ("f64", 0), ("f32", 1)],
                         ids=["f64_resident", "f64_per_colour", "f32_resident"])
@pytest.mark.parametrize("name", list(CASES))
def test_mc_equilibrium_averages_match_the_random_order_oracle(name, prec, resident):
    g, h, T, n_th, n_s = CASES[name]
    c = B.Context(g, h, prec)
    c.set_option("mc_resident", resident)
    x = torch.stack([c.spins(s) for s in _starts(c.N)]).contiguous()
    cone, st = c.mc_sweeps(x, [T] * R, n_th, seed=11, target_accept=0.5, sample=False)
    st.zero_()
    cone, st = c.mc_sweeps(x, [T] * R, n_s, seed=11, sweep0=n_th, target_accept=0.0, sample=True, cone=cone,
                           stats=st)
    gpu = _observables(st.cpu().numpy())
    ora = _oracle_obs(name)
    for k in ("E", "m", "U4"):
        a, b = gpu[k], ora[k]
        se = np.sqrt(a.var(ddof=1) / len(a) + b.var(ddof=1) / len(b))
        z = abs(a.mean() - b.mean()) / max(se, 1e-300)
        print("%s %s %s: gpu %.6g oracle %.6g (%.2f sigma)" % (name, prec, k, a.mean(), b.mean(), z))
        assert z <= NSIG, (k, a.mean(), b.mean(), se)
