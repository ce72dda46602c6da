"""The synthetic workloads and the oracle use the model parameters the paper
prints (Sec. 2.4); the KG bond made of those parameters has a sensible
equilibrium length.  Fixture: tests/golden/paper_parameters.json."""
import json
import math
import os

import numpy as np
import pytest

import oracle
import synth

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_parameters.json")))


def test_lj_workloads_use_the_papers_cutoff_and_units():
    g = GOLD["lj_fluid"]
    for w in (synth.lj_fluid_4000(), synth.lj_box_4m()):
        assert w.rc == g["rc"]
        assert w.rho == pytest.approx(g["rho"], abs=5e-4)


def test_kg_workload_uses_wca_and_fene_of_eqs_10_11():
    g = GOLD["kg_melt"]
    w = synth.kg_melt_200x100()
    assert w.rc ** 6 == pytest.approx(g["wca_rc_over_sigma_pow6"], rel=1e-12)
    assert (w.fene_k, w.fene_R0) == (g["fene_k"], g["fene_R0"])


def test_kg_bond_force_vanishes_just_below_one_sigma():
    """FENE (Eq. 11, k = 30, R0 = 1.5) plus the WCA repulsion (Eq. 10 at
    rc = 2^(1/6)) give a bond whose force changes sign once, near r = 0.96:
    attractive FENE balances the steep repulsion below sigma."""
    g = GOLD["kg_melt"]
    rc = g["wca_rc_over_sigma_pow6"] ** (1 / 6)
    p = oracle.params(10.0, 0.0, rc, fene_k=g["fene_k"], fene_R0=g["fene_R0"])
    rs = np.linspace(0.85, 1.1, 251)
    fx = []
    for r in rs:
        pos = np.array([[2.0, 2.0, 2.0], [2.0 + r, 2.0, 2.0]])
        fx.append(oracle.forces(p, 0.0, pos, [[0, 1]])[1][1, 0])
    fx = np.array(fx)
    crossings = np.nonzero(np.diff(np.sign(fx)))[0]
    assert crossings.size == 1
    r0 = rs[crossings[0]]
    assert 0.95 < r0 < 0.98


def test_table1_derived_rates_are_consistent():
    """Particle-steps/s implied by Table 1 (context numbers for the benchmark)."""
    t = GOLD["table1_runtime_s_per_1000_steps"]
    rates = [2.56e6 * 1000 / s for s in t["lebc"]]
    assert rates[0] == pytest.approx(2.37e7, rel=0.01)
    assert rates[-1] == pytest.approx(1.16e9, rel=0.01)
