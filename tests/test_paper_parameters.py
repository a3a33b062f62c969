"""The synthetic workloads use the material and task parameters the paper
prints wherever they follow the paper's tasks (the fixture
tests/golden/paper_parameters.txt cites each value).  The benchmark's own
drive settings (3.0 / 3.4 GHz at 100 mT in plane, 5 nm cells) are the
benchmark configurations' and are not checked here."""
import os

import numpy as np
import pytest

import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def paper():
    vals = {}
    with open(os.path.join(HERE, "golden", "paper_parameters.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                name, value, cite = line.split(None, 2)
                assert cite.strip(), name
                vals[name] = float(value)
    return vals


def test_every_workload_uses_the_sigmoid_sharpness(paper):
    insts = [W.film32(), W.particle64(nsteps=10), W.demux256(0, nsteps=10), W.thick512(nsteps=10),
             W.sw_particle(levels=3, hold=2), W.random_small(8, 6)] + W.batch64(nsteps=10, candidates=1)
    for i in insts:
        assert i.problem.sigmoid_a == paper["sigmoid_a"], i.tag


def test_permalloy_tasks(paper):
    for i in (W.particle64(nsteps=10), W.sw_particle(levels=3, hold=2), W.film32()):
        assert i.problem.Ms == paper["permalloy_Ms"] and i.problem.A == paper["permalloy_A"], i.tag


def test_yig_demultiplexers(paper):
    for i in W.batch64(nsteps=10, candidates=1) + [W.demux256(0, nsteps=10), W.demux256(1, nsteps=10)]:
        assert i.problem.Ms == paper["yig_Ms"] and i.problem.A == paper["yig_A"], i.tag


def test_stoner_wohlfarth_task(paper):
    levels = 30
    for reg in (False, True):
        i = W.sw_particle(levels=levels, hold=2, regularised=reg)
        p = i.problem
        assert p.dx == p.dy == p.dz == paper["particle_cell"]
        design = int(paper["particle_design_cells"])
        assert p.ny == design and int(i.mask.sum()) == design * design
        # targets: M/Ms = b H / Ms at the levels' fields H_j = 0.3 Ms j / levels
        js = np.arange(1, levels + 1)
        assert np.allclose(p.sample_targets, paper["sw_slope_b"] * 0.3 * js / levels, rtol=0, atol=1e-15)
        w = np.asarray(p.sample_weights) * levels * np.asarray(p.sample_targets)
        if reg:
            assert np.allclose(w, paper["sw_zeta"])
            assert p.penalty_w == paper["sw_xi"] and p.centre_w == paper["sw_nu"]
        else:
            assert np.allclose(w, 1.0) and p.penalty_w == 0.0 and p.centre_w == 0.0
