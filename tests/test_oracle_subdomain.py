"""Pins of the oracle's sub-domain labels (Sec. 4.2-4.3): the edge labels
that build a neighbour's halo and the migration labels of a one-dimensional
decomposition along x, and the (label, id) order the radix sort gives them.

The pins: the paper's worked example of Sec. 4.3 (labels and sorted ids),
the edge's defining property (every particle with a neighbour across a
sub-domain boundary lies in that boundary's edge, found by brute force over
all pairs), closed-form edge sizes on a lattice, and the boundary
conventions at exactly 2h.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1210_1017_gb300 import cases


def _oracle(case):
    return oracle.Oracle(case.params())


def _example_positions(halo, xlo, xhi, h):
    """Positions whose edge labels are the example's: label 1 at 0.5h past
    the left boundary, 2 at 0.5h before the right one, 0 in the middle."""
    xs = {0: 0.5 * (xlo + xhi), 1: xlo + 0.5 * h, 2: xhi - 0.5 * h}
    pos = np.zeros((len(halo), 3))
    pos[:, 0] = [xs[v] for v in halo]
    pos[:, 1] = 0.05 + 0.01 * np.arange(len(halo))
    pos[:, 2] = 0.05
    return pos


def test_worked_example_labels_and_order(golden_dir):
    g = json.load(open(os.path.join(golden_dir, "radix_sort_halo_example.json")))
    c = cases.random_block(64, seed=1)
    O = _oracle(c)
    h = c.h
    xlo = 0.02
    xhi = xlo + 5 * h                  # wider than the two edges together (4h)
    pos = _example_positions(g["halo"], xlo, xhi, h)
    ids = np.array(g["id"], np.uint32)
    lab, counts, sel = O.subdomain_select(pos, ids, 0, xlo, xhi)
    assert lab.tolist() == g["halo"]
    perm = O.sort_by_key_id(lab, ids)
    assert lab[perm].tolist() == g["sorted_halo"]
    assert ids[perm].tolist() == g["sorted_id"]
    # what the sub-domain sends: labels 1 then 2, each in ascending id
    assert ids[sel].tolist() == [2, 3, 5, 8]
    assert counts.tolist() == [4, 3, 1]


def test_edges_hold_every_particle_with_a_neighbour_across_the_boundary():
    """Sec. 4.2: the halo of a sub-domain is built from the neighbours'
    edges, so a particle with any neighbour (|r_ij| < 2h) beyond a boundary
    must be in that boundary's edge; and an edge particle is within 2h of the
    boundary.  Brute force over all pairs of a jittered block."""
    c = cases.random_block(2500, seed=17, jitter=0.45)
    O = _oracle(c)
    h = c.h
    x = c.pos[:, 0]
    span = x.max() - x.min()
    for xlo, xhi in ((x.min() + 0.2 * span, x.max() - 0.25 * span),
                     (x.min() + 0.31 * span, x.min() + 0.31 * span + 4.0 * h)):
        lab = O.subdomain_labels(c.pos, 0, xlo, xhi)
        inside = (x >= xlo) & (x < xhi)
        d2 = ((c.pos[:, None, :] - c.pos[None, :, :]) ** 2).sum(-1)
        nb = d2 < (2 * h) ** 2
        np.fill_diagonal(nb, False)
        left_nb = (nb & (x[None, :] < xlo)).any(1) & inside
        right_nb = (nb & (x[None, :] >= xhi)).any(1) & inside
        assert left_nb.sum() > 0 and right_nb.sum() > 0
        assert np.all(lab[left_nb] == 1)
        assert np.all(lab[right_nb] == 2)
        assert np.all(x[lab == 1] - xlo < 2 * h) and np.all(xhi - x[lab == 2] <= 2 * h)
        assert np.all(lab[~inside] == 0)


def test_edge_sizes_on_a_lattice():
    """Lattice planes at (i + 1/2) dp: with 2h = 2.6 dp a boundary at a
    plane gap has three planes in its edge on each side."""
    dp, nx, ny, nz = 0.02, 20, 4, 3
    ii, jj, kk = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    pos = np.stack([(ii.ravel() + 0.5) * dp, (jj.ravel() + 0.5) * dp,
                    (kk.ravel() + 0.5) * dp], axis=1)
    c = cases.random_block(64, seed=2)
    p = c.params()
    p.update(dmin=(-0.1, -0.1, -0.1), dmax=(1.0, 1.0, 1.0))
    O = oracle.Oracle(p)
    lab = O.subdomain_labels(pos, 0, 5 * dp, 15 * dp)
    plane = ny * nz
    assert (lab == 1).sum() == 3 * plane and (lab == 2).sum() == 3 * plane
    assert set(np.round(pos[lab == 1, 0] / dp - 0.5).astype(int)) == {5, 6, 7}
    assert set(np.round(pos[lab == 2, 0] / dp - 0.5).astype(int)) == {12, 13, 14}
    mig = O.subdomain_labels(pos, 1, 5 * dp, 15 * dp)
    assert (mig == 1).sum() == 5 * plane and (mig == 2).sum() == 5 * plane


def test_boundary_conventions_at_exactly_2h():
    c = cases.random_block(64, seed=3)
    p = c.params()
    h = 0.25                    # dyadic: every threshold is exact
    p.update(dmin=(-1.0, -1.0, -1.0), dmax=(3.0, 1.0, 1.0), h=h)
    O = oracle.Oracle(p)
    xlo, xhi = 0.0, 2.0
    xs = [xlo - 1e-9, xlo, xlo + 2 * h - 1e-12, xlo + 2 * h, 1.0,
          xhi - 2 * h - 1e-12, xhi - 2 * h, xhi - 1e-12, xhi]
    pos = np.array([[v, 0.0, 0.0] for v in xs])
    assert O.subdomain_labels(pos, 0, xlo, xhi).tolist() == [0, 1, 1, 0, 0, 0, 2, 2, 0]
    assert O.subdomain_labels(pos, 1, xlo, xhi).tolist() == [1, 0, 0, 0, 0, 0, 0, 0, 2]


def test_excluded_particles_are_never_selected():
    c = cases.random_block(300, seed=8)
    pos = c.pos.copy()
    pos[3, 0] = c.dmin[0] - 1.0        # outside the cell grid, left of xlo
    pos[4, 2] = np.nan
    O = _oracle(c)
    x = pos[:, 0]
    xlo, xhi = np.nanmin(c.pos[:, 0]) + 0.05, np.nanmax(c.pos[:, 0]) - 0.02
    lab, counts, sel = O.subdomain_select(pos, c.ids, 1, xlo, xhi)
    assert lab[3] == 0 and lab[4] == 0
    assert counts.sum() == c.n - 2
    assert 3 not in sel and 4 not in sel
    want = np.where(x < xlo, 1, np.where(x >= xhi, 2, 0))
    want[[3, 4]] = 0
    assert np.array_equal(lab, want)
