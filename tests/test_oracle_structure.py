"""Pins of the oracle's structural observables (Sec. III): common-neighbour analysis, the
central-atom pair-distance histogram and the mean squared displacement, each against facts fixed
by geometry (textbook CNA signatures of fcc, hcp and the icosahedron; the shell counts of the fcc
lattice, enumerated here by brute force; closed forms of the displacement)."""
import numpy as np
import pytest

import oracle
from paper_1210_3559_gb300 import inputs

A = 3.52          # Ni lattice constant (A)
NN = A / np.sqrt(2.0)


def hcp_block(nx=8, ny=8, nz=8, d=NN):
    """Ideal hcp (c/a = sqrt(8/3)), layers ABAB..., centred on its centroid."""
    pts = []
    c_half = d * np.sqrt(2.0 / 3.0)
    for k in range(nz):
        sx, sy = (0.0, 0.0) if k % 2 == 0 else (d / 2.0, d / (2.0 * np.sqrt(3.0)))
        for j in range(ny):
            for i in range(nx):
                pts.append([(i + 0.5 * j) * d + sx, j * d * np.sqrt(3.0) / 2.0 + sy, k * c_half])
    p = np.array(pts)
    return p - p.mean(axis=0)


def bcc_block(n=6, a=2.8):
    g = np.arange(n) * a
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    corner = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    p = np.concatenate([corner, corner + a / 2.0])
    return p - p.mean(axis=0)


def fcc_shells(kmax):
    """Number of fcc sites (a/2)(i, j, k), i + j + k even, at squared distance s (a/2)^2, s = 2, 4, ..."""
    r = int(np.ceil(np.sqrt(kmax))) + 1
    g = np.arange(-r, r + 1)
    I, J, K = np.meshgrid(g, g, g, indexing="ij")
    even = (I + J + K) % 2 == 0
    s = (I * I + J * J + K * K)[even]
    return {int(v): int(np.sum(s == v)) for v in range(2, kmax + 1, 2) if np.sum(s == v) > 0}


def interior(pos, depth):
    r = np.linalg.norm(pos - pos.mean(axis=0), axis=1)
    return r < r.max() - depth


# ---------------------------------------------------------------- CNA
def test_cna_signatures_fcc_hcp_icosahedron():
    fcc = inputs.fcc_sphere(1000)
    c = int(np.argmin(np.linalg.norm(fcc, axis=1)))
    nbrs = np.where((np.linalg.norm(fcc - fcc[c], axis=1) < 3.0) & (np.arange(len(fcc)) != c))[0]
    assert len(nbrs) == 12
    assert {oracle.cna_signature(fcc, c, int(j)) for j in nbrs} == {(4, 2, 1)}
    hcp = hcp_block()
    c = int(np.argmin(np.linalg.norm(hcp, axis=1)))
    nbrs = np.where((np.linalg.norm(hcp - hcp[c], axis=1) < 3.0) & (np.arange(len(hcp)) != c))[0]
    sig = sorted(oracle.cna_signature(hcp, c, int(j)) for j in nbrs)
    assert sig == [(4, 2, 1)] * 6 + [(4, 2, 2)] * 6
    ico = inputs.mackay_icosahedron(3, 2.49)
    nbrs = np.where((np.linalg.norm(ico - ico[0], axis=1) < 3.0) & (np.arange(len(ico)) != 0))[0]
    assert np.allclose(ico[0], 0.0) and len(nbrs) == 12
    assert {oracle.cna_signature(ico, 0, int(j)) for j in nbrs} == {(5, 5, 5)}


def test_cna_classes_of_ideal_structures():
    fcc = inputs.fcc_sphere(2000)
    cls, nnb = oracle.cna(fcc)
    inner = interior(fcc, 2 * 3.0)
    assert np.all(cls[inner] == oracle.CNA_FCC)
    assert np.all(cls[nnb != 12] == oracle.CNA_OTHER)
    hcp = hcp_block(12, 12, 10)
    cls, _ = oracle.cna(hcp)
    inner = np.linalg.norm(hcp, axis=1) < 5.0  # two neighbour shells inside the block
    assert inner.sum() > 20 and np.all(cls[inner] == oracle.CNA_HCP)
    ico = inputs.mackay_icosahedron(3, 2.49)
    cls, _ = oracle.cna(ico)
    assert cls[0] == oracle.CNA_ICO
    cls, nnb = oracle.cna(bcc_block())  # 8 + 6 neighbours inside 3 A: never 12
    assert np.all(cls == oracle.CNA_OTHER) and nnb.max() == 14


def test_cna_invariances():
    rng = np.random.default_rng(4)
    pos = inputs.jitter(inputs.fcc_sphere(600), 0.08, 9)
    cls, nnb = oracle.cna(pos)
    assert 0 < np.sum(cls == oracle.CNA_FCC) < len(pos)
    perm = rng.permutation(len(pos))
    c2, n2 = oracle.cna(pos[perm])
    assert np.array_equal(c2, cls[perm]) and np.array_equal(n2, nnb[perm])
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    c3, _ = oracle.cna(pos @ q.T + np.array([5.0, -3.0, 2.0]))
    # a rotation moves no distance by more than a few ulps; no pair lies that close to 3 A here
    r = np.linalg.norm(pos[:, None] - pos[None], axis=2)
    assert np.min(np.abs(r - 3.0)) > 1e-9
    assert np.array_equal(c3, cls)


# ---------------------------------------------------------------- pair-distance histogram
def test_rdf_of_the_centre_atom_is_the_fcc_shell_count():
    pos = inputs.fcc_sphere(2000)  # radius ~17 A: complete shells out to 7.5 A
    m = inputs.masses(len(pos))
    counts, nc = oracle.rdf(pos, m, r_core=0.5, bin_A=0.1, nbins=76)
    assert nc == 1
    shells = fcc_shells(24)  # r = (a/2) sqrt(s) up to 8.6 A
    assert [shells[s] for s in (2, 4, 6, 8, 10, 12, 14, 16)] == [12, 6, 24, 12, 24, 8, 48, 6]
    expect = np.zeros(76, dtype=np.int64)
    for s, n in shells.items():
        r = 0.5 * A * np.sqrt(s)
        if r < 7.6:
            expect[int(r / 0.1)] += n
    assert np.array_equal(counts, expect)


def test_rdf_counts_every_core_pair_once():
    pos = inputs.jitter(inputs.fcc_sphere(400), 0.1, 3)
    m = inputs.masses(len(pos))
    counts, nc = oracle.rdf(pos, m, r_core=4.0, bin_A=0.25, nbins=400)  # 100 A: every pair
    X = pos.mean(axis=0)
    core = np.linalg.norm(pos - X, axis=1) < 4.0
    assert nc == core.sum() and counts.sum() == nc * (len(pos) - 1)
    d = np.linalg.norm(pos[core][:, None] - pos[None], axis=2)
    d = d[d > 0]
    assert np.array_equal(counts, np.bincount((d / 0.25).astype(int), minlength=400))


# ---------------------------------------------------------------- mean squared displacement
def test_msd_closed_forms():
    pos = inputs.fcc_sphere(300)
    m = inputs.masses(300)
    v, n = oracle.msd(pos + np.array([1.5, -2.0, 0.25]), pos, m)
    assert n == 300 and v == pytest.approx(0.0, abs=1e-20)  # a rigid translation moves the COM only
    d = np.array([0.3, -0.4, 1.2])
    far = int(np.argmax(np.linalg.norm(pos - pos.mean(axis=0), axis=1)))
    moved = pos.copy()
    moved[far] += d
    v, _ = oracle.msd(moved, pos, m)
    N = len(pos)
    assert v == pytest.approx(np.dot(d, d) * (N - 1) / N ** 2, rel=1e-12)
    v, n = oracle.msd(moved, pos, m, r_core=5.0)  # the moved atom is outside the core
    core = np.linalg.norm(pos - pos.mean(axis=0), axis=1) < 5.0
    assert not core[far] and n == core.sum()
    assert v == pytest.approx(np.dot(d, d) / N ** 2, rel=1e-12)
    assert np.allclose(oracle.com(pos, m), pos.mean(axis=0), atol=1e-13)
