"""Pins of the FP64 oracle to facts fixed by the paper and the mathematics.

Each test checks the oracle against something other than itself: closed forms
(Chebyshev, cut-off, Legendre addition theorem), brute force written here in
numpy, finite differences, invariances and special cases with closed-form
answers.  A dropped term, a wrong sign or a transposed index anywhere in the
oracle should fail at least one of them.
"""
import math

import numpy as np
import pytest
from numpy.polynomial import legendre

from paper_2507_00528_gb300 import synth


def small_cfg(O, four_body=False, **kw):
    base = dict(nq_r=3, nq_a=3, k_r=5, k_a=5, hidden=6, four_body=four_body)
    base.update(kw)
    return O.Cfg(**base)


def small_batch(seed=5):
    rng = np.random.default_rng(seed)
    return synth.make_batch([12, 10], [2, 1], rng)


# ---------------------------------------------------------------- App. A

@pytest.mark.parametrize("theta", [0.1, 0.7, 1.3, 2.2, 3.0])
def test_chebyshev_closed_form(oracle, theta):
    """A1.1: T_k(cos t) = cos(k t); A1.3-A1.5: T_k' = k U_{k-1} = k sin(kt)/sin t."""
    K = 14
    T, dT = oracle.chebyshev(K, math.cos(theta))
    for k in range(K):
        assert T[k] == pytest.approx(math.cos(k * theta), abs=1e-12)
        assert dT[k] == pytest.approx(k * math.sin(k * theta) / math.sin(theta), abs=1e-10)
    assert np.all(np.abs(T) <= 1 + 1e-15)


def test_cutoff_values(oracle):
    """A2.1/A2.2: f_c(0)=1, f_c(rc/2)=1/2, f_c(rc)=f_c'(rc)=0, zero beyond rc."""
    rc = 4.0
    assert oracle.cutoff(rc, 0.0) == pytest.approx((1.0, 0.0), abs=1e-15)
    fc, fcp = oracle.cutoff(rc, rc / 2)
    assert fc == pytest.approx(0.5, abs=1e-15)
    assert fcp == pytest.approx(-math.pi / (2 * rc), rel=1e-14)
    fc, fcp = oracle.cutoff(rc, rc)
    assert abs(fc) < 1e-15 and abs(fcp) < 1e-15
    assert oracle.cutoff(rc, rc + 0.1) == (0.0, 0.0)


def test_radial_basis_derivative_fd(oracle):
    """f_k' of the basis equals a central difference of f_k (Eq. 6, A1.2-A2.2)."""
    K, rc, h = 13, 7.0, 1e-6
    for r in [0.9, 2.5, 4.1, 6.3, 6.99]:
        f, fp = oracle.radial_basis(K, rc, r)
        fpl, _ = oracle.radial_basis(K, rc, r + h)
        fmi, _ = oracle.radial_basis(K, rc, r - h)
        np.testing.assert_allclose(fp, (fpl - fmi) / (2 * h), rtol=1e-7, atol=1e-9)
        # f_k = (T_k(xi) + 1)/2 * f_c with xi = 2 (r/rc - 1)^2 - 1
        xi = 2 * (r / rc - 1) ** 2 - 1
        fc = 0.5 * (1 + math.cos(math.pi * r / rc))
        theta = math.acos(xi)
        ref = np.array([(math.cos(k * theta) + 1) / 2 * fc for k in range(K)])
        np.testing.assert_allclose(f, ref, atol=1e-13)
    f, _ = oracle.radial_basis(K, rc, rc)
    assert np.all(np.abs(f) < 1e-15)


# ---------------------------------------------------------------- App. B

def _unit(rng):
    v = rng.normal(size=3)
    return v / np.linalg.norm(v)


def test_blm_addition_theorem(oracle):
    """sum_m C_lm B_lm(u) B_lm(v) = P_l(u.v) and sum_m C_lm B_lm(u)^2 = 1, for
    every l = 1..8 (B1-B8 with the C_lm reading)."""
    C = oracle.clm(8)
    rng = np.random.default_rng(0)
    first = [l * l - 1 for l in range(1, 10)]
    for _ in range(20):
        u, v = _unit(rng), _unit(rng)
        r1, r2 = rng.uniform(0.5, 5), rng.uniform(0.5, 5)
        Bu, _ = oracle.blm(u * r1, 8)
        Bv, _ = oracle.blm(v * r2, 8)
        for l in range(1, 9):
            s = slice(first[l - 1], first[l])
            P = legendre.legval(u @ v, [0] * l + [1])
            assert np.sum(C[s] * Bu[s] * Bv[s]) == pytest.approx(P, abs=1e-12)
            assert np.sum(C[s] * Bu[s] ** 2) == pytest.approx(1.0, abs=1e-12)


def test_blm_gradient_fd_and_homogeneity(oracle):
    """B9.2 equals a central difference of B9.1; B_lm depends on direction only."""
    rng = np.random.default_rng(1)
    h = 1e-6
    for _ in range(10):
        d = rng.normal(size=3) * 2
        B, dB = oracle.blm(d, 8)
        for c in range(3):
            e = np.zeros(3); e[c] = h
            fd = (oracle.blm(d + e, 8)[0] - oracle.blm(d - e, 8)[0]) / (2 * h)
            np.testing.assert_allclose(dB[:, c], fd, rtol=1e-6, atol=1e-7)
        B2, _ = oracle.blm(3.7 * d, 8)
        np.testing.assert_allclose(B, B2, atol=1e-11)


def test_blm_printed_forms(oracle):
    """Spot values of B1-B4 at u = (1,2,2)/3 from the printed polynomials."""
    x, y, z = 1 / 3, 2 / 3, 2 / 3
    B, _ = oracle.blm(np.array([x, y, z]) * 2.0)
    assert B[0] == pytest.approx(z)
    assert B[3] == pytest.approx(3 * z * z - 1)
    assert B[7] == pytest.approx(2 * x * y)
    assert B[8] == pytest.approx(5 * z ** 3 - 3 * z)
    assert B[14] == pytest.approx((3 * x * x - y * y) * y)
    assert B[15] == pytest.approx(35 * z ** 4 - 30 * z * z + 3)
    assert B[18] == pytest.approx((7 * z * z - 1) * (x * x - y * y))
    assert B[23] == pytest.approx(4 * x ** 3 * y - 4 * x * y ** 3)


def _printed_blm():
    """The 80 printed forms of the fixtures (B1.1-B4.9 and B5.1-B8.17) as
    (index, equation, function of x, y, z, r)."""
    import ast
    import pathlib
    out = []
    gold = pathlib.Path(__file__).parent / "golden"
    lines = (gold / "blm_cartesian_l1_4.txt").read_text().splitlines() + \
        (gold / "blm_cartesian_l5_8.txt").read_text().splitlines()
    for line in lines:
        if not line.strip() or line.startswith("#"):
            continue
        l, m, eq, expr = line.split(maxsplit=3)
        tree = ast.parse(expr, mode="eval")
        names = {n.id for n in ast.walk(tree) if isinstance(n, ast.Name)}
        assert names <= {"x", "y", "z", "r"}, (eq, names)
        code = compile(tree, eq, "eval")
        out.append(((int(l) ** 2 - 1) + int(m), eq, lambda x, y, z, r, c=code: eval(c, {"__builtins__": {}},
                                                                                    dict(x=x, y=y, z=z, r=r))))
    return out


def test_blm_all_printed_forms_of_appendix_b(oracle):
    """All 80 printed b_lm of App. B (B1.1-B8.17, fixtures
    tests/golden/blm_cartesian_l1_4.txt and blm_cartesian_l5_8.txt): the
    oracle's components, in its (l, m) order, equal the printed forms at unit
    vectors, and, by homogeneity of degree l, |d|^l times them at any vector d."""
    forms = _printed_blm()
    assert sorted(q for q, _, _ in forms) == list(range(80))
    rng = np.random.default_rng(8)
    for d in rng.standard_normal((12, 3)) * rng.uniform(0.5, 3.0, (12, 1)):
        B, _ = oracle.blm(d, 8)
        r = float(np.linalg.norm(d))
        u = d / r
        for q, eq, f in forms:
            l = int(np.floor(np.sqrt(q + 1)))
            assert B[q] == pytest.approx(f(*u, 1.0), rel=1e-12, abs=1e-12), eq
            assert r ** l * B[q] == pytest.approx(f(*d, r), rel=1e-11, abs=1e-11 * r ** l), eq


def test_clm_normalisation_closed_forms(oracle):
    """The quadrature behind C_lm reproduces the l <= 4 values, and for m = 0,
    where b_l0(u) = k_l P_l(u_z) with k_l the ratio of the printed leading
    coefficient of z^l to the Legendre one (2l)! / (2^l l!^2),
    C_l0 = 1 / k_l^2 (the addition theorem at u = v = z-axis)."""
    from math import factorial
    C = oracle.clm(8)
    for q in range(24):
        assert oracle.clm_quadrature(q) == pytest.approx(C[q], rel=1e-13)
    lead = {1: 1, 2: 3, 3: 5, 4: 35, 5: 63, 6: 231, 7: 429, 8: 6435}  # printed coefficient of z^l (B1.1-B8.1)
    for l in range(1, 9):
        # the printed b_l0 at u = z-axis: the sum of its z, r^2 coefficients
        B, _ = oracle.blm(np.array([0.0, 0.0, 1.0]), 8)
        k = B[l * l - 1]  # = k_l P_l(1) = k_l
        assert k == pytest.approx(lead[l] / (factorial(2 * l) / (2 ** l * factorial(l) ** 2)), rel=1e-14)
        assert C[l * l - 1] == pytest.approx(1.0 / k ** 2, rel=1e-13)


# ---------------------------------------------------------------- Eq. 2

def _numpy_neighbors(batch, rc, extra=1):
    """Independent brute force: every atom pair and image within a wider range."""
    out = []
    for s in range(batch.n_struct):
        a0, a1 = batch.struct_off[s], batch.struct_off[s + 1]
        H = batch.cell[s]
        P = batch.pos[a0:a1]
        widths = abs(np.linalg.det(H)) / np.linalg.norm(np.cross(H[[1, 2, 0]], H[[2, 0, 1]]), axis=1)
        k = (np.floor(rc / widths) + 1 + extra).astype(int)
        sh = np.stack(np.meshgrid(*[np.arange(-kk, kk + 1) for kk in k], indexing="ij"), -1).reshape(-1, 3)
        for i in range(a1 - a0):
            d = P[None, :, None, :] + (sh @ H)[None, None, :, :] - P[i][None, None, None, :]
            d2 = np.sum(d[0] ** 2, axis=-1)
            jj, ss = np.nonzero(d2 < rc * rc)
            for j_, s_ in zip(jj, ss):
                if j_ == i and not sh[s_].any():
                    continue
                out.append((a0 + i, a0 + j_, *sh[s_]))
    return sorted(out)


@pytest.mark.parametrize("rc", [7.0, 4.0])
def test_neighbors_brute_force(oracle, rc):
    """Eq. 2 against a numpy brute force over a wider image range; canonical order."""
    rng = np.random.default_rng(2)
    b = synth.make_batch([32, 20, 9], [0, 2, 1], rng)
    off, j, sh = oracle.neighbors(b, rc)
    mine = []
    for i in range(b.n_atoms):
        lst = [(i, int(j[p]), *map(int, sh[p])) for p in range(off[i], off[i + 1])]
        assert lst == sorted(lst), "canonical order: j ascending then shift"
        mine.extend(lst)
    assert sorted(mine) == _numpy_neighbors(b, rc)
    # pair symmetry (i, j, n) <-> (j, i, -n)
    s = set(mine)
    assert all((jj, ii, -a, -bb, -cc) in s for (ii, jj, a, bb, cc) in mine)


def test_neighbor_counts_density(oracle):
    """Mean neighbour count ~ rho 4/3 pi rc^3 on rocksalt at rho = 0.033."""
    b = synth.make_config(1, n_struct=4)
    for rc, lo, hi in [(7.0, 40, 52), (4.0, 5.0, 10.0)]:
        off, j, _ = oracle.neighbors(b, rc)
        assert lo < len(j) / b.n_atoms < hi


# ---------------------------------------------------------------- Eqs. 5-8

@pytest.mark.parametrize("l_max", [4, 6, 8])
def test_q_nl_legendre_double_sum(oracle, l_max):
    """Eqs. 7-8 with the addition theorem: q_nl = sum_jk g_n g_n P_l(cos t_jik),
    for l up to l_max."""
    O = oracle
    cfg = small_cfg(O, l_max=l_max)
    b = small_batch()
    P = synth.uniform_params(cfg.n_params, 3).astype(np.float64)
    G = O.descriptors(cfg, P, b)
    off, jj, sh = O.neighbors(b, cfg.rc_a)
    nd = cfg.n_des
    base_cA = cfg.n_species * (nd * cfg.hidden + 2 * cfg.hidden + 1) + \
        cfg.n_species ** 2 * cfg.nq_r * cfg.k_r
    cA = P[base_cA:].reshape(cfg.n_species, cfg.n_species, cfg.nq_a, cfg.k_a)
    for i in [0, 7, 15]:
        s = np.searchsorted(b.struct_off, i, side="right") - 1
        vecs, gs = [], []
        for p in range(off[i], off[i + 1]):
            d = b.pos[jj[p]] + sh[p] @ b.cell[s] - b.pos[i]
            f, _ = O.radial_basis(cfg.k_a, cfg.rc_a, np.linalg.norm(d))
            vecs.append(d / np.linalg.norm(d))
            gs.append(cA[b.types[i], b.types[jj[p]]] @ f)
        vecs, gs = np.array(vecs), np.array(gs)
        cos = vecs @ vecs.T
        for n in range(cfg.nq_a):
            for l in range(1, l_max + 1):
                ref = np.sum(np.outer(gs[:, n], gs[:, n]) * legendre.legval(cos, [0] * l + [1]))
                assert G[i, cfg.nq_r + n * l_max + l - 1] == pytest.approx(ref, rel=1e-10, abs=1e-12)


def test_four_body_triple_sum_and_rotation(oracle):
    """4-body reading: tr(Q^3) equals the brute-force triple sum and is rotation invariant."""
    O = oracle
    cfg = small_cfg(O, four_body=True)
    b = small_batch()
    P = synth.uniform_params(cfg.n_params, 3).astype(np.float64)
    G = O.descriptors(cfg, P, b)
    off, jj, sh = O.neighbors(b, cfg.rc_a)
    nd = cfg.n_des
    base_cA = cfg.n_species * (nd * cfg.hidden + 2 * cfg.hidden + 1) + \
        cfg.n_species ** 2 * cfg.nq_r * cfg.k_r
    cA = P[base_cA:].reshape(cfg.n_species, cfg.n_species, cfg.nq_a, cfg.k_a)
    for i in [1, 12, 20]:
        s = np.searchsorted(b.struct_off, i, side="right") - 1
        As, gs = [], []
        for p in range(off[i], off[i + 1]):
            d = b.pos[jj[p]] + sh[p] @ b.cell[s] - b.pos[i]
            u = d / np.linalg.norm(d)
            f, _ = O.radial_basis(cfg.k_a, cfg.rc_a, np.linalg.norm(d))
            As.append(1.5 * np.outer(u, u) - 0.5 * np.eye(3))
            gs.append(cA[b.types[i], b.types[jj[p]]] @ f)
        As, gs = np.array(As), np.array(gs)
        for n in range(cfg.nq_a):
            ref = np.einsum("j,k,m,jab,kbc,mca->", gs[:, n], gs[:, n], gs[:, n], As, As, As)
            assert G[i, cfg.nq_r + cfg.nq_a * 4 + n] == pytest.approx(ref, rel=1e-10, abs=1e-13)
    # rotation invariance of every descriptor
    R = _rotation(np.random.default_rng(4))
    br = synth.Batch(b.struct_off, b.pos @ R.T, b.types, b.cell @ R.T)
    np.testing.assert_allclose(O.descriptors(cfg, P, br), G, rtol=1e-10, atol=1e-12)


def _rotation(rng):
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    if np.linalg.det(q) < 0:
        q[:, 0] *= -1
    return q


def test_dimer_closed_form(oracle):
    """Two atoms in a large box: q_n = g_n^R(r), q_nl = g_n^A(r)^2, q4_n = 3/4 g_n^A(r)^3."""
    O = oracle
    cfg = small_cfg(O, four_body=True)
    r = 2.9
    d = np.array([0.3, -0.5, 0.8]); d = d / np.linalg.norm(d) * r
    pos = np.array([[10.0, 10.0, 10.0], 10.0 + d])
    b = synth.Batch(np.array([0, 2], dtype=np.int32), pos, np.array([0, 1], dtype=np.int32),
                    np.eye(3)[None] * 30.0)
    P = synth.uniform_params(cfg.n_params, 8).astype(np.float64)
    G = O.descriptors(cfg, P, b)
    nd = cfg.n_des
    base_cR = cfg.n_species * (nd * cfg.hidden + 2 * cfg.hidden + 1)
    cR = P[base_cR:base_cR + 4 * cfg.nq_r * cfg.k_r].reshape(2, 2, cfg.nq_r, cfg.k_r)
    cA = P[base_cR + 4 * cfg.nq_r * cfg.k_r:].reshape(2, 2, cfg.nq_a, cfg.k_a)
    fR, _ = O.radial_basis(cfg.k_r, cfg.rc_r, r)
    fA, _ = O.radial_basis(cfg.k_a, cfg.rc_a, r)
    for i, (I, J) in enumerate([(0, 1), (1, 0)]):
        gR = cR[I, J] @ fR
        gA = cA[I, J] @ fA
        exp = np.concatenate([gR, np.repeat(gA ** 2, 4), 0.75 * gA ** 3])
        np.testing.assert_allclose(G[i], exp, rtol=1e-12, atol=1e-14)
    # forces: equal and opposite, along the bond, = -dE/dr by FD of the distance
    s = np.ones(nd)
    Ea, Es, F, W = O.forward(cfg, P, s, b)
    np.testing.assert_allclose(F[0] + F[1], 0, atol=1e-12)
    assert abs(np.dot(F[1], d) / (np.linalg.norm(F[1]) * r)) == pytest.approx(1.0, abs=1e-12)
    h = 1e-6
    def e_at(rr):
        p2 = np.array([[10.0, 10.0, 10.0], 10.0 + d / r * rr])
        bb = synth.Batch(b.struct_off, p2, b.types, b.cell)
        return O.forward(cfg, P, s, bb)[1][0]
    dEdr = (e_at(r + h) - e_at(r - h)) / (2 * h)
    assert np.dot(F[1], d / r) == pytest.approx(-dEdr, rel=1e-7)
    # isolated cluster: W = sum_i r_i (x) F_i (symmetrised)
    Wf = np.einsum("ia,ib->ab", pos, F)
    Ws = 0.5 * (Wf + Wf.T)
    exp = [Ws[0, 0], Ws[1, 1], Ws[2, 2], Ws[0, 1], Ws[1, 2], Ws[2, 0]]
    np.testing.assert_allclose(W[0], exp, rtol=1e-9, atol=1e-12)


# ---------------------------------------------------------------- D1.1-D1.6

def test_ann_derivatives_fd(oracle):
    """D1.5 and D1.6 against central differences of D1.1 (with the input scale)."""
    O = oracle
    cfg = small_cfg(O, four_body=True)
    P = synth.uniform_params(cfg.n_params, 11).astype(np.float64)
    rng = np.random.default_rng(3)
    G = rng.normal(size=cfg.n_des)
    s = rng.uniform(0.5, 2.0, size=cfg.n_des)
    E, Ep, Epp = O.ann(cfg, P, s, 1, G)
    h = 1e-6
    for v in range(cfg.n_des):
        e = np.zeros(cfg.n_des); e[v] = h
        Eph, Epph, _ = O.ann(cfg, P, s, 1, G + e)
        Emh, Epmh, _ = O.ann(cfg, P, s, 1, G - e)
        assert Ep[v] == pytest.approx((Eph - Emh) / (2 * h), rel=1e-7, abs=1e-10)
        np.testing.assert_allclose(Epp[:, v], (Epph - Epmh) / (2 * h), rtol=1e-6, atol=1e-9)
    # D1.1 by hand for element 1
    nd, H = cfg.n_des, cfg.hidden
    off = nd * H + 2 * H + 1
    W0 = P[off:off + nd * H].reshape(H, nd)
    b0 = P[off + nd * H: off + nd * H + H]
    w1 = P[off + nd * H + H: off + nd * H + 2 * H]
    b1 = P[off + nd * H + 2 * H]
    assert E == pytest.approx(w1 @ np.tanh(W0 @ (s * G) + b0) + b1, rel=1e-14)


# ---------------------------------------------------------------- Eqs. 1, 3, 4

@pytest.mark.parametrize("four_body,l_max", [(False, 4), (True, 4), (False, 8)])
def test_forces_are_minus_energy_gradient(oracle, four_body, l_max):
    """Eq. 3: F = -dE/dr (central differences, h = 1e-5 A) and sum F = 0."""
    O = oracle
    cfg = small_cfg(O, four_body=four_body, l_max=l_max)
    b = small_batch()
    P = synth.uniform_params(cfg.n_params, 3).astype(np.float64)
    s = O.descriptor_scale(cfg, P, b)
    _, Es, F, _ = O.forward(cfg, P, s, b)
    for st in range(b.n_struct):
        np.testing.assert_allclose(F[b.struct_off[st]:b.struct_off[st + 1]].sum(0), 0, atol=1e-10)
    h = 1e-5
    for i in [0, 5, 13, 21]:
        for x in range(3):
            p = b.pos.copy(); p[i, x] += h
            Ep = O.forward(cfg, P, s, synth.Batch(b.struct_off, p, b.types, b.cell))[1].sum()
            p[i, x] -= 2 * h
            Em = O.forward(cfg, P, s, synth.Batch(b.struct_off, p, b.types, b.cell))[1].sum()
            assert F[i, x] == pytest.approx(-(Ep - Em) / (2 * h), rel=1e-7, abs=1e-9)


@pytest.mark.parametrize("four_body", [False, True])
def test_virial_is_strain_derivative(oracle, four_body):
    """Eq. 4 summed: W = -dE/d(eps) for a homogeneous strain of cell and positions."""
    O = oracle
    cfg = small_cfg(O, four_body=four_body)
    b = small_batch()
    P = synth.uniform_params(cfg.n_params, 3).astype(np.float64)
    s = O.descriptor_scale(cfg, P, b)
    _, _, _, W = O.forward(cfg, P, s, b)
    h = 1e-5
    for q, (a, c) in enumerate([(0, 0), (1, 1), (2, 2), (0, 1), (1, 2), (2, 0)]):
        e = np.zeros((3, 3)); e[a, c] += 0.5; e[c, a] += 0.5
        def en(t):
            M = np.eye(3) + t * e
            return O.forward(cfg, P, s, synth.Batch(b.struct_off, b.pos @ M, b.types, b.cell @ M))[1]
        np.testing.assert_allclose(W[:, q], -(en(h) - en(-h)) / (2 * h), rtol=1e-7, atol=1e-8)


def test_invariances(oracle):
    """Translation, rotation and permutation invariance of E; F co-rotates."""
    O = oracle
    cfg = small_cfg(O, four_body=True)
    b = small_batch()
    P = synth.uniform_params(cfg.n_params, 3).astype(np.float64)
    s = O.descriptor_scale(cfg, P, b)
    Ea, Es, F, W = O.forward(cfg, P, s, b)
    bt = synth.Batch(b.struct_off, b.pos + np.array([0.31, -1.7, 2.2]), b.types, b.cell)
    np.testing.assert_allclose(O.forward(cfg, P, s, bt)[1], Es, rtol=1e-12)
    R = _rotation(np.random.default_rng(9))
    br = synth.Batch(b.struct_off, b.pos @ R.T, b.types, b.cell @ R.T)
    _, Es2, F2, _ = O.forward(cfg, P, s, br)
    np.testing.assert_allclose(Es2, Es, rtol=1e-11)
    np.testing.assert_allclose(F2, F @ R.T, atol=1e-10)
    perm = np.concatenate([np.random.default_rng(1).permutation(12),
                           12 + np.random.default_rng(2).permutation(10)])
    bp = synth.Batch(b.struct_off, b.pos[perm], b.types[perm], b.cell)
    Ea3, Es3, F3, _ = O.forward(cfg, P, s, bp)
    np.testing.assert_allclose(Es3, Es, rtol=1e-12)
    np.testing.assert_allclose(F3, F[perm], atol=1e-11)
    np.testing.assert_allclose(Ea3, Ea[perm], rtol=1e-12)


# ---------------------------------------------------------------- Eqs. 9-16

def _labels(O, cfg, b, s, **kw):
    teacher = synth.uniform_params(cfg.n_params, 99).astype(np.float64)
    return O.teacher_labels(cfg, teacher, s, b, **kw)


@pytest.mark.parametrize("four_body,form,l_max", [(False, 0, 4), (True, 0, 4), (True, 1, 4), (True, 0, 6),
                                                  (False, 0, 8)])
def test_gradient_matches_finite_differences(oracle, four_body, form, l_max):
    """dL/dtheta by the explicit App. C/D route vs central FD of the loss (h = 1e-5)."""
    O = oracle
    cfg = small_cfg(O, four_body=four_body, l_max=l_max)
    b = small_batch()
    P = synth.uniform_params(cfg.n_params, 3).astype(np.float64)
    s = O.descriptor_scale(cfg, P, b)
    y = _labels(O, cfg, b, s, lambda_e=1.0, lambda_f=1.0, lambda_v=0.1,
                lambda_l2=0.01, loss_form=form)
    _, g = O.loss_grad(cfg, P, s, b, y)
    idx = np.random.default_rng(7).choice(cfg.n_params, 64, replace=False)
    h = 1e-5
    gmax = np.abs(g).max()
    for k in idx:
        Pp = P.copy(); Pp[k] += h
        Lp = O.loss(cfg, Pp, s, b, y)[0]
        Pp[k] -= 2 * h
        Lm = O.loss(cfg, Pp, s, b, y)[0]
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * (abs(g[k]) + gmax), (k, fd, g[k])


@pytest.mark.parametrize("term", ["f", "v"])
def test_gradient_force_and_virial_terms_alone(oracle, term):
    """The mixed second-derivative terms on their own (lambda_e = 0) against FD."""
    O = oracle
    cfg = small_cfg(O, four_body=True)
    b = small_batch(seed=11)
    P = synth.uniform_params(cfg.n_params, 4).astype(np.float64)
    s = O.descriptor_scale(cfg, P, b)
    lam = dict(lambda_e=0.0, lambda_f=1.0 if term == "f" else 0.0,
               lambda_v=1.0 if term == "v" else 0.0)
    y = _labels(O, cfg, b, s, **lam)
    _, g = O.loss_grad(cfg, P, s, b, y)
    h = 1e-5
    gmax = np.abs(g).max()
    assert gmax > 0
    for k in np.random.default_rng(8).choice(cfg.n_params, 40, replace=False):
        Pp = P.copy(); Pp[k] += h
        Lp = O.loss(cfg, Pp, s, b, y)[0]
        Pp[k] -= 2 * h
        Lm = O.loss(cfg, Pp, s, b, y)[0]
        assert abs((Lp - Lm) / (2 * h) - g[k]) <= 1e-6 * (abs(g[k]) + gmax)


def test_gradient_b1_closed_form(oracle):
    """dL/db1_e = lambda_e 2/N_str sum_s (E_s/N_s - E_tar) N_{s,e}/N_s; the force and
    virial terms contribute nothing (D1.15)."""
    O = oracle
    cfg = small_cfg(O)
    b = small_batch()
    P = synth.uniform_params(cfg.n_params, 3).astype(np.float64)
    s = O.descriptor_scale(cfg, P, b)
    y = _labels(O, cfg, b, s, lambda_e=0.7, lambda_f=1.0, lambda_v=0.3)
    _, g = O.loss_grad(cfg, P, s, b, y)
    _, Es, _, _ = O.forward(cfg, P, s, b)
    ns = np.diff(b.struct_off)
    net = cfg.n_des * cfg.hidden + 2 * cfg.hidden + 1
    for e in range(2):
        nse = np.array([np.sum(b.types[b.struct_off[t]:b.struct_off[t + 1]] == e) for t in range(b.n_struct)])
        exp = 0.7 * 2 / b.n_struct * np.sum((Es / ns - y.energy) * nse / ns)
        assert g[e * net + net - 1] == pytest.approx(exp, rel=1e-12, abs=1e-15)


def test_loss_terms_definition(oracle):
    """Eqs. 9-12 on the returned terms, and the RMSE form."""
    O = oracle
    cfg = small_cfg(O)
    b = small_batch()
    P = synth.uniform_params(cfg.n_params, 3).astype(np.float64)
    s = O.descriptor_scale(cfg, P, b)
    y = _labels(O, cfg, b, s, lambda_e=0.5, lambda_f=2.0, lambda_v=0.25, lambda_l2=0.1)
    _, Es, F, W = O.forward(cfg, P, s, b)
    ns = np.diff(b.struct_off)
    Le = np.mean((Es / ns - y.energy) ** 2)
    Lf = np.mean((F - y.force) ** 2)
    Lv = np.mean((W / ns[:, None] - y.virial) ** 2)
    l2 = 0.1 * np.sum(P ** 2) / len(P)
    t = O.loss(cfg, P, s, b, y)
    np.testing.assert_allclose(t[1:], [Le, Lf, Lv], rtol=1e-12)
    assert t[0] == pytest.approx(0.5 * Le + 2.0 * Lf + 0.25 * Lv + l2, rel=1e-12)
    y.loss_form = 1
    t = O.loss(cfg, P, s, b, y)
    assert t[0] == pytest.approx(0.5 * Le ** 0.5 + 2.0 * Lf ** 0.5 + 0.25 * Lv ** 0.5 + l2, rel=1e-12)
    # the teacher's own labels give zero data loss
    teacher = synth.uniform_params(cfg.n_params, 99).astype(np.float64)
    y.loss_form = 0
    t = O.loss(cfg, teacher, s, b, y)
    assert np.all(np.abs(t[1:]) < 1e-24)


# ---------------------------------------------------------------- Adam, Eq. 17

def test_adam_first_step(oracle):
    """Kingma & Ba: the first bias-corrected step is -lr g / (|g| + eps)."""
    rng = np.random.default_rng(0)
    g = rng.normal(size=50)
    th = rng.normal(size=50); th0 = th.copy()
    m = np.zeros(50); v = np.zeros(50)
    oracle.adam(th, m, v, g, 1, 1e-3)
    np.testing.assert_allclose(th - th0, -1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    # second step by hand
    g2 = rng.normal(size=50)
    th1 = th.copy()
    oracle.adam(th, m, v, g2, 2, 1e-3)
    m2 = 0.9 * (0.1 * g) + 0.1 * g2
    v2 = 0.999 * (0.001 * g * g) + 0.001 * g2 * g2
    step = (m2 / (1 - 0.9 ** 2)) / (np.sqrt(v2 / (1 - 0.999 ** 2)) + 1e-8)
    np.testing.assert_allclose(th - th1, -1e-3 * step, rtol=1e-10)


def test_lr_schedule_eq17(oracle):
    """Eq. 17: lr(0) = lr_stop, lr(N_warmup) = lr_start, lr(N_total) = lr_stop."""
    a, z = 1e-3, 1e-5
    assert oracle.lr(a, z, 0, 10, 100) == pytest.approx(z)
    assert oracle.lr(a, z, 5, 10, 100) == pytest.approx(z + 0.5 * (a - z))
    assert oracle.lr(a, z, 10, 10, 100) == pytest.approx(a)
    assert oracle.lr(a, z, 55, 10, 100) == pytest.approx(z + (a - z) * 0.5)
    assert oracle.lr(a, z, 100, 10, 100) == pytest.approx(z)


def test_descriptor_scale_on_a_hand_made_set(oracle):
    """The input scale reading (none in the paper): s_v = 1 / (max_v - min_v)
    over the set's atoms, 1 for a constant component.  A hand-made G with a
    positive, a negative, a constant and a single-outlier column; the scaled
    columns then span exactly 1."""
    G = np.array([[1.0, -3.0, 2.5, 0.0],
                  [4.0, -1.0, 2.5, 0.0],
                  [2.0, -2.0, 2.5, 8.0]])
    s = oracle.scale_from_descriptors(G)
    np.testing.assert_array_equal(s, [1.0 / 3.0, 0.5, 1.0, 0.125])
    span = (s * G).max(axis=0) - (s * G).min(axis=0)
    np.testing.assert_allclose(span[[0, 1, 3]], 1.0, rtol=1e-15)
    # and on real descriptors it is that function of the oracle's G
    from paper_2507_00528_gb300 import synth
    cfg = oracle.Cfg()
    P = synth.uniform_params(cfg.n_params, 3).astype(np.float64)
    b = synth.make_batch([12, 9], [0, 1], np.random.default_rng(2))
    Gb = oracle.descriptors(cfg, P, b)
    np.testing.assert_array_equal(oracle.descriptor_scale(cfg, P, b),
                                  1.0 / (Gb.max(axis=0) - Gb.min(axis=0)))


# ------------------------------------------------------------ MD (Sec. III use)

def _md_cfg(oracle):
    return oracle.Cfg(nq_r=5, nq_a=5, k_r=9, k_a=9, hidden=30)


def test_md_free_flight(oracle):
    """An atom alone in a 30 A cell has no neighbours, so no force: it moves
    at constant velocity and is wrapped back into the cell."""
    from types import SimpleNamespace
    cfg = _md_cfg(oracle)
    P = np.random.default_rng(1).uniform(-0.5, 0.5, cfg.n_params)
    b = SimpleNamespace(struct_off=np.array([0, 1], dtype=np.int32), pos=np.array([[29.0, 0.5, 15.0]]),
                        types=np.array([1], dtype=np.int32), cell=np.eye(3)[None] * 30.0)
    v0 = np.array([[0.3, -0.2, 0.01]])
    traj = oracle.md_verlet(cfg, P, np.ones(cfg.n_des), b, v0, np.array([1 / 127.6]), 2.0, 5)
    x, v, F, _ = traj[-1]
    np.testing.assert_array_equal(F, 0.0)
    np.testing.assert_allclose(v, v0, rtol=0, atol=0)
    np.testing.assert_allclose(x, np.mod(b.pos + 10.0 * v0, 30.0), rtol=0, atol=1e-12)


def _md_problem(oracle):
    from paper_2507_00528_gb300 import synth
    cfg = _md_cfg(oracle)
    P = synth.uniform_params(cfg.n_params, 21).astype(np.float64)
    b = synth.make_batch([10, 7], [0, 1], np.random.default_rng(31))
    s = oracle.descriptor_scale(cfg, P, b)
    rng = np.random.default_rng(4)
    inv_m = 1.0 / np.where(b.types == 0, 121.76, 127.6)
    v0 = rng.standard_normal((b.n_atoms, 3)) * 0.004
    return cfg, P, s, b, v0, inv_m


def test_md_first_step_is_the_taylor_step(oracle):
    """After one step x = x0 + dt v0 + dt^2/2 F0/m (wrapped)."""
    cfg, P, s, b, v0, inv_m = _md_problem(oracle)
    F0 = oracle.forward(cfg, P, s, b)[2]
    x1 = oracle.md_verlet(cfg, P, s, b, v0, inv_m, 1.5, 1)[0][0]
    acc = oracle.EV_PER_A_AMU_IN_A_PER_FS2 * inv_m[:, None]
    ref = oracle.wrap(b, b.pos + 1.5 * v0 + 0.5 * 1.5 ** 2 * acc * F0)
    np.testing.assert_allclose(x1, ref, rtol=0, atol=1e-12)


def test_md_time_reversible_and_second_order(oracle):
    """Velocity Verlet is time reversible (n steps, reversed velocities, n
    steps back to the start) and its energy error is second order in dt."""
    from types import SimpleNamespace
    cfg, P, s, b, v0, inv_m = _md_problem(oracle)
    fwd = oracle.md_verlet(cfg, P, s, b, v0, inv_m, 1.0, 6)
    x6, v6 = fwd[-1][0], fwd[-1][1]
    b6 = SimpleNamespace(struct_off=b.struct_off, pos=x6, types=b.types, cell=b.cell)
    back = oracle.md_verlet(cfg, P, s, b6, -v6, inv_m, 1.0, 6)
    d = back[-1][0] - b.pos
    for k in range(b.n_struct):  # minimum image
        a0, a1 = b.struct_off[k], b.struct_off[k + 1]
        H = b.cell[k]
        f = d[a0:a1] @ np.linalg.inv(H)
        d[a0:a1] = (f - np.round(f)) @ H
    assert np.abs(d).max() < 1e-10
    np.testing.assert_allclose(-back[-1][1], v0, rtol=0, atol=1e-12)

    def drift(dt, n):
        m = 1.0 / inv_m
        e0 = oracle.forward(cfg, P, s, b)[1] + np.add.reduceat(
            0.5 * m * (v0 * v0).sum(1) / oracle.EV_PER_A_AMU_IN_A_PER_FS2, b.struct_off[:-1])
        out = 0.0
        for x, v, F, Es in oracle.md_verlet(cfg, P, s, b, v0, inv_m, dt, n):
            ke = np.add.reduceat(0.5 * m * (v * v).sum(1) / oracle.EV_PER_A_AMU_IN_A_PER_FS2, b.struct_off[:-1])
            out = max(out, np.abs(Es + ke - e0).max())
        return out
    d1, d2 = drift(2.0, 10), drift(1.0, 20)
    assert 2.8 < d1 / d2 < 5.5, (d1, d2)
