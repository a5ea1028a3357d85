"""Oracle against hand-worked cases stored under tests/golden/.

Each fixture states its source equations and the hand derivation of every
stored value (exact fractions); none of the values comes from code.  The
cases are chosen so that a plausible slip in the oracle fails one of them: a
wrong scaled distance or scale parameter in Eq. bh-scaled, a wrong exponent
pairing in Eq. bh-u, a wrong nucleus-type lookup, the cusp prefactor, the
pivot weighting w_g w_h, the argmax tie rule, the gradient-channel product
t1 t2, the fusion order, and the index placement and derivative side of
Eqs. K1-isdf and K3-isdf.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

from synth.workloads import Jastrow, radial_jastrow
from oracle import jastrow, pivots, wbuild

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _frac(s: str) -> float:
    return float(Fraction(s))


def _rows(s: str) -> np.ndarray:
    return np.array([[_frac(x) for x in r.split()] for r in s.split("|")])


def _data_lines(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.rstrip("\n") for ln in f if ln.strip() and not ln.startswith("#")]


def _blocks(name):
    out, cur = [], {}
    with open(os.path.join(GOLDEN, name)) as f:
        for ln in f:
            if ln.startswith("#"):
                continue
            if not ln.strip():
                if cur:
                    out.append(cur)
                cur = {}
                continue
            k, v = ln.split(":", 1)
            cur[k.strip()] = v.strip()
    if cur:
        out.append(cur)
    return out


BH_ROWS = [ln.split() for ln in _data_lines("bh_terms.txt")]

R_I = np.array([[3.0, 0.0, 0.0]])
R_J = np.array([[0.0, 4.0, 0.0]])


def _bh_case(row) -> Jastrow:
    kind, b0, b1, d, m, n, o, c0, c1 = row[:9]
    d = _frac(d)
    if kind == "cusp":
        return Jastrow(nuc_xyz=np.zeros((1, 3)), nuc_type=np.zeros(1, np.int32),
                       mno=np.zeros((0, 3), np.int32), coef=np.zeros((1, 0)),
                       b=np.array([_frac(b0)]), d=d, cusp=True)
    mno = np.array([[int(m), int(n), int(o)]], np.int32)
    if kind == "one":
        return Jastrow(nuc_xyz=np.zeros((1, 3)), nuc_type=np.zeros(1, np.int32), mno=mno,
                       coef=np.array([[_frac(c0)]]), b=np.array([_frac(b0)]), d=d,
                       cusp=False)
    assert kind == "two"
    return Jastrow(nuc_xyz=np.array([[0.0, 0.0, 0.0], [3.0, 4.0, 0.0]]),
                   nuc_type=np.array([0, 1], np.int32), mno=mno,
                   coef=np.array([[_frac(c0)], [_frac(c1)]]),
                   b=np.array([_frac(b0), _frac(b1)]), d=d, cusp=False)


@pytest.mark.parametrize("row", BH_ROWS, ids=["-".join(r[:7]) for r in BH_ROWS])
def test_bh_value_and_gradient_against_hand_fractions(row):
    jas = _bh_case(row)
    u_exp = _frac(row[9])
    g_exp = np.array([_frac(x) for x in row[10:13]])
    u = jastrow.u_value(R_I, R_J, jas)[0, 0]
    g = jastrow.grad1_u(R_I, R_J, jas)[:, 0, 0]
    assert abs(u - u_exp) <= 4e-16 * max(1.0, abs(u_exp))
    assert np.max(np.abs(g - g_exp)) <= 4e-16
    # the kernels K_c of the W build are this gradient
    K = jastrow.kernels(R_I, R_J, jas)
    assert np.max(np.abs(K[:3, 0, 0] - g_exp)) <= 4e-16
    assert abs(K[3, 0, 0] - float(np.sum(g_exp * g_exp))) <= 4e-16


PHI = np.array([[1.0, 0.0, 1.0], [0.0, 1.0, 1.0]])   # [n_orb][n_g]


@pytest.mark.parametrize("case", _blocks("pivots_three_points.txt"), ids=lambda c: c["case"])
def test_pivots_against_hand_steps(case):
    w = np.array([_frac(x) for x in case["w"].split()])
    dphi = np.zeros((3, 2, 3))
    dphi[0] = _rows(case["dphi_x"])
    res = pivots.select(PHI, dphi, w, int(case["n_mu"]), mode=case["mode"])
    exp = [int(x) for x in case["pivots"].split()]
    assert res.pivots.tolist() == exp
    assert res.rank_exhausted == bool(int(case["exhausted"]))
    if "num" not in case:
        return
    dstar = np.array([_frac(x) for x in case["dstar"].split()])
    L_exp = _rows(case["num"]) / np.sqrt(dstar)[:, None]
    L = res.L_s if case["mode"] == "scalar" else res.L_v
    assert L.shape == L_exp.shape
    assert np.max(np.abs(L - L_exp)) <= 1e-15


def test_fused_channel_lists():
    """Fused run of the last fixture case: the scalar channel took points 2
    and 0, the gradient channel point 1 (one step each way, scalar first)."""
    case = _blocks("pivots_three_points.txt")[-1]
    dphi = np.zeros((3, 2, 3))
    dphi[0] = _rows(case["dphi_x"])
    res = pivots.select(PHI, dphi, np.ones(3), 3, mode="fused")
    assert res.piv_s.tolist() == [2, 0]
    assert res.piv_v.tolist() == [1]


def test_w_two_points_against_hand_fractions():
    f = _blocks("w_two_points.txt")[0]
    grid = _rows(f["points"])
    w = np.array([_frac(x) for x in f["w"].split()])
    xi = _rows(f["xi"])
    xit = np.stack([_rows(f["xit_x"]), _rows(f["xit_y"]), _rows(f["xit_z"])])
    W_exp = np.stack([_rows(f[k]) for k in ("W_x", "W_y", "W_z", "W_sq")])
    jas = radial_jastrow(np.zeros((1, 3)))
    W, _ = wbuild.build(grid, w, xi, xit, jas)
    assert np.max(np.abs(W - W_exp)) <= 1e-17
    assert np.max(np.abs(wbuild.brute_force(grid, w, xi, xit, jas) - W_exp)) <= 1e-17


@pytest.mark.parametrize("case", _blocks("pivots_fixed_rank.txt"),
                         ids=lambda c: f"{c['n_phi']}-{c['n_grad']}")
def test_fixed_rank_fusion_against_hand_steps(case):
    """The paper's fusion: each channel to its own rank, then the union."""
    dphi = np.zeros((3, 2, 3))
    dphi[0] = _rows("0 2 0 | 0 0 1")
    res = pivots.select_ranks(PHI, dphi, np.ones(3), int(case["n_phi"]), int(case["n_grad"]))
    assert res.pivots.tolist() == [int(x) for x in case["pivots"].split()]
    assert res.rank_exhausted == bool(int(case["exhausted"]))


def _sparse(s, shape):
    a = np.zeros(shape)
    for item in s.split():
        parts = item.split(",")
        idx = tuple(int(x) for x in parts[:-1])
        a[idx] = _frac(parts[-1])
    return a


def test_mlp_forward_against_hand_fractions():
    """Oracle forward pass of the proposer network on a sparse dyadic network
    whose activations were worked by hand (some ReLUs on, some off)."""
    from oracle import mlp
    f = _blocks("mlp_forward.txt")[0]
    H, F = mlp.H, mlp.F
    theta = np.concatenate([_sparse(f["W1"], (H, F)).ravel(), _sparse(f["b1"], (H,)),
                            _sparse(f["W2"], (H, H)).ravel(), _sparse(f["b2"], (H,)),
                            _sparse(f["W3"], (H,)), [_frac(f["b3"])]])
    assert theta.size == mlp.N_PARAMS
    x = _rows(f["x"])
    for rounding in (True, False):   # dyadic weights are exact in BF16
        s, (_, _, h1, _, h2) = mlp.forward(theta, x, rounding=rounding)
        assert s.tolist() == [_frac(v) for v in f["s"].split()]
        for r, (e1, e2) in enumerate(zip(f["h1"].split("|"), f["h2"].split("|"))):
            assert np.array_equal(h1[r], _sparse(e1, (H,)))
            assert np.array_equal(h2[r], _sparse(e2, (H,)))


def test_mlp_features_against_hand_values():
    from oracle import mlp
    f = _blocks("mlp_features.txt")[0]
    phi = np.array([[_frac(v)] for v in f["phi"].split()])            # [n_orb][1]
    dphi = np.stack([np.array([[_frac(v)] for v in f[k].split()])
                     for k in ("dphi_x", "dphi_y", "dphi_z")])         # [3][n_orb][1]
    w = np.array([_frac(f["w"])])
    nuc = _rows(f["nuclei"])
    got = mlp.features(phi, dphi, w, np.zeros((1, 3)), nuc)[0]
    exp = np.array([_frac(v) for v in f["features"].split()])
    assert np.max(np.abs(got - exp)) <= 1e-15


def test_tie_margin_on_hand_case():
    """The near-tie measure used when two machines' pivot lists differ: in the
    unit case points 0 and 1 tie at step 1 (d = 3/4 each), while at step 0
    point 0 trails point 2 by (4 - 1)/4."""
    dphi = np.zeros((3, 2, 3))
    assert pivots.tie_margin(PHI, dphi, np.ones(3), [2, 0, 1], [2, 1, 0], "scalar") == (1, 0.0)
    assert pivots.tie_margin(PHI, dphi, np.ones(3), [2, 0, 1], [0, 1, 2], "scalar") == (0, 0.75)
    assert pivots.tie_margin(PHI, dphi, np.ones(3), [2, 0, 1], [2, 0, 1], "scalar") == (None, 0.0)
