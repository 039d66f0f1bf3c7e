"""Pins of the oracle's BF16 precision contract for f_theta (mode 1).

The contract (Sec. 2.2's network as the tensor cores evaluate it): every
weight is rounded to BF16, the activations entering the two hidden-to-hidden
layers are rounded to BF16, and the features, the biases, the first layer's
sums, the activations entering the output layer and the output stay at full
precision; the gradient passes the roundings straight through.

Special networks make the 5 -> 64 -> 64 -> 64 -> 1 model collapse to a chain
of scalar operations on one unit, computed here by hand: W2 and W3 are
identities, W4 picks one unit, and the weights are BF16 numbers.  Where each
rounding sits (and where none may sit) then shows in the output to the last
bit.  The BF16 rounding used here is written independently of the oracle's:
the nearer of the two BF16 neighbours of the FP32 value, found with exact
rational arithmetic, ties to the even one.
"""
import math
import struct
from fractions import Fraction

import numpy as np
import pytest

SIZES = [5, 64, 64, 64, 1]
OFF_W1, OFF_B1 = 0, 320
OFF_W2, OFF_B2 = 384, 4480
OFF_W3, OFF_B3 = 4544, 8640
OFF_W4, OFF_B4 = 8704, 8768
N_PARAMS = 8769


def f32_bits(x):
    return struct.unpack("<I", struct.pack("<f", x))[0]


def from_bits(u):
    return struct.unpack("<f", struct.pack("<I", u))[0]


def bf16_nearest(x):
    """x (a double) to FP32, then to the nearer BF16 neighbour (ties: even)."""
    f = float(np.float32(x))
    if f == 0.0 or not math.isfinite(f):
        return f
    u = f32_bits(f)
    lo_bits = u & 0xFFFF0000
    lo = from_bits(lo_bits)
    if lo == f:
        return f
    hi = from_bits(lo_bits + 0x10000)  # next BF16 away from zero (same sign)
    d_lo, d_hi = abs(Fraction(f) - Fraction(lo)), abs(Fraction(hi) - Fraction(f))
    if d_lo < d_hi:
        return lo
    if d_hi < d_lo:
        return hi
    return lo if ((lo_bits >> 16) & 1) == 0 else hi


def silu(z):
    return z / (1.0 + math.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + math.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def chain_network(k, w1, b1, b2, b3, w4, b4):
    """Parameters whose output is the chain through unit k: row k of W1 is w1
    (BF16 numbers), W2 = W3 = I, W4 = w4 e_k; the other units' biases are
    zero, so they carry silu(0) = 0."""
    p = np.zeros(N_PARAMS)
    p[OFF_W1 + 5 * k: OFF_W1 + 5 * k + 5] = w1
    p[OFF_B1 + k] = b1
    for i in range(64):
        p[OFF_W2 + 64 * i + i] = 1.0
        p[OFF_W3 + 64 * i + i] = 1.0
    p[OFF_B2 + k] = b2
    p[OFF_B3 + k] = b3
    p[OFF_W4 + k] = w4
    p[OFF_B4] = b4
    return p


def chain_out(x, w1, b1, b2, b3, w4, b4, rounded):
    r = bf16_nearest if rounded else (lambda v: v)
    z1 = float(np.dot(w1, x)) + b1
    z2 = r(silu(z1)) + b2
    z3 = r(silu(z2)) + b3
    return w4 * silu(z3) + b4, (z1, z2, z3)


def test_independent_bf16_rounding_agrees_with_known_values():
    assert bf16_nearest(1.0 + 2.0 ** -8) == 1.0  # tie, even
    assert bf16_nearest(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6  # tie, up to even
    assert bf16_nearest(0.1) == 0.10009765625
    assert bf16_nearest(-0.1) == -0.10009765625


@pytest.mark.parametrize("k", [0, 37, 63])
def test_contract_rounds_exactly_the_hidden_to_hidden_inputs(orc, k):
    rng = np.random.default_rng(900 + k)
    # BF16 weights (the contract rounds weights; these are already BF16)
    w1 = np.array([bf16_nearest(v) for v in rng.uniform(-1.5, 1.5, 5)])
    w4 = bf16_nearest(rng.uniform(0.5, 2.0))
    # features and biases that are not BF16 numbers (they must stay exact)
    X = rng.uniform(-1.0, 1.0, (16, 5)) + 1e-7
    b1, b2, b3, b4 = 0.3141592653589793, -0.2718281828459045, 0.1234567890123, 0.0987654321
    prm = chain_network(k, w1, b1, b2, b3, w4, b4)
    got1 = orc.mlp_forward(SIZES, prm, X, mode=1)
    got0 = orc.mlp_forward(SIZES, prm, X, mode=0)
    for i, x in enumerate(X):
        ref1, _ = chain_out(x, w1, b1, b2, b3, w4, b4, rounded=True)
        ref0, _ = chain_out(x, w1, b1, b2, b3, w4, b4, rounded=False)
        assert abs(got1[i] - ref1) <= 1e-15 * max(1.0, abs(ref1)), (i, got1[i], ref1)
        assert abs(got0[i] - ref0) <= 1e-15 * max(1.0, abs(ref0)), (i, got0[i], ref0)
    # the roundings matter here: the two modes differ in most rows
    assert np.count_nonzero(np.abs(got1 - got0) > 1e-9) >= 8


def test_contract_rounds_every_weight(orc):
    # a weight that is not a BF16 number enters as its BF16 value, in every
    # layer (first, hidden, output)
    k = 5
    x = np.array([0.5, -0.25, 0.125, 1.0, -1.0])
    w1 = np.array([0.3, 0.0, 0.0, 0.0, 0.0])  # 0.3 is not a BF16 number
    prm = chain_network(k, w1, 0.0, 0.0, 0.0, 1.0, 0.0)
    prm[OFF_W2 + 64 * k + k] = 1.01  # not BF16
    prm[OFF_W3 + 64 * k + k] = 0.99  # not BF16
    prm[OFF_W4 + k] = 1.7  # not BF16
    got = orc.mlp_forward(SIZES, prm, x[None, :], mode=1)[0]
    r = bf16_nearest
    z1 = r(0.3) * 0.5
    z2 = r(1.01) * r(silu(z1))
    z3 = r(0.99) * r(silu(z2))
    ref = r(1.7) * silu(z3)
    assert abs(got - ref) <= 1e-15, (got, ref)


def test_contract_gradient_passes_roundings_straight_through(orc):
    # L = mean (f - y)^2 through unit k; with straight-through roundings the
    # derivative of each rounded activation is that of the unrounded one:
    #   dL/db4 = 2 mean(res), dL/dW4[k] = 2 mean(res silu(z3)),
    #   dL/db3[k] = 2 mean(res w4 silu'(z3)),
    #   dL/db2[k] = 2 mean(res w4 silu'(z3) silu'(z2)),
    #   dL/db1[k] = 2 mean(res w4 silu'(z3) silu'(z2) silu'(z1)),
    # with z1, z2, z3 those of the rounded forward.
    k = 21
    rng = np.random.default_rng(950)
    w1 = np.array([bf16_nearest(v) for v in rng.uniform(-1.0, 1.0, 5)])
    w4 = bf16_nearest(1.25)
    b1, b2, b3, b4 = 0.2, -0.3, 0.1, 0.05
    prm = chain_network(k, w1, b1, b2, b3, w4, b4)
    X = rng.uniform(-1.0, 1.0, (12, 5))
    Y = rng.normal(size=12) * 0.1
    L, g = orc.mlp_loss_grad(SIZES, prm, X, Y, mode=1)
    res, hz3, d3, d2, d1 = [], [], [], [], []
    for x, y in zip(X, Y):
        f, (z1, z2, z3) = chain_out(x, w1, b1, b2, b3, w4, b4, rounded=True)
        res.append(f - y)
        hz3.append(silu(z3))
        d3.append(w4 * dsilu(z3))
        d2.append(w4 * dsilu(z3) * dsilu(z2))
        d1.append(w4 * dsilu(z3) * dsilu(z2) * dsilu(z1))
    res = np.array(res)
    assert abs(L - np.mean(res ** 2)) <= 1e-15
    checks = {
        OFF_B4: 2 * np.mean(res),
        OFF_W4 + k: 2 * np.mean(res * np.array(hz3)),
        OFF_B3 + k: 2 * np.mean(res * np.array(d3)),
        OFF_B2 + k: 2 * np.mean(res * np.array(d2)),
        OFF_B1 + k: 2 * np.mean(res * np.array(d1)),
    }
    for idx, ref in checks.items():
        assert abs(g[idx] - ref) <= 1e-13 * max(1.0, abs(ref)), (idx, g[idx], ref)
    # first-layer weights: dL/dW1[k][j] = 2 mean(res w4 silu'(z3) silu'(z2) silu'(z1) x_j)
    for j in range(5):
        ref = 2 * np.mean(res * np.array(d1) * X[:, j])
        assert abs(g[OFF_W1 + 5 * k + j] - ref) <= 1e-13 * max(1.0, abs(ref))


def test_flip_variants_round_the_near_boundary_activation_the_other_way(orc):
    """mlp_flip_variants returns, for an activation within rel_eps of a BF16
    rounding boundary, the output with that activation rounded to its other
    BF16 neighbour; on the chain network the expected value is computed by
    hand with the independent rounding above."""
    k = 5
    rng = np.random.default_rng(950)
    w1 = np.array([bf16_nearest(v) for v in rng.uniform(-1.0, 1.0, 5)])
    w4, b2, b3, b4 = bf16_nearest(1.25), -0.2718281828459045, 0.1234567890123, 0.0987654321
    x = rng.uniform(-1.0, 1.0, 5)
    # first activation just below the midpoint of the BF16 pair (lo, lo + 2^-7) near 1.3
    lo = bf16_nearest(1.3)
    mid = lo + 2.0 ** -8
    h_target = mid * (1.0 - 1e-7)
    z1 = 1.3
    for _ in range(60):  # Newton on silu(z) = h_target
        z1 -= (silu(z1) - h_target) / dsilu(z1)
    b1 = z1 - float(np.dot(w1, x))
    prm = chain_network(k, w1, b1, b2, b3, w4, b4)
    _, (z1c, _, _) = chain_out(x, w1, b1, b2, b3, w4, b4, rounded=True)
    h1 = silu(z1c)
    assert bf16_nearest(h1) == lo and abs(h1 - mid) < 1e-6 * mid
    # the same chain with the first activation rounded up instead of down
    z2 = (lo + 2.0 ** -7) + b2
    z3 = bf16_nearest(silu(z2)) + b3
    flipped = w4 * silu(z3) + b4
    alts = orc.mlp_flip_variants(SIZES, prm, x, 1e-6)
    assert np.min(np.abs(alts - flipped)) <= 1e-15 * max(1.0, abs(flipped)), (alts, flipped)
    base = orc.mlp_forward(SIZES, prm, x[None, :], mode=1)[0]
    assert abs(flipped - base) > 1e-4
    # a tolerance below the activation's distance to the boundary gives no
    # variant of it
    alts_tight = orc.mlp_flip_variants(SIZES, prm, x, 1e-9)
    assert alts_tight.size == 0 or np.min(np.abs(alts_tight - flipped)) > 1e-9
