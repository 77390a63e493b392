"""Pins of the oracle's learned-gamma parts (an extension of the method; the
paper searches gamma per ray, sec. 2.4): tile features, tile labels and the
40-64-64-1 MLP with its gradient."""
import numpy as np
import pytest

import oracle
import synth

RNG = np.random.default_rng(99)
NP = 64 * 40 + 64 + 64 * 64 + 64 + 64 + 1


def rand_theta(scale=0.3):
    return RNG.normal(0, scale, NP)


def unpack(th):
    o = 0
    W1 = th[o:o + 64 * 40].reshape(64, 40); o += 64 * 40
    b1 = th[o:o + 64]; o += 64
    W2 = th[o:o + 64 * 64].reshape(64, 64); o += 64 * 64
    b2 = th[o:o + 64]; o += 64
    w3 = th[o:o + 64]; o += 64
    return W1, b1, W2, b2, w3, th[o]


def test_parameter_count():
    assert oracle.mlp_nparams() == NP == 6849


def test_forward_zero_weights_gives_output_bias():
    th = np.zeros(NP)
    th[-1] = -3.25
    x = RNG.normal(size=(7, 40))
    assert np.all(oracle.mlp_forward(th, x) == -3.25)


def test_forward_linear_region_is_matrix_product():
    # positive weights and biases and non-negative inputs keep every ReLU in its linear
    # region, where the network is the composed affine map
    th = np.abs(rand_theta(0.1))
    W1, b1, W2, b2, w3, b3 = unpack(th)
    x = np.abs(RNG.normal(size=(5, 40)))
    expect = (x @ (w3 @ W2 @ W1).T) + w3 @ (W2 @ b1 + b2) + b3
    assert np.allclose(oracle.mlp_forward(th, x), expect, rtol=1e-12)


def test_forward_relu_cuts_negative_units():
    th = np.zeros(NP)
    W1, b1, W2, b2, w3, b3 = [np.asarray(a) for a in unpack(th)]
    # unit 0 of layer 1 copies feature 0, unit 1 copies minus feature 0; layer 2 sums both; output reads it
    th[0] = 1.0            # W1[0, 0]
    th[40] = -1.0          # W1[1, 0]
    o2 = 64 * 40 + 64
    th[o2 + 0] = 1.0       # W2[0, 0]
    th[o2 + 1] = 1.0       # W2[0, 1]
    o3 = o2 + 64 * 64 + 64
    th[o3 + 0] = 1.0       # w3[0]
    x = np.zeros((2, 40))
    x[0, 0], x[1, 0] = 2.5, -1.5
    assert np.allclose(oracle.mlp_forward(th, x), [2.5, 1.5])  # |x0|


def test_gradient_matches_finite_differences():
    th = rand_theta(0.2)
    x = RNG.normal(size=(9, 40))
    y = RNG.normal(size=9)
    valid = np.array([1, 1, 0, 1, 1, 1, 0, 1, 1], dtype=np.int32)
    loss, g = oracle.mlp_loss_grad(th, x, y, valid)
    pred = oracle.mlp_forward(th, x)
    m = valid.sum()
    assert loss == pytest.approx(np.sum(valid * (pred - y) ** 2) / m, rel=1e-12)
    idx = RNG.choice(NP, 80, replace=False)
    idx = np.concatenate([idx, [NP - 1, NP - 2, 0, 64 * 40]])
    h = 1e-6
    for i in idx:
        tp, tm = th.copy(), th.copy()
        tp[i] += h
        tm[i] -= h
        fd = (oracle.mlp_loss_grad(tp, x, y, valid)[0] - oracle.mlp_loss_grad(tm, x, y, valid)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), (i, fd, g[i])


def test_invalid_rows_do_not_contribute():
    th = rand_theta()
    x = RNG.normal(size=(4, 40))
    y = RNG.normal(size=4)
    l1, g1 = oracle.mlp_loss_grad(th, x[:2], y[:2])
    l2, g2 = oracle.mlp_loss_grad(th, x, y, np.array([1, 1, 0, 0], dtype=np.int32))
    assert l1 == pytest.approx(l2) and np.allclose(g1, g2)
    l3, g3 = oracle.mlp_loss_grad(th, x, y, np.zeros(4, dtype=np.int32))
    assert l3 == 0.0 and np.all(g3 == 0)


def test_tile_labels_lower_median():
    W, H = 20, 17  # two tile columns (16 + 4), two rows (16 + 1)
    k = 2
    g = RNG.uniform(0, 1, (k, W * H))
    nts = RNG.integers(0, 3, (k, W * H))
    g[0, :5] = 0.0  # gamma 0 -> floor 2^-20
    labels, valid = oracle.tile_labels(g, nts, W, H)
    for e in range(k):
        for t in range(4):
            tx, ty = t % 2, t // 2
            vals = []
            for j in range(ty * 16, min(H, ty * 16 + 16)):
                for i in range(tx * 16, min(W, tx * 16 + 16)):
                    p = j * W + i
                    if nts[e, p] > 0:
                        vals.append(np.log2(max(g[e, p], 2.0 ** -20)))
            assert valid[e, t] == (len(vals) > 0)
            if vals:
                assert labels[e, t] == sorted(vals)[(len(vals) - 1) // 2]


def test_tile_features_homogeneous_volume():
    # constant volume and table: every sample has the same opacity a', so the histogram
    # has one full bin; first non-transparent depth 0; every ray with samples counts
    dims = (24, 24, 24)
    vol = np.full(dims, 0.5, dtype=np.float32)
    lut = np.zeros((256, 4), dtype=np.float32)
    lut[:, :3] = 0.5
    lut[:, 3] = 0.3
    cam = synth.orbit(dims, 1, 32, 32, 9)[0]
    boxes = oracle.split_boxes(dims, (1, 2, 1))
    F, valid = oracle.tile_features(vol, boxes, lut, cam, 0.5, 1.0, 12)
    a = 1 - (1 - float(np.float32(0.3))) ** 0.5
    b = int(np.floor(a * 64))
    for e in range(2):
        for t in range(4):
            if not valid[e, t]:
                assert np.all(F[e, t] == 0)
                continue
            assert F[e, t, b] == pytest.approx(1.0) and F[e, t, :32].sum() == pytest.approx(1.0)
            assert F[e, t, 32] == 0.0 and F[e, t, 33] == 0.0  # first sample is non-transparent
            assert F[e, t, 37] == 12 / 64 and F[e, t, 38] == 1.0
            assert F[e, t, 39] == 0.0  # no colour variation
    assert valid.sum() >= 4


def test_tile_features_relations_real_volume(tiny_workload):
    w = tiny_workload
    cam = w["cams"][0]
    F, valid = oracle.tile_features(w["vol"], w["boxes"], w["lut"], cam, w["step"], w["ref_len"], 8)
    nz = valid.astype(bool)
    hs = F[..., :32].sum(-1)
    assert np.all((np.abs(hs[nz] - 1) < 1e-12) | (hs[nz] == 0))
    assert np.all(F[..., 34][nz] >= F[..., 32][nz])  # last back >= first front
    assert np.all((F[..., 38] >= 0) & (F[..., 38] <= 1))
    assert np.all(F[..., 33] >= 0) and np.all(F[..., 35] >= 0)
    # the non-transparent count feature matches the gamma = 0 counts of generation
    cnt0, _, _, _ = oracle.generate(w["vol"], w["boxes"], w["lut"], cam, w["step"], w["ref_len"], 10 ** 6, 0.0,
                                    maxrec=1, records=False)
    W = cam.width
    for e in range(2):
        for t in range(0, 64, 7):
            tx, ty = t % 8, t // 8
            pix = [(ty * 16 + jj) * W + tx * 16 + ii for jj in range(0, 16, 2) for ii in range(0, 16, 2)]
            # rays with owned samples are not known here; the mean over rays with a non-transparent
            # sample bounds the feature from above
            tot = cnt0[e, pix].sum()
            with_nt = (cnt0[e, pix] > 0).sum()
            if with_nt and valid[e, t]:
                assert np.log1p(tot / with_nt) / 8 >= F[e, t, 36] - 1e-12
