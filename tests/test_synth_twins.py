"""The torch twins of the seeded list generators (used to build full-size
device inputs) reproduce the C generators (used to regenerate sampled pixels
for the oracle) bit for bit.  Runs on the CPU."""
import numpy as np

import synth
from gpu_run import pack_f16_records
from synth import gpu_lists


def test_lists_twin_matches_c():
    import torch

    pix = torch.tensor([0, 1, 2, 99, 12345, 4194303], dtype=torch.int64)
    for dense, n_s in ((False, 20), (True, 32), (False, 64)):
        cnt, fb, rgba = gpu_lists.lists(13, 5, 7, pix, n_s, dense)
        for i, p in enumerate(pix.tolist()):
            f2, c2 = synth.one_list(13, 5, 7, p, n_s, dense)
            n = len(f2)
            assert int(cnt[i]) == n
            assert np.array_equal(fb[i, :n].numpy(), f2) and np.array_equal(rgba[i, :n].numpy(), c2)
            assert not fb[i, n:].any() and not rgba[i, n:].any()


def test_pool_and_picks_twin_match_c():
    import torch

    fb, rgba = gpu_lists.pool(13, 21, chunk=8, device="cpu")
    for r in (0, 7, 8, 20):
        f2, c2 = synth.one_list(13, synth.POOL_REQ, 0, r, synth.POOL_RUN, dense=True)
        assert np.array_equal(fb[r * 64:(r + 1) * 64].numpy(), f2)
        assert np.array_equal(rgba[r * 64:(r + 1) * 64].numpy(), c2)
    pix = torch.arange(0, 3000, dtype=torch.int64)
    for req, e, n_s, runs in ((0, 0, 8, 21), (63, 31, 64, 1 << 22), (17, 3, 37, 1000003)):
        n, first = gpu_lists.pool_picks(13, req, e, pix, n_s, runs)
        for p in (0, 1, 17, 2999):
            hn, hr, hs = synth.pool_pick(13, req, e, p, n_s, runs)
            assert (hn, hr * 64 + hs) == (int(n[p]), int(first[p]))
            assert 0 <= hs and hs + hn <= 64 and 0 <= hn <= n_s
    # a pooled list is a window of its run
    lists = synth.pooled_lists(13, 2, 1, [5, 6], 30, 21)
    for (f, c), p in zip(lists, (5, 6)):
        hn, hr, hs = synth.pool_pick(13, 2, 1, p, 30, 21)
        assert np.array_equal(f, fb[hr * 64 + hs:hr * 64 + hs + hn].numpy())


def test_dense_set_and_f16_pack():
    c, o, fb, rgba = gpu_lists.dense_set(0xC5, 0, 3, 50, 8, chunk=16, device="cpu")
    assert c.tolist() == [8] * 50 and o[-1].item() == 400
    f2, c2 = synth.one_list(0xC5, 0, 3, 33, 8, dense=True)
    assert np.array_equal(fb[33 * 8:34 * 8].numpy(), f2) and np.array_equal(rgba[33 * 8:34 * 8].numpy(), c2)
    pk = gpu_lists.pack_f16(fb, rgba, chunk=100).numpy()
    ref = pack_f16_records(fb.numpy(), rgba.numpy())
    # depths and colour bytes identical; tau computed in float32 against float64 may round to the
    # neighbouring binary16 value where the two straddle a rounding boundary
    assert np.array_equal(pk[:, 0:3], ref[:, 0:3])
    h_g = np.ascontiguousarray(pk[:, 3]).view(np.uint16).reshape(-1, 2)
    h_r = np.ascontiguousarray(ref[:, 3]).view(np.uint16).reshape(-1, 2)
    assert np.array_equal(h_g[:, 0], h_r[:, 0])
    t_g = h_g[:, 1].astype(np.int64)
    t_r = h_r[:, 1].astype(np.int64)
    assert np.abs(t_g - t_r).max() <= 1 and np.mean(t_g == t_r) > 0.99


def test_request_table():
    t = synth.requests(64)
    assert len(t) == 64 and t == synth.requests(64)
    for w, h, k, n_s in t:
        assert 256 <= w <= 1920 and 256 <= h <= 1080 and 2 <= k <= 32 and 8 <= n_s <= 64
    assert len({x[2] for x in t}) > 10
