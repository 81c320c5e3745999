"""Many images of uneven size answered in one launch (sfc_multi_*), through
the C-ABI (needs a GB300).

Bars: every target's pick and cost equal, bit for bit, to the single-image
query of its own index (sfc_query_batch), and sampled targets equal to the
oracle's query against that image's index (picks equal, costs within 1e-5);
a launch captured into a CUDA graph replays to the same results; invalid
image numbers are flagged; indices built with other parameters are refused.
The full-size case is the batched workload: 256 RGB images with sides
log-uniform in 256..2048 (~2.1e8 pixels), 9x9x3 patches, every image's front
targets (a seeded 512 per image) in one launch.
"""
import concurrent.futures as cf
import multiprocessing as mp

import numpy as np
import pytest
import torch

import oracle as O
from paper_1712_06326_gb300 import synth

pytestmark = pytest.mark.gpu

COST_RTOL = 1e-5
K = 9
PRM = dict(K=K, curves=8, dims=8, bits=16, window=64, pca_sample=16384)


@pytest.fixture(scope="module")
def S():
    import __graft_entry__

    __graft_entry__.build()
    from paper_1712_06326_gb300 import sfc

    torch.cuda.set_device(0)
    sfc.sfc_status()
    return sfc


def make_batch(sizes, cap):
    # a spawned pool (never forked after CUDA starts)
    n = len(sizes)
    with cf.ProcessPoolExecutor(max_workers=16, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(synth.batch_case, range(n), sizes, [K] * n, [cap] * n))


def run_batch(S, imgs, prm):
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    gds = [dev(g) for g, _, _ in imgs]
    mds = [dev(m) for _, m, _ in imgs]
    ixs = [S.sfc_index_build(gd, md, **prm) for gd, md in zip(gds, mds)]
    # the targets of all images, interleaved (round robin) so that neighbouring
    # CTAs work on different images
    order = []
    for k in range(max(len(t) for _, _, t in imgs)):
        order += [(i, k) for i, (_, _, t) in enumerate(imgs) if k < len(t)]
    img_of = np.array([i for i, _ in order], np.int32)
    cen = np.stack([imgs[i][2][k] for i, k in order]).astype(np.int32)
    mu = S.Multi(ixs, gds, mds)
    pk, cs = mu.query(dev(img_of), dev(cen))
    return gds, mds, ixs, mu, img_of, cen, pk, cs


def check_against_single(S, imgs, gds, mds, ixs, img_of, cen, pk, cs):
    pk, cs = pk.cpu().numpy(), cs.cpu().numpy()
    for i in range(len(imgs)):
        sel = np.flatnonzero(img_of == i)
        if len(sel) == 0:
            continue
        p1, c1 = S.sfc_query_batch(ixs[i], gds[i], mds[i], torch.from_numpy(cen[sel]).cuda())
        assert np.array_equal(pk[sel], p1.cpu().numpy())
        assert np.array_equal(cs[sel].view(np.uint32), c1.cpu().numpy().view(np.uint32))
    return pk, cs


def check_sampled_oracle(S, imgs, ixs, img_of, cen, pk, cs, count, seed):
    rng = np.random.default_rng(seed)
    for q in rng.choice(len(img_of), count, replace=False):
        i = int(img_of[q])
        g, m, _ = imgs[i]
        ex = S.sfc_index_export(ixs[i])
        ndim, ext, ch = O.geometry(g)
        oq = dict(ndim=ndim, ext=ext, ch=ch, K=K, C=PRM["curves"], D=PRM["dims"], bits=PRM["bits"], dict=ex["dict"],
                  N=len(ex["dict"]), subset=np.ascontiguousarray(ex["subsets"]), m=ex["subsets"].shape[1],
                  basis=ex["basis"], mean=ex["mean"], lo=ex["lo"], scale=ex["scale"], skeys=ex["skeys"],
                  sids=ex["sids"], shifts=None)
        r = O.query(oq, g, m, int(O.centres_to_lin(cen[q:q + 1], ext)[0]), PRM["window"])
        assert pk[q] == r["pick"]
        assert abs(float(cs[q]) - r["cost"]) <= COST_RTOL * r["cost"] and (cs[q] == 0) == (r["cost"] == 0)


def test_multi_small_batch_graph_and_errors(S):
    sizes = synth.batch_sizes(12, cfg=4, lo=64, hi=192, seed_sub=1)
    imgs = make_batch(sizes, cap=40)
    gds, mds, ixs, mu, img_of, cen, pk, cs = run_batch(S, imgs, PRM)
    pk, cs = check_against_single(S, imgs, gds, mds, ixs, img_of, cen, pk, cs)
    check_sampled_oracle(S, imgs, ixs, img_of, cen, pk, cs, 24, 0)
    assert S.sfc_status() == 0
    # one launch captured into a CUDA graph and replayed
    im_d = torch.from_numpy(img_of).cuda()
    cen_d = torch.from_numpy(cen).cuda()
    pb = torch.empty(len(img_of), dtype=torch.int64, device="cuda")
    cb = torch.empty(len(img_of), dtype=torch.float32, device="cuda")
    mu.query(im_d, cen_d, pb, cb)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        mu.query(im_d, cen_d, pb, cb)
    pb.fill_(-7)
    graph.replay()
    torch.cuda.synchronize()
    assert np.array_equal(pb.cpu().numpy(), pk) and np.array_equal(cb.cpu().numpy().view(np.uint32), cs.view(np.uint32))
    # image numbers outside [0, n)
    bad = im_d.clone()
    bad[0] = len(imgs)
    bad[1] = -1
    p2, c2 = mu.query(bad, cen_d)
    p2 = p2.cpu().numpy()
    assert p2[0] == -1 and p2[1] == -1 and np.array_equal(p2[2:], pk[2:])
    assert S.sfc_status() == S.SFC_EDEVICE
    assert S.sfc_status() == 0
    # indices built with other parameters
    other = S.sfc_index_build(gds[0], mds[0], **dict(PRM, window=32))
    with pytest.raises(RuntimeError, match="other parameters"):
        S.Multi([ixs[0], other], gds[:2], mds[:2])
    mu.close()


def test_multi_full_size_batch(S):
    sizes = synth.batch_sizes(256, cfg=4)
    imgs = make_batch(sizes, cap=512)
    gds, mds, ixs, mu, img_of, cen, pk, cs = run_batch(S, imgs, PRM)
    assert len(img_of) > 100_000
    pk, cs = check_against_single(S, imgs, gds, mds, ixs, img_of, cen, pk, cs)
    assert np.all(pk >= 0)
    check_sampled_oracle(S, imgs, ixs, img_of, cen, pk, cs, 16, 1)
    assert S.sfc_status() == 0
    mu.close()
