"""The batched BF16 form: many pairs of uneven sizes per call, the CUDA-graph capture of
a batch signature and the autotuner.

Launch shape (strip height, N slice) and graph replay change nothing in the arithmetic of
an output element (same MMAs in the same K order), so outputs must be bit-identical to the
eager, untuned call; the eager call itself is checked against the oracle in
test_gpu_bf16.py."""
import os

import numpy as np
import pytest
import torch

import oracle
import parity
from paper_2305_11566_gb300 import binding, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def batch():
    pairs = synth.batch_uneven(6, seed=9100)
    return [p for p, _ in pairs], [binding.to_device(p, D) for p, D in pairs]


def make_ctx(shape=synth.NET_WIDE, k=9):
    c = binding.Context(shape, k, "bf16")
    c.set_weights(synth.he_normal_weights(shape, 7))
    return c


def run(ctx, dps, stream):
    with torch.cuda.stream(stream):
        outs = ctx.pipeline(dps)
    stream.synchronize()
    ctx.synchronize(stream)
    return [o.clone() for o in outs]


def test_graph_replay_equals_eager(svlib, batch):
    pairs, dps = batch
    s = torch.cuda.Stream()
    eager = make_ctx()
    graph = make_ctx()
    try:
        eager.set_option("graphs", 0)
        ref = run(eager, dps, s)
        outs = [torch.empty_like(r) for r in ref]
        with torch.cuda.stream(s):
            graph.pipeline(dps, out=outs)        # capture + first replay
            n0 = graph.launch_count()
            for o in outs:
                o.fill_(-1)
            graph.pipeline(dps, out=outs)        # replay
            n1 = graph.launch_count()
        s.synchronize()
        graph.synchronize(s)
        for a, b in zip(outs, ref):
            assert torch.equal(a, b)
        assert n1 - n0 > len(dps)                # the replay counts its kernels
        # a different output buffer is a different signature: recaptured, same result
        outs2 = [torch.empty_like(r) for r in ref]
        with torch.cuda.stream(s):
            graph.pipeline(dps, out=outs2)
        s.synchronize()
        for a, b in zip(outs2, ref):
            assert torch.equal(a, b)
        # every pair of the replayed graph against the oracle, outside the reach of WTA near ties
        params = synth.he_normal_weights(synth.NET_WIDE, 7)
        coarse = graph.coarse_match(dps)
        for p, dp, o, d in zip(pairs, dps, outs, coarse):
            Y_o, disp_o, best_o, sec_o = oracle.pipeline(synth.NET_WIDE, params, p.left, p.right, 9, dp.max_disp)
            keep = parity.keep_mask(parity.wta_differences(d.cpu().numpy(), disp_o, best_o, sec_o), p.height, p.width)
            parity.compare_refined(o.cpu().numpy(), Y_o, keep, 0.05, 0.01, p.gt, 0.01, f"graph {p.width}x{p.height}")
    finally:
        eager.close()
        graph.close()


def test_autotune_keeps_results_and_caches(svlib, batch, tmp_path):
    pairs, dps = batch
    s = torch.cuda.Stream()
    base = make_ctx()
    tuned = make_ctx()
    again = make_ctx()
    try:
        ref = run(base, dps, s)
        cache = os.path.join(tmp_path, "tune.jsonl")
        choice = tuned.autotune(dps, cache, stream=s)
        assert all(u > 0 for u in choice["us"])
        out = run(tuned, dps, s)
        for a, b in zip(out, ref):
            assert torch.equal(a, b)
        assert os.path.exists(cache)
        loaded = again.autotune(dps, cache, stream=s)
        assert loaded["rows"] == choice["rows"] and loaded["nt"] == choice["nt"] and loaded["ctas"] == choice["ctas"]
        assert all(u == -1.0 for u in loaded["us"])
        out2 = run(again, dps, s)
        for a, b in zip(out2, ref):
            assert torch.equal(a, b)
        # the unfused decoder tail under the tuned plan (its own launch shapes) as well
        base.set_option("fused_final", 0)
        tuned.set_option("fused_final", 0)
        for a, b in zip(run(tuned, dps, s), run(base, dps, s)):
            assert torch.equal(a, b)
    finally:
        base.close()
        tuned.close()
        again.close()


def test_autotune_rejects_plain_form(svlib, batch):
    _, dps = batch
    c = binding.Context(synth.NET_SMALL, 9, "fp32")
    try:
        with pytest.raises(binding.SvError) as ei:
            c.autotune(dps)
        assert ei.value.status == binding.SV_ERR_UNSUPPORTED
    finally:
        c.close()


@pytest.mark.parametrize("pinned,mode", [(True, 0), (True, 1), (True, 2), (False, 2)])
def test_pipeline_host_buffers(svlib, batch, pinned, mode):
    """sv_pipeline_host: host images in, host disparity maps out, through copy calls (mode
    0), a gather kernel (1) or gather and scatter kernels (2) over the CPU-GPU link for
    pinned buffers; pageable buffers always take copy calls.  All must give exactly the
    device-buffer pipeline's result (same kernels).
    Odd pitches and an unaligned row start exercise the byte-wise copy path."""
    pairs, dps = batch
    s = torch.cuda.Stream()
    ctx = make_ctx()
    try:
        ref = run(ctx, dps, s)
        ctx.set_option("host_copy", mode)
        Ls, Rs, outs, Ws, Hs, ps, Ds = [], [], [], [], [], [], []
        for i, (p, dp) in enumerate(zip(pairs, dps)):
            H, W = p.left.shape
            extra = 3 if i % 2 else 16                 # odd pitch for every other pair
            lh = np.zeros((H, W + extra), np.uint8)
            rh = np.zeros((H, W + extra), np.uint8)
            lh[:, :W] = p.left
            rh[:, :W] = p.right
            o = np.zeros((H, W), np.float32)
            if pinned:
                lh = torch.from_numpy(lh).pin_memory()
                rh = torch.from_numpy(rh).pin_memory()
                o = torch.from_numpy(o).pin_memory()
            Ls.append(lh)
            Rs.append(rh)
            outs.append(o)
            Ws.append(W)
            Hs.append(H)
            ps.append(W + extra)
            Ds.append(dp.max_disp)
        ctx.pipeline_host(Ls, Rs, Ws, Hs, ps, Ds, outs, stream=s)
        for o, r in zip(outs, ref):
            got = o.numpy() if pinned else o
            assert np.array_equal(got, r.cpu().numpy())
    finally:
        ctx.close()


def test_pipeline_host_two_halves(svlib):
    """16 or more pairs: sv_pipeline_host computes the batch in two halves and copies the
    first half's results back while the second half computes; the result must equal the
    device-buffer pipeline's for every pair."""
    pairs = synth.batch_uneven(16, seed=9300)
    dps = [binding.to_device(p, D) for p, D in pairs]
    s = torch.cuda.Stream()
    ctx = make_ctx()
    try:
        ref = run(ctx, dps, s)
        Ls = [torch.from_numpy(synth.pitched(p.left)).pin_memory() for p, _ in pairs]
        Rs = [torch.from_numpy(synth.pitched(p.right)).pin_memory() for p, _ in pairs]
        outs = [torch.zeros((p.height, p.width), dtype=torch.float32).pin_memory() for p, _ in pairs]
        ctx.pipeline_host(Ls, Rs, [p.width for p, _ in pairs], [p.height for p, _ in pairs],
                          [x.shape[1] for x in Ls], [D for _, D in pairs], outs, stream=s)
        for o, r in zip(outs, ref):
            assert torch.equal(o, r.cpu())
    finally:
        ctx.close()


def test_signature_replay_across_batches_and_options(svlib, batch):
    """Graphs replayed from the call signature alone (no table preparation): alternating two
    batches replays each one's own graph (outputs and the per-pair activation offsets of the
    replayed batch), and a changed launch option (the fused decoder tail off) is a new
    signature, not a stale replay."""
    pairs, dps = batch
    other = synth.batch_uneven(4, seed=9200)
    dps2 = [binding.to_device(p, D) for p, D in other]
    s = torch.cuda.Stream()
    ctx = make_ctx()
    try:
        a1 = run(ctx, dps, s)
        b1 = run(ctx, dps2, s)
        a2 = run(ctx, dps, s)
        for x, y in zip(a1, a2):
            assert torch.equal(x, y)
        # the replayed batch's activation offsets: pair 1 of the first batch reads its e1 shape
        H, W = pairs[1].left.shape
        L1 = oracle.level_sizes(H, W)[1]
        e1 = ctx.debug_activation(0, 1, (*L1, synth.NET_WIDE.enc[0]))
        b2 = run(ctx, dps2, s)
        for x, y in zip(b1, b2):
            assert torch.equal(x, y)
        run(ctx, dps, s)
        assert np.array_equal(ctx.debug_activation(0, 1, (*L1, synth.NET_WIDE.enc[0])), e1)
        # the last decoder activation stays on chip with the fused tail; with it off it is kept
        with pytest.raises(binding.SvError):
            ctx.debug_activation(6, 0, (*pairs[0].left.shape, synth.NET_WIDE.dec[2]))
        ctx.set_option("fused_final", 0)
        a3 = run(ctx, dps, s)
        d3 = ctx.debug_activation(6, 0, (*pairs[0].left.shape, synth.NET_WIDE.dec[2]))
        assert np.isfinite(d3).all() and np.abs(d3).max() > 0
        for x, y in zip(a1, a3):  # the unfused tail: same layers, FP32 final conv on CUDA cores
            assert torch.allclose(x, y, atol=0.05, rtol=0)
    finally:
        ctx.close()
