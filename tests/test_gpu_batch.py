"""Batched contractions: every problem of a batch equals the same problem
run alone (bit for bit: the same kernels and plan), and a sample matches the
oracle; the batch replays correctly from a captured CUDA graph."""
import pytest
import torch

import paper_1802_02619_gb300 as lco
import synth
from gpu_util import assert_contract_matches

pytestmark = pytest.mark.gpu


def _dev(T):
    if isinstance(T["liv"], torch.Tensor):
        return lco.LcoTensor(list(T["dims"]), list(T["sig"]), T["liv"].cuda(), T["val"].cuda())
    return lco.LcoTensor.from_host(T, "cuda")


def _host(T):
    if isinstance(T["liv"], torch.Tensor):
        return {"dims": T["dims"], "sig": T["sig"], "liv": T["liv"].cpu().numpy(), "val": T["val"].cpu().numpy()}
    return T


def _small_batch(count=32, seed=7):
    return synth.batch_problems(count=count, seed=seed, fd2d=(5, 24), fd3d=(4, 10), rmat_nnz=(200, 5000))


def test_batch_equals_single_calls_and_oracle():
    probs = _small_batch()
    items = [(_dev(A), _dev(B), ma, mb) for A, B, ma, mb, _ in probs]
    b = lco.Batch(items, nstreams=8)
    b.run()
    outs = b.results()
    for i, ((A, B, ma, mb, kind), C) in enumerate(zip(probs, outs)):
        ref = lco.contract(items[i][0], items[i][1], ma, mb)
        assert torch.equal(C.liv, ref.liv), f"problem {i} ({kind}) pattern differs from the single call"
        assert torch.equal(C.val.view(torch.int64), ref.val.view(torch.int64)), f"problem {i} values differ"
        if i % 4 == 0:
            assert_contract_matches(C, _host(A), _host(B), ma, mb)


def test_batch_graph_replay():
    probs = _small_batch(count=16, seed=9)
    items = [(_dev(A), _dev(B), ma, mb) for A, B, ma, mb, _ in probs]
    b = lco.Batch(items, nstreams=4)
    b.run()
    first = [(C.liv.clone(), C.val.clone()) for C in b.results()]
    b.c_liv_all.zero_()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            b.run()
    torch.cuda.current_stream().wait_stream(s)
    g.replay()
    torch.cuda.synchronize()
    for (l0, v0), C in zip(first, b.results()):
        assert torch.equal(l0, C.liv) and torch.equal(v0, C.val)


def test_tuner_choices_are_correct():
    from paper_1802_02619_gb300.tune import Tuner
    probs = _small_batch(count=8, seed=11)
    items = [(_dev(A), _dev(B), ma, mb) for A, B, ma, mb, _ in probs]
    t = Tuner(cache_path=None, reps=1)
    choice = t.tune_batch(items, per_class=1)
    b = lco.Batch([it + tuple(c) for it, c in zip(items, choice)], nstreams=4)
    b.run()
    for (A, B, ma, mb, _), C in zip(probs, b.results()):
        assert_contract_matches(C, _host(A), _host(B), ma, mb)
