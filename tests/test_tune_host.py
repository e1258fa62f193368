"""Host logic of the autotuner (no GPU): the candidate list, the grouping of
a batch by signature, the sampling per group, the JSON cache and its reuse.
The timing of a configuration is replaced by a fixed table, so these tests
check which configurations the tuner asks for and what it does with the
answers, not the GPU timings themselves."""
import json
from collections import namedtuple

import pytest

import synth
from paper_1802_02619_gb300 import ContractPlan
from paper_1802_02619_gb300.tune import COL_ALGS, ROW_ALGS, Tuner

# the tuner reads only dims, sig and nnz of its operands on the host
Op = namedtuple("Op", "dims sig nnz")


def _op(T):
    return Op(list(T["dims"]), list(T["sig"]), int(T["liv"].shape[0]))


@pytest.fixture(scope="module")
def problems():
    fd = synth.config_fd2d(16)
    na = synth.config_rmat_na(bits=(8, 8, 6), nnz=2000)
    dc = synth.config_rmat_dcsr(bits=(10, 10, 6), nnz=5000)
    return {"fd": (_op(fd["A"]), _op(fd["B"]), fd["modes_a"], fd["modes_b"]),
            "na": (_op(na["A"]), _op(na["B"]), na["modes_a"], na["modes_b"]),
            "dc": (_op(dc["A"]), _op(dc["B"]), dc["modes_a"], dc["modes_b"])}


def _fake_times(calls, best):
    """time_config stand-in: `best` is fastest, every call is recorded."""
    def time_config(self, A, B, ma, mb, alg, bits, order=0):
        calls.append((alg, bits, order))
        return 1.0 if (alg, bits, order) == best else 2.0 + bits / 100.0 + order / 10.0
    return time_config


def test_candidates_start_with_table4_choice_and_cover_every_algorithm(problems):
    t = Tuner(cache_path=None)
    for A, B, ma, mb in problems.values():
        base = ContractPlan(A.dims, A.sig, A.nnz, B.dims, B.sig, B.nnz, ma, mb).info["alg"]
        cands = t.candidates(A, B, ma, mb)
        assert cands[0][0] == base
        assert {c[0] for c in cands} == set(ROW_ALGS + COL_ALGS)
        assert len(set(cands)) == len(cands)
        for alg, bits, order in cands:
            p = ContractPlan(A.dims, A.sig, A.nnz, B.dims, B.sig, B.nnz, ma, mb, alg=alg)
            if p.info["permute_a"] or p.info["permute_b"]:
                # operands to rearrange: digit caps x sort orders
                assert bits in (0, 6, 11) and order in (0, 1)
            else:
                assert (bits, order) == (0, 0)


def test_signature_separates_classes_and_sizes(problems):
    t = Tuner(cache_path=None)
    sigs = {k: t.signature(*v) for k, v in problems.items()}
    assert len(set(sigs.values())) == 3
    A, B, ma, mb = problems["fd"]
    bigger = Op(A.dims, A.sig, A.nnz * 64)
    assert t.signature(bigger, B, ma, mb) != sigs["fd"]
    assert t.signature(A, B, ma, mb) == sigs["fd"]


def test_tune_batch_groups_samples_and_caches(problems, tmp_path, monkeypatch):
    cache = tmp_path / "tune.json"
    A, B, ma, mb = problems["na"]
    best = ("CSR", 0, 0)
    calls = []
    monkeypatch.setattr(Tuner, "time_config", _fake_times(calls, best))
    items = [problems["na"]] * 5 + [problems["fd"]] * 3
    t = Tuner(cache_path=str(cache), reps=1)
    out = t.tune_batch(items, per_class=2)
    assert len(out) == len(items)
    # two signatures, two samples each, every candidate timed once per sample
    n_na = len(t.candidates(*problems["na"]))
    n_fd = len(t.candidates(*problems["fd"]))
    assert len(calls) == 2 * n_na + 2 * n_fd
    assert all(o == best for o in out)
    saved = json.loads(cache.read_text())
    assert set(saved) == {t.signature(*problems["na"]), t.signature(*problems["fd"])}
    for entry in saved.values():
        assert entry["choice"] == "CSR/0/0"
        assert entry["ms"]["CSR/0/0"] == 2.0    # summed over the two samples
    # a new tuner on the same cache times nothing for known signatures
    calls.clear()
    t2 = Tuner(cache_path=str(cache), reps=1)
    assert t2.tune_batch(items) == out
    assert calls == []
    # a new signature is tuned, the known ones are not
    out3 = t2.tune_batch(items + [problems["dc"]], per_class=1)
    assert len(calls) == len(t2.candidates(*problems["dc"]))
    assert out3[:-1] == out


def test_cache_entries_without_a_sort_order_read_as_order_zero(problems, tmp_path, monkeypatch):
    A, B, ma, mb = problems["fd"]
    t = Tuner(cache_path=None)
    cache = tmp_path / "old.json"
    cache.write_text(json.dumps({t.signature(A, B, ma, mb): {"choice": "CSRNA/6", "ms": {}}}))
    monkeypatch.setattr(Tuner, "time_config", _fake_times([], ("CSR", 0, 0)))
    assert Tuner(cache_path=str(cache)).tune_batch([problems["fd"]]) == [("CSRNA", 6, 0)]
