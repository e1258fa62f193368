"""Sorting and addition on the GPU against the oracle (bit for bit: LIV
order is unique up to stable ties, and each value is alpha*a, beta*b or
their sum, each operation rounded once on both sides), and the Eq. 4
combinatorial Laplacian chain of Sec. 6."""
import numpy as np
import pytest
import torch

import oracle
import paper_1802_02619_gb300 as lco
import synth
from gpu_util import dev
from paper_1802_02619_gb300.laplacian import combinatorial_laplacian

pytestmark = pytest.mark.gpu


def _rand(dims, nnz, seed):
    rng = np.random.default_rng(seed)
    total = int(np.prod(dims))
    liv = np.sort(rng.choice(total, size=min(nnz, total), replace=False)).astype(np.int64)
    return {"dims": list(dims), "sig": list(range(len(dims) - 1, -1, -1)), "liv": liv,
            "val": rng.uniform(-1, 1, liv.shape[0])}


def _host(T):
    return T.liv.cpu().numpy(), T.val.cpu().numpy()


@pytest.mark.parametrize("nnz", [0, 1, 2047, 2048, 2049, 100003, 1 << 20])
def test_sort_matches_oracle(nnz):
    T = _rand([97, 101, 103, 107], max(nnz, 1), nnz)
    perm = np.random.default_rng(nnz + 1).permutation(len(T["liv"]))[:nnz]
    U = {"dims": T["dims"], "sig": T["sig"], "liv": T["liv"][perm], "val": T["val"][perm]}
    S = lco.sort(dev(U))
    rl, rv = oracle.sort(U["liv"], U["val"])
    gl, gv = _host(S)
    assert np.array_equal(gl, rl) and np.array_equal(gv.view(np.int64), rv.view(np.int64))


def test_sort_keeps_equal_livs_in_input_order():
    rng = np.random.default_rng(9)
    liv = rng.integers(0, 300, 50000).astype(np.int64)
    val = np.arange(50000, dtype=np.float64)
    S = lco.sort(lco.LcoTensor([1000], [0], torch.tensor(liv, device="cuda"), torch.tensor(val, device="cuda")))
    rl, rv = oracle.sort(liv, val)
    gl, gv = _host(S)
    assert np.array_equal(gl, rl) and np.array_equal(gv, rv)


@pytest.mark.parametrize("na,nb,alpha,beta", [(5000, 7000, 1.0, 1.0), (2048, 2048, 2.0, -0.5),
                                              (0, 3000, 1.0, 3.0), (3000, 0, -1.0, 1.0), (0, 0, 1.0, 1.0),
                                              (300000, 250000, 0.75, 1.25)])
def test_add_matches_oracle(na, nb, alpha, beta):
    A, B = _rand([200, 300, 50], max(na, 1), na), _rand([200, 300, 50], max(nb, 1), nb + 7)
    A = {**A, "liv": A["liv"][:na], "val": A["val"][:na]}
    B = {**B, "liv": B["liv"][:nb], "val": B["val"][:nb]}
    C = lco.add(dev(A), dev(B), alpha, beta)
    rl, rv = oracle.add(alpha, A, beta, B)
    gl, gv = _host(C)
    assert np.array_equal(gl, rl) and np.array_equal(gv.view(np.int64), rv.view(np.int64))


def test_add_cancellation_keeps_explicit_zeros():
    A = _rand([64, 64, 64], 40000, 11)
    C = lco.add(dev(A), dev(A), 1.0, -1.0)
    gl, gv = _host(C)
    assert np.array_equal(gl, A["liv"]) and np.all(gv == 0.0)


def _oracle_chain(N):
    """The Eq. 4 chain by the oracle, with the per-entry bound sum |a||b|
    of each term carried through the same permutation and addition."""
    d, dl = synth.fd_matrix(N), synth.kronecker_delta(N)
    rm = [3, 2, 1, 0]
    by = dict(zip(("liv", "val"), oracle.contract(d, dl, [], [])[:2]), dims=[N] * 4, sig=rm)
    cl, cv, cab = oracle.contract(by, d, [1], [0])
    cy = {"liv": cl, "val": cv, "dims": [N] * 4, "sig": rm}
    pl, pv = oracle.permute([N] * 4, [2, 3, 0, 1], rm, cl, cv)
    pl2, pab = oracle.permute([N] * 4, [2, 3, 0, 1], rm, cl, cab)
    assert np.array_equal(pl, pl2)
    al, av = oracle.add(1.0, cy, 1.0, {"liv": pl, "val": pv})
    bl, bab = oracle.add(1.0, {"liv": cl, "val": cab}, 1.0, {"liv": pl, "val": pab})
    assert np.array_equal(al, bl)
    return al, av, bab


@pytest.mark.parametrize("N", [15, 31])
def test_laplacian_chain_matches_oracle(N):
    a = combinatorial_laplacian(dev(synth.fd_matrix(N)), dev(synth.kronecker_delta(N)))
    rl, rv, rab = _oracle_chain(N)
    gl, gv = _host(a)
    assert np.array_equal(gl, rl)
    # each term within 1e-13 sum |a||b| of its products; the sum adds both bounds
    err = np.abs(gv - rv)
    assert np.all(err <= 1e-13 * rab), f"worst {err.max()}"


@pytest.mark.parametrize("N", [31, 2047])
def test_laplacian_maps_quadratics_to_four(N):
    """a_ijkl x_kl with x_kl = k^2 + l^2 is exactly 4 everywhere (Eq. 1 is
    exact on quadratics); at N = 2047 (the paper's largest image) a has
    ~25M entries."""
    a = combinatorial_laplacian(dev(synth.fd_matrix(N)), dev(synth.kronecker_delta(N)))
    y = lco.contract(a, dev(synth.quadratic_field(N)), [3, 2], [0, 1])
    assert y.nnz == N * N
    assert torch.equal(y.liv, torch.arange(N * N, device="cuda"))
    assert bool((y.val == 4.0).all())
