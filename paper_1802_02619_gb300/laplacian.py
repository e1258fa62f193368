"""The combinatorial Laplacian of Eq. 4 through the library's public calls,
evaluated left to right as Sec. 2 describes:

    a_ijkl = d_ii' delta_jl d_i'k  +  d_jj' delta_ik d_j'l

Each term is an outer product with the Kronecker delta followed by the
Eq. 17 product, b_ii'jl d_i'k; the second term's product comes out named
(j,i,k,l), is re-sorted into the first term's order (i,j,l,k) -- the
permutation of Sec. 3.2 -- and the two are added."""
from __future__ import annotations

from . import LcoTensor, add, contract, radix_permute

ROW_MAJOR4 = [3, 2, 1, 0]
# the second term's product, read with the first term's mode names (i,j,l,k):
# its most significant mode j is mode 1, then i (0), k (3), l (2)
SECOND_TERM_SIG = [2, 3, 0, 1]


def first_term(d: LcoTensor, delta: LcoTensor) -> LcoTensor:
    """c_ijlk = (d_ii' delta_jl) d_i'k."""
    b = contract(d, delta, [], [])          # b_ii'jl
    return contract(b, d, [1], [0])         # modes (i, j, l, k)


def combinatorial_laplacian(d: LcoTensor, delta: LcoTensor) -> LcoTensor:
    """a_ijkl of Eq. 4 with modes named (i, j, l, k), row-major."""
    cy = first_term(d, delta)
    cx = first_term(d, delta)               # c_jikl: the same steps along the other axis
    cx_named = LcoTensor(list(cx.dims), SECOND_TERM_SIG, cx.liv, cx.val)
    cx_sorted = radix_permute(cx_named, ROW_MAJOR4)
    return add(cy, cx_sorted)
