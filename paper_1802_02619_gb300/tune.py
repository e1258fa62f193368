"""Autotuner for the contraction path.

For a problem the tuner times candidate configurations of the library --
the algorithm (Table 4's choice and the alternatives that are always
correct on the GPU: CSR, CSRNA, DCSR, SOP and, for column-major inputs, the
column variants), and for the operand permutations the radix digit-width
cap (the tile's bucket count) and the sort order (LSD passes only, or high
digit first with each high-digit bucket sorted inside one CTA when the
device finds the buckets small enough) -- on the problem's own data, and
keeps the fastest.  For a batch it groups
problems by a signature (sparsity classes, which operands need rearranging,
size bucket) and tunes a few samples per group; decisions are cached in a
JSON file (``LCO_TUNE_CACHE``) keyed by the signature.
"""
from __future__ import annotations

import json
import math
import os
import statistics

import torch

from . import ContractPlan, LcoTensor

ROW_ALGS = ("CSR", "CSRNA", "DCSR", "SOP")
COL_ALGS = ("CSC", "CSCNA", "DCSC")


def _bucket(n: int) -> int:
    return int(math.log2(max(n, 1)) // 2)


class Tuner:
    def __init__(self, cache_path: str | None = None, reps: int = 3):
        self.cache_path = cache_path or os.environ.get("LCO_TUNE_CACHE")
        self.reps = reps
        self.cache = {}
        if self.cache_path and os.path.exists(self.cache_path):
            with open(self.cache_path) as fh:
                self.cache = json.load(fh)

    def save(self):
        if self.cache_path:
            tmp = self.cache_path + ".tmp"
            with open(tmp, "w") as fh:
                json.dump(self.cache, fh, indent=1, sort_keys=True)
            os.replace(tmp, self.cache_path)

    def signature(self, A: LcoTensor, B: LcoTensor, modes_a, modes_b) -> str:
        p = ContractPlan(A.dims, A.sig, A.nnz, B.dims, B.sig, B.nnz, modes_a, modes_b)
        i = p.info
        return (f"{i['alg']}|ca{i['class_a']}|cb{i['class_b']}|pa{i['permute_a']}|pb{i['permute_b']}"
                f"|na{_bucket(A.nnz)}|nb{_bucket(B.nnz)}")

    def candidates(self, A, B, modes_a, modes_b):
        """(alg, max_digit_bits, radix_order) triples to time."""
        base = ContractPlan(A.dims, A.sig, A.nnz, B.dims, B.sig, B.nnz, modes_a, modes_b)
        algs = [base.info["alg"]] + [a for a in ROW_ALGS + COL_ALGS if a != base.info["alg"]]
        out = []
        for alg in algs:
            p = ContractPlan(A.dims, A.sig, A.nnz, B.dims, B.sig, B.nnz, modes_a, modes_b, alg=alg)
            if p.info["permute_a"] or p.info["permute_b"]:
                out += [(alg, b, o) for b in (0, 6, 11) for o in (0, 1)]
            else:
                out.append((alg, 0, 0))
        return out

    def time_config(self, A, B, modes_a, modes_b, alg, bits, order=0) -> float:
        p = ContractPlan(A.dims, A.sig, A.nnz, B.dims, B.sig, B.nnz, modes_a, modes_b, alg=alg,
                         max_digit_bits=bits, radix_order=order)
        p.ensure_workspace(0, A.liv.device)
        p.symbolic(A, B)
        f = p.result()["f"]
        p.ensure_workspace(f, A.liv.device)
        c_liv = torch.empty(max(f, 1), dtype=torch.int64, device=A.liv.device)
        c_val = torch.empty(max(f, 1), dtype=torch.float64, device=A.liv.device)
        p.run(A, B, c_liv[:f], c_val[:f])
        torch.cuda.synchronize()
        ts = []
        for _ in range(self.reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            p.run(A, B, c_liv[:f], c_val[:f])
            e1.record()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        if p.result()["status"] != 0:
            return float("inf")
        return statistics.median(ts)

    def tune(self, A, B, modes_a, modes_b):
        """(alg, max_digit_bits, radix_order, {config: ms}) for one problem."""
        times = {}
        for alg, bits, order in self.candidates(A, B, modes_a, modes_b):
            times[f"{alg}/{bits}/{order}"] = self.time_config(A, B, modes_a, modes_b, alg, bits, order)
        best = min(times, key=times.get)
        alg, bits, order = best.split("/")
        return alg, int(bits), int(order), times

    def tune_batch(self, items, per_class: int = 2):
        """Per item (alg, max_digit_bits, radix_order): groups by signature,
        tunes up to per_class samples of each new group, reuses cached
        decisions."""
        groups = {}
        for idx, (A, B, ma, mb) in enumerate(items):
            groups.setdefault(self.signature(A, B, ma, mb), []).append(idx)
        decision = {}
        for sig, idxs in groups.items():
            if sig not in self.cache:
                totals = {}
                for idx in idxs[:per_class]:
                    A, B, ma, mb = items[idx]
                    *_, times = self.tune(A, B, ma, mb)
                    for k, v in times.items():
                        totals[k] = totals.get(k, 0.0) + v
                best = min(totals, key=totals.get)
                self.cache[sig] = {"choice": best, "ms": totals}
            parts = self.cache[sig]["choice"].split("/")
            alg, bits, order = parts[0], int(parts[1]), int(parts[2]) if len(parts) > 2 else 0
            for idx in idxs:
                decision[idx] = (alg, bits, order)
        self.save()
        return [decision[i] for i in range(len(items))]
