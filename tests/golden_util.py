"""Readers for the text fixtures under tests/golden (each line cites the paper)."""

import os

import torch

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_complex_matrix(name: str) -> torch.Tensor:
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if not line:
                continue
            row = []
            for tok in line.split():
                re, im = tok.split(",")
                row.append(complex(float(re), float(im)))
            rows.append(row)
    return torch.tensor(rows, dtype=torch.complex128)


def read_numbers(name: str = "paper_numbers.txt") -> dict:
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if not line:
                continue
            k, v = line.split()
            out[k] = float(v)
    return out
