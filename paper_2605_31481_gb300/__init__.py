"""Batched Featherstone rigid-body dynamics on GB300 (sm_103a).

The compute path is libfst.so (hand-written CUDA, C ABI in include/fst.h);
`api` is its thin PyTorch binding. Importing the package does not load the
library; the first call does, and fails loudly if it has not been built.
"""
from .api import Model, MultiBatch, fk, jacobian, rnea, crba, aba, eval, soa, aos  # noqa: F401

__all__ = ["Model", "MultiBatch", "fk", "jacobian", "rnea", "crba", "aba", "eval", "soa", "aos"]
