"""GB300-native optimal cycle mean solver (Howard policy iteration on CUDA).

The compute path is the hand-written sm_103a CUDA library ``libocm.so``
(C ABI in ``include/ocm.h``); this package builds it in-tree and binds it.
"""
from . import autotune, shard
from ._native import build, load
from .ocm import (OCM_MAX, OCM_MIN, BatchSolution, OCMError, OCMFunction, SccSolution, Solution,
                  backward, backward_batch, make_workspace, scc, solve, solve_batch, solve_scc,
                  workspace_bytes, workspace_bytes_batch)

__all__ = ["shard", "build", "load", "solve", "solve_batch", "solve_scc", "scc", "backward",
           "backward_batch", "OCMFunction", "OCMError", "Solution", "BatchSolution", "SccSolution",
           "make_workspace", "workspace_bytes", "workspace_bytes_batch", "OCM_MAX", "OCM_MIN"]
