"""GB300-native optimal cycle mean solver (Howard policy iteration on CUDA).

The compute path is the hand-written sm_103a CUDA library ``libocm.so``
(C ABI in ``include/ocm.h``); this package builds it in-tree and binds it.
"""
from ._native import build, load
from .ocm import (OCM_MAX, OCM_MIN, OCMError, OCMFunction, Solution, backward, make_workspace,
                  solve, workspace_bytes)

__all__ = ["build", "load", "solve", "backward", "OCMFunction", "OCMError", "Solution",
           "make_workspace", "workspace_bytes", "OCM_MAX", "OCM_MIN"]
