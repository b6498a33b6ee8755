"""GB300-native OCD soft-output detection for massive MU-MIMO-OFDM.

The detector (Algorithm 1 of arXiv 1611.08779 with the Eq. 9 soft output)
runs in the CUDA library libocd.so; this package is its Python binding plus
the seeded input generator and the subcarrier partition used by the benchmark.
"""
from ._native import OcdError  # noqa: F401
from .api import (bits_per_symbol, fault_status, make_staging, ocd_detect,  # noqa: F401
                  ocd_detect_host, version)
from .batched import (BatchedGraph, Cell, Tune, make_cell, make_workspace,  # noqa: F401
                      ocd_autotune_batched, ocd_detect_batched, ocd_detect_batched_static)
from .shard import shard_range  # noqa: F401
from .unfolded import UnfoldedBCE, UnfoldedOCD, unfolded_bce_loss, unfolded_ocd  # noqa: F401
