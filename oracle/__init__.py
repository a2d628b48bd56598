"""FP64 CPU oracle for the EvoL force step -- TEST INFRASTRUCTURE ONLY.

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package.  The CUDA library never calls it and has no fallback to it.
"""
from .oracle import (  # noqa: F401
    build_oracle, lib, kernels, OracleTree, force_step, kdk, eta_from_nnei, hash_id, ewald,
    TimeStep, timestep_criteria, global_timestep, run, Bins, run_bins, step_ticks, active_force_step,
)
