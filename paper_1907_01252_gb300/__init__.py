"""GB300 implementation of the data-parallel hot path of Parareal time stepping
for monolithic ALE fluid-structure interaction (Margenberg & Richter).

The CUDA library (csrc/, C ABI in include/fsi.h) does all the arithmetic; the
binding in `fsi.py` (import it as a submodule) only marshals arguments.
`workloads.py` describes the synthetic inputs.
"""
