"""GB300 (sm_103a) frozen Gaussian approximation of the acoustic wave equation.

The compute path is libfga (CUDA kernels behind the C ABI of include/fga.h);
`fga` is its Python binding and `workloads` builds seeded synthetic inputs.
Importing the package does not load the CUDA library; `fga.load()` does.
"""

__all__ = ["fga", "workloads", "build"]
