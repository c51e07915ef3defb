"""GB300-native matrix-free multigrid solver for pressurised phase-field fracture.

The compute path lives in the CUDA library built from csrc/ (C ABI declared in include/pff.h);
`paper_1902_08112_gb300.pff` is a thin ctypes binding with the same call names.  Importing this
package does not load the library; the first call through `pff` does, and raises if the
library is missing.
"""
__all__ = ["pff", "workloads"]
