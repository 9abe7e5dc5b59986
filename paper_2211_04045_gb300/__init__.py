"""GB300 (sm_103a) implementation of the two-way continuous collision handling
step of Wang et al., "Fast GPU-Based Two-Way Continuous Collision Handling"
(arXiv 2211.04045).

``cch`` is the binding of the C ABI in ``include/cch.h`` (the CUDA library
``libcch.so``); ``scenes`` generates the seeded synthetic inputs.  Importing the
package loads nothing; the library is loaded on first use.
"""
__all__ = ["cch", "scenes", "build"]
