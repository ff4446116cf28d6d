"""GB300 (sm_103a) implementation of the FC2T2 transform (Lange & Kutz, arXiv 2111.00110).

* ``capi``       -- ctypes binding of the C ABI in ``include/fc2t2.h`` (library in ``_build/``)
* ``transform``  -- ``Plan`` and the differentiable explicit layer ``fc2t2`` (needs torch)
* ``accessor``   -- the expansion's accessor: values, first and second partials at points or on
                    a meshgrid (``Plan.expand``)
* ``workloads``  -- seeded synthetic inputs
* ``build``      -- nvcc build of the CUDA library

Submodules are imported lazily so that ``workloads`` works without the CUDA library.
"""
__all__ = ["capi", "transform", "accessor", "workloads", "build"]
