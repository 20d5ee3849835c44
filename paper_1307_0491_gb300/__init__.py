"""GB300 (sm_103a) time stepper for the Saint-Venant--Exner system with the
relaxation-solver fluxes of arXiv:1307.0491.

* ``paper_1307_0491_gb300.sve``       -- Python binding of the C ABI
  (include/sve.h) of ``libsve.so`` and a ``Solver`` convenience class.
* ``paper_1307_0491_gb300.build``     -- in-tree nvcc build of ``libsve.so``.
* ``paper_1307_0491_gb300.workloads`` -- seeded synthetic inputs.

Importing the package loads nothing; ``sve.load()`` loads the CUDA library
and fails loudly if it has not been built.
"""
__all__ = ["sve", "build", "workloads"]
