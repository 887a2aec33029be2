"""FP64 CPU oracle for GeRaF's lensless RF rendering hot path.

TEST INFRASTRUCTURE ONLY: importable by ``tests/``, ``__graft_entry__.smoke()``
and the benchmark's CPU-baseline / reference leg, never by the CUDA product
package. See ``geraf_oracle.py`` for the definitions and their paper passages.
"""
