"""FP64 CPU oracle for STEM-EELS maps (Brown, Ciston & Ophus, arXiv 1908.07628).

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The CUDA library never imports, links or calls it, and this package
imports nothing from the CUDA library: the only code the two sides share is the
seeded input generator in ``specimen``.

Contents
* ``multislice``  -- the conventional quadratic algorithm (Sec. III, first
  algorithm listing), written plainly with numpy FFTs.  This is the definition
  every other result is compared against.
* ``linear``      -- the scattering-matrix (PRISM-EELS) algorithm (Sec. III,
  second listing) in its exact store-and-stream form, FP64, used to check the
  paper's statement that the linear algorithm adds no error.
* ``dense``       -- the same physics with every operator written as an explicit
  dense matrix (DFT matrices, diagonals, interpolation kernels), for grids of
  16-32 pixels; shares no FFT call with the others.

Every function is pinned by a ``-m "not gpu"`` test against something other than
itself (closed forms, brute force, invariants, printed numbers of the paper).
"""
from . import multislice, linear, dense  # noqa: F401
