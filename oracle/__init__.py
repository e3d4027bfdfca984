"""FP64 CPU oracle for complex-Jacobian gain calibration (Smirnov & Tasse, arXiv:1502.06974).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call or link this
package: only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
(and its ``--impl reference`` arm) use it.  It shares no code with the CUDA library.

Modules
  wirtinger    explicit complex Jacobians (Sect. 1 eq. JJ; Sect. 2 eq. JJ:di; Sect. 2.5;
               Sect. 4 eq. JJ:pol with the 4x4 forms of App. B), J^H J, J^H r, and the full
               GN / LM solvers of App. C.
  blocks       closed forms of the per-antenna blocks of J^H J and J^H r / J^H d that the
               approximate-inverse methods use (eqs. JHJ:DI:tf, JHR:DI:tf, JHJ:DD:unpol,
               JHR:DD:unpol, JHJ:pol and the polarized J^H R).
  diagonal     the paper's approximate-inverse iterations step by step: StefCal (eq. stefcal,
               eq. stefcal-lambda-average), polarized StefCal (eq. update:DI:diag:pol, read as
               [sum D Y^H][sum Y Y^H]^-1) and CohJones (Sect. 3.2.2).
  smooth       smoothing in time and frequency (Sect. 3.4): per-sample gains from the ratio of two
               kernel convolutions (eq. JHJ:diag:smooth), scalar and 2x2.
  cpu_lm.cpp   the same StefCal + LM method in FP64 C++/OpenMP (the all-core CPU comparator).
  gauge        gauge alignment and the relative gain error used for parity.

Every function works in complex128 / float64 whatever the input precision.
"""
