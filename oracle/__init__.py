"""FP64 CPU oracle for the high-order lattice Boltzmann step with Hermite body sources.

TEST INFRASTRUCTURE.  This package is the independent reference the CUDA path
is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import, call,
link or execute anything under ``oracle/``; the product package never does.
It shares no code, header, table or constant generator with the CUDA path.

Modules:
  lattice   velocity sets and Gauss-Hermite weights (Sec. 4.1, Table 1)
  hlbm_oracle.c / solver   the FP64 time step (Eqs. 2.2, 3.3, 3.7, 3.8, 3.12,
            4.4, 4.5; Table 2), two-pass, periodic or between Tamm-Mott-Smith
            walls (Sec. 4.3, Eqs. 4.7-4.8)
  eos       equations of state and the Maxwell equal-area construction (Sec. 5.4)
  analytic  closed forms used as physics pins
  adjoint   discrete adjoint of the body-force step (FP64, reverse mode)
"""
