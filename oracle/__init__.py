"""FP64 CPU oracle of one two-fluid FlIC/Godunov time step (Kulikov 2013, GPUPEGAS).

This package is TEST INFRASTRUCTURE.  Only the test suite, the package smoke check
and the benchmark's CPU-baseline leg may import it.  The CUDA library never calls it
and the CUDA path shares no code with it.

Everything is plain numpy in float64, written to be checked against the paper by
eye: periodic shifts are ``np.roll``, every stage is a whole-array expression, and
the discrete Fourier transform is numpy's library FFT (a primitive, not part of the
method).  Section and equation references are to the paper:

* Sec. 2 (gas and Boltzmann-moment equations, the uniform grid),
* Sec. 2.1 (gas Eulerian stage: linearised Riemann face solution; Lagrangian stage:
  face-flux transport),
* Sec. 2.2 (Boltzmann-moment Eulerian stage: closed-form face solution of the 6x6
  linear system),
* Sec. 2.3 (Poisson equation with the 27-point stencil, solved by FFT),
* Sec. 2.4 (correctness checks kappa_gas, kappa_bme and the energy balance).

Where the paper is silent or garbled the oracle follows the readings listed in
``READINGS`` (module ``flic_oracle``); the CUDA path implements the same readings.
"""
from .flic_oracle import *  # noqa: F401,F403
