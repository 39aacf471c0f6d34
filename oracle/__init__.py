"""Plain, slow FP64 CPU oracle of the channel-flow time step.

TEST INFRASTRUCTURE ONLY.  Nothing in the library imports this package; only
the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may call it.  It shares no code with the CUDA path.

The oracle spells out the discretisation of the method step by step with
dense operators and library primitives (numpy matrix products, dense LU via
``numpy.linalg.solve``), without blocking, fusion or fast transforms:

* ``spectral``  Chebyshev (wall-normal) and Fourier (wall-parallel) operators.
* ``channel``   one RK3 / Crank-Nicolson step of the velocity-vorticity
  formulation, the wall action, observation, wall shear and reward.
* ``stability`` the Orr-Sommerfeld eigenvalue problem used to pin the linear
  dynamics (Tollmien-Schlichting growth rate at Re = 10^4, alpha = 1).
* ``policy``    the shared agent policy (a multilayer perceptron on the
  sensing-plane window above each actuator, Sec. 3.2) of the on-device
  control mode.

Every function cites the part of the paper it follows.  The paper fixes the
Fourier x Chebyshev basis (Sec. 3.1), the RK3 + Crank-Nicolson time scheme
(Sec. 3.1), the wall blowing/suction action with its linear ramp and clip
(Sec. 3.2), the sensing plane snapped up to a Chebyshev node (Sec. 3.2), the
wall-shear reward (Sec. 3.2) and the opposition-control law (Sec. 4.1,
equation for v_w).  Where it is silent this oracle takes these readings: a
closed channel y in [-1, 1] with the action on the lower wall (an open channel
with a free-slip top as the option top_bc = 1), the SMR low-storage RK3 with
alpha = beta, the 3/2 rule, and the velocity-vorticity form with the v problem
solved as one coupled dense system.
"""

from . import spectral, channel, stability, policy  # noqa: F401
