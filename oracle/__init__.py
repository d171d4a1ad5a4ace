"""FP64 CPU oracle of the Kinetic Compressive Sensing hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it.  It shares no code with the CUDA path
(no kernels, headers, tables or helpers) and imports nothing from it.

Every function is a plain restatement of the paper (Scipioni et al., "Kinetic
Compressive Sensing"), in float64, written for a reader to check by eye:

* ``projector``  Joseph system matrix p_vd and its transpose (Eq. 2 sums).
* ``kinetics``   FDG two-tissue irreversible model, frame-integrated, and its
                 Jacobian (Sec. II-C "Fast parallel GPU implementation").
* ``osl``        OS-MAP-OSL update with the kinetics-derived prior (Eq. 2-3).
* ``lm``         Huber potential (Eq. 5-6) and the MAP Levenberg-Marquardt
                 step (Eq. 4).
* ``icm``        the ICM alternation (Sec. II-D).

Parity status of every function is listed in each module's header.
"""
from . import projector, kinetics, osl, lm, icm  # noqa: F401
