"""Plain FP64 CPU oracle for the N-component free-energy lattice Boltzmann method.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only the tests, the smoke check of `__graft_entry__`
and the CPU-baseline / reference leg of `bench.py` use it.  It shares no code,
table or constant with the CUDA library; the only inputs both sides see come
from `nfe_workloads` (seeded initial fields and parameters).

What it computes (arXiv 2605.22214, Rennick, Zhang, Bingert, Krause and
Kusumaatmaja):
  * `thermo`      -- Sec. II: beta/kappa from sigma and D, the alpha/gamma
                     system (Eqs. 8-9), chemical potentials (Eq. 7), the
                     reduction-consistency term phi_j with its Lambda solves
                     (Eqs. 13-15), the stabiliser xi_j with its Theta solves
                     (Eqs. 16-19), and the flux potential of Eq. 12, both
                     literally and in the factored form C_i q_i(C) + (3D/4) lap C_i.
  * `lbm`         -- Sec. III: the D2Q9/D3Q19 populations f_k and g_{i,k},
                     isotropic stencils (Eqs. 35-36), the conservative force
                     (Eq. 34) and the non-conservative one (Eq. 31), moments
                     (Eqs. 37-38), TRT/BGK collision with forcing (Eqs. 22-30),
                     the Cahn-Hilliard LBE (Eqs. 39-43), halfway bounce-back
                     and the wall-gradient rule (Eqs. 44-45), periodic edges.
  * `observables` -- Sec. IV: Neumann angles (Eq. 51), the layered-Poiseuille
                     profile (Eqs. 53-58), Laplace pressure and lens angles
                     measured from fields, and the domain size L_i.
  * `boundaries`  -- Sec. III C on D2Q9: solid nodes inside the grid, velocity
                     and volume-fraction inlets and the convective outflow (the
                     conditions of the applications in Sec. V).

Every floating-point value is numpy float64.  The time stepper keeps all Q
populations f_k (f_0 included) and all (N-1) Q populations g_{i,k} with a
general tau_g, streams them, and bounces them back, in the order of Sec. III.
"""
from . import poly, thermo, lbm, observables, boundaries  # noqa: F401
