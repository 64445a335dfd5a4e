"""Plain, slow FP64 CPU oracle for the Brillouin-kernel overlap operator.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute anything in this package; only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.
It shares no code with the CUDA library (no kernels, headers, tables or
helpers); the only common code is the seeded input generator
``synthetic_fields``, which holds none of the method's arithmetic.

Everything is numpy in complex128 and follows Duerr & Koutsou, "On the
suitability of the Brillouin action as a kernel to the overlap procedure"
(arXiv:1701.00726):

  conventions  lattice indexing, chiral gamma basis, the 81-offset numbering
               (App. C)
  links        off-axis links W_d(n) as the literal average over all k!
               shortest paths (App. C, Brillouin operator flop count)
  dirac        D_wil and D_bri (Eqs. def_wils / def_bril, stencil weights from
               the momentum forms of App. A), clover term
  kl           diagonal / upper-diagonal Kenney-Laub rationals (Sec. 3,
               Eqs. def_gell, KLnn_parfrac, Tabs. 1, 2, 5, 6)
  mscg         multi-shift CG (Sec. 3.3, App. B) in the Jegerlehner form
  overlap      D_ov = rho (1 + gamma5 f_nn(H)) (Eq. def_over) and its massive
               forms (Eqs. def_mass_traditional, upshot_complete)
  dense        dense matrices and eigendecomposition on tiny lattices
  freefield    momentum-space closed forms (App. A)
  grad         gradient of Re<eta, D_ov psi> (adjoint by the chain rule)

Parity status: the clover term follows the standard clover-leaf reading
(the paper does not define sigma_{mu nu} F_{mu nu}); it is pinned by
hermiticity, gauge covariance and its vanishing on the free field, and is
"parity unpinned" against the paper itself.
"""
