"""FP64 CPU oracle for Monte-Carlo line-by-line ray tracing (test infrastructure).

This package is test infrastructure only.  It is imported, called, linked or
executed by the tests, by ``__graft_entry__.smoke()`` and by the benchmark's
CPU-baseline leg, and by nothing else: the product path (the CUDA library and
its Python binding) never routes through it and shares no code with it.

What it computes, following Collange, Daumas and Defour, "Graphic processors
to speed-up simulations for the design of high performance solar receptors"
(Section 3):

* ``physics``  -- Eq. (S) line intensity at temperature, number density of the
  absorber, Lorentz / Doppler widths, Lorentz and Voigt profiles f, and the
  Planck function of Eq. (planck), all in float64.
* ``kappa``    -- Eq. (tau): the absorption coefficient kappa(nu_j, T_k) as the
  direct sum over lines within the wing cutoff (single absorbing gas).
* ``trace``    -- the Monte-Carlo ray-tracing estimator through finite volumes
  (Section 3, Fig. "Monte-Carlo ray-tracing"): Philox4x32-10 draws, emission
  weights from Eq. (planck), cell-by-cell walk with the Beer-Lambert first term
  of Eq. (I), per-cell absorbed-power tally and energy balance.  The walk is in
  plain C (``trace.c``) because it is a per-ray loop.
* ``mlp``      -- float64 forward / backward of the surrogate network that can
  stand in for the kappa lookup.

Every function names the equation or section it follows.  Parity status of
each function is stated in its own docstring; all of them are pinned by the
CPU tests to closed forms, invariants, brute force or an independent library.
"""
