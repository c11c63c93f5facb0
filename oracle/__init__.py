"""Plain CPU FP64 oracle of the asynchronous DG (ADG / ADG-AT) method.

TEST INFRASTRUCTURE ONLY. This package is the slow, obviously-correct restatement of the
method that the CUDA path is checked against. Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / reference leg of ``bench.py`` may import it. The product path
(``paper_2404_03399_gb300``) never imports it, and it never imports the product path.

Modules:

* ``operators`` -- LGL nodes and weights, Lagrange basis, the reference-element matrices
  M, S, K-, K+, K_l, K_r (Section 2, Eq. matrices-reference).
* ``delays``    -- the paper's delay emulation: a uniform draw per PE boundary per step,
  binned by the probability set (Section 6.1), driven by SplitMix64.
* ``atflux``    -- asynchrony-tolerant flux coefficients solved from the Taylor
  constraints (Section 5, Eq. at-flux-constraints) in exact rational arithmetic.
* ``dg``        -- the fully discrete DG / ADG / ADG-AT solver (Eqs. DGscheme,
  asyncEulerDG, asyncEulerDGconserved, at-flux-gen) with explicit RK schemes, in torch
  float64 on the CPU so that autograd supplies an independent discrete gradient.
* ``fourier``   -- amplification matrices of the synchronous and asynchronous schemes
  (Section 4.2) and a Fourier-space recurrence for the stage-consistent delayed scheme.

Parity pins live in ``tests/test_oracle_*.py``. Functions that no pin fixes say
"parity unpinned" in their docstring.
"""
