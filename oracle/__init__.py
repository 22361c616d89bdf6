"""CPU FP64 oracle for the sparse-monomial engine and the affine-normal direction.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, calls or links
this package: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` use it.  It shares no code with the CUDA library; the only
common module is the seeded input generator ``paper_2604_06575_b300.workloads``,
which draws inputs and does none of the method's arithmetic.

Each function is the plain definition of what the method computes, written for
a reader to check against the paper by eye (slow on purpose):

* ``engine``  -- variable-id alignment, product expansion, simplify (Sec. 3.2,
  Sec. 2 "simplify", Table "coresemantics"); canonical monomial order (Sec. 3.1).
* ``derivs``  -- value, gradient, Hessian and third-derivative tensor of a
  polynomial by falling factorials (Sec. 3.3).
* ``affine``  -- the affine-normal direction (Sec. 5): the 'ad' route (full
  third tensor) and the stochastic log-det route (Hutchinson + CG).
* ``rng``     -- the SplitMix64 counter-based generator used for probes.
* ``mlp``     -- FP64 forward/backward of the learned preconditioner network.

Pins (tests marked ``not gpu``) tie every function to something other than
itself: the paper's printed examples, closed forms, brute force, finite
differences and the geometric invariants of the affine normal.
"""
